// Pipelined per-tile kernels of the BF16 form for FC and ResNet networks.
//
// The general fused kernels (fused.cu) run each contraction of a tile and
// then its epilogue, one after the other: the tensor cores wait while the
// epilogue warps read the accumulator, apply the activation and write the
// next operand, and the epilogue warps wait while the next contraction runs.
// Here the two overlap within one tile:
//   * TMEM holds two accumulators of 256 columns, used by alternate
//     contractions (phase q writes buffer q % 2), so contraction q + 1 can
//     run while the epilogue of phase q still reads buffer q % 2;
//   * contraction q + 1 reads its operand tile 64 columns (one K slice) at a
//     time, and the epilogue of phase q releases the operand slab by slab
//     (mbarrier `slab[s]`): the contraction of layer l + 1 starts as soon as
//     the first 64 columns of h_l are written, not when all 256 are;
//   * the ResNet residual of the forward sweep is the BF16 operand tile
//     itself (h_l = bf16(h_{l-1} + act(a_l)), the recomputation of the
//     backward kernel does the same), while y = w_o^T h_L + b_o is
//     accumulated in FP32 from every layer's act(a_l) (h_L = h_0 +
//     sum_l act(a_l)), so the BF16 rounding of the stream enters y only
//     through the contractions' operands;
//   * the reverse (Z) sweep's residual g_{l-1} = g_l + W_l^T e_l is
//     accumulated by the tensor cores: the epilogue copies g_l into the next
//     contraction's buffer before releasing the first slab, and the
//     contraction adds W_l^T e_l onto it.
// Four epilogue warpgroups (16 warps) share the columns: in every 64-column
// slab, warpgroup g owns columns 16 g .. 16 g + 15 of all 128 rows (one TMEM
// lane per thread).  Warpgroup 0 holds the producer (weight slices through a
// TMA ring), the MMA issuer (one thread), and the store warp (TMA stores of
// the operand stacks, the next tile's input rows, and the release of the
// operand tile for the next phase's writes).
//
// Every wait is bounded and also gives up once another role has aborted; a
// role that gives up sets the device error flag (fbsde_check_finite reports
// FBSDE_ERR_TIMEOUT), and before TMEM is released each role waits (bounded)
// for the asynchronous work it issued: the producer for its last TMA loads,
// the MMA issuer for its last tcgen05.mma (a commit to a drain barrier), the
// store warp for its input loads and bulk stores.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <string>
#include <type_traits>

#include "fused_common.cuh"

namespace fbsde {

constexpr int kPGroups = 4;                      // epilogue warpgroups
constexpr int kPThreads = 128 * (1 + kPGroups);  // warpgroup 0: producer, MMA, store warp, spare
constexpr int kPStages = 3;                      // weight ring stages of the forward kernel (32 KB each)
constexpr int kPBwdStages = 3;                   // the backward kernel's ring (its two operand tiles take 128 KB)
// 20 warps: 5 per SM sub-partition, 96 registers per thread at launch;
// warpgroup 0 then drops to kPRegsCtl and the epilogue warpgroups rise to
// kPRegsEpi (setmaxnreg).
constexpr int kPRegsLaunch = 96;
constexpr uint32_t kPRegsCtl = 32, kPRegsEpi = 112;
static_assert(128u * kPRegsCtl + 128u * kPGroups * kPRegsEpi <= (uint32_t)kPThreads * kPRegsLaunch,
              "register split exceeds the launch allocation");
static_assert(kPRegsCtl + kPGroups * kPRegsEpi <= 512, "register split exceeds an SM sub-partition");
static_assert(16384 / ((kPThreads / 32 + 3) / 4 * 32) >= kPRegsLaunch, "launch registers per sub-partition");

// Barriers and flags of one CTA (shared memory).
struct PipeBars {
    uint64_t bfull[kPStages > kPBwdStages ? kPStages : kPBwdStages], bempty[kPStages > kPBwdStages ? kPStages : kPBwdStages];
    uint64_t accf[2];   // contraction into TMEM buffer b complete
    uint64_t slab[4];   // 64-column slab s of the operand tile written (one arrival per epilogue warp)
    uint64_t tfree;     // the operand tile may be written by the next phase (store warp)
    uint64_t xfull;     // this tile's input rows have arrived
    uint64_t ybar;      // Y partial sums of the four warpgroups are in place (one arrival per warp)
    uint64_t gate;      // never completed: the test hook's first wait
    uint64_t drain;     // MMA issuer: its last contractions have completed
    uint64_t tread;     // backward: every epilogue warp has read its TMEM columns of an up-sweep phase
    uint32_t tslot;
    int abort_flag;
};

// Bounded wait that also gives up as soon as another role has aborted (the
// flag's shared-memory address in abort_s).  32-bit clock arithmetic: the
// control warps run on 32 registers, and a budget below 2^31 cycles (about
// a second) is exact under one wrap of the counter.
__device__ __forceinline__ bool try_wait_s(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool pwait(uint32_t bar, uint32_t parity, uint32_t budget, uint32_t abort_s) {
    if (try_wait_s(bar, parity)) return true;
    const uint32_t t0 = (uint32_t)clock();
    while (true) {
        if (try_wait_s(bar, parity)) return true;
        uint32_t ab;
        asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(ab) : "r"(abort_s) : "memory");
        if (ab) return false;
        if ((uint32_t)clock() - t0 > budget) return false;
    }
}

__device__ __forceinline__ bool pwait(uint64_t* bar, uint32_t parity, uint32_t budget, uint32_t abort_s) {
    return pwait(tc::smem_u32(bar), parity, budget, abort_s);
}

__device__ __forceinline__ void pfail(int* err, uint32_t abort_s) {
    if (err) atomicExch(err, 2);
    asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(abort_s), "r"(1u) : "memory");
}

// A wait budget for pwait (at most 2^31 - 1 cycles).
__host__ __device__ __forceinline__ uint32_t pbudget(long long b) {
    return (uint32_t)(b < 0x7fffffffLL ? (b > 0 ? b : 0) : 0x7fffffffLL);
}

// The waits at the end, for asynchronous work already issued: bounded, and
// not cut short by the abort flag.
constexpr long long kDrainBudget = 400000000LL;  // ~0.2 s

__device__ __forceinline__ void st_tile16_packed(uint8_t* tile, int row, int col, const uint32_t (&u)[8]) {
    uint8_t* base = tile + (col >> 6) * 16384;
    *reinterpret_cast<uint4*>(base + tc::sw128_offset(row, (col & 63) >> 3)) = make_uint4(u[0], u[1], u[2], u[3]);
    *reinterpret_cast<uint4*>(base + tc::sw128_offset(row, ((col & 63) >> 3) + 1)) = make_uint4(u[4], u[5], u[6], u[7]);
}
__device__ __forceinline__ void ld_tile16_packed(const uint8_t* tile, int row, int col, uint32_t (&u)[8]) {
    const uint8_t* base = tile + (col >> 6) * 16384;
    const uint4 a = *reinterpret_cast<const uint4*>(base + tc::sw128_offset(row, (col & 63) >> 3));
    const uint4 b = *reinterpret_cast<const uint4*>(base + tc::sw128_offset(row, ((col & 63) >> 3) + 1));
    u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
    u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
}
__device__ __forceinline__ void tmem_ld16w(uint32_t taddr, uint32_t (&r)[16]) { tc::tmem_ld16(taddr, r); }

// Copy this thread's accumulator columns (16 per slab, nkw slabs) from TMEM
// buffer `from` to buffer `to` (same lanes), two slabs per round trip.
__device__ __forceinline__ void tmem_copy64(uint32_t from, uint32_t to, int eg, int nkw) {
#pragma unroll
    for (int s = 0; s < 4; s += 2) {
        if (s < nkw) {
            uint32_t u[16], v[16];
            tc::tmem_ld16(from + (uint32_t)(s * 64 + eg * 16), u);
            if (s + 1 < nkw) tc::tmem_ld16(from + (uint32_t)((s + 1) * 64 + eg * 16), v);
            tc::tmem_wait_ld_regs(u);
            tc::tmem_wait_ld_regs(v);
            tc::tmem_st16(to + (uint32_t)(s * 64 + eg * 16), u);
            if (s + 1 < nkw) tc::tmem_st16(to + (uint32_t)((s + 1) * 64 + eg * 16), v);
        }
    }
    tc::tmem_wait_st();
}

// The warp's part of an operand slab is written: every lane orders its shared-
// memory writes for the async proxy (the tensor cores read them next) and its
// TMEM accesses before the synchronisation, then one lane arrives for the
// warp (512 single-thread arrivals on one barrier word serialise).
__device__ __forceinline__ void slab_release(uint64_t* bar, int lane) {
    tc::fence_async_shared();
    tc::tc_fence_before();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(bar);
}
// 8 floats of a read-only table in global memory (L1-cached)
__device__ __forceinline__ void ld_f8g(const float* src, float* v) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(src)), b = __ldg(reinterpret_cast<const float4*>(src) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
// Sixteen consecutive floats from a 16-byte-aligned shared-memory address.
__device__ __forceinline__ void ld_f16v(const float* src, float (&v)[16]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 q = reinterpret_cast<const float4*>(src)[k];
        v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
}

// Per-tile blocks of the pipelined kernels (the forward's act' scratch and
// g_l, the backward's act' and S scratch), 8-column-group-major: the 8 BF16
// values of columns c0 .. c0+7 (c0 % 8 == 0) of `row` are 16 contiguous bytes
// at word ((c0 / 8) * 128 + row) * 4, so one 16-byte access per thread of a
// warp covers 512 consecutive bytes (whole 32-byte sectors).
__device__ __forceinline__ uint32_t* g8_at(uint32_t* blk, int row, int c0) {
    return blk + ((size_t)(c0 >> 3) * 128 + row) * 4;
}
__device__ __forceinline__ void st_g8h(uint32_t* blk, int row, int c0, const uint32_t (&u)[4], uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(g8_at(blk, row, c0)), "r"(u[0]),
                 "r"(u[1]), "r"(u[2]), "r"(u[3]), "l"(pol) : "memory");
}
// Columns c0 .. c0+15 (c0 % 16 == 0): two 8-column groups.
__device__ __forceinline__ void st_g16h(uint32_t* blk, int row, int c0, const uint32_t (&u)[8], uint64_t pol) {
    st_g8h(blk, row, c0, {u[0], u[1], u[2], u[3]}, pol);
    st_g8h(blk, row, c0 + 8, {u[4], u[5], u[6], u[7]}, pol);
}
__device__ __forceinline__ void ld_g16(const uint32_t* blk, int row, int c0, uint32_t (&u)[8]) {
    // through L2 only: L1 keeps the register spills and the parameter table
    const uint4 a = __ldcg(reinterpret_cast<const uint4*>(g8_at(const_cast<uint32_t*>(blk), row, c0)));
    const uint4 b = __ldcg(reinterpret_cast<const uint4*>(g8_at(const_cast<uint32_t*>(blk), row, c0 + 8)));
    u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
    u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
}

// For each j < 8 the sum of v[j] over the 32 lanes of a warp, by a fixed
// butterfly (the same additions in the same order on every call): lane l
// returns the sum for j = (l >> 2) & 7.
__device__ __forceinline__ float warp_colsum8(const float (&v)[8], int lane) {
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    float a4[4], b2[2];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        a4[j] = (u16 ? v[j + 4] : v[j]) + __shfl_xor_sync(0xffffffffu, u16 ? v[j] : v[j + 4], 16);
#pragma unroll
    for (int j = 0; j < 2; ++j)
        b2[j] = (u8 ? a4[j + 2] : a4[j]) + __shfl_xor_sync(0xffffffffu, u8 ? a4[j] : a4[j + 2], 8);
    float c = (u4 ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, u4 ? b2[0] : b2[1], 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// ---------------------------------------------------------------- forward + Z

// Phase q of a tile: 0 lift, 1..L layers, L+1..2L reverse through layer
// 2L+1-q, 2L+1 the Z contraction.  Phases 0..2L write the operand tile.
struct PipeFwdPlan {
    const FwdZArgs* a;
    __device__ int nq() const { return 2 * a->L + 2; }
    __device__ const CUtensorMap* map(int q) const {
        const int L = a->L;
        if (q <= L) return &a->wf[q];
        if (q <= 2 * L) return &a->wr[2 * L + 1 - q];
        return &a->wr[0];
    }
    __device__ int nk(int q) const { return q == 0 ? a->Dp / 64 : a->wp / 64; }
    __device__ int K(int q) const { return q == 0 ? a->D : a->w; }
    __device__ int N(int q) const { return q == 2 * a->L + 1 ? a->Dn : a->w; }
};

template <int ACT, bool RES>
__device__ __forceinline__ void fwdp_body(const FwdZArgs& a, const int cta, const int nctas) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* tile = smem;
    uint8_t* ring = smem + kFTileBytes;
    float* ptab = (float*)(ring + kPStages * kFStageBytes);
    const int L = a.L;
    const int prows = param_rows(L, 0);
    float* ysum = ptab + prows * a.w;
    PipeBars* B = (PipeBars*)(((uintptr_t)(ysum + kPGroups * 128) + 15) & ~(uintptr_t)15);
    const uint32_t abort_s = tc::smem_u32(&B->abort_flag);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PipeFwdPlan plan{&a};
    const int nq = plan.nq();
    const int nkw = a.wp / 64;
    const uint32_t budget = pbudget(a.wait_budget);

    stage_params(ptab, a.theta, a.off, L, a.w, a.D + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kPStages; ++s) {
            tc::mbar_init(&B->bfull[s], 1);
            tc::mbar_init(&B->bempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) tc::mbar_init(&B->accf[b], 1);
        for (int s = 0; s < 4; ++s) tc::mbar_init(&B->slab[s], 4 * kPGroups);
        tc::mbar_init(&B->tfree, 1);
        tc::mbar_init(&B->xfull, 1);
        tc::mbar_init(&B->ybar, 4 * kPGroups);
        tc::mbar_init(&B->gate, 1);
        tc::mbar_init(&B->drain, 1);
        B->abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&B->tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = B->tslot;

    if (warp < 4) {
        tc::setmaxnreg_dec<kPRegsCtl>();
        if (warp == 0 && lane == 0) {
            // ---- producer: the weight slices of every phase through the ring
            int it = 0;
            bool ok = !a.gate || pwait(&B->gate, 0, budget, abort_s);
            for (int t = cta; ok && t < a.ntiles; t += nctas)
                for (int q = 0; ok && q < nq; ++q) {
                    const CUtensorMap* m = plan.map(q);
                    const uint32_t bytes = (uint32_t)plan.N(q) * 128u;
                    for (int kc = 0; kc < plan.nk(q); ++kc, ++it) {
                        const int s = it % kPStages;
                        if (!pwait(&B->bempty[s], ((uint32_t)(it / kPStages) & 1u) ^ 1u, budget, abort_s)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_expect_tx(&B->bfull[s], bytes);
                        tc::tma_load_2d(ring + s * kFStageBytes, m, &B->bfull[s], kc * 64, 0);
                    }
                }
            if (!ok) pfail(a.err, abort_s);
            // drain: the loads of the last stages issued
            for (int j = it - 1; j >= 0 && j >= it - kPStages; --j)
                tc::mbar_wait(&B->bfull[j % kPStages], (uint32_t)(j / kPStages) & 1u, kDrainBudget);
        } else if (warp == 1 && lane == 0) {
            // ---- MMA issuer
            int it = 0, tl = 0;
            bool ok = !a.gate || pwait(&B->gate, 0, budget, abort_s);
            const uint32_t tile_addr = tc::smem_u32(tile), ring_addr = tc::smem_u32(ring);
            // (a bulk L2 prefetch of each reverse phase's act' block measured slower)
            for (int t = cta; ok && t < a.ntiles; t += nctas, ++tl) {
                for (int q = 0; ok && q < nq; ++q) {
                    const int buf = q & 1;
                    const uint32_t d = tmem + (uint32_t)(buf * 256);
                    const uint32_t idesc = tc::idesc_bf16(128, plan.N(q), 0, 0);
                    const bool accumulate = RES && q > L && q <= 2 * L;
                    if (q == 0 && !pwait(&B->xfull, (uint32_t)tl & 1u, budget, abort_s)) { ok = false; break; }
                    const uint32_t spar = (uint32_t)(tl * (2 * L + 1) + q - 1) & 1u;
                    const int K = plan.K(q);
                    for (int kc = 0; kc < plan.nk(q); ++kc, ++it) {
                        const int s = it % kPStages;
                        if (!pwait(&B->bfull[s], (uint32_t)(it / kPStages) & 1u, budget, abort_s) ||
                            (q > 0 && !pwait(&B->slab[kc], spar, budget, abort_s))) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const int nsteps = min(4, (K - kc * 64 + 15) / 16);
                        // four K steps unrolled, the ones past K skipped (a loop with a
                        // run-time trip count spills this role's registers)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (k < nsteps) {
                                const uint64_t ad = tc::sdesc_sw128(tile_addr + (uint32_t)kc * 16384u + 32u * k, 16u);
                                const uint64_t bd = tc::sdesc_sw128(ring_addr + (uint32_t)s * kFStageBytes + 32u * k, 16u);
                                tc::mma_bf16(d, ad, bd, idesc, (accumulate || kc > 0 || k > 0) ? 1u : 0u);
                            }
                        }
                        tc::mma_commit(&B->bempty[s]);
                    }
                    if (ok) tc::mma_commit(&B->accf[buf]);
                }
            }
            if (!ok) pfail(a.err, abort_s);
            // drain: every contraction issued has completed
            tc::mma_commit(&B->drain);
            tc::mbar_wait(&B->drain, 0, kDrainBudget);
        } else if (warp == 2 && lane == 0) {
            // ---- store warp: operand-stack stores, input rows, tile release
            const uint64_t pol_stream = tc::l2_policy_evict_first();
            bool ok = !a.gate || pwait(&B->gate, 0, budget, abort_s);
            int tl = 0, xl = 0;  // tiles processed, input loads issued
            auto load_x = [&](int t) {
                tc::mbar_expect_tx(&B->xfull, (uint32_t)(a.Dp / 64) * 16384u);
                for (int k = 0; k < a.Dp / 64; ++k)
                    tc::tma_load_2d(tile + k * 16384, &a.xin, &B->xfull, k * 64, t * 128);
                ++xl;
            };
            if (ok) {
                tc::mbar_arrive(&B->tfree);  // the first phase may write
                if (cta < a.ntiles) load_x(cta);
            }
            for (int t = cta; ok && t < a.ntiles; t += nctas, ++tl) {
                for (int q = 0; ok && q <= 2 * L; ++q) {
                    const uint32_t par = (uint32_t)(tl * (2 * L + 1) + q) & 1u;
                    const bool store = a.for_grad && q >= L;
                    for (int s = 0; s < nkw; ++s) {
                        if (!pwait(&B->slab[s], par, budget, abort_s)) { ok = false; break; }
                        if (store) {
                            tc::tma_store_3d_hint(&a.eb, tile + s * 16384, s * 64, t * 128, 2 * L - q, pol_stream);
                            tc::tma_store_commit();
                        }
                    }
                    if (!ok) break;
                    tc::tma_store_wait_read<0>();
                    tc::mbar_arrive(&B->tfree);
                }
                if (!ok) break;
                // the Z contraction reads e_0 from the tile; the next tile's
                // input rows replace it once that contraction has completed
                const uint32_t zpar = (uint32_t)((tl * nq + 2 * L + 1) >> 1) & 1u;
                if (!pwait(&B->accf[1], zpar, budget, abort_s)) { ok = false; break; }
                if (t + nctas < a.ntiles) load_x(t + nctas);
            }
            if (!ok) pfail(a.err, abort_s);
            // drain: bulk stores, and the last input load if nobody consumed it
            tc::tma_store_wait_all<0>();
            if (xl > 0) tc::mbar_wait(&B->xfull, (uint32_t)(xl - 1) & 1u, kDrainBudget);
        }
    } else {
        tc::setmaxnreg_inc<kPRegsEpi>();
        // ---- epilogue: warpgroup eg owns columns 64 s + 16 eg .. + 15 of slab s
        const int eg = (warp - 4) >> 2, lg = warp & 3;
        const int row = lg * 32 + lane;
        const uint32_t tlane = tmem + ((uint32_t)(lg * 32) << 16);
        const float* wo = ptab + (L + 1) * a.w;
        const float* win0 = ptab + (L + 2) * a.w;
        const size_t blk = (size_t)(a.w / 2) * 128;
        uint32_t* scr = a.scratch + (size_t)cta * L * blk;
        // derivative scratch at normal L2 priority: 97 MB over the grid does not fit
        // beside the streamed stacks, and evict-last measured slower
        const uint64_t pol_keep = tc::l2_policy_evict_normal(), pol_stream = tc::l2_policy_evict_first();
        bool ok = !a.gate || pwait(&B->gate, 0, budget, abort_s);
        int tl = 0;

        // wait for contraction q (TMEM buffer q % 2) and, when the phase writes
        // the operand tile, for the tile's release
        auto begin = [&](int q) -> bool {
            if (!pwait(&B->accf[q & 1], (uint32_t)((tl * nq + q) >> 1) & 1u, budget, abort_s)) return false;
            tc::tc_fence_after();
            if (q <= 2 * L && !pwait(&B->tfree, (uint32_t)(tl * (2 * L + 1) + q) & 1u, budget, abort_s))
                return false;
            return true;
        };

        // forward layer l (phase q = l): a = acc + b_l (+ t W_in[:,0] at the
        // lift); h_l = [h_{l-1}] + act(a) in BF16 to the tile (the operand of
        // the next contraction), act'(a_l) to the scratch; y accumulates
        // w_o^T act(a_l) in FP32 (ResNet: every layer, since h_L = h_0 +
        // sum_l act(a_l); FC: the top layer); at the top e_L = act'(a_L) w_o.
        // LIFT: l = 0 (no residual read).
        auto fwd_layer = [&](auto lift_tag, int l, float tval, float& ypart) {
            constexpr bool LIFT = decltype(lift_tag)::value;
            const uint32_t tb = tlane + (uint32_t)((l & 1) * 256);
            const float* bias = ptab + l * a.w;
            uint32_t* sc = scr + (size_t)l * blk;
            const bool top = l == L;
            if (RES && top && L >= 1) {
                // g_L = w_o seeds the reverse sweep's accumulation (next buffer)
                const uint32_t tn = tlane + (uint32_t)(((l + 1) & 1) * 256);
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int c0 = s * 64 + eg * 16;
                    if (s < nkw && c0 < a.w) {
                        uint32_t u[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) u[j] = __float_as_uint(wo[c0 + j]);
                        tc::tmem_st16(tn + (uint32_t)c0, u);
                    }
                }
                tc::tmem_wait_st();
            }
            // one slab per iteration, not unrolled: the registers of a slab
            // are not held across slabs
#pragma unroll 1
            for (int s = 0; s < nkw; ++s) {
                {
                    const int c0 = s * 64 + eg * 16;
                    uint32_t rb[16];
                    tmem_ld16w(tb + (uint32_t)c0, rb);
                    tc::tmem_wait_ld_regs(rb);
                    uint32_t dpk[8];
                    if (c0 < a.w) {
                        uint32_t hi[8], out[8];
                        if (RES && !LIFT) ld_tile16_packed(tile, row, c0, hi);
                        float bv[16], wv[16];
                        ld_f16v(bias + c0, bv);
                        if (LIFT) {
                            float tw[16];
                            ld_f16v(win0 + c0, tw);
#pragma unroll
                            for (int j = 0; j < 16; ++j) bv[j] = fmaf(tval, tw[j], bv[j]);
                        }
                        if (RES || top) ld_f16v(wo + c0, wv);
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const float a0 = __uint_as_float(rb[2 * k]) + bv[2 * k];
                            const float a1 = __uint_as_float(rb[2 * k + 1]) + bv[2 * k + 1];
                            const Act3 f0 = act3_sfu<ACT>(a0), f1 = act3_sfu<ACT>(a1);
                            if (RES || top) {
                                ypart = fmaf(f0.f, wv[2 * k], ypart);
                                ypart = fmaf(f1.f, wv[2 * k + 1], ypart);
                            }
                            if (!top) {
                                float h0 = f0.f, h1 = f1.f;
                                if (RES && !LIFT) {
                                    const float2 hh = unpack_bf16x2(hi[k]);
                                    h0 += hh.x;
                                    h1 += hh.y;
                                }
                                out[k] = pack_bf16x2(h0, h1);
                                dpk[k] = pack_bf16x2(f0.d1, f1.d1);
                            } else {
                                out[k] = pack_bf16x2(f0.d1 * wv[2 * k], f1.d1 * wv[2 * k + 1]);
                            }
                        }
                        st_tile16_packed(tile, row, c0, out);
                    }
                    slab_release(&B->slab[s], lane);
                    if (!top && c0 < a.w) st_g16h(sc, row, c0, dpk, pol_keep);
                }
            }
        };

        // reverse through layer l (phase q = 2L+1-l): the buffer holds g_{l-1}
        // (g_l + W_l^T e_l for ResNet, W_l^T e_l for FC); e_{l-1} = act'(a_{l-1})
        // g_{l-1} to the tile, bf16(g_{l-1}) to G for the gradient
        auto reverse = [&](int q, int t) -> bool {
            const int l = 2 * L + 1 - q;
            const uint32_t tb = tlane + (uint32_t)((q & 1) * 256);
            const uint32_t* sc = scr + (size_t)(l - 1) * blk;
            uint32_t* gout = a.G + (size_t)t * blk + (size_t)(l - 1) * a.G_words;
            // act' words of the first slab are requested before the wait for the
            // contraction, those of the next slab (and its accumulator columns)
            // before the current slab is processed
            uint32_t gn[16], dn[8];
            if (eg * 16 < a.w) ld_g16(sc, row, eg * 16, dn);
            if (!begin(q)) return false;
            // ResNet: g_{l-1} seeds the next reverse contraction's buffer
            if (RES && q < 2 * L) tmem_copy64(tb, tlane + (uint32_t)(((q + 1) & 1) * 256), eg, nkw);
            tmem_ld16w(tb + (uint32_t)(eg * 16), gn);
#pragma unroll 1
            for (int s = 0; s < nkw; ++s) {
                const int c0 = s * 64 + eg * 16;
                tc::tmem_wait_ld_regs(gn);
                uint32_t g[16], du[8];
#pragma unroll
                for (int k = 0; k < 16; ++k) g[k] = gn[k];
#pragma unroll
                for (int k = 0; k < 8; ++k) du[k] = dn[k];
                if (s + 1 < nkw) {
                    if (c0 + 64 < a.w) ld_g16(sc, row, c0 + 64, dn);
                    tmem_ld16w(tb + (uint32_t)(c0 + 64), gn);
                }
                uint32_t gp[8];
                if (c0 < a.w) {
                    uint32_t out[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float2 d = unpack_bf16x2(du[k]);
                        const float g0 = __uint_as_float(g[2 * k]), g1 = __uint_as_float(g[2 * k + 1]);
                        out[k] = pack_bf16x2(d.x * g0, d.y * g1);
                        gp[k] = pack_bf16x2(g0, g1);
                    }
                    st_tile16_packed(tile, row, c0, out);
                }
                slab_release(&B->slab[s], lane);
                if (a.for_grad && c0 < a.w) st_g16h(gout, row, c0, gp, pol_stream);
            }
            return true;
        };

        for (int t = cta; ok && t < a.ntiles; t += nctas, ++tl) {
            const int p = t * 128 + row;
            const bool valid = p < a.P;
            const float tval = valid ? (float)(p / a.M) * a.dt : 0.f;
            float ypart = 0.f;
            // lift, hidden layers
            if (!(ok = begin(0))) break;
            fwd_layer(std::true_type{}, 0, tval, ypart);
            for (int l = 1; ok && l <= L; ++l) {
                if (!(ok = begin(l))) break;
                fwd_layer(std::false_type{}, l, tval, ypart);
            }
            if (!ok) break;
            // y = b_o + the warpgroups' partial sums, added in a fixed order
            ysum[eg * 128 + row] = ypart;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&B->ybar);
            if (eg == 0) {
                if (!(ok = pwait(&B->ybar, (uint32_t)tl & 1u, budget, abort_s))) break;
                float y = __ldg(a.theta + a.off.bo);
                for (int g2 = 0; g2 < kPGroups; ++g2) y += ysum[g2 * 128 + row];
                if (valid) a.Y[p] = y;
            }
            // reverse sweep
            for (int q = L + 1; ok && q <= 2 * L; ++q) ok = reverse(q, t);
            if (!ok) break;
            // Z = W_in[:,1:]^T e_0
            const int qz = 2 * L + 1;
            if (!(ok = begin(qz))) break;
            const uint32_t tb = tlane + (uint32_t)((qz & 1) * 256);
            for (int c0 = eg * 16; c0 < a.Dn; c0 += 16 * kPGroups) {
                uint32_t rv[16];
                tmem_ld16w(tb + (uint32_t)c0, rv);
                tc::tmem_wait_ld_regs(rv);
                if (valid) {
                    float* zr = a.Z + (size_t)p * a.D + c0;
                    if ((a.D & 3) == 0 && c0 + 16 <= a.D) {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            reinterpret_cast<float4*>(zr)[k] =
                                make_float4(__uint_as_float(rv[4 * k]), __uint_as_float(rv[4 * k + 1]),
                                            __uint_as_float(rv[4 * k + 2]), __uint_as_float(rv[4 * k + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < a.D) zr[j] = __uint_as_float(rv[j]);
                    }
                }
            }
        }
        if (!ok) pfail(a.err, abort_s);
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

template <int ACT, bool RES>
__global__ void __launch_bounds__(kPThreads, 1) k_fwd_pipe(const __grid_constant__ FwdZArgs a) {
    fwdp_body<ACT, RES>(a, (int)blockIdx.x, (int)gridDim.x);
}

template <int ACT, bool RES>
__global__ void __launch_bounds__(kPThreads, 1)
    k_fwd_pipe_group(const FwdZArgs* __restrict__ all, const int* __restrict__ cta_begin, int n) {
    int i = 0;
    while (i + 1 < n && (int)blockIdx.x >= cta_begin[i + 1]) ++i;
    fwdp_body<ACT, RES>(all[i], (int)blockIdx.x - cta_begin[i], cta_begin[i + 1] - cta_begin[i]);
}

// ---------------------------------------------------------------- tangent + adjoint

// Phase q of a tile: 0..L the forward recomputation and the tangent of layer
// q together (one weight stream, two accumulators: TMEM buffer 0 and 1);
// L+1..2L the adjoint through layer 2L+1-q (buffer q % 2).  Every phase
// writes the operand tiles: h_l (tile_h) and h'_l (tile_d) in the up-sweep,
// abar (tile_h) in the adjoint sweep.
//
// An up-sweep contraction fills both TMEM buffers, so it cannot run into the
// other buffer while the previous epilogue works: it starts once every
// epilogue warp has read its accumulator columns (barrier `tread`), each K
// slice waiting for its slab of the operand tiles.  The top phase also sums
// alpha h_L + h'_L over the tile's rows (the read-out gradient) into per-tile
// partials.  The derivative scratch (act'(a_l), S_l) and the g_l blocks are
// dropped from L2 once read (`discard.global.L2`), so dead scratch is never
// written back to HBM.
struct PipeBwdPlan {
    const BwdArgs* a;
    __device__ int nq() const { return 2 * a->L + 1; }
    __device__ const CUtensorMap* map(int q) const {
        return q <= a->L ? &a->wf[q] : &a->wr[2 * a->L + 1 - q];
    }
    __device__ int nk(int q) const { return q == 0 ? a->Dp / 64 : a->wp / 64; }
    __device__ int K(int q) const { return q == 0 ? a->D : a->w; }
};

template <int ACT, bool RES>
__device__ __forceinline__ void bwdp_body(const BwdArgs& a, const int cta, const int nctas) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* tile_h = smem;                  // h_l in the up-sweep, abar_l in the adjoint sweep
    uint8_t* tile_d = smem + kFTileBytes;    // h'_l
    uint8_t* ring = smem + 2 * kFTileBytes;
    // the per-column parameters are read from the table in global memory (held
    // in L1): shared memory holds the two operand tiles and a ring of three
    // weight slices, so the contraction of an up-sweep phase finds its first
    // three K slices loaded
    const float* ptab = a.pvec;
    const int L = a.L;
    PipeBars* B = (PipeBars*)(ring + kPBwdStages * kFStageBytes);
    const uint32_t abort_s = tc::smem_u32(&B->abort_flag);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PipeBwdPlan plan{&a};
    const int nq = plan.nq();
    const int nkw = a.wp / 64, nkx = a.Dp / 64;
    const uint32_t budget = pbudget(a.wait_budget);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPBwdStages; ++s) {
            tc::mbar_init(&B->bfull[s], 1);
            tc::mbar_init(&B->bempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) tc::mbar_init(&B->accf[b], 1);
        for (int s = 0; s < 4; ++s) tc::mbar_init(&B->slab[s], 4 * kPGroups);
        tc::mbar_init(&B->tfree, 1);
        tc::mbar_init(&B->xfull, 1);
        tc::mbar_init(&B->ybar, 1);  // the tangent inputs (v rows) of a tile have arrived
        tc::mbar_init(&B->tread, 4 * kPGroups);
        tc::mbar_init(&B->gate, 1);
        tc::mbar_init(&B->drain, 1);
        B->abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(&B->tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = B->tslot;
    uint64_t* vfull = &B->ybar;

    if (warp < 4) {
        tc::setmaxnreg_dec<kPRegsCtl>();
        if (warp == 0 && lane == 0) {
            // ---- producer
            int it = 0;
            bool ok = !a.gate || pwait(&B->gate, 0, budget, abort_s);
            for (int t = cta; ok && t < a.ntiles; t += nctas)
                for (int q = 0; ok && q < nq; ++q) {
                    if (q < L) {
                        // into L2 about one phase ahead of its reader: g_q, read by the
                        // epilogue of up-sweep phase q
                        const size_t blk = (size_t)(a.w / 2) * 128;
                        tc::prefetch_l2_bulk(a.G + (size_t)q * a.G_words + (size_t)t * blk, (uint32_t)(blk * 4));
                    }
                    if (q > L) {
                        // into L2 about one phase ahead of the adjoint epilogue of phase
                        // q: this CTA's act' and S blocks of layer 2L - q
                        const size_t blk = (size_t)(a.w / 2) * 128;
                        const uint32_t* d1b = a.scratch + ((size_t)cta * 2 * L + (2 * L - q)) * blk;
                        tc::prefetch_l2_bulk(d1b, (uint32_t)(blk * 4));
                        tc::prefetch_l2_bulk(d1b + (size_t)L * blk, (uint32_t)(blk * 4));
                    }
                    const CUtensorMap* m = plan.map(q);
                    const uint32_t bytes = (uint32_t)a.w * 128u;
                    for (int kc = 0; kc < plan.nk(q); ++kc, ++it) {
                        const int s = it % kPBwdStages;
                        if (!pwait(&B->bempty[s], ((uint32_t)(it / kPBwdStages) & 1u) ^ 1u, budget, abort_s)) {
                            ok = false;
                            break;
                        }
                        tc::mbar_expect_tx(&B->bfull[s], bytes);
                        tc::tma_load_2d(ring + s * kFStageBytes, m, &B->bfull[s], kc * 64, 0);
                    }
                }
            if (!ok) pfail(a.err, abort_s);
            for (int j = it - 1; j >= 0 && j >= it - kPBwdStages; --j)
                tc::mbar_wait(&B->bfull[j % kPBwdStages], (uint32_t)(j / kPBwdStages) & 1u, kDrainBudget);
        } else if (warp == 1 && lane == 0) {
            // ---- MMA issuer (few live values: the control warps run on 32
            // registers, and a spilled value reloaded after a long wait costs a
            // round trip to L2)
            int it = 0, tl = 0;
            bool ok = !a.gate || pwait(&B->gate, 0, budget, abort_s);
            const uint32_t idesc = tc::idesc_bf16(128, a.w, 0, 0);
            // shared-memory descriptors: the fields but the start address, and
            // start addresses in 16-byte units (+2 per 16-element K step)
            const uint64_t dfix = tc::sdesc_sw128(0u, 16u);
            const uint32_t th16 = tc::smem_u32(tile_h) >> 4, td16 = tc::smem_u32(tile_d) >> 4;
            const uint32_t rg16 = tc::smem_u32(ring) >> 4;
            // barrier addresses in shared memory (32 bits)
            const uint32_t Bs = tc::smem_u32(B);
            const uint32_t bfull_s = Bs + (uint32_t)offsetof(PipeBars, bfull), slab_s = Bs + (uint32_t)offsetof(PipeBars, slab);
            for (int t = cta; ok && t < a.ntiles; t += nctas, ++tl) {
                for (int q = 0; ok && q < nq; ++q) {
                    const bool up = q <= L;
                    const uint32_t spar = (uint32_t)(tl * nq + q - 1) & 1u;
                    if (q == 0) {
                        if (!pwait(&B->xfull, (uint32_t)tl & 1u, budget, abort_s) ||
                            !pwait(vfull, (uint32_t)tl & 1u, budget, abort_s)) { ok = false; break; }
                    } else if (up) {
                        // the contraction overwrites both accumulators: every epilogue
                        // warp of the last phase has read them (each K slice then waits
                        // for its slab of the operand tiles below), so the first K
                        // slices run while the last slab is still being computed
                        if (!pwait(Bs + (uint32_t)offsetof(PipeBars, tread), (uint32_t)(tl * L + q - 1) & 1u, budget, abort_s)) { ok = false; break; }
                    } else if (q == L + 1) {
                        // accumulates onto the adjoint the top phase seeded: every slab done
                        for (int s = 0; s < nkw && ok; ++s) ok = pwait(slab_s + 8u * s, spar, budget, abort_s);
                        if (!ok) break;
                    }
                    const uint32_t d = tmem + (up ? 0u : (uint32_t)((q & 1) * 256));
                    const bool kslab = q >= 1 && q != L + 1;
                    const int nk = plan.nk(q), K = plan.K(q);
                    for (int kc = 0; kc < nk; ++kc, ++it) {
                        const int s = it % kPBwdStages;
                        if (!pwait(bfull_s + 8u * s, (uint32_t)(it / kPBwdStages) & 1u, budget, abort_s) ||
                            (kslab && !pwait(slab_s + 8u * kc, spar, budget, abort_s))) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const int nsteps = min(4, (K - kc * 64 + 15) / 16);
                        const uint32_t b16 = rg16 + (uint32_t)s * (kFStageBytes >> 4);
                        const uint32_t a16 = (uint32_t)kc * (16384u >> 4);
                        // four K steps unrolled, the ones past K skipped (a loop with a
                        // run-time trip count spills this role's registers)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (k < nsteps) {
                                const uint32_t en = ((!up && RES) || kc > 0 || k > 0) ? 1u : 0u;
                                const uint64_t bd = dfix | (b16 + 2u * k);
                                tc::mma_bf16(d, dfix | (th16 + a16 + 2u * k), bd, idesc, en);
                                if (up) tc::mma_bf16(tmem + 256u, dfix | (td16 + a16 + 2u * k), bd, idesc, en);
                            }
                        }
                        tc::mma_commit(&B->bempty[s]);
                    }
                    if (ok) tc::mma_commit(&B->accf[(tl * nq + q) & 1]);
                }
            }
            if (!ok) pfail(a.err, abort_s);
            tc::mma_commit(&B->drain);
            tc::mbar_wait(&B->drain, 0, kDrainBudget);
        } else if (warp == 2 && lane == 0) {
            // ---- store warp: operand-stack stores, input rows, tile release
            const uint64_t pol_stream = tc::l2_policy_evict_first();
            bool ok = !a.gate || pwait(&B->gate, 0, budget, abort_s);
            int tl = 0, xl = 0, vl = 0;
            auto load_x = [&](int t) {
                tc::mbar_expect_tx(&B->xfull, (uint32_t)nkx * 16384u);
                for (int k = 0; k < nkx; ++k) tc::tma_load_2d(tile_h + k * 16384, &a.xb, &B->xfull, k * 64, t * 128);
                ++xl;
            };
            auto load_v = [&](int t) {
                tc::mbar_expect_tx(vfull, (uint32_t)nkx * 16384u);
                for (int k = 0; k < nkx; ++k) tc::tma_load_2d(tile_d + k * 16384, &a.vb, vfull, k * 64, t * 128);
                ++vl;
            };
            if (ok) {
                tc::mbar_arrive(&B->tfree);
                if (cta < a.ntiles) { load_x(cta); load_v(cta); }
            }
            for (int t = cta; ok && t < a.ntiles; t += nctas, ++tl) {
                for (int q = 0; ok && q < nq; ++q) {
                    const uint32_t par = (uint32_t)(tl * nq + q) & 1u;
                    for (int s = 0; s < nkw; ++s) {
                        if (!pwait(&B->slab[s], par, budget, abort_s)) { ok = false; break; }
                        if (q < L) {
                            tc::tma_store_3d_hint(&a.hb, tile_h + s * 16384, s * 64, t * 128, q, pol_stream);
                            tc::tma_store_3d_hint(&a.hdb, tile_d + s * 16384, s * 64, t * 128, q, pol_stream);
                        } else if (q == L) {
                            tc::tma_store_3d_hint(&a.abb, tile_h + s * 16384, s * 64, t * 128, L, pol_stream);
                        } else {
                            tc::tma_store_3d_hint(&a.abb, tile_h + s * 16384, s * 64, t * 128, 2 * L - q, pol_stream);
                        }
                        tc::tma_store_commit();
                    }
                    if (!ok) break;
                    tc::tma_store_wait_read<0>();
                    // tile_d's last reader in this tile was the store above (q == L):
                    // the next tile's v rows may replace it; tile_h's last reader is
                    // the store of abar_0 (q == 2L)
                    if (q == L && t + nctas < a.ntiles) load_v(t + nctas);
                    if (q == 2 * L && t + nctas < a.ntiles) load_x(t + nctas);
                    tc::mbar_arrive(&B->tfree);
                }
            }
            if (!ok) pfail(a.err, abort_s);
            tc::tma_store_wait_all<0>();
            if (xl > 0) tc::mbar_wait(&B->xfull, (uint32_t)(xl - 1) & 1u, kDrainBudget);
            if (vl > 0) tc::mbar_wait(vfull, (uint32_t)(vl - 1) & 1u, kDrainBudget);
        }
    } else {
        tc::setmaxnreg_inc<kPRegsEpi>();
        const int eg = (warp - 4) >> 2, lg = warp & 3;
        const int row = lg * 32 + lane;
        const uint32_t tlane = tmem + ((uint32_t)(lg * 32) << 16);
        const float* wo = ptab + (size_t)(L + 1) * a.w;
        const float* win0 = ptab + (size_t)(L + 2) * a.w;
        const size_t blk = (size_t)(a.w / 2) * 128;
        uint32_t* scr_d1 = a.scratch + (size_t)cta * 2 * L * blk;  // act'(a_l), l < L
        uint32_t* scr_S = scr_d1 + (size_t)L * blk;                 // S_l, l < L
        const uint64_t pol_keep = tc::l2_policy_evict_normal();  // as in the forward kernel
        bool ok = !a.gate || pwait(&B->gate, 0, budget, abort_s);
        int tl = 0;

        auto begin = [&](int q) -> bool {
            const int G = tl * nq + q;
            if (!pwait(&B->accf[G & 1], (uint32_t)(G >> 1) & 1u, budget, abort_s)) return false;
            tc::tc_fence_after();
            return pwait(&B->tfree, (uint32_t)G & 1u, budget, abort_s);
        };

        // up-sweep layer l: a = acc + b_l (+ t W_in[:,0]), t = act(a):
        //   h_l = [h_{l-1}] + t,  h'_l = [h'_{l-1}] + act'(a) a',  S_l = act''(a) a' g_l
        // (l < L: act'(a_l) and S_l to the scratch); at the top (g_L = w_o):
        //   hbar_L = alpha w_o,  abar_L = act'(a_L) hbar_L + S_L
        // Each 16-column slab is taken as two halves of 8 columns.
        auto up = [&](auto lift_tag, int l, float tval, float alpha_p, int t, bool valid, int p) -> bool {
            constexpr bool LIFT = decltype(lift_tag)::value;
            const bool top = l == L;
            const float* bias = ptab + (size_t)l * a.w;
            const uint32_t* gin = a.G + (size_t)t * blk + (size_t)l * a.G_words;
            if (!begin(l)) return false;
#pragma unroll 1
            for (int s = 0; s < nkw; ++s) {
                const int c0 = s * 64 + eg * 16;
                uint32_t gw[8];
                if (!top && c0 < a.w) ld_g16(gin, row, c0, gw);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int cc = c0 + half * 8;
                    uint32_t ra[8], rt[8];
                    tc::tmem_ld8(tlane + (uint32_t)cc, ra);
                    tc::tmem_ld8(tlane + 256u + (uint32_t)cc, rt);
                    tc::tmem_wait_ld();
                    if (!top && half == 1 && s == nkw - 1) {
                        // this warp's last TMEM read of the phase: the next contraction may
                        // overwrite the accumulators
                        tc::tc_fence_before();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&B->tread);
                    }
                    if (c0 < a.w) {
                        float bv[8], g[8], hp[8], hdp[8];
                        ld_f8g(bias + cc, bv);
                        if (LIFT) {
                            float tw[8];
                            ld_f8g(win0 + cc, tw);
#pragma unroll
                            for (int j = 0; j < 8; ++j) bv[j] = fmaf(tval, tw[j], bv[j]);
                        }
                        if (top) ld_f8g(wo + cc, g);
                        else {
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const float2 f = unpack_bf16x2(gw[half * 4 + k]);
                                g[2 * k] = f.x; g[2 * k + 1] = f.y;
                            }
                        }
                        if (RES && !LIFT) {
                            ld_tile8(tile_h, row, cc, hp);
                            ld_tile8(tile_d, row, cc, hdp);
                        }
                        float h[8], hd[8], d1[8], S[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float av = __uint_as_float(ra[j]) + bv[j];
                            const Act3 f = act3_sfu<ACT>(av);
                            const float ad = __uint_as_float(rt[j]);
                            h[j] = ((RES && !LIFT) ? hp[j] : 0.f) + f.f;
                            hd[j] = ((RES && !LIFT) ? hdp[j] : 0.f) + f.d1 * ad;
                            S[j] = f.d2 * ad * g[j];
                            d1[j] = f.d1;
                        }
                        if (!top) st_tile8(tile_d, row, cc, hd);
                        if (!top) {
                            st_tile8(tile_h, row, cc, h);
                            uint32_t w1[4], w2[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                w1[k] = pack_bf16x2(d1[2 * k], d1[2 * k + 1]);
                                w2[k] = pack_bf16x2(S[2 * k], S[2 * k + 1]);
                            }
                            st_g8h(scr_d1 + (size_t)l * blk, row, cc, w1, pol_keep);
                            st_g8h(scr_S + (size_t)l * blk, row, cc, w2, pol_keep);
                        } else {
                            // dw_o = sum over points of alpha h_L + h'_L: this warp's 32 rows
                            // summed by a fixed butterfly, one partial per tile, row group and
                            // column (the sum over tiles follows in a fixed order)
                            float cv[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) cv[j] = valid ? fmaf(alpha_p, h[j], hd[j]) : 0.f;
                            const float csum = warp_colsum8(cv, lane);
                            if ((lane & 3) == 0) a.wopart[((size_t)t * 4 + lg) * a.w + cc + ((lane >> 2) & 7)] = csum;
                            float ab[8], hb[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                hb[j] = alpha_p * g[j];
                                ab[j] = d1[j] * hb[j] + S[j];
                            }
                            st_tile8(tile_h, row, cc, ab);
                            if (RES && L >= 1) {
                                // hbar_L seeds the adjoint sweep's accumulation (buffer (L+1) % 2)
                                uint32_t u[8];
#pragma unroll
                                for (int j = 0; j < 8; ++j) u[j] = __float_as_uint(hb[j]);
                                tc::tmem_st8(tlane + (uint32_t)(((L + 1) & 1) * 256 + cc), u);
                            }
                        }
                    }
                }
                if (RES && top) tc::tmem_wait_st();
                slab_release(&B->slab[s], lane);
                if (!top && c0 < a.w) {
                    // this slab's g_l lines are dead once read: drop them from L2
                    __syncwarp();
                    if (lane < 8) {
                        const size_t grp = (size_t)(c0 >> 3) + ((lane >> 2) & 1);
                        const uint8_t* line =
                            reinterpret_cast<const uint8_t*>(gin + (grp * 128 + (size_t)lg * 32) * 4) + (lane & 3) * 128;
                        asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
                    }
                }
            }
            return true;
        };

        // adjoint through layer l (phase q = 2L+1-l): the buffer holds
        // hbar_{l-1} (ResNet: hbar_l + W_l^T abar_l, accumulated onto the
        // seeded buffer; FC: W_l^T abar_l); abar_{l-1} = act'(a_{l-1}) hbar_{l-1} + S_{l-1}
        auto adj = [&](int q) -> bool {
            const int l = 2 * L + 1 - q;
            const uint32_t tb = tlane + (uint32_t)((q & 1) * 256);
            const uint32_t* d1src = scr_d1 + (size_t)(l - 1) * blk;
            const uint32_t* Ssrc = scr_S + (size_t)(l - 1) * blk;
            // the first slab's act' and S words are requested before the wait
            uint32_t hn[16], dn[8], sn[8];
            if (eg * 16 < a.w) {
                ld_g16(d1src, row, eg * 16, dn);
                ld_g16(Ssrc, row, eg * 16, sn);
            }
            if (!begin(q)) return false;
            if (RES && q < 2 * L) tmem_copy64(tb, tlane + (uint32_t)(((q + 1) & 1) * 256), eg, nkw);
            tmem_ld16w(tb + (uint32_t)(eg * 16), hn);
#pragma unroll 1
            for (int s = 0; s < nkw; ++s) {
                const int c0 = s * 64 + eg * 16;
                tc::tmem_wait_ld_regs(hn);
                uint32_t hb[16], du[8], su[8];
#pragma unroll
                for (int k = 0; k < 16; ++k) hb[k] = hn[k];
#pragma unroll
                for (int k = 0; k < 8; ++k) { du[k] = dn[k]; su[k] = sn[k]; }
                if (s + 1 < nkw) {
                    if (c0 + 64 < a.w) {
                        ld_g16(d1src, row, c0 + 64, dn);
                        ld_g16(Ssrc, row, c0 + 64, sn);
                    }
                    tmem_ld16w(tb + (uint32_t)(c0 + 64), hn);
                }
                if (c0 < a.w) {
                    uint32_t out[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float2 d = unpack_bf16x2(du[k]), S = unpack_bf16x2(su[k]);
                        out[k] = pack_bf16x2(fmaf(d.x, __uint_as_float(hb[2 * k]), S.x),
                                             fmaf(d.y, __uint_as_float(hb[2 * k + 1]), S.y));
                    }
                    st_tile16_packed(tile_h, row, c0, out);
                }
                slab_release(&B->slab[s], lane);
                if (c0 < a.w) {
                    // this slab's act' and S lines are dead once read (the next tile
                    // rewrites them): drop them from L2 without a write-back.  Per
                    // block, the warp's 32 rows of the two 8-column groups are eight
                    // 128-byte lines; lanes 0-7 take the act' block's, 8-15 the S block's.
                    __syncwarp();
                    if (lane < 16) {
                        const uint32_t* base = lane < 8 ? d1src : Ssrc;
                        const size_t grp = (size_t)(c0 >> 3) + ((lane >> 2) & 1);
                        const uint8_t* line =
                            reinterpret_cast<const uint8_t*>(base + (grp * 128 + (size_t)lg * 32) * 4) + (lane & 3) * 128;
                        asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
                    }
                }
            }
            return true;
        };

        for (int t = cta; ok && t < a.ntiles; t += nctas, ++tl) {
            const int p = t * 128 + row;
            const bool valid = p < a.P;
            const float tval = valid ? (float)(p / a.M) * a.dt : 0.f;
            const float alpha_p = valid ? __ldg(a.alpha + p) : 0.f;
            ok = up(std::true_type{}, 0, tval, alpha_p, t, valid, p);
            for (int l = 1; ok && l <= L; ++l) ok = up(std::false_type{}, l, tval, alpha_p, t, valid, p);
            for (int q = L + 1; ok && q <= 2 * L; ++q) ok = adj(q);
        }
        if (!ok) pfail(a.err, abort_s);
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

template <int ACT, bool RES>
__global__ void __launch_bounds__(kPThreads, 1) k_bwd_pipe(const __grid_constant__ BwdArgs a) {
    bwdp_body<ACT, RES>(a, (int)blockIdx.x, (int)gridDim.x);
}

template <int ACT, bool RES>
__global__ void __launch_bounds__(kPThreads, 1)
    k_bwd_pipe_group(const BwdArgs* __restrict__ all, const int* __restrict__ cta_begin, int n) {
    int i = 0;
    while (i + 1 < n && (int)blockIdx.x >= cta_begin[i + 1]) ++i;
    bwdp_body<ACT, RES>(all[i], (int)blockIdx.x - cta_begin[i], cta_begin[i + 1] - cta_begin[i]);
}

// ---------------------------------------------------------------- host side

size_t fwd_pipe_smem_bytes(int L, int w) {
    return 1024 + kFTileBytes + (size_t)kPStages * kFStageBytes + (size_t)param_rows(L, 0) * w * 4 +
           (size_t)kPGroups * 128 * 4 + 16 + sizeof(PipeBars);
}

int fwd_pipe_threads() { return kPThreads; }

template <class K>
static cudaError_t prepare_pipe(K kernel, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the smallest shared-memory configuration that holds the block (196 of 228
    // KB when it fits, as for the forward kernel): the rest of the SM's 256 KB
    // is L1
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 85);
    if (e != cudaSuccess) return e;
    // the register split assumes exactly kPRegsLaunch registers per thread at launch
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != kPRegsLaunch || fa.maxThreadsPerBlock < kPThreads) return cudaErrorInvalidConfiguration;
    return cudaSuccess;
}

cudaError_t launch_fwd_pipe(const FwdZArgs& a, int act_tanh, int res, int grid, cudaStream_t st) {
    const size_t smem = fwd_pipe_smem_bytes(a.L, a.w);
    cudaError_t e;
#define FBSDE_PIPE_LAUNCH(A, R)                                            \
    do {                                                                   \
        e = prepare_pipe(k_fwd_pipe<A, R>, smem);                          \
        if (e == cudaSuccess) k_fwd_pipe<A, R><<<grid, kPThreads, smem, st>>>(a); \
    } while (0)
    if (act_tanh) {
        if (res) FBSDE_PIPE_LAUNCH(FBSDE_TANH, true);
        else FBSDE_PIPE_LAUNCH(FBSDE_TANH, false);
    } else {
        if (res) FBSDE_PIPE_LAUNCH(FBSDE_SIN, true);
        else FBSDE_PIPE_LAUNCH(FBSDE_SIN, false);
    }
#undef FBSDE_PIPE_LAUNCH
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

size_t bwd_pipe_smem_bytes(int L, int w) {
    (void)L;
    (void)w;
    return 1024 + 2 * kFTileBytes + (size_t)kPBwdStages * kFStageBytes + sizeof(PipeBars);
}

cudaError_t launch_bwd_pipe(const BwdArgs& a, int act_tanh, int res, int grid, cudaStream_t st) {
    const size_t smem = bwd_pipe_smem_bytes(a.L, a.w);
    cudaError_t e;
#define FBSDE_PIPE_LAUNCH(A, R)                                            \
    do {                                                                   \
        e = prepare_pipe(k_bwd_pipe<A, R>, smem);                          \
        if (e == cudaSuccess) k_bwd_pipe<A, R><<<grid, kPThreads, smem, st>>>(a); \
    } while (0)
    if (act_tanh) {
        if (res) FBSDE_PIPE_LAUNCH(FBSDE_TANH, true);
        else FBSDE_PIPE_LAUNCH(FBSDE_TANH, false);
    } else {
        if (res) FBSDE_PIPE_LAUNCH(FBSDE_SIN, true);
        else FBSDE_PIPE_LAUNCH(FBSDE_SIN, false);
    }
#undef FBSDE_PIPE_LAUNCH
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_bwd_pipe_group(const BwdArgs* all, const int* beg, int n, int act_tanh, int res, int grid,
                                  size_t smem, cudaStream_t st) {
    cudaError_t e;
#define FBSDE_PIPE_LAUNCH(A, R)                                                     \
    do {                                                                            \
        e = prepare_pipe(k_bwd_pipe_group<A, R>, smem);                             \
        if (e == cudaSuccess) k_bwd_pipe_group<A, R><<<grid, kPThreads, smem, st>>>(all, beg, n); \
    } while (0)
    if (act_tanh) {
        if (res) FBSDE_PIPE_LAUNCH(FBSDE_TANH, true);
        else FBSDE_PIPE_LAUNCH(FBSDE_TANH, false);
    } else {
        if (res) FBSDE_PIPE_LAUNCH(FBSDE_SIN, true);
        else FBSDE_PIPE_LAUNCH(FBSDE_SIN, false);
    }
#undef FBSDE_PIPE_LAUNCH
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_fwd_pipe_group(const FwdZArgs* all, const int* beg, int n, int act_tanh, int res, int grid,
                                  size_t smem, cudaStream_t st) {
    cudaError_t e;
#define FBSDE_PIPE_LAUNCH(A, R)                                                     \
    do {                                                                            \
        e = prepare_pipe(k_fwd_pipe_group<A, R>, smem);                             \
        if (e == cudaSuccess) k_fwd_pipe_group<A, R><<<grid, kPThreads, smem, st>>>(all, beg, n); \
    } while (0)
    if (act_tanh) {
        if (res) FBSDE_PIPE_LAUNCH(FBSDE_TANH, true);
        else FBSDE_PIPE_LAUNCH(FBSDE_TANH, false);
    } else {
        if (res) FBSDE_PIPE_LAUNCH(FBSDE_SIN, true);
        else FBSDE_PIPE_LAUNCH(FBSDE_SIN, false);
    }
#undef FBSDE_PIPE_LAUNCH
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace fbsde
