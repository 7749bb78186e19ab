// Shared pieces of the per-tile fused kernels of the BF16 form: tile and
// ring sizes, the operand-layout helpers (128-byte-swizzled shared-memory
// tiles, column-pair-major global blocks), the per-column parameter table and
// the launch arguments of the forward (Y, Z) and backward (tangent, adjoint)
// kernels.  Included by fused.cu (the general kernels, NAIS-Net and FP8) and
// fused_pipe.cu (the pipelined FC / ResNet kernels).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "bf16_work.cuh"
#include "tc_common.cuh"

namespace fbsde {
constexpr uint32_t kFStageBytes = 32768;  // one weight slice: up to 256 rows x 128 B
constexpr uint32_t kFTileBytes = 65536;   // activation tile: 4 x [128 x 64] BF16
// Epilogue warp groups (4 warps each, one thread per TMEM lane per group) of
// the two kernels.  Each SM sub-partition holds 16K registers.  The forward
// kernel (warps 0-1 producer and MMA, 3 groups: 14 warps) stays within 128
// registers per thread.  The backward kernel reserves warpgroup 0 (producer,
// MMA, two idle warps) and runs 2 epilogue warpgroups: launched at 168
// registers per thread, warpgroup 0 drops to kBwdRegsCtl and the epilogue
// warpgroups rise to kBwdRegsEpi (setmaxnreg), room for the accumulator
// columns of the next chunk in flight.
constexpr int kFwdGroups = 3;
constexpr int kBwdGroups = 2;
constexpr int kFDepth = 4;  // chunks of global operands kept in flight per thread
__host__ __device__ constexpr int fused_threads(int groups) { return 64 + 128 * groups; }
__host__ __device__ constexpr int bwd_threads() { return 128 + 128 * kBwdGroups; }
constexpr int kBwdRegsLaunch = (65536 / bwd_threads()) & ~7;
constexpr uint32_t kBwdRegsCtl = 40, kBwdRegsEpi = 232;
static_assert(kBwdRegsLaunch == 168, "backward launch register budget");
static_assert(128 * kBwdRegsCtl + 128 * kBwdGroups * kBwdRegsEpi <= (uint32_t)bwd_threads() * kBwdRegsLaunch,
              "register split exceeds the launch allocation");
static_assert(kBwdRegsCtl + kBwdGroups * kBwdRegsEpi <= 512, "register split exceeds an SM sub-partition");
constexpr int kFwdStages = 4;
constexpr int kBwdStages = 2;
// Backward epilogue: chunk iterations per thread that make up one 64-column
// slab (8 chunks of 8 columns shared by the groups).
constexpr int kSlabIters = 8 / kBwdGroups;
static_assert(kSlabIters * kBwdGroups == 8 && kSlabIters % 2 == 0, "slab / group split");

struct FGemm {
    const CUtensorMap* map;
    int nk, K, N, asel;  // K slices, contraction length, output columns, A tile (0 or 1)
    int dual;            // 1: also multiply tile 1 by the same weights into TMEM columns 256..
    int dcol = 0;        // TMEM column of the accumulator
    int acc = 0;         // 1: add to the accumulator's contents (a residual kept there)
    int f8 = 0;          // 1: E4M3 operands (K slices of 128, K = 32 per instruction)
    // NAIS-Net blocks: after the nk slices over the tile, nx slices of 64 over
    // the network input.  Each takes two ring stages: the weight slice (map
    // wx, N rows) and then the BF16 input rows of this tile (map xa; with
    // `dual`, map xb beside them at +16 KB for the second accumulator).
    int nx = 0, Kx = 0;
    const CUtensorMap* wx = nullptr;
    const CUtensorMap* xa = nullptr;
    const CUtensorMap* xb = nullptr;
    // then a second contraction of the same tile (NAIS-Net: B_l[:,1:]^T e_l
    // into the Z accumulator): nk2 weight slices of map2, N2 output columns
    // at TMEM column dcol2, added to its contents when acc2
    const CUtensorMap* map2 = nullptr;
    int nk2 = 0, N2 = 0, dcol2 = 0, acc2 = 0;
};

// ---------------------------------------------------------------- small helpers

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack_bf16x2(uint32_t u) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}

// Columns col..col+7 (col % 8 == 0) of `row` into / out of a swizzled tile.
__device__ __forceinline__ void st_tile8(uint8_t* tile, int row, int col, const float* v) {
    uint4 u;
    u.x = pack_bf16x2(v[0], v[1]); u.y = pack_bf16x2(v[2], v[3]);
    u.z = pack_bf16x2(v[4], v[5]); u.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + (col >> 6) * 16384 + tc::sw128_offset(row, (col & 63) >> 3)) = u;
}
__device__ __forceinline__ void ld_tile8(const uint8_t* tile, int row, int col, float* v) {
    const uint4 u = *reinterpret_cast<const uint4*>(tile + (col >> 6) * 16384 + tc::sw128_offset(row, (col & 63) >> 3));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = unpack_bf16x2(w[i]);
        v[2 * i] = f.x; v[2 * i + 1] = f.y;
    }
}

// Columns col..col+7 (col % 8 == 0) of `row`, times s, into a tile of E4M3
// operands: 128-column slices of 16 KB, 128-byte swizzled rows, each 16-byte
// unit holding 16 values (RN, saturating to the finite range).
__device__ __forceinline__ void st_tile8_e4m3(uint8_t* tile, int row, int col, const float* v, float s) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        w[i] = (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(v[2 * i] * s, v[2 * i + 1] * s), __NV_SATFINITE,
                                                  __NV_E4M3);
    uint8_t* dst = tile + (col >> 7) * 16384 + tc::sw128_offset(row, (col & 127) >> 4) + ((col >> 3) & 1) * 8;
    *reinterpret_cast<uint2*>(dst) = make_uint2(w[0] | (w[1] << 16), w[2] | (w[3] << 16));
}

__device__ __forceinline__ void st_bf16x16(bf16* dst, const float* v) {
    uint4 u0, u1;
    u0.x = pack_bf16x2(v[0], v[1]);   u0.y = pack_bf16x2(v[2], v[3]);
    u0.z = pack_bf16x2(v[4], v[5]);   u0.w = pack_bf16x2(v[6], v[7]);
    u1.x = pack_bf16x2(v[8], v[9]);   u1.y = pack_bf16x2(v[10], v[11]);
    u1.z = pack_bf16x2(v[12], v[13]); u1.w = pack_bf16x2(v[14], v[15]);
    reinterpret_cast<uint4*>(dst)[0] = u0;
    reinterpret_cast<uint4*>(dst)[1] = u1;
}
__device__ __forceinline__ void ld_bf16x16(const bf16* src, float* v) {
    const uint4 u0 = reinterpret_cast<const uint4*>(src)[0];
    const uint4 u1 = reinterpret_cast<const uint4*>(src)[1];
    const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 f = unpack_bf16x2(w[i]);
        v[2 * i] = f.x; v[2 * i + 1] = f.y;
    }
}

__device__ __forceinline__ void tmem_st_f16(uint32_t taddr, const float* v) {
    uint32_t u[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) u[j] = __float_as_uint(v[j]);
    tc::tmem_st16(taddr, u);
}

__device__ __forceinline__ void tmem_st_f8(uint32_t taddr, const float* v) {
    uint32_t u[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) u[j] = __float_as_uint(v[j]);
    tc::tmem_st8(taddr, u);
}
// Eight consecutive floats from a 16-byte-aligned address.
__device__ __forceinline__ void ld_f8(const float* src, float* v) {
    const float4 a = reinterpret_cast<const float4*>(src)[0];
    const float4 b = reinterpret_cast<const float4*>(src)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void st_bf16x8(bf16* dst, const float* v) {
    uint4 u;
    u.x = pack_bf16x2(v[0], v[1]); u.y = pack_bf16x2(v[2], v[3]);
    u.z = pack_bf16x2(v[4], v[5]); u.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(dst) = u;
}

// Column-pair-major 128-row blocks (per-CTA scratch, g_l): the BF16 pair of
// columns (2k, 2k+1) of row r is 32-bit word k * 128 + r, so the 32 rows of a
// warp touch one 128-byte line per access instead of 32 lines.
__device__ __forceinline__ void st_pm16(uint32_t* blk, int row, int c0, const float* v) {
    uint32_t* q = blk + (c0 >> 1) * 128 + row;
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k * 128] = pack_bf16x2(v[2 * k], v[2 * k + 1]);
}
__device__ __forceinline__ void ld_pm16_raw(const uint32_t* blk, int row, int c0, uint32_t (&u)[8]) {
    const uint32_t* q = blk + (c0 >> 1) * 128 + row;
#pragma unroll
    for (int k = 0; k < 8; ++k) u[k] = q[k * 128];
}
__device__ __forceinline__ void st_pm8(uint32_t* blk, int row, int c0, const float* v) {
    uint32_t* q = blk + (c0 >> 1) * 128 + row;
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k * 128] = pack_bf16x2(v[2 * k], v[2 * k + 1]);
}
// Cache-hinted variants (L2 eviction policy `pol`).
__device__ __forceinline__ void st_pm8h(uint32_t* blk, int row, int c0, const float* v, uint64_t pol) {
    uint32_t* q = blk + (c0 >> 1) * 128 + row;
#pragma unroll
    for (int k = 0; k < 4; ++k) tc::st_global_hint(q + k * 128, pack_bf16x2(v[2 * k], v[2 * k + 1]), pol);
}
__device__ __forceinline__ void ld_pm8h(const uint32_t* blk, int row, int c0, uint32_t (&u)[4], uint64_t pol) {
    const uint32_t* q = blk + (c0 >> 1) * 128 + row;
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = tc::ld_global_hint(q + k * 128, pol);
}
__device__ __forceinline__ void ld_pm8_raw(const uint32_t* blk, int row, int c0, uint32_t (&u)[4]) {
    const uint32_t* q = blk + (c0 >> 1) * 128 + row;
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = q[k * 128];
}
__device__ __forceinline__ void unpack8(const uint32_t (&u)[4], float* v) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = unpack_bf16x2(u[k]);
        v[2 * k] = f.x; v[2 * k + 1] = f.y;
    }
}
__device__ __forceinline__ void unpack16(const uint32_t (&u)[8], float* v) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 f = unpack_bf16x2(u[k]);
        v[2 * k] = f.x; v[2 * k + 1] = f.y;
    }
}

// Walk the chunks first, first + step, ... < n with the global operands of the
// next kFDepth chunks in flight: load(ch, words) issues the loads of chunk ch,
// body(ch, words) consumes them.  Register indices stay static (unrolled).
template <int NW, class Load, class Body, int DEPTH = kFDepth>
__device__ __forceinline__ void chunk_loop(int first, int step, int n, Load load, Body body) {
    uint32_t buf[DEPTH][NW];
#pragma unroll
    for (int d = 0; d < DEPTH; ++d)
        if (first + d * step < n) load(first + d * step, buf[d]);
    for (int base = 0; first + base * step < n; base += DEPTH) {
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            const int ch = first + (base + d) * step;
            if (ch < n) {
                uint32_t cur[NW];
#pragma unroll
                for (int k = 0; k < NW; ++k) cur[k] = buf[d][k];
                const int nxt = ch + DEPTH * step;
                if (nxt < n) load(nxt, buf[d]);
                body(ch, cur);
            }
        }
    }
}

// chunk_loop with the accumulator columns of each chunk read from TMEM one
// chunk ahead: loadt(ch, regs) issues the (up to two 8-column) TMEM loads of
// chunk ch, and the wait for them comes only when chunk ch is next, so the
// TMEM latency overlaps the body of the chunk before.  DEPTH must be even.
// The chunks come in `nblocks` blocks of DEPTH per thread (the same count in
// every thread, whatever its share of the n chunks); block(b) runs after
// block b.
template <int NW, int DEPTH, class LoadG, class LoadT, class Body, class Block>
__device__ __forceinline__ void chunk_loop_t(int first, int step, int n, int nblocks, LoadG loadg, LoadT loadt,
                                             Body body, Block block) {
    static_assert(DEPTH % 2 == 0, "TMEM double buffer indexing needs an even depth");
    uint32_t gb[DEPTH][NW];
    uint32_t tb[2][16];
#pragma unroll
    for (int d = 0; d < DEPTH; ++d)
        if (first + d * step < n) loadg(first + d * step, gb[d]);
    if (first < n) loadt(first, tb[0]);
    for (int b = 0; b < nblocks; ++b) {
        const int base = b * DEPTH;
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            const int ch = first + (base + d) * step;
            if (ch < n) {
                tc::tmem_wait_ld_regs(tb[d & 1]);
                uint32_t cg[NW], ct[16];
#pragma unroll
                for (int k = 0; k < NW; ++k) cg[k] = gb[d][k];
#pragma unroll
                for (int k = 0; k < 16; ++k) ct[k] = tb[d & 1][k];
                if (ch + step < n) loadt(ch + step, tb[(d + 1) & 1]);
                if (ch + DEPTH * step < n) loadg(ch + DEPTH * step, gb[d]);
                body(ch, cg, ct);
            }
        }
        block(b);
    }
}

// Tiles leave shared memory by TMA bulk stores issued by one epilogue thread.
// Before a phase writes tiles, the storing thread waits until earlier stores
// have read them and opens `tfree` (bounded wait for all).  The forward
// kernel stores after a phase: every epilogue thread fences its writes for
// the async proxy and arrives on `wdone`, which the storing thread waits for
// (bounded) before it issues the stores.  The backward kernel stores each
// 64-column slab as soon as a named barrier says all its chunks are written,
// and hands the tiles to the MMA issuer with handoff().
struct StoreSync {
    uint64_t* tfree;  // count 1: the storing thread
    uint64_t* wdone;  // count: every epilogue thread
    bool st_thread;
    uint32_t tphase, wphase;
    __device__ bool before_write() {
        if (st_thread) {
            tc::tma_store_wait_read<0>();
            tc::mbar_arrive(tfree);
        }
        return tc::mbar_wait(tfree, (tphase++) & 1u, tc::kWaitBudget);
    }
    // every epilogue thread: the tiles written (and fenced for the async
    // proxy) go to the MMA issuer; no stores wait on this
    __device__ void handoff(uint64_t* aready) {
        tc::tmem_wait_st();
        tc::tc_fence_before();
        tc::mbar_arrive(aready);
    }
    // returns false on timeout; the storing thread may issue stores after it.
    // With `aready`, every thread also hands the tiles to the MMA issuer
    // before the storing thread waits, so the next contraction does not wait
    // for the stores to be issued (both only read the tiles).
    __device__ bool after_write(uint64_t* aready = nullptr) {
        tc::fence_async_shared();
        tc::mbar_arrive(wdone);
        if (aready) {
            tc::tmem_wait_st();
            tc::tc_fence_before();
            tc::mbar_arrive(aready);
        }
        bool ok = true;
        if (st_thread) ok = tc::mbar_wait(wdone, wphase & 1u, tc::kWaitBudget);
        ++wphase;
        return ok;
    }
};

// Per-layer vectors staged in shared memory once per CTA:
// [l * w] bias of layer l (l = 0: b_in; NAIS-Net: C_l), [(L+1) w] w_o,
// [(L+2) w] W_in[:, 0], and for NAIS-Net [(L+2+l) w] B_l[:, 0], l = 1..L
// (the weights of t, which enters every block).
struct ParamOffsets {
    unsigned long long bin, Win, wo, bo, b[kFusedMaxDepth + 1], B[kFusedMaxDepth + 1];
    int nais;
};

__host__ __device__ __forceinline__ int param_rows(int L, int nais) { return nais ? 2 * L + 3 : L + 3; }

__device__ __forceinline__ float param_value(const float* th, const ParamOffsets& o, int L, int l, int c, int K0) {
    if (l <= L) return th[(l == 0 ? o.bin : o.b[l]) + c];
    if (l == L + 1) return th[o.wo + c];
    if (l == L + 2) return th[o.Win + (size_t)c * K0];
    return th[o.B[l - (L + 2)] + (size_t)c * K0];
}

__device__ __forceinline__ void stage_params(float* ptab, const float* th, const ParamOffsets& o, int L, int w,
                                             int K0) {
    const int n = param_rows(L, o.nais) * w;
    for (int i = threadIdx.x; i < n; i += blockDim.x) ptab[i] = param_value(th, o, L, i / w, i % w, K0);
}

struct FwdZArgs {
    CUtensorMap wf[kFusedMaxDepth + 1];  // forward weights: [0] W_in[:,1:] (box {64, w}), [l] W_l
    CUtensorMap wr[kFusedMaxDepth + 1];  // reverse weights: [0] W_in[:,1:]^T (box {64, Dn}), [l] W_l^T
    CUtensorMap eb;                      // e_l stack [L+1][P x wp] (TMA stores), when for_grad
    CUtensorMap xin;                     // BF16 copy of X, [P x Dp], box {64, 128} (TMA loads)
    const float* X;                      // [P x D]
    const float* theta;
    float* Y;                            // [P], zeroed before the launch
    float* Z;                            // [P x D]
    uint32_t* G;                         // g_l, l < L: word l * G_words + (tile * w/2 + k) * 128 + row
    unsigned long long G_words;
    uint32_t* scratch;                   // per CTA: L column-pair-major blocks (act'(a_l), l < L)
    int for_grad;                        // also write g_l and e_l for the gradient
    ParamOffsets off;
    int P, M, D, Dp, Dn, w, wp, L, ntiles;
    float dt;
    int* err;
    // FP8 hidden layers: E4M3 W_l (box {128, w}) and the per-layer inverse
    // scales of the accumulators; h_l for l < L is written to the tile in E4M3
    int f8;
    CUtensorMap wf8[kFusedMaxDepth + 1];
    const float* f8inv;
    // NAIS-Net: B_l[:, 1:] (box {64, w}), streamed beside the X rows, its
    // transpose (box {64, Dn}) for the Z terms, and the step h
    CUtensorMap wbx[kFusedMaxDepth + 1];
    CUtensorMap wbxT[kFusedMaxDepth + 1];
    float hs;
    long long wait_budget;  // SM clock cycles a bounded wait may spin before it gives up
    int gate;               // test hook: every role's first wait is on a barrier nothing completes
};

struct BwdArgs {
    CUtensorMap wf[kFusedMaxDepth + 1];
    CUtensorMap wr[kFusedMaxDepth + 1];
    CUtensorMap hb, hdb, abb;  // operand stacks [L+1][P x wp] (TMA stores)
    CUtensorMap xb, vb;        // BF16 copies of X and V, [P x Dp], box {64, 128} (TMA loads)
    const float* X;
    const float* V;            // d loss / d Z_n  [P x D]
    const float* alpha;        // d loss / d Y_n  [P]
    const float* theta;
    const uint32_t* G;         // g_l, l < L, column-pair-major per tile (from k_fused_fwdz)
    unsigned long long G_words;
    bf16* HbL;                 // h_L rows of wp (its tile slot holds abar_L); general kernels
    float* wopart;             // pipelined kernels: [ntiles][4][w] partial sums of alpha h_L + h'_L
    uint32_t* scratch;         // per CTA: act'(a_l) and S_l, l < L, column-pair-major
    ParamOffsets off;
    const float* pvec;  // [param_rows x w]: b_0..b_L, w_o, W_in[:,0] (NAIS-Net: B_l[:,0])
    int P, M, D, Dp, w, wp, L, ntiles;
    int res;            // ResNet, NAIS-Net: hbar accumulates in place in TMEM columns 256..
    float dt;
    int* err;
    CUtensorMap wbx[kFusedMaxDepth + 1];  // NAIS-Net: B_l[:, 1:] (box {64, w})
    float hs;                             // NAIS-Net step h
    long long wait_budget;  // SM clock cycles a bounded wait may spin before it gives up
    int gate;               // test hook: every role's first wait is on a barrier nothing completes
};

// The pipelined FC / ResNet kernels (fused_pipe.cu).
size_t fwd_pipe_smem_bytes(int L, int w);
cudaError_t launch_fwd_pipe(const FwdZArgs& a, int act_tanh, int res, int grid, cudaStream_t st);
cudaError_t launch_fwd_pipe_group(const FwdZArgs* all, const int* beg, int n, int act_tanh, int res, int grid,
                                  size_t smem, cudaStream_t st);
size_t bwd_pipe_smem_bytes(int L, int w);
cudaError_t launch_bwd_pipe(const BwdArgs& a, int act_tanh, int res, int grid, cudaStream_t st);
cudaError_t launch_bwd_pipe_group(const BwdArgs* all, const int* beg, int n, int act_tanh, int res, int grid,
                                  size_t smem, cudaStream_t st);

}  // namespace fbsde
