// Per-tile fused kernels of the BF16 form (FC, ResNet and NAIS-Net networks).
//
// Both kernels walk one tile of 128 points (persistent CTAs, one per SM)
// through a fixed sequence of layer contractions without leaving the SM:
//   * activation tiles (BF16, 128 rows x up to 256 columns) live in shared
//     memory in the 128-byte-swizzled K-major layout the tensor cores read,
//     and each layer's epilogue rewrites them in place;
//   * the forward kernel keeps the residual stream (FP32) in TMEM columns
//     256..511 next to the accumulator (columns 0..255); the backward kernel
//     holds two accumulators there (forward recomputation and tangent) and
//     accumulates the adjoint h-bar in place;
//   * the weights stream from L2 through a TMA ring, one 64-wide K slice per
//     stage, in the order the layers consume them (NAIS-Net blocks: then the
//     B_l slices, each beside this tile's input rows in the next stage);
//   * per-layer derivatives needed later in the tile go to a per-CTA scratch
//     region that the same CTA reads back within microseconds.
// Warp 0 issues the weight TMA loads and warp 1 allocates TMEM and issues
// tcgen05.mma from one thread; the epilogue warpgroups (three in the forward
// kernel from warp 2, two in the backward kernel from warp 4, each covering
// the 128 TMEM lanes) take alternating 8-column chunks.  The MMA of
// contraction q+1 starts when every epilogue thread has finished contraction
// q (mbarrier `aready`): they have read its accumulator and written the
// operand the next contraction reads.  Every wait is bounded.
//
// k_fused_fwdz (Section 2.2: Y = u(t, X) and Z = grad_x u by the reverse
// pass): lift, L layers, the reverse sweep through the L layers and the Z
// contraction; outputs Y, Z and g_l (BF16, l < L) for the gradient.  Its F8
// variant runs the hidden-layer forward contractions on E4M3 operands.
//
// k_fused_bwd (the derivative of the loss of Eq. "loss" through Y_n and Z_n):
// per layer the forward contraction (recomputed) and the tangent contraction
// along (0, v), then the adjoint sweep down the layers; outputs the operands
// of the weight-gradient contractions: h_l, h'_l, abar_l (BF16).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>

#include "bf16_work.cuh"
#include "fused_common.cuh"
#include "tc_common.cuh"

namespace fbsde {


// ---------------------------------------------------------------- producer / MMA roles

// Warp 0, one lane: stream the weight slices of every contraction of every
// tile of this CTA through the ring.
// XS: the schedule may contain input slices (FGemm::nx).
template <bool XS, class Sched>
__device__ void producer_role(const Sched& sch, int ntiles, int nstages, uint8_t* ring, uint64_t* bfull,
                              uint64_t* bempty, volatile int* abort_flag, int* err) {
    int it = 0;
    bool ok = true;
    for (int t = sch.cta; t < ntiles && ok; t += sch.nctas) {
        for (int q = 0; q < sch.nq() && ok; ++q) {
            const FGemm g = sch.gemm(q);
            const int nload = XS ? g.nk + 2 * g.nx + g.nk2 : g.nk;
            for (int kc = 0; kc < nload; ++kc, ++it) {
                const int s = it % nstages;
                const uint32_t ph = (uint32_t)(it / nstages) & 1u;
                if (*abort_flag || !tc::mbar_wait(&bempty[s], ph ^ 1u, tc::kWaitBudget)) {
                    ok = false;
                    break;
                }
                if (!XS || kc < g.nk) {
                    tc::mbar_expect_tx(&bfull[s], (uint32_t)g.N * 128u);
                    tc::tma_load_2d(ring + s * kFStageBytes, g.map, &bfull[s], kc * 64, 0);
                } else if (kc >= g.nk + 2 * g.nx) {
                    tc::mbar_expect_tx(&bfull[s], (uint32_t)g.N2 * 128u);
                    tc::tma_load_2d(ring + s * kFStageBytes, g.map2, &bfull[s], (kc - g.nk - 2 * g.nx) * 64, 0);
                } else if (((kc - g.nk) & 1) == 0) {
                    tc::mbar_expect_tx(&bfull[s], (uint32_t)g.N * 128u);
                    tc::tma_load_2d(ring + s * kFStageBytes, g.wx, &bfull[s], ((kc - g.nk) >> 1) * 64, 0);
                } else {
                    const int x = ((kc - g.nk) >> 1) * 64;
                    tc::mbar_expect_tx(&bfull[s], g.xb ? 32768u : 16384u);
                    tc::tma_load_2d(ring + s * kFStageBytes, g.xa, &bfull[s], x, t * 128);
                    if (g.xb) tc::tma_load_2d(ring + s * kFStageBytes + 16384, g.xb, &bfull[s], x, t * 128);
                }
            }
        }
    }
    if (!ok) {
        if (err) atomicExch(err, 2);
        *abort_flag = 1;
    }
}

// Warp 1, one lane: per contraction wait for the operand tile, then issue
// K = 16 MMAs slice by slice, releasing each ring stage and finally
// signalling the accumulator.
// F8: the schedule may contain E4M3 contractions (FGemm::f8); without it
// the loop is the BF16 one only.
template <bool F8, bool XS, class Sched>
__device__ void mma_role(const Sched& sch, int ntiles, int nstages, uint32_t abase0, uint32_t abase1,
                         uint32_t rbase, uint32_t tmem, uint64_t* bfull, uint64_t* bempty, uint64_t* accf,
                         uint64_t* aready, volatile int* abort_flag, int* err) {
    int it = 0, qg = 0;
    bool ok = true;
    for (int t = sch.cta; t < ntiles && ok; t += sch.nctas) {
        for (int q = 0; q < sch.nq() && ok; ++q, ++qg) {
            if (*abort_flag || !tc::mbar_wait(aready, (uint32_t)qg & 1u, tc::kWaitBudget)) {
                ok = false;
                break;
            }
            tc::tc_fence_after();
            const FGemm g = sch.gemm(q);
            sch.prefetch(q, t);
            const uint32_t abase = g.asel ? abase1 : abase0;
            const bool f8 = F8 && g.f8 != 0;
            const uint32_t idesc = f8 ? tc::idesc_e4m3(128, g.N) : tc::idesc_bf16(128, g.N, 0, 0);
            const bool dual = g.dual != 0;
            for (int kc = 0; kc < g.nk; ++kc, ++it) {
                const int s = it % nstages;
                const uint32_t ph = (uint32_t)(it / nstages) & 1u;
                if (*abort_flag || !tc::mbar_wait(&bfull[s], ph, tc::kWaitBudget)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                // K per slice 64 (BF16) or 128 (E4M3); one K step is 32 bytes of
                // the 128-byte swizzled rows for both types
                const int nsteps = f8 ? min(4, (g.K - kc * 128 + 31) / 32) : min(4, (g.K - kc * 64 + 15) / 16);
                for (int k = 0; k < nsteps; ++k) {
                    const uint64_t ad = tc::sdesc_sw128(abase + (uint32_t)kc * 16384u + 32u * k, 16u);
                    const uint64_t bd = tc::sdesc_sw128(rbase + (uint32_t)s * kFStageBytes + 32u * k, 16u);
                    if (F8 && f8) {
                        tc::mma_f8(tmem + (uint32_t)g.dcol, ad, bd, idesc, (g.acc || kc > 0 || k > 0) ? 1u : 0u);
                        continue;
                    }
                    tc::mma_bf16(tmem + (uint32_t)g.dcol, ad, bd, idesc, (g.acc || kc > 0 || k > 0) ? 1u : 0u);
                    if (dual) {
                        const uint64_t ad1 = tc::sdesc_sw128(abase1 + (uint32_t)kc * 16384u + 32u * k, 16u);
                        tc::mma_bf16(tmem + 256u, ad1, bd, idesc, (kc > 0 || k > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&bempty[s]);
            }
            // input slices: weights in one stage, the input rows in the next;
            // both accumulate onto the tile's contraction
            for (int j = 0; XS && ok && j < g.nx; ++j, it += 2) {
                const int s1 = it % nstages, s2 = (it + 1) % nstages;
                if (*abort_flag || !tc::mbar_wait(&bfull[s1], (uint32_t)(it / nstages) & 1u, tc::kWaitBudget) ||
                    !tc::mbar_wait(&bfull[s2], (uint32_t)((it + 1) / nstages) & 1u, tc::kWaitBudget)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const int nsteps = min(4, (g.Kx - j * 64 + 15) / 16);
                for (int k = 0; k < nsteps; ++k) {
                    const uint64_t bd = tc::sdesc_sw128(rbase + (uint32_t)s1 * kFStageBytes + 32u * k, 16u);
                    const uint64_t ad = tc::sdesc_sw128(rbase + (uint32_t)s2 * kFStageBytes + 32u * k, 16u);
                    tc::mma_bf16(tmem + (uint32_t)g.dcol, ad, bd, idesc, 1u);
                    if (dual) {
                        const uint64_t ad1 = tc::sdesc_sw128(rbase + (uint32_t)s2 * kFStageBytes + 16384u + 32u * k, 16u);
                        tc::mma_bf16(tmem + 256u, ad1, bd, idesc, 1u);
                    }
                }
                tc::mma_commit(&bempty[s1]);
                tc::mma_commit(&bempty[s2]);
            }
            // second contraction of the tile
            for (int kc = 0; XS && ok && kc < g.nk2; ++kc, ++it) {
                const int s = it % nstages;
                if (*abort_flag || !tc::mbar_wait(&bfull[s], (uint32_t)(it / nstages) & 1u, tc::kWaitBudget)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t idesc2 = tc::idesc_bf16(128, g.N2, 0, 0);
                const int nsteps = min(4, (g.K - kc * 64 + 15) / 16);
                for (int k = 0; k < nsteps; ++k) {
                    const uint64_t ad = tc::sdesc_sw128(abase + (uint32_t)kc * 16384u + 32u * k, 16u);
                    const uint64_t bd = tc::sdesc_sw128(rbase + (uint32_t)s * kFStageBytes + 32u * k, 16u);
                    tc::mma_bf16(tmem + (uint32_t)g.dcol2, ad, bd, idesc2, (g.acc2 || kc > 0 || k > 0) ? 1u : 0u);
                }
                tc::mma_commit(&bempty[s]);
            }
            if (ok) tc::mma_commit(accf);
        }
    }
    if (!ok) {
        if (err) atomicExch(err, 2);
        *abort_flag = 1;
    }
}

// ---------------------------------------------------------------- forward + Z


struct FwdZSched {
    const FwdZArgs* a;
    int cta, nctas;  // this CTA among the CTAs that share the tiles
    __device__ int nq() const { return 2 * a->L + 2; }
    // 0: lift, 1..L: layers, L+1..2L: reverse through layer 2L+1-q, 2L+1: Z
    __device__ FGemm gemm(int q) const {
        FGemm g;
        const int L = a->L;
        g.asel = 0;
        g.dual = 0;
        if (q == 0) { g.map = &a->wf[0]; g.nk = a->Dp / 64; g.K = a->D; g.N = a->w; }
        else if (q <= L && a->f8) { g.map = &a->wf8[q]; g.nk = (a->w + 127) / 128; g.K = a->w; g.N = a->w; g.f8 = 1; }
        else if (q <= L) {
            g.map = &a->wf[q]; g.nk = a->wp / 64; g.K = a->w; g.N = a->w;
            if (a->off.nais) { g.nx = a->Dp / 64; g.Kx = a->D; g.wx = &a->wbx[q]; g.xa = &a->xin; }
        }
        else if (q <= 2 * L) {
            const int l = 2 * L + 1 - q;
            g.map = &a->wr[l]; g.nk = a->wp / 64; g.K = a->w; g.N = a->w;
            if (a->off.nais) {
                // g_{l-1} = g_l + A_l^T e_l accumulates in place (columns 0..),
                // Z += B_l[:,1:]^T e_l in columns 256..
                g.acc = 1;
                g.map2 = &a->wbxT[l]; g.nk2 = a->wp / 64; g.N2 = a->Dn; g.dcol2 = 256; g.acc2 = l < L;
            }
        }
        else {
            g.map = &a->wr[0]; g.nk = a->wp / 64; g.K = a->w; g.N = a->Dn;
            if (a->off.nais) { g.dcol = 256; g.acc = L > 0; }
        }
        return g;
    }
    // into L2 while contraction q runs: the act' block its epilogue reads
    __device__ void prefetch(int q, int) const {
        const int L = a->L;
        if (q > L && q <= 2 * L) {
            const int l = 2 * L + 1 - q;
            const size_t blk = (size_t)(a->w / 2) * 128;
            tc::prefetch_l2_bulk(a->scratch + ((size_t)cta * L + (l - 1)) * blk, (uint32_t)(blk * 4));
        }
    }
};

// NAIS: NAIS-Net blocks (h_l = h_{l-1} + h act(A_l h_{l-1} + B_l u + C_l), Section 3.1).
// The CTA is number `cta` of the `nctas` CTAs that walk this instance's tiles.
template <int ACT, bool RES, bool F8, bool NAIS>
__device__ __forceinline__ void fwdz_body(const FwdZArgs& a, const int cta, const int nctas) {
    constexpr int NG = kFwdGroups, NE = 128 * NG;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* tile = smem;
    uint8_t* ring = smem + kFTileBytes;
    float* ptab = (float*)(ring + kFwdStages * kFStageBytes);
    const int prows = param_rows(a.L, NAIS);
    uint64_t* bfull = (uint64_t*)(ptab + prows * a.w);
    uint64_t* bempty = bfull + kFwdStages;
    uint64_t* accf = bempty + kFwdStages;
    uint64_t* aready = accf + 1;
    uint64_t* tfree = aready + 1;
    uint64_t* wdone = tfree + 1;
    uint64_t* xfull = wdone + 1;
    uint64_t* ybar = xfull + 1;
    uint32_t* tslot = (uint32_t*)(ybar + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);
    float* ysum = (float*)(smem + kFTileBytes + kFwdStages * kFStageBytes) + prows * a.w + 64;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = a.L;
    const FwdZSched sch{&a, cta, nctas};

    stage_params(ptab, a.theta, a.off, L, a.w, a.D + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kFwdStages; ++s) {
            tc::mbar_init(&bfull[s], 1);
            tc::mbar_init(&bempty[s], 1);
        }
        tc::mbar_init(accf, 1);
        tc::mbar_init(aready, NE);
        tc::mbar_init(tfree, 1);
        tc::mbar_init(wdone, NE);
        tc::mbar_init(xfull, 1);
        tc::mbar_init(ybar, NE);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) producer_role<NAIS>(sch, a.ntiles, kFwdStages, ring, bfull, bempty, abort_flag, a.err);
    } else if (warp == 1) {
        if (lane == 0)
            mma_role<F8, NAIS>(sch, a.ntiles, kFwdStages, tc::smem_u32(tile), tc::smem_u32(tile), tc::smem_u32(ring), tmem,
                     bfull, bempty, accf, aready, abort_flag, a.err);
    } else {
        const int eg = (warp - 2) >> 2;  // epilogue group: chunks eg, eg + NG, ...
        const int lg = warp & 3;         // TMEM lane group of this warp
        const int row = lg * 32 + lane;
        const uint32_t tacc = tmem + ((uint32_t)(lg * 32) << 16);
        const uint32_t tres = tacc + 256u;
        const float* wo = ptab + (L + 1) * a.w;
        const float* win0 = ptab + (L + 2) * a.w;
        const size_t blk = (size_t)(a.w / 2) * 128;  // words of one column-pair-major 128-row block
        uint32_t* scr = a.scratch + (size_t)cta * L * blk;
        StoreSync ss{tfree, wdone, warp == 2 && lane == 0, 0u, 0u};
        // L2 policies: per-CTA scratch stays (re-read within microseconds),
        // the g_l / e_l streams go out first (read by later kernels)
        const uint64_t pol_keep = tc::l2_policy_evict_last(), pol_stream = tc::l2_policy_evict_first();
        const int nq = sch.nq();
        const int nkw = a.wp / 64;
        const int nch = a.w / 8;
        int qg = 0, tcount = 0;
        bool ok = true;
        // network input (t enters as a per-row bias): the BF16 X rows by TMA,
        // requested for the next tile as soon as the Z contraction has read
        // the current one, so that the load overlaps the Z epilogue
        auto request_x = [&](int tile_index) {
            if (ss.st_thread) {
                tc::mbar_expect_tx(xfull, (uint32_t)(a.Dp / 64) * 16384u);
                for (int k = 0; k < a.Dp / 64; ++k)
                    tc::tma_load_2d(tile + k * 16384, &a.xin, xfull, k * 64, tile_index * 128);
            }
        };
        bool requested = false;
        for (int t = cta; t < a.ntiles && ok; t += nctas) {
            const int p = t * 128 + row;
            const bool valid = p < a.P;
            const float tval = valid ? (float)(p / a.M) * a.dt : 0.f;
            uint32_t* gtile = a.G + (size_t)t * blk;
            if (!requested) {
                if (!ss.before_write()) { ok = false; break; }
                request_x(t);
            }
            requested = false;
            if (!tc::mbar_wait(xfull, (uint32_t)tcount & 1u, tc::kWaitBudget)) { ok = false; break; }
            ++tcount;
            if (!ss.after_write(aready)) { ok = false; break; }
            for (int q = 0; q < nq; ++q, ++qg) {
                if (!tc::mbar_wait(accf, (uint32_t)qg & 1u, tc::kWaitBudget)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const bool writes_tile = q <= 2 * L;
                if (writes_tile && !ss.before_write()) { ok = false; break; }
                if (q == nq - 1 && t + nctas < a.ntiles) {
                    if (!ss.before_write()) { ok = false; break; }
                    request_x(t + nctas);
                    requested = true;
                }
                int store_layer = -1;  // e_l stored from the tile after this phase
                if (q <= L) {
                    // forward layer l: a = acc + b_l (+ t W_in[:,0]); h_l = [h_{l-1}] + act(a)
                    const int l = q;
                    const float* bias = ptab + l * a.w;
                    const float* bt = ptab + (L + 2 + l) * a.w;  // NAIS: B_l[:, 0]
                    const bool blk_nais = NAIS && l >= 1;
                    uint32_t* sc = scr + (size_t)l * blk;
                    float ypart = 0.f;
                    // FP8 hidden layers: the accumulator of layer l >= 1 carries the
                    // scales of its E4M3 operands; h_l (l < L) goes out in E4M3
                    const bool f8 = F8 && a.f8 != 0;
                    const float ascale = (F8 && f8 && l >= 1) ? __ldg(a.f8inv + l) : 1.f;
                    const float hscale = F8 ? e4m3_act_scale(l, RES) : 1.f;
                    for (int ch = eg; ch < nch; ch += NG) {
                        const int c0 = ch * 8;
                        uint32_t rv[8], rr[8];
                        tc::tmem_ld8(tacc + (uint32_t)c0, rv);
                        if (RES && l >= 1) tc::tmem_ld8(tres + (uint32_t)c0, rr);
                        tc::tmem_wait_ld();
                        float h[8], d1[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float av = F8 ? fmaf(__uint_as_float(rv[j]), ascale, bias[c0 + j])
                                          : __uint_as_float(rv[j]) + bias[c0 + j];
                            if (l == 0) av = fmaf(tval, win0[c0 + j], av);
                            if (blk_nais) av = fmaf(tval, bt[c0 + j], av);
                            const Act3 f = act3_sfu<ACT>(av);
                            h[j] = ((RES && l >= 1) ? __uint_as_float(rr[j]) : 0.f) + (blk_nais ? a.hs * f.f : f.f);
                            d1[j] = blk_nais ? a.hs * f.d1 : f.d1;
                        }
                        if (l < L) {
                            if (F8 && f8) st_tile8_e4m3(tile, row, c0, h, hscale);
                            else st_tile8(tile, row, c0, h);
                            st_pm8h(sc, row, c0, d1, pol_keep);
                            if (RES) tmem_st_f8(tres + (uint32_t)c0, h);
                        } else {
                            // top: y = w_o^T h_L + b_o and e_L = act'(a_L) w_o
                            float e[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                ypart = fmaf(h[j], wo[c0 + j], ypart);
                                e[j] = d1[j] * wo[c0 + j];
                            }
                            st_tile8(tile, row, c0, e);
                            // NAIS-Net: g_L = w_o seeds the in-place accumulation of g
                            if (NAIS) tmem_st_f8(tacc + (uint32_t)c0, wo + c0);
                        }
                    }
                    if (l == L) {
                        // y = b_o + the groups' partial sums, added in a fixed order
                        ysum[eg * 128 + row] = ypart;
                        tc::mbar_arrive(ybar);
                        if (eg == 0) {
                            if (!tc::mbar_wait(ybar, (uint32_t)(tcount - 1) & 1u, tc::kWaitBudget)) { ok = false; break; }
                            float y = __ldg(a.theta + a.off.bo);
                            for (int g2 = 0; g2 < NG; ++g2) y += ysum[g2 * 128 + row];
                            if (valid) a.Y[p] = y;
                        }
                        store_layer = L;
                    }
                } else if (q <= 2 * L) {
                    // reverse through layer l: g_{l-1} = [g_l] + W_l^T e_l, e_{l-1} = act'(a_{l-1}) g_{l-1}
                    const int l = 2 * L + 1 - q;
                    const uint32_t* sc = scr + (size_t)(l - 1) * blk;
                    uint32_t* gout = gtile + (size_t)(l - 1) * a.G_words;
                    chunk_loop<4>(eg, NG, nch,
                        [&](int ch, uint32_t (&u)[4]) { ld_pm8_raw(sc, row, ch * 8, u); },
                        [&](int ch, const uint32_t (&du)[4]) {
                            const int c0 = ch * 8;
                            float d1[8];
                            unpack8(du, d1);
                            // ResNet: g_l from the FP32 residual columns; NAIS-Net: the
                            // contraction accumulated g_{l-1} in place
                            constexpr bool RRES = RES && !NAIS;
                            uint32_t rv[8], rr[8];
                            tc::tmem_ld8(tacc + (uint32_t)c0, rv);
                            if (RRES && l < L) tc::tmem_ld8(tres + (uint32_t)c0, rr);
                            tc::tmem_wait_ld();
                            float g[8], e[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const float gl = RRES ? (l == L ? wo[c0 + j] : __uint_as_float(rr[j])) : 0.f;
                                g[j] = gl + __uint_as_float(rv[j]);
                                e[j] = d1[j] * g[j];
                            }
                            if (a.for_grad) st_pm8h(gout, row, c0, g, pol_stream);
                            st_tile8(tile, row, c0, e);
                            if (RRES) tmem_st_f8(tres + (uint32_t)c0, g);
                        });
                    store_layer = l - 1;
                } else {
                    // Z = W_in[:,1:]^T e_0 (NAIS-Net: + sum_l B_l[:,1:]^T e_l, columns 256..)
                    for (int ch = eg; ch < a.Dn / 8; ch += NG) {
                        const int c0 = ch * 8;
                        uint32_t rv[8];
                        tc::tmem_ld8(tacc + (NAIS ? 256u : 0u) + (uint32_t)c0, rv);
                        tc::tmem_wait_ld();
                        if (valid) {
                            float* zr = a.Z + (size_t)p * a.D + c0;
                            if ((a.D & 3) == 0 && c0 + 8 <= a.D) {
                                reinterpret_cast<float4*>(zr)[0] = make_float4(
                                    __uint_as_float(rv[0]), __uint_as_float(rv[1]), __uint_as_float(rv[2]),
                                    __uint_as_float(rv[3]));
                                reinterpret_cast<float4*>(zr)[1] = make_float4(
                                    __uint_as_float(rv[4]), __uint_as_float(rv[5]), __uint_as_float(rv[6]),
                                    __uint_as_float(rv[7]));
                            } else {
#pragma unroll
                                for (int j = 0; j < 8; ++j)
                                    if (c0 + j < a.D) zr[j] = __uint_as_float(rv[j]);
                            }
                        }
                    }
                }
                if (writes_tile) {
                    if (!ss.after_write(q < nq - 1 ? aready : nullptr)) { ok = false; break; }
                    if (ss.st_thread && a.for_grad && store_layer >= 0) {
                        for (int k = 0; k < nkw; ++k)
                            tc::tma_store_3d_hint(&a.eb, tile + k * 16384, k * 64, t * 128, store_layer, pol_stream);
                        tc::tma_store_commit();
                    }
                } else if (q < nq - 1) {
                    tc::tmem_wait_st();
                    tc::tc_fence_before();
                    tc::mbar_arrive(aready);
                }
            }
        }
        if (ss.st_thread) tc::tma_store_wait_all<0>();
        if (!ok) {
            if (a.err) atomicExch(a.err, 2);
            *abort_flag = 1;
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

template <int ACT, bool RES, bool F8, bool NAIS>
__global__ void __launch_bounds__(fused_threads(kFwdGroups), 1) k_fused_fwdz(const __grid_constant__ FwdZArgs a) {
    fwdz_body<ACT, RES, F8, NAIS>(a, (int)blockIdx.x, (int)gridDim.x);
}

// One launch for the forward kernels of several instances (a group): CTAs
// cta_begin[i] .. cta_begin[i+1]-1 walk the tiles of instance i, whose
// arguments (tensor maps included) sit in global memory.
template <int ACT, bool RES, bool F8, bool NAIS>
__global__ void __launch_bounds__(fused_threads(kFwdGroups), 1)
    k_fused_fwdz_group(const FwdZArgs* __restrict__ all, const int* __restrict__ cta_begin, int n) {
    int i = 0;
    while (i + 1 < n && (int)blockIdx.x >= cta_begin[i + 1]) ++i;
    fwdz_body<ACT, RES, F8, NAIS>(all[i], (int)blockIdx.x - cta_begin[i], cta_begin[i + 1] - cta_begin[i]);
}

// ---------------------------------------------------------------- tangent + adjoint


struct BwdSched {
    const BwdArgs* a;
    int cta, nctas;  // this CTA among the CTAs that share the tiles
    __device__ int nq() const { return 2 * a->L + 1; }
    // l = q (0..L): forward and tangent contractions of layer l together (two
    // accumulators, one weight stream); q = L+1+j: adjoint through layer L-j
    __device__ FGemm gemm(int q) const {
        FGemm g;
        const int L = a->L;
        if (q <= L) {
            g.asel = 0;
            g.dual = 1;
            g.map = &a->wf[q];
            g.nk = (q == 0 ? a->Dp : a->wp) / 64;
            g.K = q == 0 ? a->D : a->w;
            g.N = a->w;
            if (q > 0 && a->off.nais) {
                // forward B_l x and tangent B_l v from the same weight slices
                g.nx = a->Dp / 64; g.Kx = a->D; g.wx = &a->wbx[q]; g.xa = &a->xb; g.xb = &a->vb;
            }
        } else {
            const int l = L - (q - (L + 1));
            g.asel = 0;
            g.dual = 0;
            g.dcol = a->res ? 256 : 0;
            g.acc = a->res;
            g.map = &a->wr[l];
            g.nk = a->wp / 64;
            g.K = a->w;
            g.N = a->w;
        }
        return g;
    }
    // into L2 while contraction q runs: the blocks its epilogue reads
    __device__ void prefetch(int q, int t) const {
        const int L = a->L;
        const size_t blk = (size_t)(a->w / 2) * 128;
        if (q < L) {
            tc::prefetch_l2_bulk(a->G + (size_t)q * a->G_words + (size_t)t * blk, (uint32_t)(blk * 4));
        } else if (q > L) {
            const int l = L - (q - (L + 1));
            const uint32_t* d1 = a->scratch + (size_t)cta * 2 * L * blk + (size_t)(l - 1) * blk;
            tc::prefetch_l2_bulk(d1, (uint32_t)(blk * 4));
            tc::prefetch_l2_bulk(d1 + (size_t)L * blk, (uint32_t)(blk * 4));
        }
    }
};

// The backward recomputes the forward with the BF16 skip path of the tile (the
// FP32 residual of k_fused_fwdz has no room here: TMEM holds both the forward
// and the tangent accumulators), and carries the tangent h' in BF16 as well.
template <int ACT, bool RES, bool NAIS>
__device__ __forceinline__ void bwd_body(const BwdArgs& a, const int cta, const int nctas) {
    constexpr int NG = kBwdGroups, NE = 128 * NG;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* tile_h = smem;                  // h_l in the up-sweep, abar_l in the down-sweep
    uint8_t* tile_d = smem + kFTileBytes;    // h'_l
    uint8_t* ring = smem + 2 * kFTileBytes;
    float* ptab = (float*)(ring + kBwdStages * kFStageBytes);
    const int prows = param_rows(a.L, NAIS);
    uint64_t* bfull = (uint64_t*)(ptab + prows * a.w);
    uint64_t* bempty = bfull + kBwdStages;
    uint64_t* accf = bempty + kBwdStages;
    uint64_t* aready = accf + 1;
    uint64_t* tfree = aready + 1;
    uint64_t* wdone = tfree + 1;
    uint64_t* xfull = wdone + 1;
    uint32_t* tslot = (uint32_t*)(xfull + 1);
    volatile int* abort_flag = (volatile int*)(tslot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = a.L;
    const BwdSched sch{&a, cta, nctas};

    for (int k = threadIdx.x; k < prows * a.w / 4; k += blockDim.x)
        reinterpret_cast<float4*>(ptab)[k] = __ldg(reinterpret_cast<const float4*>(a.pvec) + k);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kBwdStages; ++s) {
            tc::mbar_init(&bfull[s], 1);
            tc::mbar_init(&bempty[s], 1);
        }
        tc::mbar_init(accf, 1);
        tc::mbar_init(aready, NE);
        tc::mbar_init(tfree, 1);
        tc::mbar_init(wdone, NE);
        tc::mbar_init(xfull, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp < 4) {
        tc::setmaxnreg_dec<kBwdRegsCtl>();
        if (warp == 0) {
            if (lane == 0) producer_role<NAIS>(sch, a.ntiles, kBwdStages, ring, bfull, bempty, abort_flag, a.err);
        } else if (warp == 1) {
            if (lane == 0)
                mma_role<false, NAIS>(sch, a.ntiles, kBwdStages, tc::smem_u32(tile_h), tc::smem_u32(tile_d), tc::smem_u32(ring),
                         tmem, bfull, bempty, accf, aready, abort_flag, a.err);
        }
    } else {
        tc::setmaxnreg_inc<kBwdRegsEpi>();
        const int eg = (warp - 4) >> 2;
        const int lg = warp & 3;
        const int row = lg * 32 + lane;
        const uint32_t tacc = tmem + ((uint32_t)(lg * 32) << 16);
        const uint32_t tsec = tacc + 256u;  // tangent accumulator in the up-sweep, hbar in the down-sweep
        // per-column parameters (biases, w_o, W_in[:,0]; NAIS-Net: B_l[:,0]):
        // 16-byte broadcast loads from the table staged in shared memory at
        // the start (copied from the table k_stage_pvec forms each step)
        const float* wo = ptab + (size_t)(L + 1) * a.w;
        const float* win0 = ptab + (size_t)(L + 2) * a.w;
        const size_t blk = (size_t)(a.w / 2) * 128;
        uint32_t* scr_d1 = a.scratch + (size_t)cta * 2 * L * blk;  // act'(a_l), l < L
        uint32_t* scr_S = scr_d1 + (size_t)L * blk;                       // S_l, l < L
        StoreSync ss{tfree, wdone, warp == 4 && lane == 0, 0u, 0u};
        // L2 policies: per-CTA scratch stays (re-read within microseconds),
        // g_l and the operand stacks stream
        const uint64_t pol_keep = tc::l2_policy_evict_last(), pol_stream = tc::l2_policy_evict_first();
        const int nq = sch.nq();
        const int nch = a.w / 8;
        const int nkw = a.wp / 64, nkx = a.Dp / 64;
        int qg = 0, tcount = 0;
        bool v_requested = false;
        bool ok = true;
        // A wait that runs out of budget clears `ok` but the thread still
        // goes through the phase (the named barriers of the slab stores need
        // every epilogue thread); at the end of each phase all of them take
        // the same decision, so none is left waiting at a barrier.
        for (int t = cta; t < a.ntiles && ok; t += nctas) {
            const int p = t * 128 + row;
            const bool valid = p < a.P;
            const float tval = valid ? (float)(p / a.M) * a.dt : 0.f;
            const float alpha_p = valid ? __ldg(a.alpha + p) : 0.f;
            const uint32_t* gtile = a.G + (size_t)t * blk;
            // inputs: (t, X) for the forward, (0, v) for the tangent, BF16 rows
            // by TMA; the v rows were requested during the previous tile's
            // adjoint sweep (tile_d is free once the up-sweep is done)
            if (ok) ok = ss.before_write();
            if (ss.st_thread) {
                tc::mbar_expect_tx(xfull, (uint32_t)nkx * (v_requested ? 1u : 2u) * 16384u);
                for (int k = 0; k < nkx; ++k) {
                    tc::tma_load_2d(tile_h + k * 16384, &a.xb, xfull, k * 64, t * 128);
                    if (!v_requested) tc::tma_load_2d(tile_d + k * 16384, &a.vb, xfull, k * 64, t * 128);
                }
            }
            v_requested = false;
            if (ok) ok = tc::mbar_wait(xfull, (uint32_t)tcount & 1u, tc::kWaitBudget);
            ++tcount;
            if (ok) ok = ss.after_write(aready);
            for (int q = 0; q < nq; ++q, ++qg) {
                if (ok) ok = tc::mbar_wait(accf, (uint32_t)qg & 1u, tc::kWaitBudget);
                tc::tc_fence_after();
                if (ok) ok = ss.before_write();
                if (q == L + 1 && t + nctas < a.ntiles) {
                    // the last reader of tile_d was the dual contraction of
                    // layer L and its stores have drained (before_write)
                    if (ss.st_thread) {
                        tc::mbar_expect_tx_only(xfull, (uint32_t)nkx * 16384u);
                        for (int k = 0; k < nkx; ++k)
                            tc::tma_load_2d(tile_d + k * 16384, &a.vb, xfull, k * 64, (t + nctas) * 128);
                    }
                    v_requested = true;
                }
                if (q <= L) {
                    // layer l forward and tangent:
                    //   a = acc + b (+ t W_in[:,0]),  h_l = [h_{l-1}] + act(a)
                    //   h'_l = [h'_{l-1}] + act'(a) a',  S_l = act''(a) a' g_l
                    // at the top (l = L) also abar_L = act'(a_L) alpha w_o + S_L and hbar_L = alpha w_o
                    const int l = q;
                    const float* bias = ptab + (size_t)l * a.w;
                    const float* bt = ptab + (size_t)(L + 2 + l) * a.w;  // NAIS: B_l[:, 0]
                    const bool blk_nais = NAIS && l >= 1;
                    const uint32_t* gin = gtile + (size_t)l * a.G_words;
                    auto loadt = [&](int ch, uint32_t (&r)[16]) {
                        tc::tmem_ld8(tacc + (uint32_t)(ch * 8), *reinterpret_cast<uint32_t(*)[8]>(r));
                        tc::tmem_ld8(tsec + (uint32_t)(ch * 8), *reinterpret_cast<uint32_t(*)[8]>(r + 8));
                    };
                    auto body = [&](int ch, const uint32_t (&gq)[4], const uint32_t (&rt)[16]) {
                        const int c0 = ch * 8;
                        float g[8], bv[8], hp[8], hdp[8];
                        ld_f8(bias + c0, bv);
                        if (l < L) unpack8(gq, g);
                        else ld_f8(wo + c0, g);
                        if (RES && l >= 1) {
                            ld_tile8(tile_h, row, c0, hp);
                            ld_tile8(tile_d, row, c0, hdp);
                        }
                        if (l == 0 || blk_nais) {
                            float w0[8];
                            ld_f8((l == 0 ? win0 : bt) + c0, w0);
#pragma unroll
                            for (int j = 0; j < 8; ++j) bv[j] = fmaf(tval, w0[j], bv[j]);
                        }
                        float h[8], hd[8], d1[8], S[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float av = __uint_as_float(rt[j]) + bv[j];
                            Act3 f = act3_sfu<ACT>(av);
                            if (blk_nais) {
                                f.f *= a.hs; f.d1 *= a.hs; f.d2 *= a.hs;
                            }
                            const float ad = __uint_as_float(rt[8 + j]);
                            h[j] = ((RES && l >= 1) ? hp[j] : 0.f) + f.f;
                            hd[j] = ((RES && l >= 1) ? hdp[j] : 0.f) + f.d1 * ad;
                            S[j] = f.d2 * ad * g[j];
                            d1[j] = f.d1;
                        }
                        st_tile8(tile_d, row, c0, hd);
                        if (l < L) {
                            st_tile8(tile_h, row, c0, h);
                            st_pm8h(scr_d1 + (size_t)l * blk, row, c0, d1, pol_keep);
                            st_pm8h(scr_S + (size_t)l * blk, row, c0, S, pol_keep);
                        } else {
                            if (valid) st_bf16x8(a.HbL + (size_t)p * a.wp + c0, h);
                            float ab[8], hb[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                hb[j] = alpha_p * g[j];  // g = w_o at the top
                                ab[j] = d1[j] * hb[j] + S[j];
                            }
                            st_tile8(tile_h, row, c0, ab);
                            if (RES) tmem_st_f8(tsec + (uint32_t)c0, hb);
                        }
                    };
                    // each finished 64-column slab leaves by TMA while the
                    // epilogue goes on with the next one
                    auto slab = [&](int k) {
                        tc::fence_async_shared();
                        tc::named_bar(1, NE);
                        if (ss.st_thread) {
                            tc::tma_store_3d_hint(&a.hdb, tile_d + k * 16384, k * 64, t * 128, l, pol_stream);
                            if (l < L) tc::tma_store_3d_hint(&a.hb, tile_h + k * 16384, k * 64, t * 128, l, pol_stream);
                            else tc::tma_store_3d_hint(&a.abb, tile_h + k * 16384, k * 64, t * 128, L, pol_stream);
                            tc::tma_store_commit();
                        }
                    };
                    if (l < L)
                        chunk_loop_t<4, kSlabIters>(eg, NG, nch, nkw,
                                                    [&](int ch, uint32_t (&u)[4]) { ld_pm8h(gin, row, ch * 8, u, pol_stream); },
                                                    loadt, body, slab);
                    else
                        chunk_loop_t<4, kSlabIters>(eg, NG, nch, nkw,
                                                    [&](int, uint32_t (&u)[4]) { u[0] = u[1] = u[2] = u[3] = 0; },
                                                    loadt, body, slab);
                    if (q < nq - 1) ss.handoff(aready);
                } else {
                    // adjoint through layer l: hbar_{l-1} = [hbar_l] + W_l^T abar_l,
                    // abar_{l-1} = act'(a_{l-1}) hbar_{l-1} + S_{l-1}
                    const int l = L - (q - (L + 1));
                    const uint32_t* d1src = scr_d1 + (size_t)(l - 1) * blk;
                    const uint32_t* Ssrc = scr_S + (size_t)(l - 1) * blk;
                    auto ld_adj = [&](int ch, uint32_t (&u)[8]) {
                        uint32_t* uu = u;
                        ld_pm8_raw(d1src, row, ch * 8, *reinterpret_cast<uint32_t(*)[4]>(uu));
                        ld_pm8_raw(Ssrc, row, ch * 8, *reinterpret_cast<uint32_t(*)[4]>(uu + 4));
                    };
                    // ResNet: the contraction added W_l^T abar_l to hbar_l in
                    // place (columns 256..), so the accumulator is hbar_{l-1}
                    const uint32_t thb = RES ? tsec : tacc;
                    auto ldt_adj = [&](int ch, uint32_t (&r)[16]) {
                        tc::tmem_ld8(thb + (uint32_t)(ch * 8), *reinterpret_cast<uint32_t(*)[8]>(r));
                    };
                    auto body_adj = [&](int ch, const uint32_t (&u)[8], const uint32_t (&rt)[16]) {
                        const int c0 = ch * 8;
                        float d1[8], S[8], ab[8];
                        unpack8(*reinterpret_cast<const uint32_t(*)[4]>(u), d1);
                        unpack8(*reinterpret_cast<const uint32_t(*)[4]>(u + 4), S);
#pragma unroll
                        for (int j = 0; j < 8; ++j) ab[j] = d1[j] * __uint_as_float(rt[j]) + S[j];
                        st_tile8(tile_h, row, c0, ab);
                    };
                    auto slab = [&](int k) {
                        tc::fence_async_shared();
                        tc::named_bar(1, NE);
                        if (ss.st_thread) {
                            tc::tma_store_3d_hint(&a.abb, tile_h + k * 16384, k * 64, t * 128, l - 1, pol_stream);
                            tc::tma_store_commit();
                        }
                    };
                    chunk_loop_t<8, kSlabIters>(eg, NG, nch, nkw, ld_adj, ldt_adj, body_adj, slab);
                    if (q < nq - 1) ss.handoff(aready);
                }
                ok = tc::named_bar_and(1, NE, ok);
                if (!ok) break;
            }
        }
        if (ss.st_thread) tc::tma_store_wait_all<0>();
        if (!ok) {
            if (a.err) atomicExch(a.err, 2);
            *abort_flag = 1;
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

template <int ACT, bool RES, bool NAIS>
__global__ void __launch_bounds__(bwd_threads(), 1) k_fused_bwd(const __grid_constant__ BwdArgs a) {
    bwd_body<ACT, RES, NAIS>(a, (int)blockIdx.x, (int)gridDim.x);
}

// The backward kernels of a group in one launch (as k_fused_fwdz_group).
template <int ACT, bool RES, bool NAIS>
__global__ void __launch_bounds__(bwd_threads(), 1)
    k_fused_bwd_group(const BwdArgs* __restrict__ all, const int* __restrict__ cta_begin, int n) {
    int i = 0;
    while (i + 1 < n && (int)blockIdx.x >= cta_begin[i + 1]) ++i;
    bwd_body<ACT, RES, NAIS>(all[i], (int)blockIdx.x - cta_begin[i], cta_begin[i + 1] - cta_begin[i]);
}

// ---------------------------------------------------------------- host launchers

static size_t fwdz_smem_bytes(int L, int w, int nais) {
    return 1024 + kFTileBytes + (size_t)kFwdStages * kFStageBytes + (size_t)param_rows(L, nais) * w * 4 + 256 +
           (size_t)kFwdGroups * 128 * 4 + 64;
}
static size_t bwd_smem_bytes(int L, int w, int nais) {
    return 1024 + 2 * kFTileBytes + (size_t)kBwdStages * kFStageBytes + (size_t)param_rows(L, nais) * w * 4 + 128;
}

// `launch_regs` > 0: the kernel moves registers between warpgroups, which
// needs exactly that many registers per thread at launch; any other count is
// refused here rather than launched.
template <class K, class A>
static cudaError_t launch_fused(K kernel, const A& args, int grid, int threads, size_t smem, cudaStream_t st,
                                int launch_regs = 0) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (launch_regs > 0) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, kernel);
        if (e != cudaSuccess) return e;
        if (fa.numRegs != launch_regs || fa.maxThreadsPerBlock < threads) return cudaErrorInvalidConfiguration;
    }
    kernel<<<grid, threads, smem, st>>>(args);
    return cudaGetLastError();
}

static ParamOffsets param_offsets(const fbsde_ctx* c) {
    ParamOffsets o;
    std::memset(&o, 0, sizeof(o));
    o.bin = c->pl.bin; o.Win = c->pl.Win; o.wo = c->pl.wo; o.bo = c->pl.bo;
    o.nais = c->akind == FBSDE_NAIS ? 1 : 0;
    for (int l = 1; l <= c->L; ++l) {
        o.b[l] = c->pl.b[l];
        if (o.nais) o.B[l] = c->pl.B[l];
    }
    return o;
}

// Wait budget of a launch under the test hook: its first wait (on a barrier
// nothing completes) gives up after about 10 us.
constexpr long long kGateBudget = 20000LL;

// The pipelined kernels serve FC and ResNet networks in BF16 (not NAIS-Net,
// not the FP8 form).
static bool pipelined(const fbsde_ctx* c) { return c->akind != FBSDE_NAIS && !c->bf->f8; }

// Arguments of one instance's forward kernel.
static void fwd_args(fbsde_ctx* c, const float* theta, bool for_grad, FwdZArgs& a) {
    Bf16Work* b = c->bf;
    std::memset(&a, 0, sizeof(a));
    a.wf[0] = b->mWinx;
    a.wr[0] = b->mWinxT;
    for (int l = 1; l <= c->L; ++l) {
        a.wf[l] = b->mW[l];
        a.wr[l] = b->mWT[l];
    }
    a.eb = b->sEb;
    a.xin = b->mXb;
    a.X = c->X; a.theta = theta; a.Y = c->Y; a.Z = c->Z;
    a.G = (uint32_t*)b->G; a.G_words = b->G_stride / 2; a.scratch = (uint32_t*)b->scratch;
    a.for_grad = for_grad ? 1 : 0;
    a.off = param_offsets(c);
    a.P = (int)c->P(); a.M = c->M; a.D = c->D; a.Dp = b->Dp; a.Dn = b->Dn; a.w = c->w; a.wp = b->wp;
    a.L = c->L; a.ntiles = (a.P + 127) / 128; a.dt = (float)(c->T / c->N); a.err = b->err;
    a.f8 = b->f8 ? 1 : 0;
    if (b->f8) {
        for (int l = 1; l <= c->L; ++l) a.wf8[l] = b->mW8[l];
        a.f8inv = b->f8inv;
    }
    const bool nais = c->akind == FBSDE_NAIS;
    if (nais) {
        for (int l = 1; l <= c->L; ++l) a.wbx[l] = b->mBx[l];
        for (int l = 1; l <= c->L; ++l) a.wbxT[l] = b->mBxT[l];
        a.hs = (float)c->h;
    }
    a.wait_budget = b->gate_fwd ? kGateBudget : tc::kWaitBudget;
    a.gate = b->gate_fwd;
}

fbsde_status fused_forward(fbsde_ctx* c, const float* theta, bool for_grad) {
    Bf16Work* b = c->bf;
    FwdZArgs a;
    fwd_args(c, theta, for_grad, a);
    const bool nais = c->akind == FBSDE_NAIS;
    const int cap = c->grid_cap > 0 && c->grid_cap < b->grid ? c->grid_cap : b->grid;
    const int grid = a.ntiles < cap ? a.ntiles : cap;
    const size_t smem = fwdz_smem_bytes(c->L, c->w, nais ? 1 : 0);
    const int FT = fused_threads(kFwdGroups);
    const bool res = c->akind == FBSDE_RESNET;
    const int tok = prof_begin(c, PROF_POINTS);
    cudaError_t e;
    if (pipelined(c)) {
        e = launch_fwd_pipe(a, c->act == FBSDE_TANH, res, grid, c->stream);
    } else if (nais) {
        e = c->act == FBSDE_TANH ? launch_fused(k_fused_fwdz<FBSDE_TANH, true, false, true>, a, grid, FT, smem, c->stream)
                                 : launch_fused(k_fused_fwdz<FBSDE_SIN, true, false, true>, a, grid, FT, smem, c->stream);
    } else if (b->f8) {
        if (c->act == FBSDE_TANH)
            e = res ? launch_fused(k_fused_fwdz<FBSDE_TANH, true, true, false>, a, grid, FT, smem, c->stream)
                    : launch_fused(k_fused_fwdz<FBSDE_TANH, false, true, false>, a, grid, FT, smem, c->stream);
        else
            e = res ? launch_fused(k_fused_fwdz<FBSDE_SIN, true, true, false>, a, grid, FT, smem, c->stream)
                    : launch_fused(k_fused_fwdz<FBSDE_SIN, false, true, false>, a, grid, FT, smem, c->stream);
    } else {
        e = cudaErrorInvalidConfiguration;  // FC / ResNet in BF16 always take the pipelined kernel
    }
    // algorithmic flops: lift + L layers forward (NAIS-Net: + B_l x), L reverse
    // layers and the Z contraction
    const double P = a.P, w = a.w, D = a.D;
    prof_end(c, PROF_POINTS, tok, 2.0 * P * w * (2.0 * D + 2.0 * c->L * w + (nais ? c->L * D : 0.0)));
    b->gate_fwd = 0;
    if (e != cudaSuccess) return set_err(c, FBSDE_ERR_CUDA, std::string("fused forward: ") + cudaGetErrorString(e));
    ++c->n_launch;
    return FBSDE_OK;
}

// Per-column parameters of the backward (b_0..b_L, w_o, W_in[:,0]) gathered
// into one aligned table.
__global__ void k_stage_pvec(const float* __restrict__ th, ParamOffsets o, int L, int w, int K0,
                             float* __restrict__ pvec) {
    const int n = param_rows(L, o.nais) * w;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        pvec[i] = param_value(th, o, L, i / w, i % w, K0);
}

// Arguments of one instance's backward kernel.
static void bwd_args(fbsde_ctx* c, const float* theta, BwdArgs& a) {
    Bf16Work* b = c->bf;
    std::memset(&a, 0, sizeof(a));
    a.wf[0] = b->mWinx;
    for (int l = 1; l <= c->L; ++l) {
        a.wf[l] = b->mW[l];
        a.wr[l] = b->mWT[l];
    }
    a.hb = b->sHb; a.hdb = b->sHDb; a.abb = b->sABb; a.xb = b->mXb; a.vb = b->mVb;
    a.X = c->X; a.V = c->V; a.alpha = c->alpha; a.theta = theta;
    a.G = (const uint32_t*)b->G; a.G_words = b->G_stride / 2;
    a.HbL = b->Hb[c->L];
    a.wopart = b->wopart;
    a.scratch = (uint32_t*)b->scratch;
    a.off = param_offsets(c);
    a.P = (int)c->P(); a.M = c->M; a.D = c->D; a.Dp = b->Dp; a.w = c->w; a.wp = b->wp;
    a.L = c->L; a.ntiles = (a.P + 127) / 128; a.dt = (float)(c->T / c->N); a.err = b->err;
    a.pvec = b->pvec;
    const bool nais = c->akind == FBSDE_NAIS;
    a.res = c->akind != FBSDE_FC ? 1 : 0;
    if (nais) {
        for (int l = 1; l <= c->L; ++l) a.wbx[l] = b->mBx[l];
        a.hs = (float)c->h;
    }
    a.wait_budget = b->gate_bwd ? kGateBudget : tc::kWaitBudget;
    a.gate = b->gate_bwd;
}

// The per-column parameter table of the backward, from Theta (one small launch).
static fbsde_status stage_pvec(fbsde_ctx* c, const float* theta, cudaStream_t st) {
    const ParamOffsets off = param_offsets(c);
    k_stage_pvec<<<4, 256, 0, st>>>(theta, off, c->L, c->w, c->D + 1, c->bf->pvec);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return set_err(c, FBSDE_ERR_CUDA, std::string("parameter table: ") + cudaGetErrorString(le));
    ++c->n_launch;
    return FBSDE_OK;
}

fbsde_status fused_backward(fbsde_ctx* c, const float* theta) {
    Bf16Work* b = c->bf;
    BwdArgs a;
    bwd_args(c, theta, a);
    const bool nais = c->akind == FBSDE_NAIS;
    FBSDE_TRY(stage_pvec(c, theta, c->stream));
    const int cap = c->grid_cap > 0 && c->grid_cap < b->grid ? c->grid_cap : b->grid;
    const int grid = a.ntiles < cap ? a.ntiles : cap;
    const size_t smem = bwd_smem_bytes(c->L, c->w, nais ? 1 : 0);
    const int FT = bwd_threads(), R = kBwdRegsLaunch;
    const bool res = c->akind == FBSDE_RESNET;
    const int tok = prof_begin(c, PROF_POINTS);
    cudaError_t e;
    if (pipelined(c))
        e = launch_bwd_pipe(a, c->act == FBSDE_TANH, res, grid, c->stream);
    else if (nais)
        e = c->act == FBSDE_TANH ? launch_fused(k_fused_bwd<FBSDE_TANH, true, true>, a, grid, FT, smem, c->stream, R)
                                 : launch_fused(k_fused_bwd<FBSDE_SIN, true, true>, a, grid, FT, smem, c->stream, R);
    else if (c->act == FBSDE_TANH)
        e = res ? launch_fused(k_fused_bwd<FBSDE_TANH, true, false>, a, grid, FT, smem, c->stream, R)
                : launch_fused(k_fused_bwd<FBSDE_TANH, false, false>, a, grid, FT, smem, c->stream, R);
    else
        e = res ? launch_fused(k_fused_bwd<FBSDE_SIN, true, false>, a, grid, FT, smem, c->stream, R)
                : launch_fused(k_fused_bwd<FBSDE_SIN, false, false>, a, grid, FT, smem, c->stream, R);
    // algorithmic flops: tangent (lift + L layers, NAIS-Net: + B_l v) and
    // adjoint (L layers); the forward recomputation is overhead and not counted
    const double P = a.P, w = a.w, D = a.D;
    prof_end(c, PROF_POINTS, tok, 2.0 * P * w * (D + 2.0 * c->L * w + (nais ? c->L * D : 0.0)));
    b->gate_bwd = 0;
    if (e != cudaSuccess) return set_err(c, FBSDE_ERR_CUDA, std::string("fused backward: ") + cudaGetErrorString(e));
    ++c->n_launch;
    return FBSDE_OK;
}

// Test hook: arm the gate of the next pipelined forward and backward launch.
fbsde_status arm_timeout_test(fbsde_ctx* c) {
    if (c->prec == FBSDE_FP32 || !c->bf || !c->bf->fused || !pipelined(c))
        return set_err(c, FBSDE_ERR_UNSUPPORTED, "the timeout test hook serves the pipelined FC / ResNet BF16 kernels");
    c->bf->gate_fwd = 1;
    c->bf->gate_bwd = 1;
    return FBSDE_OK;
}

// ---------------------------------------------------------------- grouped launches

// Kernel variant of an instance (activation x network kind); instances of one
// grouped launch share it.
int fused_variant(const fbsde_ctx* c) {
    return (c->act == FBSDE_TANH ? 1 : 0) | (c->akind == FBSDE_RESNET ? 2 : c->akind == FBSDE_NAIS ? 4 : 0);
}

bool fused_groupable(const fbsde_ctx* c) {
    return c->prec != FBSDE_FP32 && c->bf && c->bf->fused && !c->bf->f8;
}

fbsde_status fused_group_alloc(FusedGroupBuf* g, int n) {
    fused_group_free(g);
    g->bytes = (size_t)n * (sizeof(FwdZArgs) + sizeof(BwdArgs)) + (size_t)(n + 1) * sizeof(int);
    g->host = std::malloc(g->bytes);
    g->last = std::malloc(g->bytes);
    if (!g->host || !g->last || cudaMalloc(&g->dev, g->bytes) != cudaSuccess) {
        fused_group_free(g);
        return FBSDE_ERR_OOM;
    }
    g->cap = n;
    g->valid = false;
    return FBSDE_OK;
}

void fused_group_free(FusedGroupBuf* g) {
    std::free(g->host);
    std::free(g->last);
    if (g->dev) cudaFree(g->dev);
    g->host = g->last = nullptr;
    g->dev = nullptr;
    g->cap = 0;
    g->valid = false;
}

// Layout of the argument block: n forward arguments, n backward arguments
// (both 64-byte aligned: they hold tensor maps), then the n + 1 CTA offsets.
static FwdZArgs* fwd_block(void* base) { return reinterpret_cast<FwdZArgs*>(base); }
static BwdArgs* bwd_block(void* base, int cap) {
    return reinterpret_cast<BwdArgs*>(static_cast<char*>(base) + (size_t)cap * sizeof(FwdZArgs));
}
static int* begin_block(void* base, int cap) {
    return reinterpret_cast<int*>(static_cast<char*>(base) + (size_t)cap * (sizeof(FwdZArgs) + sizeof(BwdArgs)));
}

fbsde_status fused_group_prepare(fbsde_ctx* const* c, const float* const* theta, int n, FusedGroupBuf* g,
                                 cudaStream_t st) {
    if (n < 1 || n > g->cap) return FBSDE_ERR_INVALID;
    std::memset(g->host, 0, g->bytes);
    FwdZArgs* fa = fwd_block(g->host);
    BwdArgs* ba = bwd_block(g->host, g->cap);
    int* beg = begin_block(g->host, g->cap);
    beg[0] = 0;
    g->smem_fwd = g->smem_bwd = 0;
    for (int i = 0; i < n; ++i) {
        fwd_args(c[i], theta[i], true, fa[i]);
        bwd_args(c[i], theta[i], ba[i]);
        const int cap = c[i]->grid_cap > 0 && c[i]->grid_cap < c[i]->bf->grid ? c[i]->grid_cap : c[i]->bf->grid;
        beg[i + 1] = beg[i] + std::max(1, std::min(cap, fa[i].ntiles));
        const int nais = c[i]->akind == FBSDE_NAIS ? 1 : 0;
        g->smem_fwd = std::max(g->smem_fwd, pipelined(c[i]) ? fwd_pipe_smem_bytes(c[i]->L, c[i]->w)
                                                             : fwdz_smem_bytes(c[i]->L, c[i]->w, nais));
        g->smem_bwd = std::max(g->smem_bwd, pipelined(c[i]) ? bwd_pipe_smem_bytes(c[i]->L, c[i]->w)
                                                             : bwd_smem_bytes(c[i]->L, c[i]->w, nais));
    }
    for (int i = 0; i < n; ++i) c[i]->bf->gate_fwd = c[i]->bf->gate_bwd = 0;  // the test hook serves solo launches
    g->n = n;
    g->grid = beg[n];
    if (g->valid && std::memcmp(g->host, g->last, g->bytes) == 0) return FBSDE_OK;
    // new arguments: the device copy must not change under a launch in
    // flight, and a graph being captured must find it already in place
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FBSDE_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return FBSDE_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpy(g->dev, g->host, g->bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return FBSDE_ERR_CUDA;
    std::memcpy(g->last, g->host, g->bytes);
    g->valid = true;
    return FBSDE_OK;
}

template <class K, class A>
static cudaError_t launch_group(K kernel, const A* all, const int* beg, int n, int grid, int threads, size_t smem,
                                cudaStream_t st, int launch_regs) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (launch_regs > 0) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, kernel);
        if (e != cudaSuccess) return e;
        if (fa.numRegs != launch_regs || fa.maxThreadsPerBlock < threads) return cudaErrorInvalidConfiguration;
    }
    kernel<<<grid, threads, smem, st>>>(all, beg, n);
    return cudaGetLastError();
}

fbsde_status fused_group_forward(fbsde_ctx* const* c, int n, FusedGroupBuf* g, cudaStream_t st) {
    if (n != g->n || !g->valid) return FBSDE_ERR_INVALID;
    const FwdZArgs* all = fwd_block(g->dev);
    const int* beg = begin_block(g->dev, g->cap);
    const int FT = fused_threads(kFwdGroups);
    cudaError_t e;
    const int var = fused_variant(c[0]);
    switch (var) {
        case 0: case 1: case 2: case 3:
            e = launch_fwd_pipe_group(all, beg, n, var & 1, (var & 2) ? 1 : 0, g->grid, g->smem_fwd, st);
            break;
        case 4: e = launch_group(k_fused_fwdz_group<FBSDE_SIN, true, false, true>, all, beg, n, g->grid, FT, g->smem_fwd, st, 0); break;
        default: e = launch_group(k_fused_fwdz_group<FBSDE_TANH, true, false, true>, all, beg, n, g->grid, FT, g->smem_fwd, st, 0); break;
    }
    if (e != cudaSuccess) return set_err(c[0], FBSDE_ERR_CUDA, std::string("grouped fused forward: ") + cudaGetErrorString(e));
    ++c[0]->n_launch;
    return FBSDE_OK;
}

fbsde_status fused_group_stage_pvec(fbsde_ctx* c, const float* theta, cudaStream_t st) {
    return stage_pvec(c, theta, st);
}

fbsde_status fused_group_backward(fbsde_ctx* const* c, int n, FusedGroupBuf* g, cudaStream_t st) {
    if (n != g->n || !g->valid) return FBSDE_ERR_INVALID;
    const BwdArgs* all = bwd_block(g->dev, g->cap);
    const int* beg = begin_block(g->dev, g->cap);
    const int FT = bwd_threads(), R = kBwdRegsLaunch;
    cudaError_t e;
    const int var = fused_variant(c[0]);
    switch (var) {
        case 0: case 1: case 2: case 3:
            e = launch_bwd_pipe_group(all, beg, n, var & 1, (var & 2) ? 1 : 0, g->grid, g->smem_bwd, st);
            break;
        case 4: e = launch_group(k_fused_bwd_group<FBSDE_SIN, true, true>, all, beg, n, g->grid, FT, g->smem_bwd, st, R); break;
        default: e = launch_group(k_fused_bwd_group<FBSDE_TANH, true, true>, all, beg, n, g->grid, FT, g->smem_bwd, st, R); break;
    }
    if (e != cudaSuccess) return set_err(c[0], FBSDE_ERR_CUDA, std::string("grouped fused backward: ") + cudaGetErrorString(e));
    ++c[0]->n_launch;
    return FBSDE_OK;
}

}  // namespace fbsde
