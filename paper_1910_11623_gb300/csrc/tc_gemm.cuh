// Tensor-core contraction with a fused epilogue (BF16 operands, FP32
// accumulation in TMEM), the engine of the BF16 form.
//
//   NT mode: D[m][n] = sum_pairs sum_k A(m, k) B(n, k), A [rows x K] and
//            B [N x K] both K-major (rows of K contiguous): the network sweeps,
//            where m runs over points and B is a weight matrix.
//   TN mode: D[m][n] = sum_pairs sum_k A(k, m) B(k, n), A [K x rows] and
//            B [K x N] both MN-major: the weight gradients, where k runs over
//            points; blockIdx.y splits K into chunks of args.kchunk.
//
// One CTA computes a 128 x Nt tile: Nt = N for N <= 256, else blockIdx.z
// picks 256 of the N columns (weight maps of such widths have boxes of 256
// rows; the last box may run past the matrix and reads zeros).  Warp 0 streams 64-wide K
// slices of A and B into a 4-stage shared-memory ring with TMA (128-byte
// swizzle); warp 1 allocates TMEM and one of its threads issues the
// tcgen05.mma instructions (K = 16 each) and commits stage releases and the
// final accumulator; warps 2-5 (one thread per accumulator row) read the
// accumulator with tcgen05.ld in 16-column slices and call the epilogue.
// In TN mode the epilogue warps, idle during the main loop, can also sum the
// columns of pair 0's A operand over the CTA's K range (a bias gradient is
// the column sum of the same operand whose weight gradient this contracts):
// they read each ring stage after it lands and release it with the MMA.
// Every wait is bounded; a wait that gives up sets *args.err.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include "tc_common.cuh"

namespace fbsde {

constexpr int kTcStages = 4;
// operand pairs one contraction can sum (the NAIS-Net Z contraction takes L + 1)
constexpr int kTcMaxPairs = 17;

struct TcPair {
    CUtensorMap a;  // NT: [rows x K], box {64, 128}; TN: [K x rows], box {64, 64}
    CUtensorMap b;  // NT: [N x K],    box {64, min(N, 256)};   TN: [K x N],    box {64, 64}
    int K;
};

struct TcArgs {
    TcPair pr[kTcMaxPairs];
    int npairs;
    int rows;    // output rows (NT: points; TN: output features)
    int N;       // output columns: multiple of 16, 16..512 (tiles of 256 over blockIdx.z)
    int kchunk;  // TN: K range per blockIdx.y, multiple of 64
    int* err;    // device flag set when a bounded wait gives up
    // TN, optional (NULL: off): cs_part[blockIdx.y * rows + m] = sum over the
    // CTA's K range of A(k, m) of pair 0, and cs_tpart the same weighted by
    // t_k = floor(k / cs_M) * cs_dt (the time of point k)
    float* cs_part;
    float* cs_tpart;
    int cs_M;
    float cs_dt;
};

__host__ __device__ inline uint32_t tc_b_stage_bytes(int N) { return (uint32_t)((N + 63) / 64 * 64) * 128u; }
__host__ __device__ inline uint32_t tc_stage_bytes(int N) { return 16384u + tc_b_stage_bytes(N); }
inline size_t tc_smem_bytes(int N) { return 1024 + (size_t)kTcStages * tc_stage_bytes(N) + 256; }

template <bool TN, class Epi>
__global__ void __launch_bounds__(192, 1) tc_gemm_kernel(const __grid_constant__ TcArgs args, const Epi epi) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int n0 = (int)blockIdx.z * 256;          // first column of this CTA
    const int N = min(256, args.N - n0);           // its columns
    const int Nbox = min(256, args.N);             // NT: weight rows per stage
    const uint32_t stage_bytes = tc_stage_bytes(Nbox);
    uint64_t* full = (uint64_t*)(smem + kTcStages * stage_bytes);
    uint64_t* empty = full + kTcStages;
    uint64_t* accf = empty + kTcStages;
    uint32_t* tmem_slot = (uint32_t*)(accf + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 128;
    const uint32_t ncols = tc::tmem_cols_for(N);
    const int kbeg = TN ? (int)blockIdx.y * args.kchunk : 0;

    // stage release: the MMA's commit, plus one arrival per epilogue warp
    // when they read the stages for the column sums
    const bool colsums = TN && args.cs_part != nullptr && blockIdx.z == 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], colsums ? 5 : 1);
        }
        tc::mbar_init(accf, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, ncols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            for (int q = 0; q < args.npairs; ++q) {
                tc::tma_prefetch_desc(&args.pr[q].a);
                tc::tma_prefetch_desc(&args.pr[q].b);
            }
            int it = 0;
            bool ok = true;
            for (int q = 0; q < args.npairs && ok; ++q) {
                const TcPair& pr = args.pr[q];
                const int kend = TN ? min(pr.K, kbeg + args.kchunk) : pr.K;
                for (int k0 = kbeg; k0 < kend; k0 += 64, ++it) {
                    const int s = it % kTcStages;
                    const uint32_t ph = (uint32_t)(it / kTcStages) & 1u;
                    if (*abort_flag || !tc::mbar_wait(&empty[s], ph ^ 1u, tc::kWaitBudget)) {
                        ok = false;
                        break;
                    }
                    uint8_t* sa = smem + (size_t)s * stage_bytes;
                    uint8_t* sb = sa + 16384;
                    if (!TN) {
                        tc::mbar_expect_tx(&full[s], 16384u + (uint32_t)Nbox * 128u);
                        tc::tma_load_2d(sa, &pr.a, &full[s], k0, m0);
                        tc::tma_load_2d(sb, &pr.b, &full[s], k0, n0);
                    } else {
                        const int na = (args.rows - m0 > 64) ? 2 : 1;
                        const int nb = (N + 63) / 64;
                        tc::mbar_expect_tx(&full[s], (uint32_t)(na + nb) * 8192u);
                        for (int j = 0; j < na; ++j) tc::tma_load_2d(sa + j * 8192, &pr.a, &full[s], m0 + 64 * j, k0);
                        for (int j = 0; j < nb; ++j) tc::tma_load_2d(sb + j * 8192, &pr.b, &full[s], n0 + 64 * j, k0);
                    }
                }
            }
            if (!ok) {
                if (args.err) atomicExch(args.err, 1);
                *abort_flag = 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(128, N, TN ? 1 : 0, TN ? 1 : 0);
            int it = 0;
            bool ok = true;
            for (int q = 0; q < args.npairs && ok; ++q) {
                const TcPair& pr = args.pr[q];
                const int kend = TN ? min(pr.K, kbeg + args.kchunk) : pr.K;
                for (int k0 = kbeg; k0 < kend; k0 += 64, ++it) {
                    const int s = it % kTcStages;
                    const uint32_t ph = (uint32_t)(it / kTcStages) & 1u;
                    if (*abort_flag || !tc::mbar_wait(&full[s], ph, tc::kWaitBudget)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t sa = tc::smem_u32(smem + (size_t)s * stage_bytes);
                    const uint32_t sb = sa + 16384u;
                    const int nsteps = min(4, (kend - k0 + 15) / 16);
                    for (int k = 0; k < nsteps; ++k) {
                        uint64_t ad, bd;
                        if (!TN) {
                            ad = tc::sdesc_sw128(sa + 32u * k, 16u);
                            bd = tc::sdesc_sw128(sb + 32u * k, 16u);
                        } else {
                            ad = tc::sdesc_sw128(sa + 2048u * k, 8192u);
                            bd = tc::sdesc_sw128(sb + 2048u * k, 8192u);
                        }
                        tc::mma_bf16(tmem, ad, bd, idesc, (it > 0 || k > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&empty[s]);
                }
            }
            if (ok) {
                tc::mma_commit(accf);
            } else {
                if (args.err) atomicExch(args.err, 1);
                *abort_flag = 1;
            }
        }
    } else {
        const int lg = warp & 3;  // TMEM lane group of this warp
        const int row = m0 + lg * 32 + lane;
        bool cs_ok = true;
        if (colsums) {
            // feature fm of the tile: box fm / 64 of the stage's A slice, a
            // [64 points x 64 features] block with the 128-byte swizzle
            const int fm = lg * 32 + lane, box = fm >> 6, f = fm & 63;
            const bool mine = row < args.rows;
            float cs = 0.f, cst = 0.f;
            int it = 0;
            for (int q = 0; q < args.npairs && cs_ok; ++q) {
                const int kend = min(args.pr[q].K, kbeg + args.kchunk);
                for (int k0 = kbeg; k0 < kend; k0 += 64, ++it) {
                    const int s = it % kTcStages;
                    const uint32_t ph = (uint32_t)(it / kTcStages) & 1u;
                    if (*abort_flag || !tc::mbar_wait(&full[s], ph, tc::kWaitBudget)) {
                        cs_ok = false;
                        break;
                    }
                    if (q == 0 && mine) {
                        const uint8_t* sa = smem + (size_t)s * stage_bytes + box * 8192;
                        const int nk = min(64, kend - k0);
                        int n = k0 / args.cs_M, r = k0 % args.cs_M;
                        for (int kk = 0; kk < nk; ++kk) {
                            const uint32_t off = (uint32_t)kk * 128u + ((uint32_t)((f >> 3) ^ (kk & 7)) << 4) +
                                                 (uint32_t)(f & 7) * 2u;
                            const float v = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(sa + off));
                            cs += v;
                            cst = fmaf((float)n * args.cs_dt, v, cst);
                            if (++r == args.cs_M) { r = 0; ++n; }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&empty[s]);
                }
            }
            if (cs_ok && mine) {
                args.cs_part[(size_t)blockIdx.y * args.rows + row] = cs;
                if (args.cs_tpart) args.cs_tpart[(size_t)blockIdx.y * args.rows + row] = cst;
            }
        }
        const bool ok = cs_ok && tc::mbar_wait(accf, 0, tc::kWaitBudget);
        if (ok) {
            tc::tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t r[16];
                tc::tmem_ld16(tbase + (uint32_t)c0, r);
                tc::tmem_wait_ld();
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
                if (row < args.rows) epi(row, n0 + c0, v, (int)blockIdx.y);
            }
        } else if (lane == 0) {
            if (args.err) atomicExch(args.err, 1);
            *abort_flag = 1;
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, ncols);
    }
}

template <bool TN, class Epi>
inline cudaError_t tc_gemm(const TcArgs& a, int splits, const Epi& e, cudaStream_t st) {
    static bool configured = false;
    const size_t smem_max = tc_smem_bytes(256);
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(tc_gemm_kernel<TN, Epi>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (err != cudaSuccess) return err;
        configured = true;
    }
    dim3 grid((a.rows + 127) / 128, TN ? splits : 1, (a.N + 255) / 256);
    tc_gemm_kernel<TN, Epi><<<grid, 192, tc_smem_bytes(a.N < 256 ? a.N : 256), st>>>(a, e);
    return cudaGetLastError();
}

}  // namespace fbsde
