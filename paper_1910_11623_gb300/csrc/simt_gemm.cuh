// FP32 CUDA-core GEMM with a fused per-element epilogue (the FP32 form).
//
// C[m][n] = sum_{pairs q} sum_k A_q(m, k) B_q(k, n), for up to kMaxPairs
// operand pairs that share one accumulator (NAIS adds B_l (t, x) to A_l h,
// Z sums W_in^T e_0 and every B_l^T e_l).  Layouts are compile-time:
//   A_T = false: A(m, k) = A[m * lda + k]      (activations, row per point)
//   A_T = true : A(m, k) = A[k * lda + m]      (weight gradients: K = points)
//   B_KN = false: B(k, n) = B[n * ldb + k]     (W as stored, [out][in]: h W^T)
//   B_KN = true : B(k, n) = B[k * ldb + n]     (e W: reverse sweeps)
// gridDim.z > 1 splits K: split z covers [z * kchunk, (z+1) * kchunk) of every
// pair and the epilogue receives z to write a partial sum.
//
// Tile 128 x 128 x 8, 256 threads, 8 x 8 outputs per thread held in two 4 x 4
// quadrants so the shared-memory reads are float4 broadcasts.
#pragma once
#include <cuda_runtime.h>

namespace fbsde {

constexpr int kMaxPairs = 18;

struct GemmPair {
    const float* A;
    const float* B;
    int K, lda, ldb;
};

struct GemmArgs {
    GemmPair pair[kMaxPairs];
    int npairs;
    int Mrows, Ncols;
    int kchunk;  // K range per split (gridDim.z splits)
};

template <bool A_T, bool B_KN, class Epi>
__global__ void __launch_bounds__(256) simt_gemm_kernel(const GemmArgs args, const Epi epi) {
    constexpr int BM = 128, BN = 128, BK = 8;
    __shared__ __align__(16) float As[BK][BM];
    __shared__ __align__(16) float Bs[BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int z = blockIdx.z;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int q = 0; q < args.npairs; ++q) {
        const GemmPair pr = args.pair[q];
        const int kb = z * args.kchunk;
        const int ke = min(pr.K, kb + args.kchunk);
        for (int k0 = kb; k0 < ke; k0 += BK) {
            // global -> registers (4 A and 4 B elements per thread)
            float ra[4], rb[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int mm, kk;
                if (A_T) { int e = tid + 256 * j; mm = e & (BM - 1); kk = e >> 7; }
                else     { int e = tid * 4 + j;   kk = e & (BK - 1); mm = e >> 3; }
                const int gm = m0 + mm, gk = k0 + kk;
                float v = 0.f;
                if (gm < args.Mrows && gk < ke)
                    v = A_T ? pr.A[(size_t)gk * pr.lda + gm] : pr.A[(size_t)gm * pr.lda + gk];
                ra[j] = v;
                int nn, kb2;
                if (B_KN) { int e = tid + 256 * j; nn = e & (BN - 1); kb2 = e >> 7; }
                else      { int e = tid * 4 + j;   kb2 = e & (BK - 1); nn = e >> 3; }
                const int gn = n0 + nn, gk2 = k0 + kb2;
                float u = 0.f;
                if (gn < args.Ncols && gk2 < ke)
                    u = B_KN ? pr.B[(size_t)gk2 * pr.ldb + gn] : pr.B[(size_t)gn * pr.ldb + gk2];
                rb[j] = u;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (A_T) { int e = tid + 256 * j; As[e >> 7][e & (BM - 1)] = ra[j]; }
                else     { int e = tid * 4 + j;   As[e & (BK - 1)][e >> 3] = ra[j]; }
                if (B_KN) { int e = tid + 256 * j; Bs[e >> 7][e & (BN - 1)] = rb[j]; }
                else      { int e = tid * 4 + j;   Bs[e & (BK - 1)][e >> 3] = rb[j]; }
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
                const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
        }
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= args.Mrows) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (col < args.Ncols) epi(row, col, acc[i][j], z);
        }
    }
}

template <bool A_T, bool B_KN, class Epi>
inline cudaError_t simt_gemm(const GemmArgs& args, int splits, const Epi& epi, cudaStream_t st) {
    dim3 grid((args.Mrows + 127) / 128, (args.Ncols + 127) / 128, splits);
    simt_gemm_kernel<A_T, B_KN, Epi><<<grid, 256, 0, st>>>(args, epi);
    return cudaGetLastError();
}

}  // namespace fbsde
