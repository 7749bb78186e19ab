// Workspace of the BF16 tensor-core form, shared by the layered sweeps
// (tc_path.cu) and the per-tile fused kernels (fused.cu).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace fbsde {

typedef __nv_bfloat16 bf16;

// Row-major BF16 matrix [outer x inner] with row stride ld (elements), box
// {64, box_outer}, 128-byte swizzle, zero fill outside the matrix.
bool map2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_outer);

// act and its first two derivatives with fast SFU math (BF16 form).  tanh
// from e = exp(-2|a|): tanh = sign(a) (1 - e) / (1 + e), tanh' = 4 e / (1 + e)^2
// (no cancellation where tanh saturates), tanh'' = -2 tanh tanh'.
__device__ __forceinline__ Act3 act3_fast(int act, float a) {
    Act3 r;
    if (act == FBSDE_SIN) {
        float s, c;
        __sincosf(a, &s, &c);
        r.f = s; r.d1 = c; r.d2 = -s;
    } else {
        const float e = __expf(-2.f * fabsf(a));
        const float q = __fdividef(1.f, 1.f + e);
        const float t = copysignf((1.f - e) * q, a);
        r.f = t; r.d1 = 4.f * e * q * q; r.d2 = -2.f * t * r.d1;
    }
    return r;
}

// f and act' (and act'') with one SFU operation per element, for the fused
// kernels: tanh.approx (hardware tanh, relative error about 2^-11) with
// act' = 1 - f^2 and act'' = -2 f act'; sin.approx / cos.approx for sin.
__device__ __forceinline__ float tanh_sfu(float a) {
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
template <int ACT>
__device__ __forceinline__ Act3 act3_sfu(float a) {
    Act3 r;
    if (ACT == FBSDE_SIN) {
        r.f = __sinf(a); r.d1 = __cosf(a); r.d2 = -r.f;
    } else {
        r.f = tanh_sfu(a); r.d1 = fmaf(-r.f, r.f, 1.f); r.d2 = -2.f * r.f * r.d1;
    }
    return r;
}

constexpr int kFusedMaxDepth = 8;  // depth served by the per-tile fused kernels

struct Bf16Work {
    int Dp, Dn, wp;  // D padded to 64 (operand rows), D padded to 16 (MMA N), w padded to 64
    int sms = 1;     // multiprocessors of the device
    void* mem = nullptr;
    bf16 *Xb, *Vb;
    bf16 *Hb[kMaxDepth + 1], *Eb[kMaxDepth + 1], *HDb[kMaxDepth + 1], *ABb[kMaxDepth + 1];
    // layered path: FP32 residual streams h, g, h', hbar; pre-activations a
    // and the tangent terms S in BF16 (they are not accumulated)
    float *Hf[kMaxDepth + 1], *Gf[kMaxDepth + 1], *HDf[kMaxDepth + 1], *HBf[kMaxDepth + 1];
    bf16 *Af[kMaxDepth + 1], *Sf[kMaxDepth + 1];
    bf16 *Winx, *WinxT, *W[kMaxDepth + 1], *WT[kMaxDepth + 1], *Bx[kMaxDepth + 1], *BxT[kMaxDepth + 1];
    float* colpart;
    int* err;
    // NT operand maps (box rows 128)
    CUtensorMap mXb, mVb, mHb[kMaxDepth + 1], mEb[kMaxDepth + 1], mHDb[kMaxDepth + 1], mABb[kMaxDepth + 1];
    // weight maps (box rows = N of the contraction)
    CUtensorMap mWinx, mWinxT, mW[kMaxDepth + 1], mWT[kMaxDepth + 1], mBx[kMaxDepth + 1], mBxT[kMaxDepth + 1];
    // MN-major maps for the weight gradients (box {64, 64})
    CUtensorMap tX, tV, tH[kMaxDepth + 1], tE[kMaxDepth + 1], tHD[kMaxDepth + 1], tAB[kMaxDepth + 1];
    // per-tile fused kernels (FC / ResNet / NAIS-Net, depth <= kFusedMaxDepth, D <= 256)
    bool fused = false;
    CUtensorMap sHb, sHDb, sABb, sEb;  // layer stacks of the operands, box {64, 128, 1} (TMA stores)
    int grid = 0;          // persistent CTAs
    size_t OP_stride = 0;  // elements between consecutive layers of Hb, Eb, HDb, ABb
    bf16* G = nullptr;     // g_l, l < L, per 128-row tile column-pair-major (written by the fused forward)
    size_t G_stride = 0;   // elements between consecutive g_l
    bf16* scratch = nullptr;  // per-CTA activation-derivative scratch
    float* pvec = nullptr;    // [(2L+3) x w] per-column parameters of the fused backward
    // FP8 hidden layers (prec FBSDE_FP8_HIDDEN): E4M3 copies of W_l (l >= 1),
    // [w x wp8] bytes, their maps (box {128, w}) and per-layer inverse scales
    bool f8 = false;
    int wp8 = 0;
    uint8_t* W8[kMaxDepth + 1] = {};
    CUtensorMap mW8[kMaxDepth + 1];
    float* f8inv = nullptr;  // [L + 1]: 1 / (scale of h_{l-1} x scale of W_l)
    // Test hook (fbsde_test_timeout_once): the next launch of each fused kernel
    // gives up at its first wait, before it issues any copy or contraction.
    int gate_fwd = 0, gate_bwd = 0;
    // pipelined backward: per tile and 32-row group, the column sums of
    // alpha h_L + h'_L (the read-out gradient), summed in order afterwards
    float* wopart = nullptr;
};

// Scale of the E4M3 copy of h_l (the operand of layer l + 1): the largest
// power of two s with s x bound(h_l) <= 448, the largest finite E4M3 value;
// bound = l + 1 for a ResNet (h_0 = act(.) in [-1, 1], each block adds at
// most 1), 1 for an FC network (|act| <= 1 for tanh and sin).
__host__ __device__ inline float e4m3_act_scale(int l, bool res) {
    const float bound = res ? (float)(l + 1) : 1.f;
    float s = 1.f;
    while (bound * s * 2.f <= 448.f) s *= 2.f;
    return s;
}


fbsde_status fused_forward(fbsde_ctx* c, const float* theta, bool for_grad);
fbsde_status fused_backward(fbsde_ctx* c, const float* theta);

// One launch of each fused kernel for several instances (a group) that share
// the kernel variant: instance i takes its CTA count from its grid cap (one
// per SM when unset), and its arguments are uploaded to `dev` by
// fused_group_prepare (a blocking copy, only when they changed; while a graph
// is being captured they must already be in place).
struct FusedGroupBuf {
    void* host = nullptr;  // argument block being built
    void* last = nullptr;  // the block the device copy holds
    void* dev = nullptr;
    size_t bytes = 0;
    size_t smem_fwd = 0, smem_bwd = 0;
    int cap = 0, n = 0, grid = 0;
    bool valid = false;
};
int fused_variant(const fbsde_ctx* c);
bool fused_groupable(const fbsde_ctx* c);
fbsde_status fused_group_alloc(FusedGroupBuf* g, int n);
void fused_group_free(FusedGroupBuf* g);
fbsde_status fused_group_prepare(fbsde_ctx* const* c, const float* const* theta, int n, FusedGroupBuf* g,
                                 cudaStream_t st);
fbsde_status fused_group_forward(fbsde_ctx* const* c, int n, FusedGroupBuf* g, cudaStream_t st);
fbsde_status fused_group_stage_pvec(fbsde_ctx* c, const float* theta, cudaStream_t st);
fbsde_status fused_group_backward(fbsde_ctx* const* c, int n, FusedGroupBuf* g, cudaStream_t st);
fbsde_status bf16_wgrad_tail(fbsde_ctx* c, const float* theta, float* grad);

}  // namespace fbsde
