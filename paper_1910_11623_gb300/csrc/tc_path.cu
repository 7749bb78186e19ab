// BF16 form of the network sweeps: every contraction runs on the tcgen05
// tensor cores (BF16 operands, FP32 accumulation) with the per-layer
// elementwise work fused into the GEMM epilogue.  The sweeps are the ones of
// the FP32 form (forward, Z-reverse, tangent, adjoint, weight gradients; see
// fp32_path.cu); GEMM operands are stored in BF16, every residual stream,
// pre-activation and reduction stays in FP32.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "internal.cuh"
#include "tc_gemm.cuh"
#include "bf16_work.cuh"

namespace fbsde {

static inline size_t rup(size_t x, size_t m) { return (x + m - 1) / m * m; }
static inline unsigned nblk(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ tensor maps

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Row-major BF16 matrix [outer x inner] with row stride ld (elements), box
// {64, box_outer}, 128-byte swizzle, zero fill outside the matrix.
bool map2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld,
                  uint32_t box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld * sizeof(bf16)};
    cuuint32_t box[2] = {64, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row-major 8-bit matrix [outer x inner] (row stride ld bytes), box
// {128, box_outer}, 128-byte swizzle, zero fill outside the matrix.
bool map2d_u8(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld};
    cuuint32_t box[2] = {128, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Stack of `depth` row-major BF16 matrices [outer x inner] (row stride ld,
// matrix stride mstride elements), box {64, box_outer, 1}, 128-byte swizzle.
bool map3d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t depth, uint64_t ld,
           uint64_t mstride, uint32_t box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {inner, outer, depth};
    cuuint64_t strides[2] = {ld * sizeof(bf16), mstride * sizeof(bf16)};
    cuuint32_t box[3] = {64, box_outer, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ------------------------------------------------------------------ workspace

constexpr int kColSplits = 296;
// Column-sum partials: kColSplits rows of (width + 32) floats, twice (the
// weight-gradient contractions also keep a t-weighted set; their splits times
// output rows never exceed kColSplits x width).
static size_t colpart_floats(int w) { return (size_t)2 * kColSplits * (rup(w, 16) + 16); }

int* bf16_error_flag(fbsde_ctx* c) { return c->bf ? c->bf->err : nullptr; }

fbsde_status bf16_create(fbsde_ctx* c) {
    Bf16Work* b = new (std::nothrow) Bf16Work();
    if (!b) return set_err(c, FBSDE_ERR_OOM, "host allocation failed");
    c->bf = b;
    const int w = c->w, L = c->L, D = c->D;
    b->Dp = (int)rup(D, 64);
    b->Dn = (int)rup(D, 16);
    b->wp = (int)rup(w, 64);
    const size_t Pm = c->Pmax();
    b->OP_stride = rup(Pm * b->wp, 128);
    const size_t nl = (size_t)L + 1;
    // per-tile fused kernels: FC / ResNet / NAIS-Net, depth <= kFusedMaxDepth,
    // D <= 256, width <= 256 (the accumulator and the residual share TMEM)
    if (b->Dn > 256)
        return set_err(c, FBSDE_ERR_UNSUPPORTED,
                       "the BF16 forms need D <= 256 (the Z contraction's output width); use the FP32 form");
    b->fused = L <= kFusedMaxDepth && b->Dp <= 256 && w <= 256;
    b->f8 = c->prec == FBSDE_FP8_HIDDEN;
    if (b->f8 && (!b->fused || c->akind == FBSDE_NAIS || w % 32 != 0))
        return set_err(c, FBSDE_ERR_UNSUPPORTED,
                       "FP8 hidden layers need an FC or ResNet network with depth <= 8, D <= 256 and a width "
                       "that is a multiple of 32");
    b->wp8 = (int)rup(w, 128);
    c->need_V32 = !b->fused;  // the fused backward reads the BF16 v rows only
    {
        int dev = 0, sms = 0;
        FBSDE_CK(c, cudaGetDevice(&dev));
        FBSDE_CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        b->sms = sms > 0 ? sms : 1;
    }
    if (b->fused) {
        b->grid = b->sms;
        b->G_stride = rup((Pm + 127) / 128 * 128 * (size_t)w, 128);
    }
    // the layered sweeps keep FP32 copies of every per-layer tensor; the fused
    // kernels keep them on chip and need only the BF16 operands
    const bool layered_f32 = !b->fused;
    size_t bytes = 0;
    auto add = [&](size_t n) { bytes += rup(n, 256); };
    add(2 * Pm * b->Dp * sizeof(bf16));
    for (int k = 0; k < 4; ++k) add(nl * b->OP_stride * sizeof(bf16));
    if (layered_f32) {
        for (int k = 0; k < 4; ++k) add(nl * Pm * w * sizeof(float));
        for (int k = 0; k < 2; ++k) add(nl * Pm * w * sizeof(bf16));
    }
    add((size_t)w * b->Dp * 2); add((size_t)b->Dn * b->wp * 2);
    for (int l = 1; l <= L; ++l) {
        add((size_t)w * b->wp * 2); add((size_t)w * b->wp * 2);
        add((size_t)w * b->Dp * 2); add((size_t)b->Dn * b->wp * 2);
    }
    add(colpart_floats(w) * sizeof(float));
    add(256);
    if (b->fused) {
        add((size_t)(L > 0 ? L : 1) * b->G_stride * sizeof(bf16));
        add((size_t)b->grid * (2 * L + 2) * 128 * w * sizeof(bf16));
        add((size_t)(2 * L + 3) * w * sizeof(float));
        add((Pm + 127) / 128 * 4 * (size_t)w * sizeof(float));
    }
    if (b->f8) {
        for (int l = 1; l <= L; ++l) add((size_t)w * b->wp8);
        add((size_t)(L + 1) * sizeof(float));
    }
    cudaError_t e = cudaMalloc(&b->mem, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, e == cudaErrorMemoryAllocation ? FBSDE_ERR_OOM : FBSDE_ERR_CUDA,
                       std::string("cudaMalloc BF16 workspace (") + std::to_string(bytes >> 20) + " MiB): " +
                           cudaGetErrorString(e));
    }
    FBSDE_CK(c, cudaMemset(b->mem, 0, bytes));
    char* cur = (char*)b->mem;
    auto take = [&](size_t n) { char* p = cur; cur += rup(n, 256); return (void*)p; };
    b->Xb = (bf16*)take(Pm * b->Dp * sizeof(bf16));
    b->Vb = (bf16*)take(Pm * b->Dp * sizeof(bf16));
    bf16* blk[4];
    for (int k = 0; k < 4; ++k) blk[k] = (bf16*)take(nl * b->OP_stride * sizeof(bf16));
    float* fblk[4] = {};
    bf16* hblk[2] = {};
    if (layered_f32) {
        for (int k = 0; k < 4; ++k) fblk[k] = (float*)take(nl * Pm * w * sizeof(float));
        for (int k = 0; k < 2; ++k) hblk[k] = (bf16*)take(nl * Pm * w * sizeof(bf16));
    }
    for (int l = 0; l <= L; ++l) {
        b->Hb[l] = blk[0] + l * b->OP_stride; b->Eb[l] = blk[1] + l * b->OP_stride;
        b->HDb[l] = blk[2] + l * b->OP_stride; b->ABb[l] = blk[3] + l * b->OP_stride;
        if (layered_f32) {
            const size_t o = (size_t)l * Pm * w;
            b->Hf[l] = fblk[0] + o; b->Gf[l] = fblk[1] + o; b->HDf[l] = fblk[2] + o; b->HBf[l] = fblk[3] + o;
            b->Af[l] = hblk[0] + o; b->Sf[l] = hblk[1] + o;
        }
    }
    b->Winx = (bf16*)take((size_t)w * b->Dp * 2);
    b->WinxT = (bf16*)take((size_t)b->Dn * b->wp * 2);
    for (int l = 1; l <= L; ++l) {
        b->W[l] = (bf16*)take((size_t)w * b->wp * 2); b->WT[l] = (bf16*)take((size_t)w * b->wp * 2);
        b->Bx[l] = (bf16*)take((size_t)w * b->Dp * 2); b->BxT[l] = (bf16*)take((size_t)b->Dn * b->wp * 2);
    }
    b->colpart = (float*)take(colpart_floats(w) * sizeof(float));
    b->err = (int*)take(256);
    if (b->fused) {
        b->G = (bf16*)take((size_t)(L > 0 ? L : 1) * b->G_stride * sizeof(bf16));
        b->scratch = (bf16*)take((size_t)b->grid * (2 * L + 2) * 128 * w * sizeof(bf16));
        b->pvec = (float*)take((size_t)(2 * L + 3) * w * sizeof(float));
        b->wopart = (float*)take((Pm + 127) / 128 * 4 * (size_t)w * sizeof(float));
    }
    if (b->f8) {
        for (int l = 1; l <= L; ++l) b->W8[l] = (uint8_t*)take((size_t)w * b->wp8);
        b->f8inv = (float*)take((size_t)(L + 1) * sizeof(float));
    }

    bool ok = true;
    const uint64_t P64 = Pm;
    ok &= map2d(&b->mXb, b->Xb, b->Dp, P64, b->Dp, 128);
    ok &= map2d(&b->mVb, b->Vb, b->Dp, P64, b->Dp, 128);
    ok &= map2d(&b->tX, b->Xb, b->Dp, P64, b->Dp, 64);
    ok &= map2d(&b->tV, b->Vb, b->Dp, P64, b->Dp, 64);
    for (int l = 0; l <= L; ++l) {
        ok &= map2d(&b->mHb[l], b->Hb[l], b->wp, P64, b->wp, 128);
        ok &= map2d(&b->mEb[l], b->Eb[l], b->wp, P64, b->wp, 128);
        ok &= map2d(&b->mHDb[l], b->HDb[l], b->wp, P64, b->wp, 128);
        ok &= map2d(&b->mABb[l], b->ABb[l], b->wp, P64, b->wp, 128);
        ok &= map2d(&b->tH[l], b->Hb[l], b->wp, P64, b->wp, 64);
        ok &= map2d(&b->tE[l], b->Eb[l], b->wp, P64, b->wp, 64);
        ok &= map2d(&b->tHD[l], b->HDb[l], b->wp, P64, b->wp, 64);
        ok &= map2d(&b->tAB[l], b->ABb[l], b->wp, P64, b->wp, 64);
    }
    // weight maps: boxes of up to 256 rows (wider layers run in column tiles)
    const uint32_t wbox = (uint32_t)(w < 256 ? w : 256);
    ok &= map2d(&b->mWinx, b->Winx, b->Dp, w, b->Dp, wbox);
    ok &= map2d(&b->mWinxT, b->WinxT, b->wp, b->Dn, b->wp, b->Dn);
    for (int l = 1; l <= L; ++l) {
        ok &= map2d(&b->mW[l], b->W[l], b->wp, w, b->wp, wbox);
        ok &= map2d(&b->mWT[l], b->WT[l], b->wp, w, b->wp, wbox);
        ok &= map2d(&b->mBx[l], b->Bx[l], b->Dp, w, b->Dp, wbox);
        ok &= map2d(&b->mBxT[l], b->BxT[l], b->wp, b->Dn, b->wp, b->Dn);
        if (b->f8) ok &= map2d_u8(&b->mW8[l], b->W8[l], b->wp8, w, b->wp8, w);
    }
    if (b->fused) {
        ok &= map3d(&b->sHb, b->Hb[0], b->wp, P64, (uint64_t)L + 1, b->wp, b->OP_stride, 128);
        ok &= map3d(&b->sHDb, b->HDb[0], b->wp, P64, (uint64_t)L + 1, b->wp, b->OP_stride, 128);
        ok &= map3d(&b->sABb, b->ABb[0], b->wp, P64, (uint64_t)L + 1, b->wp, b->OP_stride, 128);
        ok &= map3d(&b->sEb, b->Eb[0], b->wp, P64, (uint64_t)L + 1, b->wp, b->OP_stride, 128);
    }
    if (!ok) return set_err(c, FBSDE_ERR_CUDA, "cuTensorMapEncodeTiled failed (driver entry point or arguments)");
    if (b->fused) {
        c->Xb_op = b->Xb;
        c->Vb_op = b->Vb;
        c->ld_op = b->Dp;
    }
    return FBSDE_OK;
}

void bf16_destroy(fbsde_ctx* c) {
    if (!c->bf) return;
    if (c->bf->mem) cudaFree(c->bf->mem);
    delete c->bf;
    c->bf = nullptr;
}

// ------------------------------------------------------------------ activations

__device__ __forceinline__ void ld16f(const float* p, float (&v)[16]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float4 x = __ldg(q + i);
        v[4 * i] = x.x; v[4 * i + 1] = x.y; v[4 * i + 2] = x.z; v[4 * i + 3] = x.w;
    }
}
__device__ __forceinline__ void st16f(float* p, const float (&v)[16]) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
// Sixteen BF16 values (32-byte aligned) as floats.
__device__ __forceinline__ void ld16b(const bf16* p, float (&v)[16]) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const uint4 u = __ldg(q + i);
        const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w4[k]));
            v[8 * i + 2 * k] = f.x;
            v[8 * i + 2 * k + 1] = f.y;
        }
    }
}
__device__ __forceinline__ void st16b(bf16* p, const float (&v)[16]) {
    uint4 u[2];
    uint32_t* w = reinterpret_cast<uint32_t*>(u);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    uint4* q = reinterpret_cast<uint4*>(p);
    q[0] = u[0];
    q[1] = u[1];
}

// ------------------------------------------------------------------ epilogues (16 columns per call)

struct EpiFwdB {  // a = acc + b + t tcol; h = s hprev + c act(a)
    const float* bias; const float* tcol; int K0; const float* hprev; float s, c;
    bf16* aout; float* hout; bf16* hbout; int w, wp, M; float dt; int act;
    __device__ void operator()(int row, int c0, const float (&v)[16], int) const {
        const float t = (float)(row / M) * dt;
        float a[16], h[16], hp[16];
        if (hprev) ld16f(hprev + (size_t)row * w + c0, hp);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            a[j] = v[j] + bias[c0 + j];
            if (tcol) a[j] += t * tcol[(size_t)(c0 + j) * K0];
            const float f = act3_fast(act, a[j]).f;
            h[j] = (hprev ? s * hp[j] : 0.f) + c * f;
        }
        st16b(aout + (size_t)row * w + c0, a);
        st16f(hout + (size_t)row * w + c0, h);
        st16b(hbout + (size_t)row * wp + c0, h);
    }
};

struct EpiRevB {  // g = s g_l + acc; e = c_prev act'(a_prev) g
    const float* gl; float s; const bf16* aprev; float cprev;
    float* gout; bf16* eout; int w, wp; int act;
    __device__ void operator()(int row, int c0, const float (&v)[16], int) const {
        float g[16], e[16], gv[16], ap[16];
        ld16f(gl + (size_t)row * w + c0, gv);
        ld16b(aprev + (size_t)row * w + c0, ap);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            g[j] = s * gv[j] + v[j];
            e[j] = cprev * act3_fast(act, ap[j]).d1 * g[j];
        }
        st16f(gout + (size_t)row * w + c0, g);
        st16b(eout + (size_t)row * wp + c0, e);
    }
};

struct EpiZB {  // Z (+)= acc, columns < D
    float* Z; int D; int accumulate;
    __device__ void operator()(int row, int c0, const float (&v)[16], int) const {
        float* z = Z + (size_t)row * D;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (c0 + j < D) z[c0 + j] = accumulate ? z[c0 + j] + v[j] : v[j];
    }
};

struct EpiTanB {  // h' = s h'_prev + c act'(a) a'; S = c act''(a) a' g
    const bf16* a; const float* hdprev; const float* g; float s, c;
    float* hdout; bf16* hdbout; bf16* sout; int w, wp; int act;
    __device__ void operator()(int row, int c0, const float (&v)[16], int) const {
        float av[16], gv[16], hp[16], hd[16], sv[16];
        const size_t o = (size_t)row * w + c0;
        ld16b(a + o, av);
        ld16f(g + o, gv);
        if (hdprev) ld16f(hdprev + o, hp);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const Act3 f = act3_fast(act, av[j]);
            hd[j] = (hdprev ? s * hp[j] : 0.f) + c * f.d1 * v[j];
            sv[j] = c * f.d2 * v[j] * gv[j];
        }
        st16f(hdout + o, hd);
        st16b(hdbout + (size_t)row * wp + c0, hd);
        st16b(sout + o, sv);
    }
};

struct EpiAdjB {  // hbar = s hbar_l + acc; abar_prev = c_prev act'(a_prev) hbar + S_prev
    const float* hbl; float s; const bf16* aprev; const bf16* sprev; float cprev;
    float* hbout; bf16* about; int w, wp; int act;
    __device__ void operator()(int row, int c0, const float (&v)[16], int) const {
        float hv[16], ap[16], sp[16], hb[16], ab[16];
        const size_t o = (size_t)row * w + c0;
        ld16f(hbl + o, hv);
        ld16b(aprev + o, ap);
        ld16b(sprev + o, sp);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            hb[j] = s * hv[j] + v[j];
            ab[j] = cprev * act3_fast(act, ap[j]).d1 * hb[j] + sp[j];
        }
        st16f(hbout + o, hb);
        st16b(about + (size_t)row * wp + c0, ab);
    }
};

struct EpiPartB {  // split-K partial sums part[split][row][col]
    float* part; int rows, N;
    __device__ void operator()(int row, int c0, const float (&v)[16], int split) const {
        st16f(part + ((size_t)split * rows + row) * N + c0, v);
    }
};

struct EpiStoreB {  // C[row][c0 + j] = acc for columns < N
    float* C; int ldc, N;
    __device__ void operator()(int row, int c0, const float (&v)[16], int) const {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (c0 + j < N) C[(size_t)row * ldc + c0 + j] = v[j];
    }
};

// ------------------------------------------------------------------ small kernels

// out[r][c] (row stride ldo, zero padded to rows_o x cols_o) = src(r, c) with
// src(r, c) = S[r * lds + off + c] (or S[c * lds + off + r] when transposed)
// for r < rows_v, c < cols_v.
__global__ void k_cvt_bf16(int rows_o, int cols_o, int ldo, bf16* __restrict__ out, const float* __restrict__ S,
                           int lds, int off, int rows_v, int cols_v, int transpose) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)rows_o * cols_o) return;
    const int r = (int)(i / cols_o), cc = (int)(i % cols_o);
    float x = 0.f;
    if (r < rows_v && cc < cols_v) x = transpose ? S[(size_t)cc * lds + off + r] : S[(size_t)r * lds + off + cc];
    out[(size_t)r * ldo + cc] = __float2bfloat16_rn(x);
}

// The BF16 weight copies refreshed every step, all in one launch
// (blockIdx.y = copy): out[r][c] = S[r][off + c] (or S[c][off + r] when
// transposed) for r < rows_v, c < cols_v, zero in the padding.
struct CvtJob {
    bf16* out;
    const float* S;
    int rows_o, cols_o, ldo, lds, off, rows_v, cols_v, tr;
};
constexpr int kMaxCvtJobs = 2 + 4 * kMaxDepth;
struct CvtBatch {
    CvtJob job[kMaxCvtJobs];
    int n;
};

__global__ void k_cvt_bf16_batch(const __grid_constant__ CvtBatch b) {
    const CvtJob& j = b.job[blockIdx.y];
    const size_t n = (size_t)j.rows_o * j.cols_o;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / j.cols_o), cc = (int)(i % j.cols_o);
        float x = 0.f;
        if (r < j.rows_v && cc < j.cols_v)
            x = j.tr ? j.S[(size_t)cc * j.lds + j.off + r] : j.S[(size_t)r * j.lds + j.off + cc];
        j.out[(size_t)r * j.ldo + cc] = __float2bfloat16_rn(x);
    }
}

// g_L = w_o, e_L = c_L act'(a_L) w_o (BF16)
__global__ void k_top_rev_b(size_t P, int w, int wp, const bf16* __restrict__ aL, const float* __restrict__ wo,
                            float cL, int act, float* __restrict__ gL, bf16* __restrict__ eL) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * w) return;
    const size_t p = i / w;
    const int j = (int)(i % w);
    gL[i] = wo[j];
    eL[p * wp + j] = __float2bfloat16_rn(cL * act3_fast(act, __bfloat162float(aL[i])).d1 * wo[j]);
}

// hbar_L = alpha w_o, abar_L = c_L act'(a_L) hbar_L + S_L (BF16)
__global__ void k_top_adj_b(size_t P, int w, int wp, const bf16* __restrict__ aL, const float* __restrict__ wo,
                            const float* __restrict__ alpha, const bf16* __restrict__ SL, float cL, int act,
                            float* __restrict__ hbL, bf16* __restrict__ abL) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * w) return;
    const size_t p = i / w;
    const int j = (int)(i % w);
    const float hb = alpha[p] * wo[j];
    hbL[i] = hb;
    abL[p * wp + j] = __float2bfloat16_rn(cL * act3_fast(act, __bfloat162float(aL[i])).d1 * hb +
                                          __bfloat162float(SL[i]));
}

// Partial column sums over a range of points, fixed order:
// part[split][c] = sum_{p in split} wt(p) X[p][c] (+ X2[p][c]), wt = 1 (mode 0),
// t_p (mode 1) or wts[p] (mode 2); X2 (same layout, optional) enters with
// weight 1.  256 threads: 32 column lanes x 8 row lanes; a column
// lane covers 8 consecutive columns with one 16- or 32-byte load per row (the
// vector path needs ncols and ldx multiples of 8), the row lanes stride the
// split's rows and are combined in shared memory in a fixed order.
// Eight consecutive values of a BF16 or FP32 row (16- or 32-byte aligned) as floats.
template <class T>
__device__ __forceinline__ void ld_row8(const T* src, float (&v)[8]) {
    if (sizeof(T) == 2) {
        const uint4 q = *reinterpret_cast<const uint4*>(src);
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w4[i]));
            v[2 * i] = f.x; v[2 * i + 1] = f.y;
        }
    } else {
        const float4 a = reinterpret_cast<const float4*>(src)[0];
        const float4 b = reinterpret_cast<const float4*>(src)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_colsum(size_t P, int ncols, const T* __restrict__ X, int ldx, int mode,
                                                const float* __restrict__ wts, int M, float dt,
                                                float* __restrict__ part, size_t chunk,
                                                const T* __restrict__ X2 = nullptr) {
    __shared__ float red[8][256 + 8];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int split = blockIdx.x;
    const size_t p0 = (size_t)split * chunk, p1 = min(P, p0 + chunk);
    const bool vec = (ncols % 8 == 0) && (ldx % 8 == 0);
    for (int cb = 0; cb < ncols; cb += 256) {
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int c0 = cb + tx * 8;
        if (vec && c0 < ncols) {
            // four rows in flight per thread
            size_t p = p0 + ty;
            for (; p + 24 < p1; p += 32) {
                float v[4][8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const T* row = X + (p + 8 * u) * ldx;
                    if (sizeof(T) == 2) {
                        const uint4 q = *reinterpret_cast<const uint4*>(row + c0);
                        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w4[i]));
                            v[u][2 * i] = f.x; v[u][2 * i + 1] = f.y;
                        }
                    } else {
                        const float4 a = reinterpret_cast<const float4*>(row + c0)[0];
                        const float4 b = reinterpret_cast<const float4*>(row + c0)[1];
                        v[u][0] = a.x; v[u][1] = a.y; v[u][2] = a.z; v[u][3] = a.w;
                        v[u][4] = b.x; v[u][5] = b.y; v[u][6] = b.z; v[u][7] = b.w;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const size_t pu = p + 8 * u;
                    const float wt = mode == 0 ? 1.f : mode == 1 ? (float)(pu / M) * dt : wts[pu];
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[i] = fmaf(wt, v[u][i], acc[i]);
                }
                if (X2) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float v2[8];
                        ld_row8(X2 + (p + 8 * u) * ldx + c0, v2);
#pragma unroll
                        for (int i = 0; i < 8; ++i) acc[i] += v2[i];
                    }
                }
            }
            for (; p < p1; p += 8) {
                const float wt = mode == 0 ? 1.f : mode == 1 ? (float)(p / M) * dt : wts[p];
                const T* row = X + p * ldx;
                float v[8];
                if (sizeof(T) == 2) {
                    const uint4 q = *reinterpret_cast<const uint4*>(row + c0);
                    const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w4[i]));
                        v[2 * i] = f.x; v[2 * i + 1] = f.y;
                    }
                } else {
                    const float4 a = reinterpret_cast<const float4*>(row + c0)[0];
                    const float4 b = reinterpret_cast<const float4*>(row + c0)[1];
                    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = fmaf(wt, v[i], acc[i]);
                if (X2) {
                    float v2[8];
                    ld_row8(X2 + p * ldx + c0, v2);
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[i] += v2[i];
                }
            }
        } else if (!vec) {
            for (size_t p = p0 + ty; p < p1; p += 8) {
                const float wt = mode == 0 ? 1.f : mode == 1 ? (float)(p / M) * dt : wts[p];
                const T* row = X + p * ldx;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (c0 + i < ncols) {
                        acc[i] = fmaf(wt, (float)row[c0 + i], acc[i]);
                        if (X2) acc[i] += (float)X2[p * ldx + c0 + i];
                    }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) red[ty][tx * 8 + i] = acc[i];
        __syncthreads();
        const int c = cb + threadIdx.x;
        if (threadIdx.x < 256 && c < ncols) {
            float s = 0.f;
#pragma unroll
            for (int r = 0; r < 8; ++r) s += red[r][threadIdx.x];
            part[(size_t)split * ncols + c] = s;
        }
        __syncthreads();
    }
}

// One warp per column: lane i sums splits i, i+32, ... in order, then a fixed
// butterfly combines the lanes (bit-reproducible).
__global__ void k_colsum_reduce(const float* __restrict__ part, int splits, int ncols, float* __restrict__ out,
                                int ldo, int accumulate) {
    const int c = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= ncols) return;
    float s = 0.f;
    for (int k = lane; k < splits; k += 32) s += part[(size_t)k * ncols + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[(size_t)c * ldo] = accumulate ? out[(size_t)c * ldo] + s : s;
}

// The tail of one weight-gradient contraction in one launch.  Blocks [0, nred)
// reduce the split-K partials: out[r * ld + off + c] = sum_z part[z][r][c] for
// c < nc, a block per 32 consecutive columns of one row, warp g summing the
// splits z = g, g + 8, ... (one column per lane, every load in flight at once)
// and warp 0 adding the eight warps' sums in order (bit-reproducible).  Each
// later block sums, one warp per entry,
// the column-sum partials of pair 0's A operand (cs_part, then cst_part) over
// the splits, in k_colsum_reduce's order.
__global__ void __launch_bounds__(256) k_wgrad_finish(const float* __restrict__ part, int splits, int rows, int N,
                                                      int nc, float* __restrict__ out, int ld, int off, int nred,
                                                      const float* __restrict__ cs_part, float* __restrict__ cs_out,
                                                      int cs_ld, const float* __restrict__ cst_part,
                                                      float* __restrict__ cst_out, int cst_ld) {
    if ((int)blockIdx.x < nred) {
        __shared__ float red[8][33];
        const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
        const int cblocks = (nc + 31) / 32;
        const int r = blockIdx.x / cblocks, c = (blockIdx.x % cblocks) * 32 + lane;
        const size_t stride = (size_t)rows * N;
        float s = 0.f;
        if (r < rows && c < nc) {
            const float* q = part + (size_t)r * N + c;
            int z = g;
            for (; z + 24 < splits; z += 32) {
                const float a0 = __ldcs(q + (size_t)z * stride), a1 = __ldcs(q + (size_t)(z + 8) * stride);
                const float a2 = __ldcs(q + (size_t)(z + 16) * stride), a3 = __ldcs(q + (size_t)(z + 24) * stride);
                s += (a0 + a1) + (a2 + a3);
            }
            for (; z < splits; z += 8) s += __ldcs(q + (size_t)z * stride);
        }
        red[g][lane] = s;
        __syncthreads();
        if (g == 0 && r < rows && c < nc) {
            float t = red[0][lane];
#pragma unroll
            for (int k = 1; k < 8; ++k) t += red[k][lane];
            out[(size_t)r * ld + off + c] = t;
        }
        return;
    }
    const int e = ((int)blockIdx.x - nred) * 8 + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
    const bool second = e >= rows;
    const int col = second ? e - rows : e;
    const float* src = second ? cst_part : cs_part;
    if (!src || col >= rows) return;
    float s = 0.f;
    for (int k = lane; k < splits; k += 32) s += src[(size_t)k * rows + col];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        if (second) cst_out[(size_t)col * cst_ld] = s;
        else cs_out[(size_t)col * cs_ld] = s;
    }
}

// ------------------------------------------------------------------ launch helpers

template <bool TN, class Epi>
static fbsde_status tc_launch(fbsde_ctx* c, int cls, const TcArgs& a, int splits, const Epi& e, double flops) {
    const int tok = prof_begin(c, cls);
    cudaError_t err = tc_gemm<TN>(a, splits, e, c->stream);
    prof_end(c, cls, tok, flops);
    if (err != cudaSuccess) return set_err(c, FBSDE_ERR_CUDA, std::string("tcgen05 GEMM: ") + cudaGetErrorString(err));
    ++c->n_launch;
    return FBSDE_OK;
}

static TcArgs nt_args(fbsde_ctx* c, int rows, int N) {
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rows = rows; a.N = N; a.kchunk = 0; a.err = c->bf->err;
    return a;
}
static void add_pair(TcArgs& a, const CUtensorMap& A, const CUtensorMap& B, int K) {
    a.pr[a.npairs].a = A;
    a.pr[a.npairs].b = B;
    a.pr[a.npairs].K = K;
    ++a.npairs;
}

// Column sums over the P points (or over `rows` rows when given).
static fbsde_status colsum(fbsde_ctx* c, int cls, const void* X, bool is_bf16, int ldx, int ncols, int mode,
                           const float* wts, float* out, int ldo, int accumulate, const void* X2 = nullptr,
                           size_t rows = 0) {
    Bf16Work* b = c->bf;
    const size_t P = rows ? rows : c->P();
    const size_t chunk = (P + kColSplits - 1) / kColSplits;
    const int splits = (int)((P + chunk - 1) / chunk);
    const float dt = (float)(c->T / c->N);
    const int tok = prof_begin(c, cls);
    if (is_bf16)
        k_colsum<bf16><<<splits, 256, 0, c->stream>>>(P, ncols, (const bf16*)X, ldx, mode, wts, c->M, dt, b->colpart,
                                                       chunk, (const bf16*)X2);
    else
        k_colsum<float><<<splits, 256, 0, c->stream>>>(P, ncols, (const float*)X, ldx, mode, wts, c->M, dt, b->colpart,
                                                        chunk, (const float*)X2);
    FBSDE_CK_LAUNCH(c);
    k_colsum_reduce<<<nblk((size_t)ncols * 32, 256), 256, 0, c->stream>>>(b->colpart, splits, ncols, out, ldo,
                                                                        accumulate);
    prof_end(c, cls, tok, 2.0 * (double)P * ncols);
    FBSDE_CK_LAUNCH(c);
    return FBSDE_OK;
}

// Weight gradient: out[r * ld + off + j] = sum over points of the TN pairs,
// for output rows r < rows and columns j < ncols_store.  With cs_out the same
// launch also sums the columns of pair 0's A operand over all points
// (cs_out[r * cs_ld], a bias gradient) and, with cst_out, the same sums
// weighted by the point's time t (cst_out[r * cst_ld], the t column of W_in).
static fbsde_status wgrad(fbsde_ctx* c, TcArgs a, int ncols_store, float* out, int ld, int off,
                          float* cs_out = nullptr, int cs_ld = 1, float* cst_out = nullptr, int cst_ld = 1) {
    const size_t P = c->P();
    const int mblocks = (a.rows + 127) / 128;
    // one wave of CTAs (one per SM, each streaming its own range of points):
    // half the split-K partials of two waves, and measured faster than both
    // two waves and half a wave
    int want = (c->bf->sms + mblocks - 1) / mblocks;
    size_t kc = rup((P + want - 1) / want, 64);
    int splits = (int)((P + kc - 1) / kc);
    while ((size_t)splits * a.rows * a.N > c->part_floats) {
        kc *= 2;
        splits = (int)((P + kc - 1) / kc);
    }
    a.kchunk = (int)kc;
    Bf16Work* b = c->bf;
    const size_t cs_cap = colpart_floats(c->w);
    const bool cs = cs_out && (size_t)splits * a.rows * (cst_out ? 2 : 1) <= cs_cap;
    if (cs) {
        a.cs_part = b->colpart;
        a.cs_tpart = cst_out ? b->colpart + (size_t)splits * a.rows : nullptr;
        a.cs_M = c->M;
        a.cs_dt = (float)(c->T / c->N);
    }
    double flops = 0;
    for (int q = 0; q < a.npairs; ++q) flops += 2.0 * a.rows * (double)ncols_store * P;
    FBSDE_TRY(tc_launch<true>(c, PROF_WGRAD, a, splits, EpiPartB{c->part, a.rows, a.N}, flops));
    // the split-K reduction and the column sums in one launch
    const int nred = a.rows * ((ncols_store + 31) / 32);
    const int ncs = cs ? (a.rows * (cst_out ? 2 : 1) + 7) / 8 : 0;
    k_wgrad_finish<<<(unsigned)(nred + ncs), 256, 0, c->stream>>>(
        c->part, splits, a.rows, a.N, ncols_store, out, ld, off, nred, cs ? b->colpart : nullptr, cs_out, cs_ld,
        cs && cst_out ? b->colpart + (size_t)splits * a.rows : nullptr, cst_out, cst_ld);
    FBSDE_CK_LAUNCH(c);
    if (!cs && cs_out) {
        // the partial sums do not fit the scratch: a separate pass over pair 0's A
        return set_err(c, FBSDE_ERR_UNSUPPORTED, "column-sum scratch too small for this split");
    }
    return FBSDE_OK;
}

// ------------------------------------------------------------------ weights

// E4M3 copies of the hidden-layer weights W_l (l = 1..L), one block per layer:
// the block's max |W_l| sets the per-tensor scale s_W (the largest power of two
// with s_W max|W| <= 448, so the scaled values stay finite), the copy holds
// RN(s_W W_l) (satfinite), and inv[l] = 1 / (s_h(l-1) s_W) undoes both scales
// on the FP32 accumulator.
struct Fp8WeightArgs {
    const float* W[kMaxDepth + 1];
    uint8_t* W8[kMaxDepth + 1];
    int w, ld8, res;
    float* inv;
};

__global__ void __launch_bounds__(1024) k_fp8_weights(const Fp8WeightArgs a) {
    __shared__ float red[32];
    __shared__ float s_scale;
    const int l = blockIdx.x + 1;
    const float* W = a.W[l];
    const int n = a.w * a.w;
    float mx = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf(W[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[k]);
        float s = 1.f;
        if (m > 0.f) {
            while (m * s * 2.f <= 448.f && s < 1.0e30f) s *= 2.f;
            while (m * s > 448.f) s *= 0.5f;
        }
        s_scale = s;
        a.inv[l] = 1.f / (e4m3_act_scale(l - 1, a.res != 0) * s);
    }
    __syncthreads();
    const float s = s_scale;
    uint8_t* W8 = a.W8[l];
    for (int i = threadIdx.x; i < a.w * a.ld8; i += blockDim.x) {
        const int r = i / a.ld8, k = i % a.ld8;
        const float v = k < a.w ? W[(size_t)r * a.w + k] * s : 0.f;
        W8[i] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
}

fbsde_status bf16_prepare_weights(fbsde_ctx* c, const float* theta) {
    FBSDE_TRY(fp32_prepare_weights(c, theta));  // NAIS: A_l = -R^T R - eps I in FP32
    Bf16Work* b = c->bf;
    const int w = c->w, D = c->D, K0 = D + 1;
    const ParamLayout& pl = c->pl;
    CvtBatch cb;
    std::memset(&cb, 0, sizeof(cb));
    size_t most = 0;
    auto cvt = [&](bf16* out, int rows_o, int cols_o, int ldo, const float* S, int lds, int off, int rows_v,
                   int cols_v, int tr) -> fbsde_status {
        if (cb.n >= kMaxCvtJobs) return set_err(c, FBSDE_ERR_UNSUPPORTED, "too many weight copies");
        cb.job[cb.n++] = CvtJob{out, S, rows_o, cols_o, ldo, lds, off, rows_v, cols_v, tr};
        most = std::max(most, (size_t)rows_o * cols_o);
        return FBSDE_OK;
    };
    FBSDE_TRY(cvt(b->Winx, w, b->Dp, b->Dp, theta + pl.Win, K0, 1, w, D, 0));
    FBSDE_TRY(cvt(b->WinxT, b->Dn, b->wp, b->wp, theta + pl.Win, K0, 1, D, w, 1));
    for (int l = 1; l <= c->L; ++l) {
        const float* Wm = c->akind == FBSDE_NAIS ? c->Amat[l] : theta + pl.W[l];
        FBSDE_TRY(cvt(b->W[l], w, b->wp, b->wp, Wm, w, 0, w, w, 0));
        FBSDE_TRY(cvt(b->WT[l], w, b->wp, b->wp, Wm, w, 0, w, w, 1));
        if (c->akind == FBSDE_NAIS) {
            FBSDE_TRY(cvt(b->Bx[l], w, b->Dp, b->Dp, theta + pl.B[l], K0, 1, w, D, 0));
            FBSDE_TRY(cvt(b->BxT[l], b->Dn, b->wp, b->wp, theta + pl.B[l], K0, 1, D, w, 1));
        }
    }
    k_cvt_bf16_batch<<<dim3((unsigned)std::min<size_t>(nblk(most, 256), 64), (unsigned)cb.n), 256, 0, c->stream>>>(cb);
    FBSDE_CK_LAUNCH(c);
    if (b->f8) {
        Fp8WeightArgs fa;
        std::memset(&fa, 0, sizeof(fa));
        for (int l = 1; l <= c->L; ++l) {
            fa.W[l] = theta + pl.W[l];
            fa.W8[l] = b->W8[l];
        }
        fa.w = w; fa.ld8 = b->wp8; fa.res = c->akind == FBSDE_RESNET ? 1 : 0; fa.inv = b->f8inv;
        k_fp8_weights<<<c->L, 1024, 0, c->stream>>>(fa);
        FBSDE_CK_LAUNCH(c);
    }
    return FBSDE_OK;
}

// ------------------------------------------------------------------ forward

fbsde_status bf16_forward(fbsde_ctx* c, const float* theta, bool for_grad) {
    Bf16Work* b = c->bf;
    if (b->fused) return fused_forward(c, theta, for_grad);
    const int w = c->w, L = c->L, D = c->D, K0 = D + 1, act = c->act, wp = b->wp;
    const int P = (int)c->P();
    const ParamLayout& pl = c->pl;
    const float dt = (float)(c->T / c->N);
    const bool nais = c->akind == FBSDE_NAIS;
    cudaStream_t st = c->stream;

    // GEMM operand copy of X
    k_cvt_bf16<<<nblk((size_t)P * b->Dp, 256), 256, 0, st>>>(P, b->Dp, b->Dp, b->Xb, c->X, D, 0, P, D, 0);
    FBSDE_CK_LAUNCH(c);

    {   // lift
        TcArgs a = nt_args(c, P, w);
        add_pair(a, b->mXb, b->mWinx, D);
        EpiFwdB e{theta + pl.bin, theta + pl.Win, K0, nullptr, 0.f, 1.f, b->Af[0], b->Hf[0], b->Hb[0], w, wp,
                  c->M, dt, act};
        FBSDE_TRY(tc_launch<false>(c, PROF_POINTS, a, 1, e, 2.0 * P * w * (double)D));
    }
    for (int l = 1; l <= L; ++l) {
        TcArgs a = nt_args(c, P, w);
        add_pair(a, b->mHb[l - 1], b->mW[l], w);
        double fl = 2.0 * P * w * (double)w;
        if (nais) { add_pair(a, b->mXb, b->mBx[l], D); fl += 2.0 * P * w * (double)D; }
        EpiFwdB e{theta + pl.b[l], nais ? theta + pl.B[l] : nullptr, K0, b->Hf[l - 1], layer_skip(c, l),
                  layer_scale(c, l), b->Af[l], b->Hf[l], b->Hb[l], w, wp, c->M, dt, act};
        FBSDE_TRY(tc_launch<false>(c, PROF_POINTS, a, 1, e, fl));
    }
    FBSDE_TRY(launch_rowdot(c, b->Hf[L], theta, c->Y));

    k_top_rev_b<<<nblk((size_t)P * w, 256), 256, 0, st>>>(P, w, wp, b->Af[L], theta + pl.wo, layer_scale(c, L), act,
                                                          b->Gf[L], b->Eb[L]);
    FBSDE_CK_LAUNCH(c);
    for (int l = L; l >= 1; --l) {
        TcArgs a = nt_args(c, P, w);
        add_pair(a, b->mEb[l], b->mWT[l], w);
        EpiRevB e{b->Gf[l], layer_skip(c, l), b->Af[l - 1], layer_scale(c, l - 1), b->Gf[l - 1], b->Eb[l - 1], w, wp,
                  act};
        FBSDE_TRY(tc_launch<false>(c, PROF_POINTS, a, 1, e, 2.0 * P * w * (double)w));
    }
    {   // Z = W_in[:,1:]^T e_0 (+ sum_l B_l[:,1:]^T e_l): one contraction over all pairs
        TcArgs a = nt_args(c, P, b->Dn);
        add_pair(a, b->mEb[0], b->mWinxT, w);
        if (nais)
            for (int l = 1; l <= L; ++l) add_pair(a, b->mEb[l], b->mBxT[l], w);
        FBSDE_TRY(tc_launch<false>(c, PROF_POINTS, a, 1, EpiZB{c->Z, D, 0}, 2.0 * P * D * (double)w * a.npairs));
    }
    return FBSDE_OK;
}

// ------------------------------------------------------------------ backward

fbsde_status bf16_backward(fbsde_ctx* c, const float* theta, float* grad) {
    Bf16Work* b = c->bf;
    if (b->fused) {
        FBSDE_TRY(fused_backward(c, theta));
        return bf16_wgrad_tail(c, theta, grad);
    }
    const int w = c->w, L = c->L, D = c->D, K0 = D + 1, act = c->act, wp = b->wp;
    const int P = (int)c->P();
    const ParamLayout& pl = c->pl;
    const bool nais = c->akind == FBSDE_NAIS;
    cudaStream_t st = c->stream;

    k_cvt_bf16<<<nblk((size_t)P * b->Dp, 256), 256, 0, st>>>(P, b->Dp, b->Dp, b->Vb, c->V, D, 0, P, D, 0);
    FBSDE_CK_LAUNCH(c);

    {   // tangent lift along u' = (0, v)
        TcArgs a = nt_args(c, P, w);
        add_pair(a, b->mVb, b->mWinx, D);
        EpiTanB e{b->Af[0], nullptr, b->Gf[0], 0.f, 1.f, b->HDf[0], b->HDb[0], b->Sf[0], w, wp, act};
        FBSDE_TRY(tc_launch<false>(c, PROF_POINTS, a, 1, e, 2.0 * P * w * (double)D));
    }
    for (int l = 1; l <= L; ++l) {
        TcArgs a = nt_args(c, P, w);
        add_pair(a, b->mHDb[l - 1], b->mW[l], w);
        double fl = 2.0 * P * w * (double)w;
        if (nais) { add_pair(a, b->mVb, b->mBx[l], D); fl += 2.0 * P * w * (double)D; }
        EpiTanB e{b->Af[l], b->HDf[l - 1], b->Gf[l], layer_skip(c, l), layer_scale(c, l), b->HDf[l], b->HDb[l],
                  b->Sf[l], w, wp, act};
        FBSDE_TRY(tc_launch<false>(c, PROF_POINTS, a, 1, e, fl));
    }
    k_top_adj_b<<<nblk((size_t)P * w, 256), 256, 0, st>>>(P, w, wp, b->Af[L], theta + pl.wo, c->alpha, b->Sf[L],
                                                          layer_scale(c, L), act, b->HBf[L], b->ABb[L]);
    FBSDE_CK_LAUNCH(c);
    for (int l = L; l >= 1; --l) {
        TcArgs a = nt_args(c, P, w);
        add_pair(a, b->mABb[l], b->mWT[l], w);
        EpiAdjB e{b->HBf[l], layer_skip(c, l), b->Af[l - 1], b->Sf[l - 1], layer_scale(c, l - 1), b->HBf[l - 1],
                  b->ABb[l - 1], w, wp, act};
        FBSDE_TRY(tc_launch<false>(c, PROF_POINTS, a, 1, e, 2.0 * P * w * (double)w));
    }

    return bf16_wgrad_tail(c, theta, grad);
}

// Weight gradients from the BF16 operands the sweeps left in HBM: W_l, W_in
// (and NAIS B_l) by tensor-core contractions over all points, biases and the
// read-out by fixed-order column sums.
fbsde_status bf16_wgrad_tail(fbsde_ctx* c, const float* theta, float* grad) {
    Bf16Work* b = c->bf;
    const int w = c->w, L = c->L, D = c->D, K0 = D + 1, wp = b->wp;
    const int P = (int)c->P();
    const ParamLayout& pl = c->pl;
    const bool nais = c->akind == FBSDE_NAIS;
    // weight gradients: contractions over all points on the tensor cores
    for (int l = 1; l <= L; ++l) {
        TcArgs a = nt_args(c, w, w);
        add_pair(a, b->tAB[l], b->tH[l - 1], P);
        add_pair(a, b->tE[l], b->tHD[l - 1], P);
        // b_l (and for NAIS the t column of B_l) from the same pass over abar_l
        FBSDE_TRY(wgrad(c, a, w, nais ? c->gA[l] : grad + pl.W[l], w, 0, grad + pl.b[l], 1,
                        nais ? grad + pl.B[l] : nullptr, K0));
        if (nais) {
            TcArgs ax = nt_args(c, w, b->Dn);
            add_pair(ax, b->tAB[l], b->tX, P);
            add_pair(ax, b->tE[l], b->tV, P);
            FBSDE_TRY(wgrad(c, ax, D, grad + pl.B[l], K0, 1));
        }
    }
    if (nais) FBSDE_TRY(nais_chain_R(c, theta, grad));  // dR = -R (dA + dA^T)
    {
        TcArgs ax = nt_args(c, w, b->Dn);
        add_pair(ax, b->tAB[0], b->tX, P);
        add_pair(ax, b->tE[0], b->tV, P);
        // b_in and the t column of W_in from the same pass over abar_0
        FBSDE_TRY(wgrad(c, ax, D, grad + pl.Win, K0, 1, grad + pl.bin, 1, grad + pl.Win, K0));
    }
    // dw_o = sum_p alpha_p h_L(p) + h'_L(p);  db_o = sum_p alpha_p
    if (b->fused && c->akind != FBSDE_NAIS && !b->f8) {
        // the pipelined backward left one partial sum per tile, 32-row group
        // and column: sum them in a fixed order
        FBSDE_TRY(colsum(c, PROF_WGRAD, b->wopart, false, w, w, 0, nullptr, grad + pl.wo, 1, 0, nullptr,
                         (P + 127) / 128 * 4));
    } else if (b->fused) {
        FBSDE_TRY(colsum(c, PROF_WGRAD, b->Hb[L], true, wp, w, 2, c->alpha, grad + pl.wo, 1, 0, b->HDb[L]));
    } else {
        FBSDE_TRY(colsum(c, PROF_WGRAD, b->Hf[L], false, w, w, 2, c->alpha, grad + pl.wo, 1, 0, b->HDf[L]));
    }
    // db_o = sum_p alpha_p, formed with the loss (k_loss_reduce)
    FBSDE_CK(c, cudaMemcpyAsync(grad + pl.bo, c->alpha_sum, sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    return launch_check_finite(c, grad, pl.total);
}

}  // namespace fbsde

// ------------------------------------------------------------------ C ABI: the contraction engine

using namespace fbsde;

extern "C" fbsde_status fbsde_gemm_bf16(const void* A_dev, const void* B_dev, float* C_dev, int rows, int N, int K,
                                        int lda, int ldb, int ldc, int trans, void* cuda_stream) {
    if (!A_dev || !B_dev || !C_dev) return FBSDE_ERR_INVALID;
    if (rows < 1 || K < 1 || N < 16 || N > 256 || N % 16 != 0 || ldc < N) return FBSDE_ERR_INVALID;
    if (lda % 8 != 0 || ldb % 8 != 0 || ((uintptr_t)A_dev & 15) || ((uintptr_t)B_dev & 15)) return FBSDE_ERR_INVALID;
    if (trans != 0 && trans != 1) return FBSDE_ERR_INVALID;
    if (trans == 0 && (lda < K || ldb < K)) return FBSDE_ERR_INVALID;
    if (trans == 1 && (lda < rows || ldb < N)) return FBSDE_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rows = rows; a.N = N; a.npairs = 1; a.err = nullptr; a.pr[0].K = K;
    bool ok;
    if (trans == 0) {
        ok = map2d(&a.pr[0].a, A_dev, (uint64_t)K, (uint64_t)rows, (uint64_t)lda, 128) &&
             map2d(&a.pr[0].b, B_dev, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, (uint32_t)N);
    } else {
        ok = map2d(&a.pr[0].a, A_dev, (uint64_t)rows, (uint64_t)K, (uint64_t)lda, 64) &&
             map2d(&a.pr[0].b, B_dev, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, 64);
        a.kchunk = (int)rup((size_t)K, 64);
    }
    if (!ok) return FBSDE_ERR_CUDA;
    cudaError_t e = trans == 0 ? tc_gemm<false>(a, 1, EpiStoreB{C_dev, ldc, N}, st)
                               : tc_gemm<true>(a, 1, EpiStoreB{C_dev, ldc, N}, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? FBSDE_OK : FBSDE_ERR_CUDA;
}
