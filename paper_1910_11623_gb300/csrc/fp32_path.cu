// FP32 form of the network sweeps (CUDA-core FP32 GEMMs, accurate
// transcendental functions, every per-layer tensor kept in HBM).
//
// For the points p = n M + m (all paths, all times) with inputs u = (t_n, X_n):
//   forward  (Section 2.2, 3.1):  a_0 = W_in u + b_in, h_0 = act(a_0);
//            a_l = W_l h_{l-1} + b_l (+ B_l u, NAIS), h_l = s h_{l-1} + c act(a_l);
//            Y = w_o^T h_L + b_o
//   Z-reverse (Z = grad_x u):     g_L = w_o, e_l = c act'(a_l) g_l,
//            g_{l-1} = s g_l + W_l^T e_l, Z = W_in[:,1:]^T e_0 (+ sum_l B_l[:,1:]^T e_l)
//   tangent along u' = (0, v):    a'_0 = W_in u', h'_0 = act'(a_0) a'_0,
//            a'_l = W_l h'_{l-1} (+ B_l u'), h'_l = s h'_{l-1} + c act'(a_l) a'_l,
//            S_l = c act''(a_l) a'_l g_l
//   adjoint of sum_p alpha_p y_p + v_p^T Z_p:
//            hbar_L = alpha w_o, abar_l = c act'(a_l) hbar_l + S_l,
//            hbar_{l-1} = s hbar_l + W_l^T abar_l
//   weights: dW_l = sum_p abar_l h_{l-1}^T + e_l h'_{l-1}^T, db_l = sum_p abar_l, ...
// (s, c) = (0, 1) for FC and the lift, (1, 1) for ResNet, (1, h) for NAIS.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "simt_gemm.cuh"

namespace fbsde {

// Matrix acting on h in layer l >= 1: W_l, or the NAIS A_l formed per call.
static inline const float* layer_matrix(const fbsde_ctx* c, const float* theta, int l) {
    return c->akind == FBSDE_NAIS ? c->Amat[l] : theta + c->pl.W[l];
}

// ---------------------------------------------------------------- epilogues

struct EpiFwd {  // a = acc + bias + t * tcol; h = s hprev + c act(a)
    const float* bias; const float* tcol; const float* hprev;
    float s, c; float* aout; float* hout;
    int w, K0, M; float dt; int act;
    __device__ void operator()(int row, int col, float acc, int) const {
        float a = acc + bias[col];
        if (tcol) a += (float)(row / M) * dt * tcol[(size_t)col * K0];
        const size_t i = (size_t)row * w + col;
        aout[i] = a;
        const float f = act3_accurate(act, a).f;
        hout[i] = (hprev ? s * hprev[i] : 0.f) + c * f;
    }
};

struct EpiRev {  // g = s g_l + acc; e = c_prev act'(a_prev) g
    const float* gl; float s; const float* aprev; float cprev;
    float* gout; float* eout; int w; int act;
    __device__ void operator()(int row, int col, float acc, int) const {
        const size_t i = (size_t)row * w + col;
        const float g = s * gl[i] + acc;
        gout[i] = g;
        eout[i] = cprev * act3_accurate(act, aprev[i]).d1 * g;
    }
};

struct EpiStore {
    float* out; int ld;
    __device__ void operator()(int row, int col, float acc, int) const {
        out[(size_t)row * ld + col] = acc;
    }
};

struct EpiTan {  // h' = s h'_prev + c act'(a) a'; S = c act''(a) a' g
    const float* a; const float* hdprev; const float* g; float s, c;
    float* hdout; float* sout; int w; int act;
    __device__ void operator()(int row, int col, float acc, int) const {
        const size_t i = (size_t)row * w + col;
        const Act3 f = act3_accurate(act, a[i]);
        hdout[i] = (hdprev ? s * hdprev[i] : 0.f) + c * f.d1 * acc;
        sout[i] = c * f.d2 * acc * g[i];
    }
};

struct EpiAdj {  // hbar = s hbar_l + acc; abar_prev = c_prev act'(a_prev) hbar + S_prev
    const float* hbl; float s; const float* aprev; const float* sprev; float cprev;
    float* hbout; float* about; int w; int act;
    __device__ void operator()(int row, int col, float acc, int) const {
        const size_t i = (size_t)row * w + col;
        const float hb = s * hbl[i] + acc;
        hbout[i] = hb;
        about[i] = cprev * act3_accurate(act, aprev[i]).d1 * hb + sprev[i];
    }
};

struct EpiPartial {  // split-K partial sums part[z][row][col]
    float* part; int rows, cols;
    __device__ void operator()(int row, int col, float acc, int z) const {
        part[((size_t)z * rows + row) * cols + col] = acc;
    }
};

// ---------------------------------------------------------------- small kernels

// g_L = w_o (broadcast), e_L = c_L act'(a_L) w_o
__global__ void k_top_rev(size_t P, int w, const float* __restrict__ aL, const float* __restrict__ wo,
                          float cL, int act, float* __restrict__ gL, float* __restrict__ eL) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * w) return;
    const int j = (int)(i % w);
    gL[i] = wo[j];
    eL[i] = cL * act3_accurate(act, aL[i]).d1 * wo[j];
}

// hbar_L = alpha w_o, abar_L = c_L act'(a_L) hbar_L + S_L
__global__ void k_top_adj(size_t P, int w, const float* __restrict__ aL, const float* __restrict__ wo,
                          const float* __restrict__ alpha, const float* __restrict__ SL, float cL,
                          int act, float* __restrict__ hbL, float* __restrict__ abL) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * w) return;
    const int j = (int)(i % w);
    const float hb = alpha[i / w] * wo[j];
    hbL[i] = hb;
    abL[i] = cL * act3_accurate(act, aL[i]).d1 * hb + SL[i];
}

// y_p = w_o^T h_L(p) + b_o, one warp per point
__global__ void k_rowdot(size_t P, int w, const float* __restrict__ h, const float* __restrict__ wo,
                         const float* __restrict__ bo, float* __restrict__ y) {
    const size_t p = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= P) return;
    float s = 0.f;
    for (int j = lane; j < w; j += 32) s = fmaf(h[p * w + j], wo[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[p] = s + bo[0];
}

// out[r * ld + off + (c - c0)] = sum_z part[z][r][c], c in [c0, c0 + nc), fixed order
__global__ void k_reduce_part(const float* __restrict__ part, int splits, int rows, int cols,
                              int c0, int nc, float* __restrict__ out, int ld, int off) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * nc) return;
    const int r = i / nc, c = c0 + i % nc;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[((size_t)z * rows + r) * cols + c];
    out[(size_t)r * ld + off + (c - c0)] = s;
}

__global__ void k_ones_t(size_t P, int M, float dt, float* __restrict__ ot) {
    size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    ot[2 * p] = 1.f;
    ot[2 * p + 1] = (float)(p / M) * dt;
}




// w x w products of every NAIS-Net block in one launch (blockIdx.z = block
// l - 1), 32 x 32 outputs per CTA, each of the 256 threads 2 x 2 of them:
//   MODE 0: C_l = -X_l^T Y_l - eps I   (A_l = -R_l^T R_l - eps I)
//   MODE 1: C_l =  X_l^T Y_l           (R_l^T R_l for the projection)
//   MODE 2: C_l = -X_l (Y_l + Y_l^T)   (d loss / d R_l = -R_l (dA_l + dA_l^T))
struct WxwArgs {
    const float* X[kMaxDepth + 1];
    const float* Y[kMaxDepth + 1];
    float* C[kMaxDepth + 1];
    int w;
};

template <int MODE>
__global__ void __launch_bounds__(256) k_wxw(const WxwArgs a, float eps) {
    const int l = blockIdx.z + 1, w = a.w;
    const float* __restrict__ X = a.X[l];
    const float* __restrict__ Y = a.Y[l];
    __shared__ float xs[32][33];  // xs[k][m]
    __shared__ float ys[32][33];  // ys[k][n]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < w; k0 += 32) {
        for (int i = threadIdx.x; i < 1024; i += 256) {
            const int r = i >> 5, q = i & 31;
            if (MODE == 2) {  // X[m][k]
                const int m = m0 + r, k = k0 + q;
                xs[q][r] = (m < w && k < w) ? X[(size_t)m * w + k] : 0.f;
            } else {          // X[k][m]
                const int k = k0 + r, m = m0 + q;
                xs[r][q] = (m < w && k < w) ? X[(size_t)k * w + m] : 0.f;
            }
            const int k = k0 + r, n = n0 + q;
            float yv = 0.f;
            if (k < w && n < w) {
                yv = Y[(size_t)k * w + n];
                if (MODE == 2) yv += Y[(size_t)n * w + k];
            }
            ys[r][q] = yv;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float x0 = xs[kk][ty * 2], x1 = xs[kk][ty * 2 + 1];
            const float y0 = ys[kk][tx * 2], y1 = ys[kk][tx * 2 + 1];
            acc[0][0] = fmaf(x0, y0, acc[0][0]);
            acc[0][1] = fmaf(x0, y1, acc[0][1]);
            acc[1][0] = fmaf(x1, y0, acc[1][0]);
            acc[1][1] = fmaf(x1, y1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int m = m0 + ty * 2 + i, n = n0 + tx * 2 + j;
            if (m >= w || n >= w) continue;
            float v = acc[i][j];
            if (MODE == 0) v = -v - (m == n ? eps : 0.f);
            if (MODE == 2) v = -v;
            a.C[l][(size_t)m * w + n] = v;
        }
}

// Per block l (one CTA each): ||C_l||_F^2 in a fixed order, then
// scale[l] = sqrt(delta / ||C_l||_F) if the norm exceeds delta, else 1.
__global__ void k_proj_scales(int n, const WxwArgs a, float delta, float* __restrict__ scale) {
    const int l = blockIdx.x + 1;
    const float* __restrict__ G = a.C[l];
    __shared__ double sh[1024];
    float part = 0.f;  // a thread's n / 1024 squares in FP32, the tree in FP64
    for (int i = threadIdx.x; i < n; i += blockDim.x) part = fmaf(G[i], G[i], part);
    sh[threadIdx.x] = (double)part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nrm = sqrt(sh[0]);
        scale[l] = nrm > (double)delta ? (float)sqrt((double)delta / nrm) : 1.f;
    }
}

// R_l *= scale[l] for every block (blockIdx.y = l - 1); R_l passed in Y.
__global__ void k_scale_blocks(int n, const WxwArgs a, const float* __restrict__ scale) {
    const int l = blockIdx.y + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) const_cast<float*>(a.Y[l])[i] *= scale[l];
}

__global__ void k_check_finite(size_t n, const float* __restrict__ x, int* __restrict__ flag) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(x[i])) *flag = 1;
}

static inline unsigned nblk(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Algorithmic flops of a contraction: 2 per multiply-add over every pair.
static double gemm_flops(const GemmArgs& g) {
    double f = 0;
    for (int q = 0; q < g.npairs; ++q) f += 2.0 * g.Mrows * (double)g.Ncols * g.pair[q].K;
    return f;
}

#define GEMM_LAUNCH(c, cls, AT, BKN, g, splits, epi)                                    \
    do {                                                                                \
        int tok_ = prof_begin((c), (cls));                                              \
        cudaError_t e_ = simt_gemm<AT, BKN>((g), (splits), (epi), (c)->stream);          \
        prof_end((c), (cls), tok_, gemm_flops(g));                                      \
        if (e_ != cudaSuccess) return set_err((c), FBSDE_ERR_CUDA, cudaGetErrorString(e_)); \
        ++(c)->n_launch;                                                                \
    } while (0)

// ---------------------------------------------------------------- workspace

size_t fp32_workspace_floats(const fbsde_ctx* c) {
    return (size_t)8 * (c->L + 1) * c->Pmax() * c->w;
}

void fp32_carve(fbsde_ctx* c, float*& cur) {
    const size_t n = c->Pmax() * c->w;
    for (int l = 0; l <= c->L; ++l) {
        c->f32.A[l] = cur; cur += n;
        c->f32.H[l] = cur; cur += n;
        c->f32.E[l] = cur; cur += n;
        c->f32.G[l] = cur; cur += n;
        c->f32.HD[l] = cur; cur += n;
        c->f32.S[l] = cur; cur += n;
        c->f32.AB[l] = cur; cur += n;
        c->f32.HB[l] = cur; cur += n;
    }
}

static fbsde_status launch_wxw(fbsde_ctx* c, int mode, const WxwArgs& a, int cls) {
    const int w = c->w, nt = (w + 31) / 32;
    if (c->L < 1) return FBSDE_OK;
    const dim3 grid(nt, nt, c->L);
    const int tok = prof_begin(c, cls);
    if (mode == 0) k_wxw<0><<<grid, 256, 0, c->stream>>>(a, (float)c->eps);
    else if (mode == 1) k_wxw<1><<<grid, 256, 0, c->stream>>>(a, 0.f);
    else k_wxw<2><<<grid, 256, 0, c->stream>>>(a, 0.f);
    prof_end(c, cls, tok, 2.0 * w * (double)w * w * c->L);
    FBSDE_CK_LAUNCH(c);
    return FBSDE_OK;
}

// NAIS: A_l = -R_l^T R_l - eps I for every block (Section 3.1), one launch.
static fbsde_status form_nais_A(fbsde_ctx* c, const float* theta) {
    WxwArgs a{};
    a.w = c->w;
    for (int l = 1; l <= c->L; ++l) {
        a.X[l] = a.Y[l] = theta + c->pl.W[l];
        a.C[l] = c->Amat[l];
    }
    return launch_wxw(c, 0, a, PROF_OTHER);
}

fbsde_status fp32_prepare_weights(fbsde_ctx* c, const float* theta) {
    if (c->akind == FBSDE_NAIS) FBSDE_TRY(form_nais_A(c, theta));
    return FBSDE_OK;
}

// Split-K plan for a K = P contraction with an (rows x cols) output.
static void splitk_plan(size_t K, int rows, int cols, int& splits, int& kchunk, size_t part_cap) {
    const int tiles = ((rows + 127) / 128) * ((cols + 127) / 128);
    int want = (2 * 152 + tiles - 1) / tiles;
    want = want < 1 ? 1 : (want > 512 ? 512 : want);
    size_t kc = (K + want - 1) / want;
    kc = (kc + 7) / 8 * 8;
    if (kc < 8) kc = 8;
    splits = (int)((K + kc - 1) / kc);
    while ((size_t)splits * rows * cols > part_cap) {  // never exceed the partial buffer
        kc *= 2;
        splits = (int)((K + kc - 1) / kc);
    }
    kchunk = (int)kc;
}

// out[r * ld + off + j] = sum_p sum_pairs A(p, r) B(p, c0 + j) for j < nc.
static fbsde_status tn_reduce(fbsde_ctx* c, GemmArgs g, int c0, int nc, float* out, int ld, int off) {
    int splits, kchunk;
    splitk_plan((size_t)g.pair[0].K, g.Mrows, g.Ncols, splits, kchunk, c->part_floats);
    g.kchunk = kchunk;
    GEMM_LAUNCH(c, PROF_WGRAD, true, true, g, splits, (EpiPartial{c->part, g.Mrows, g.Ncols}));
    k_reduce_part<<<nblk((size_t)g.Mrows * nc, 256), 256, 0, c->stream>>>(
        c->part, splits, g.Mrows, g.Ncols, c0, nc, out, ld, off);
    FBSDE_CK_LAUNCH(c);
    return FBSDE_OK;
}

// ---------------------------------------------------------------- shared with the BF16 form

fbsde_status launch_rowdot(fbsde_ctx* c, const float* h, const float* theta, float* y) {
    const size_t P = c->P();
    k_rowdot<<<nblk(P * 32, 256), 256, 0, c->stream>>>(P, c->w, h, theta + c->pl.wo, theta + c->pl.bo, y);
    FBSDE_CK_LAUNCH(c);
    return FBSDE_OK;
}

// d loss / d R_l = -R_l (dA_l + dA_l^T) from the gradients dA_l in c->gA[l],
// every block in one launch.
fbsde_status nais_chain_R(fbsde_ctx* c, const float* theta, float* grad) {
    WxwArgs a{};
    a.w = c->w;
    for (int l = 1; l <= c->L; ++l) {
        a.X[l] = theta + c->pl.W[l];
        a.Y[l] = c->gA[l];
        a.C[l] = grad + c->pl.W[l];
    }
    return launch_wxw(c, 2, a, PROF_WGRAD);
}

fbsde_status launch_check_finite(fbsde_ctx* c, const float* x, size_t n) {
    k_check_finite<<<nblk(n, 256), 256, 0, c->stream>>>(n, x, c->nonfinite);
    FBSDE_CK_LAUNCH(c);
    return FBSDE_OK;
}

// ---------------------------------------------------------------- forward

fbsde_status fp32_forward(fbsde_ctx* c, const float* theta) {
    const int w = c->w, L = c->L, D = c->D, K0 = D + 1, act = c->act;
    const size_t P = c->P();
    const ParamLayout& pl = c->pl;
    const float dt = (float)(c->T / c->N);
    Fp32Work& f = c->f32;
    cudaStream_t st = c->stream;
    const int NOSPLIT = 1 << 30;

    // lift: a_0 = W_in[:,1:] x + t W_in[:,0] + b_in
    {
        GemmArgs g{};
        g.npairs = 1; g.Mrows = (int)P; g.Ncols = w; g.kchunk = NOSPLIT;
        g.pair[0] = {c->X, theta + pl.Win + 1, D, D, K0};
        EpiFwd e{theta + pl.bin, theta + pl.Win, nullptr, 0.f, 1.f, f.A[0], f.H[0], w, K0, c->M, dt, act};
        GEMM_LAUNCH(c, PROF_POINTS, false, false, g, 1, (e));
    }
    for (int l = 1; l <= L; ++l) {
        GemmArgs g{};
        g.Mrows = (int)P; g.Ncols = w; g.kchunk = NOSPLIT;
        g.pair[0] = {f.H[l - 1], layer_matrix(c, theta, l), w, w, w};
        g.npairs = 1;
        const float* tcol = nullptr;
        if (c->akind == FBSDE_NAIS) {
            g.pair[1] = {c->X, theta + pl.B[l] + 1, D, D, K0};
            g.npairs = 2;
            tcol = theta + pl.B[l];
        }
        EpiFwd e{theta + pl.b[l], tcol, f.H[l - 1], layer_skip(c, l), layer_scale(c, l),
                 f.A[l], f.H[l], w, K0, c->M, dt, act};
        GEMM_LAUNCH(c, PROF_POINTS, false, false, g, 1, (e));
    }
    // Y = w_o^T h_L + b_o
    k_rowdot<<<nblk(P * 32, 256), 256, 0, st>>>(P, w, f.H[L], theta + pl.wo, theta + pl.bo, c->Y);
    FBSDE_CK_LAUNCH(c);

    // Z-reverse
    k_top_rev<<<nblk(P * w, 256), 256, 0, st>>>(P, w, f.A[L], theta + pl.wo, layer_scale(c, L), act,
                                                f.G[L], f.E[L]);
    FBSDE_CK_LAUNCH(c);
    for (int l = L; l >= 1; --l) {
        GemmArgs g{};
        g.npairs = 1; g.Mrows = (int)P; g.Ncols = w; g.kchunk = NOSPLIT;
        g.pair[0] = {f.E[l], layer_matrix(c, theta, l), w, w, w};
        EpiRev e{f.G[l], layer_skip(c, l), f.A[l - 1], layer_scale(c, l - 1), f.G[l - 1], f.E[l - 1], w, act};
        GEMM_LAUNCH(c, PROF_POINTS, false, true, g, 1, (e));
    }
    // Z = W_in[:,1:]^T e_0 + sum_l B_l[:,1:]^T e_l
    {
        GemmArgs g{};
        g.Mrows = (int)P; g.Ncols = D; g.kchunk = NOSPLIT;
        g.pair[0] = {f.E[0], theta + pl.Win + 1, w, w, K0};
        g.npairs = 1;
        if (c->akind == FBSDE_NAIS)
            for (int l = 1; l <= L; ++l) g.pair[g.npairs++] = {f.E[l], theta + pl.B[l] + 1, w, w, K0};
        GEMM_LAUNCH(c, PROF_POINTS, false, true, g, 1, (EpiStore{c->Z, D}));
    }
    return FBSDE_OK;
}

// ---------------------------------------------------------------- backward

fbsde_status fp32_backward(fbsde_ctx* c, const float* theta, float* grad) {
    const int w = c->w, L = c->L, D = c->D, K0 = D + 1, act = c->act;
    const size_t P = c->P();
    const ParamLayout& pl = c->pl;
    Fp32Work& f = c->f32;
    cudaStream_t st = c->stream;
    const int NOSPLIT = 1 << 30;
    const float dt = (float)(c->T / c->N);

    k_ones_t<<<nblk(P, 256), 256, 0, st>>>(P, c->M, dt, c->ones_t);
    FBSDE_CK_LAUNCH(c);

    // tangent sweep along u' = (0, v)
    {
        GemmArgs g{};
        g.npairs = 1; g.Mrows = (int)P; g.Ncols = w; g.kchunk = NOSPLIT;
        g.pair[0] = {c->V, theta + pl.Win + 1, D, D, K0};
        EpiTan e{f.A[0], nullptr, f.G[0], 0.f, 1.f, f.HD[0], f.S[0], w, act};
        GEMM_LAUNCH(c, PROF_POINTS, false, false, g, 1, (e));
    }
    for (int l = 1; l <= L; ++l) {
        GemmArgs g{};
        g.Mrows = (int)P; g.Ncols = w; g.kchunk = NOSPLIT;
        g.pair[0] = {f.HD[l - 1], layer_matrix(c, theta, l), w, w, w};
        g.npairs = 1;
        if (c->akind == FBSDE_NAIS) { g.pair[1] = {c->V, theta + pl.B[l] + 1, D, D, K0}; g.npairs = 2; }
        EpiTan e{f.A[l], f.HD[l - 1], f.G[l], layer_skip(c, l), layer_scale(c, l), f.HD[l], f.S[l], w, act};
        GEMM_LAUNCH(c, PROF_POINTS, false, false, g, 1, (e));
    }
    // adjoint sweep
    k_top_adj<<<nblk(P * w, 256), 256, 0, st>>>(P, w, f.A[L], theta + pl.wo, c->alpha, f.S[L],
                                                layer_scale(c, L), act, f.HB[L], f.AB[L]);
    FBSDE_CK_LAUNCH(c);
    for (int l = L; l >= 1; --l) {
        GemmArgs g{};
        g.npairs = 1; g.Mrows = (int)P; g.Ncols = w; g.kchunk = NOSPLIT;
        g.pair[0] = {f.AB[l], layer_matrix(c, theta, l), w, w, w};
        EpiAdj e{f.HB[l], layer_skip(c, l), f.A[l - 1], f.S[l - 1], layer_scale(c, l - 1), f.HB[l - 1],
                 f.AB[l - 1], w, act};
        GEMM_LAUNCH(c, PROF_POINTS, false, true, g, 1, (e));
    }

    // weight gradients (contractions over all points)
    const int Pi = (int)P;
    for (int l = 1; l <= L; ++l) {
        GemmArgs g{};
        g.npairs = 2; g.Mrows = w; g.Ncols = w;
        g.pair[0] = {f.AB[l], f.H[l - 1], Pi, w, w};
        g.pair[1] = {f.E[l], f.HD[l - 1], Pi, w, w};
        float* dst = (c->akind == FBSDE_NAIS) ? c->gA[l] : grad + pl.W[l];
        FBSDE_TRY(tn_reduce(c, g, 0, w, dst, w, 0));
        // bias (and NAIS t-column of B_l) from (1, t) per point
        GemmArgs gb{};
        gb.npairs = 1; gb.Mrows = w; gb.Ncols = 2;
        gb.pair[0] = {f.AB[l], c->ones_t, Pi, w, 2};
        FBSDE_TRY(tn_reduce(c, gb, 0, 1, grad + pl.b[l], 1, 0));
        if (c->akind == FBSDE_NAIS) {
            FBSDE_TRY(tn_reduce(c, gb, 1, 1, grad + pl.B[l], K0, 0));
            GemmArgs gx{};
            gx.npairs = 2; gx.Mrows = w; gx.Ncols = D;
            gx.pair[0] = {f.AB[l], c->X, Pi, w, D};
            gx.pair[1] = {f.E[l], c->V, Pi, w, D};
            FBSDE_TRY(tn_reduce(c, gx, 0, D, grad + pl.B[l], K0, 1));
        }
    }
    if (c->akind == FBSDE_NAIS) FBSDE_TRY(nais_chain_R(c, theta, grad));  // dR = -R (dA + dA^T)
    {
        GemmArgs g{};
        g.npairs = 2; g.Mrows = w; g.Ncols = D;
        g.pair[0] = {f.AB[0], c->X, Pi, w, D};
        g.pair[1] = {f.E[0], c->V, Pi, w, D};
        FBSDE_TRY(tn_reduce(c, g, 0, D, grad + pl.Win, K0, 1));
        GemmArgs gb{};
        gb.npairs = 1; gb.Mrows = w; gb.Ncols = 2;
        gb.pair[0] = {f.AB[0], c->ones_t, Pi, w, 2};
        FBSDE_TRY(tn_reduce(c, gb, 0, 1, grad + pl.bin, 1, 0));
        FBSDE_TRY(tn_reduce(c, gb, 1, 1, grad + pl.Win, K0, 0));
    }
    {
        // dw_o = sum_p alpha_p h_L(p) + h'_L(p);  db_o = sum_p alpha_p
        GemmArgs g{};
        g.npairs = 2; g.Mrows = w; g.Ncols = 1;
        g.pair[0] = {f.H[L], c->alpha, Pi, w, 1};
        g.pair[1] = {f.HD[L], c->ones_t, Pi, w, 2};
        FBSDE_TRY(tn_reduce(c, g, 0, 1, grad + pl.wo, 1, 0));
        // db_o = sum_p alpha_p, formed with the loss (k_loss_reduce)
        FBSDE_CK(c, cudaMemcpyAsync(grad + pl.bo, c->alpha_sum, sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    k_check_finite<<<nblk(pl.total, 256), 256, 0, st>>>(pl.total, grad, c->nonfinite);
    FBSDE_CK_LAUNCH(c);
    return FBSDE_OK;
}

// ---------------------------------------------------------------- NAIS projection

// After an update: if ||R_l^T R_l||_F > delta, R_l *= sqrt(delta / ||R_l^T R_l||_F)
// (Section 3.1: projection onto the feasible set of the Frobenius-norm bound).
fbsde_status nais_project(fbsde_ctx* c, float* theta) {
    const int w = c->w, L = c->L;
    if (L < 1) return FBSDE_OK;
    // S_l = R_l^T R_l into the dA_l buffers (free once the update is done)
    WxwArgs a{};
    a.w = w;
    for (int l = 1; l <= L; ++l) {
        a.X[l] = a.Y[l] = theta + c->pl.W[l];
        a.C[l] = c->gA[l];
    }
    FBSDE_TRY(launch_wxw(c, 1, a, PROF_OTHER));
    k_proj_scales<<<L, 1024, 0, c->stream>>>(w * w, a, (float)c->delta, c->fscal);
    FBSDE_CK_LAUNCH(c);
    k_scale_blocks<<<dim3(nblk((size_t)w * w, 256), L), 256, 0, c->stream>>>(w * w, a, c->fscal);
    FBSDE_CK_LAUNCH(c);
    return FBSDE_OK;
}

}  // namespace fbsde
