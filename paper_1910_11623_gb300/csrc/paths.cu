// Steps of the hot path shared by both arithmetic forms:
//   - Brownian increments and the forward Euler-Maruyama paths
//     (Section 2.2, Eq. "disc equations", lines 1-2);
//   - Xavier parameter initialisation from Philox;
//   - the Y-residuals, loss and loss seeds alpha = dL/dY_n, v = dL/dZ_n
//     (Section 2.2, Eq. "loss"), with a fixed-order loss reduction.
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "philox.cuh"

namespace fbsde {

// One thread per (path m, dimension quad q): walks the N steps of its path,
// drawing Delta W_n from Philox counter (q, n, m, iter) and updating
// X_{n+1} = X_n + sigma(X_n) Delta W_n.  Layout: row n * M + m, column d.
// With D a multiple of 4 a quad's row pieces are written as single 16-byte
// (FP32) and 8-byte (BF16) stores.
__global__ void k_paths(ProblemDev pd, const float* __restrict__ x0, uint32_t k0, uint32_t k1,
                        uint32_t it_host, const uint64_t* __restrict__ it_dev, float* __restrict__ X,
                        float* __restrict__ dW, __nv_bfloat16* __restrict__ Xb, int ldb) {
    const uint32_t it = it_dev ? (uint32_t)*it_dev : it_host;
    const int Q = (pd.D + 3) >> 2;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)pd.M * Q) return;
    const int m = (int)(idx / Q), q = (int)(idx % Q);
    const int d0 = 4 * q;
    const int nd = min(4, pd.D - d0);
    const bool vec = (pd.D & 3) == 0 && (ldb & 3) == 0;
    float x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = (j < nd) ? x0[d0 + j] : 0.f;
    auto put = [&](float* frow, __nv_bfloat16* brow, const float* v) {
        if (vec) {
            if (frow) *reinterpret_cast<float4*>(frow) = make_float4(v[0], v[1], v[2], v[3]);
            if (brow) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
                uint2 u;
                u.x = *reinterpret_cast<uint32_t*>(&lo);
                u.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(brow) = u;
            }
        } else {
            if (frow)
                for (int j = 0; j < nd; ++j) frow[j] = v[j];
            if (brow)
                for (int j = 0; j < nd; ++j) brow[j] = __float2bfloat16_rn(v[j]);
        }
    };
    put(X ? X + (size_t)m * pd.D + d0 : nullptr, Xb ? Xb + (size_t)m * ldb + d0 : nullptr, x);
    const float sqrt2 = 1.41421356237309515f;
    // the draws of later steps do not depend on X: unrolled, their Philox
    // rounds overlap the X updates and stores of earlier ones
#pragma unroll 4
    for (int n = 0; n < pd.N; ++n) {
        u32x4 c{(uint32_t)q, (uint32_t)n, (uint32_t)m, it};
        u32x4 w = philox4x32_10(c, k0, k1);
        float z[4];
        box_muller(w.x, w.y, z[0], z[1]);
        box_muller(w.z, w.w, z[2], z[3]);
        float dw[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            dw[j] = pd.sqrt_dt * z[j];
            if (pd.kind == FBSDE_BSB) x[j] = x[j] + (pd.sigma * x[j]) * dw[j];
            else                      x[j] = x[j] + sqrt2 * dw[j];
        }
        put(dW ? dW + ((size_t)n * pd.M + m) * pd.D + d0 : nullptr, nullptr, dw);
        put(X ? X + ((size_t)(n + 1) * pd.M + m) * pd.D + d0 : nullptr,
            Xb ? Xb + ((size_t)(n + 1) * pd.M + m) * ldb + d0 : nullptr, x);
    }
}

fbsde_status launch_paths(fbsde_ctx* ctx, uint64_t iter) {
    ProblemDev pd = ctx->pdev();
    const int Q = (ctx->D + 3) / 4;
    const long n = (long)ctx->M * Q;
    const int bs = 128;
    const int tok = prof_begin(ctx, PROF_OTHER);
    k_paths<<<(unsigned)((n + bs - 1) / bs), bs, 0, ctx->stream>>>(
        pd, ctx->x0_dev, (uint32_t)ctx->seed, (uint32_t)(ctx->seed >> 32), (uint32_t)iter, ctx->step_dev,
        ctx->X, ctx->dW, ctx->Xb_op, ctx->ld_op);
    prof_end(ctx, PROF_OTHER, tok, 0.0);
    FBSDE_CK_LAUNCH(ctx);
    return FBSDE_OK;
}

// ---------------------------------------------------------------- Philox entry

__global__ void k_philox_blocks(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                                size_t count, uint32_t* __restrict__ out) {
    size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    u32x4 c{ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3]};
    u32x4 w = philox4x32_10(c, k0, k1);
    out[4 * j] = w.x; out[4 * j + 1] = w.y; out[4 * j + 2] = w.z; out[4 * j + 3] = w.w;
}

cudaError_t philox_blocks(const uint32_t* ctr, uint32_t k0, uint32_t k1, size_t count,
                          uint32_t* out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_philox_blocks<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(ctr, k0, k1, count, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- init

// theta[off + i] = std * z(off + i) with z(j) the Box-Muller normal of Philox
// block (j >> 2, 0, 0, 0) under the init key, slot j & 3.
__global__ void k_init_segment(float* __restrict__ theta, size_t off, size_t count, float std_,
                               uint32_t k0, uint32_t k1) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    size_t j = off + i;
    u32x4 c{(uint32_t)(j >> 2), 0u, 0u, 0u};
    u32x4 w = philox4x32_10(c, k0, k1);
    float z[4];
    box_muller(w.x, w.y, z[0], z[1]);
    box_muller(w.z, w.w, z[2], z[3]);
    theta[j] = std_ * z[j & 3];
}

fbsde_status launch_init(fbsde_ctx* ctx, float* theta) {
    const ParamLayout& pl = ctx->pl;
    const int w = ctx->w, Din = ctx->D + 1;
    FBSDE_CK(ctx, cudaMemsetAsync(theta, 0, pl.total * sizeof(float), ctx->stream));
    const uint32_t k0 = (uint32_t)ctx->seed ^ 0x494E4954u, k1 = (uint32_t)(ctx->seed >> 32);
    auto seg = [&](size_t off, size_t count, int fan_in, int fan_out) -> fbsde_status {
        float sd = (float)std::sqrt(2.0 / (double)(fan_in + fan_out));
        k_init_segment<<<(unsigned)((count + 255) / 256), 256, 0, ctx->stream>>>(theta, off, count,
                                                                                  sd, k0, k1);
        FBSDE_CK_LAUNCH(ctx);
        return FBSDE_OK;
    };
    FBSDE_TRY(seg(pl.Win, (size_t)w * Din, Din, w));
    for (int l = 1; l <= ctx->L; ++l) {
        FBSDE_TRY(seg(pl.W[l], (size_t)w * w, w, w));
        if (ctx->akind == FBSDE_NAIS) FBSDE_TRY(seg(pl.B[l], (size_t)w * Din, Din, w));
    }
    FBSDE_TRY(seg(pl.wo, (size_t)w, w, 1));
    if (ctx->akind == FBSDE_NAIS) FBSDE_TRY(nais_project(ctx, theta));
    return FBSDE_OK;
}

// ---------------------------------------------------------------- seeds and loss

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per path m walks n = 0..N:
//   r_n   = Y_{n+1} - Y_n - phi(X_n, Y_n, Z_n) dt - Z_n^T sigma(X_n) dW_n      (n < N)
//   r_T   = Y_N - g(X_N)
//   alpha = 2 r_{n-1} [n >= 1] - 2 r_n (1 + phi_y dt) [n < N] + 2 r_T [n = N]
//   v     = -2 r_n (phi_z dt + sigma(X_n) dW_n) [n < N] + 2 (Z_N - grad g) [n = N, term on]
// and the per-path loss sum_n r_n^2 + r_T^2 (+ |Z_N - grad g|^2), accumulated in FP64.
// Serves fbsde_residual_loss_noalloc, whose caller passes the increments.
__global__ void k_seeds(ProblemDev pd, const float* __restrict__ X, const float* __restrict__ dW,
                        const float* __restrict__ Y, const float* __restrict__ Z,
                        float* __restrict__ alpha, float* __restrict__ V,
                        double* __restrict__ path_loss, __nv_bfloat16* __restrict__ Vb, int ldb) {
    const int lane = threadIdx.x & 31;
    const int m = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (m >= pd.M) return;
    const int D = pd.D;
    const bool bsb = pd.kind == FBSDE_BSB;
    const float sqrt2 = 1.41421356237309515f;
    double pl = 0.0;
    float rprev = 0.f;
    for (int n = 0; n < pd.N; ++n) {
        const size_t p = (size_t)n * pd.M + m;
        const float* x = X + p * D;
        const float* z = Z + p * D;
        const float* dw = dW + p * D;
        float zx = 0.f, zsdw = 0.f, zz = 0.f;
        for (int d = lane; d < D; d += 32) {
            const float sdw = bsb ? pd.sigma * x[d] * dw[d] : sqrt2 * dw[d];
            zx = fmaf(z[d], x[d], zx);
            zsdw = fmaf(z[d], sdw, zsdw);
            zz = fmaf(z[d], z[d], zz);
        }
        zx = warp_sum(zx); zsdw = warp_sum(zsdw); zz = warp_sum(zz);
        const float yn = Y[p], yn1 = Y[p + pd.M];
        const float phi = bsb ? pd.r * (yn - zx) : zz;
        const float phi_y = bsb ? pd.r : 0.f;
        const float r = yn1 - yn - phi * pd.dt - zsdw;
        pl += (double)r * (double)r;
        if (lane == 0) alpha[p] = (n >= 1 ? 2.f * rprev : 0.f) - 2.f * r * (1.f + phi_y * pd.dt);
        float* vp = V + p * D;
        for (int d = lane; d < D; d += 32) {
            const float sdw = bsb ? pd.sigma * x[d] * dw[d] : sqrt2 * dw[d];
            const float phiz = bsb ? -pd.r * x[d] : 2.f * z[d];
            vp[d] = -2.f * r * (phiz * pd.dt + sdw);
            if (Vb) Vb[p * ldb + d] = __float2bfloat16_rn(vp[d]);
        }
        rprev = r;
    }
    // terminal point n = N
    const size_t p = (size_t)pd.N * pd.M + m;
    const float* x = X + p * D;
    const float* z = Z + p * D;
    float s = 0.f;
    for (int d = lane; d < D; d += 32) s = fmaf(x[d], x[d], s);
    s = warp_sum(s);
    const float g = bsb ? s : logf(0.5f * (1.f + s));
    const float rT = Y[p] - g;
    pl += (double)rT * (double)rT;
    float* vp = V + p * D;
    float zt = 0.f;
    for (int d = lane; d < D; d += 32) {
        float v = 0.f;
        if (pd.tgt) {
            const float gg = bsb ? 2.f * x[d] : 2.f * x[d] / (1.f + s);
            const float diff = z[d] - gg;
            v = 2.f * diff;
            zt = fmaf(diff, diff, zt);
        }
        vp[d] = v;
        if (Vb) Vb[p * ldb + d] = __float2bfloat16_rn(v);
    }
    zt = warp_sum(zt);
    if (pd.tgt) pl += (double)zt;
    if (lane == 0) {
        alpha[p] = (pd.N >= 1 ? 2.f * rprev : 0.f) + 2.f * rT;
        path_loss[m] = pl;
    }
}

// Fixed-order reduction of the per-path losses (one block, so the result is
// bit-reproducible), plus Y_0 = u(0, x0) (all paths start at x0, so it is the
// network value at point 0) and the non-finite flag.
// With path_alpha, the same fixed-order sum of the per-path alpha sums goes
// to *alpha_sum (the gradient in the read-out bias b_o).
__global__ void k_loss_reduce(const double* __restrict__ path_loss, int M,
                              const float* __restrict__ Y, float* __restrict__ loss_out,
                              float* __restrict__ y0_out, int* __restrict__ nonfinite,
                              const double* __restrict__ path_alpha, float* __restrict__ alpha_sum) {
    // strided sums per thread, a fixed butterfly per warp, then the warps'
    // sums in order by warp 0 (the same additions on every call)
    __shared__ double sh[32], sa[32];
    double acc = 0.0, acca = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        acc += path_loss[m];
        if (path_alpha) acca += path_alpha[m];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        acca += __shfl_xor_sync(0xffffffffu, acca, o);
    }
    if (lane == 0) { sh[wid] = acc; sa[wid] = acca; }
    __syncthreads();
    if (wid == 0) {
        const int nw = (int)(blockDim.x >> 5);
        acc = lane < nw ? sh[lane] : 0.0;
        acca = lane < nw ? sa[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
            acca += __shfl_xor_sync(0xffffffffu, acca, o);
        }
        if (lane == 0) {
            const double L = acc;
            if (loss_out) *loss_out = (float)L;
            if (y0_out) *y0_out = Y[0];
            if (path_alpha) *alpha_sum = (float)acca;
            if (!isfinite(L) || !isfinite(Y[0])) *nonfinite = 1;
        }
    }
}

__global__ void k_d2f(int n, const double* __restrict__ in, float* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

fbsde_status copy_path_loss(fbsde_ctx* ctx, float* out) {
    k_d2f<<<(ctx->M + 255) / 256, 256, 0, ctx->stream>>>(ctx->M, ctx->path_loss_d, out);
    FBSDE_CK_LAUNCH(ctx);
    return FBSDE_OK;
}

// One warp per point (n, m), n < N, forms the residual of Eq. "loss"
//   r_n = Y_{n+1} - Y_n - phi(X_n, Y_n, Z_n) dt - Z_n^T sigma(X_n) dW_n
// and the seed v_n = -2 r_n (phi_z dt + sigma(X_n) dW_n), and stores r_n;
// k_seeds_paths then forms alpha_n from r_{n-1} and r_n, the per-path loss
// (FP64, fixed order) and the terminal point.  Lane = dimension quad (16-byte
// loads when D is a multiple of 4).
__global__ void k_resid(ProblemDev pd, const float* __restrict__ X, const float* __restrict__ dW,
                        const float* __restrict__ Y, const float* __restrict__ Z, float* __restrict__ rbuf,
                        float* __restrict__ V, __nv_bfloat16* __restrict__ Vb, int ldb) {
    const int lane = threadIdx.x & 31;
    const long wp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wp >= (long)pd.N * pd.M) return;
    const size_t p = (size_t)wp;  // n * M + m
    const int D = pd.D, Q = (D + 3) >> 2;
    const bool bsb = pd.kind == FBSDE_BSB;
    const bool vec = (D & 3) == 0;
    const float sqrt2 = 1.41421356237309515f;
    const float* x = X + p * D;
    const float* z = Z + p * D;
    const float* w = dW + p * D;
    // Y_n and Y_{n+1} requested with the quads below, not after the sums
    const float yn = Y[p], yn1 = Y[p + pd.M];
    // quad q of this point: x, z and dW of dimensions 4q .. 4q+3 (zero past D)
    auto quad = [&](int q, float (&xv)[4], float (&zv)[4], float (&dw)[4]) {
        const int d0 = 4 * q;
        if (vec) {
            const float4 a = reinterpret_cast<const float4*>(x)[q];
            const float4 b = reinterpret_cast<const float4*>(z)[q];
            const float4 c = reinterpret_cast<const float4*>(w)[q];
            xv[0] = a.x; xv[1] = a.y; xv[2] = a.z; xv[3] = a.w;
            zv[0] = b.x; zv[1] = b.y; zv[2] = b.z; zv[3] = b.w;
            dw[0] = c.x; dw[1] = c.y; dw[2] = c.z; dw[3] = c.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                xv[j] = d0 + j < D ? x[d0 + j] : 0.f;
                zv[j] = d0 + j < D ? z[d0 + j] : 0.f;
                dw[j] = d0 + j < D ? w[d0 + j] : 0.f;
            }
        }
    };
    float zx = 0.f, zsdw = 0.f, zz = 0.f;
    float x0[4], z0[4], w0[4];  // this lane's first quad, kept for the second pass
    for (int q = lane; q < Q; q += 32) {
        float xv[4], zv[4], dw[4];
        quad(q, xv, zv, dw);
        if (q == lane) {
#pragma unroll
            for (int j = 0; j < 4; ++j) { x0[j] = xv[j]; z0[j] = zv[j]; w0[j] = dw[j]; }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // padded dimensions carry x = z = 0
            const float sdw = bsb ? pd.sigma * xv[j] * dw[j] : sqrt2 * dw[j];
            zx = fmaf(zv[j], xv[j], zx);
            zsdw = fmaf(zv[j], sdw, zsdw);
            zz = fmaf(zv[j], zv[j], zz);
        }
    }
    zx = warp_sum(zx); zsdw = warp_sum(zsdw); zz = warp_sum(zz);
    const float phi = bsb ? pd.r * (yn - zx) : zz;
    const float r = yn1 - yn - phi * pd.dt - zsdw;
    if (lane == 0) rbuf[p] = r;
    for (int q = lane; q < Q; q += 32) {
        float xv[4], zv[4], dw[4], v[4];
        if (q == lane) {
#pragma unroll
            for (int j = 0; j < 4; ++j) { xv[j] = x0[j]; zv[j] = z0[j]; dw[j] = w0[j]; }
        } else {
            quad(q, xv, zv, dw);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float sdw = bsb ? pd.sigma * xv[j] * dw[j] : sqrt2 * dw[j];
            const float phiz = bsb ? -pd.r * xv[j] : 2.f * zv[j];
            v[j] = -2.f * r * (phiz * pd.dt + sdw);
        }
        const int d0 = 4 * q;
        if (vec) {
            if (V) reinterpret_cast<float4*>(V + p * D)[q] = make_float4(v[0], v[1], v[2], v[3]);
            if (Vb && (ldb & 3) == 0) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
                uint2 u;
                u.x = *reinterpret_cast<uint32_t*>(&lo);
                u.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(Vb + p * ldb + d0) = u;
            } else if (Vb) {
#pragma unroll
                for (int j = 0; j < 4; ++j) Vb[p * ldb + d0 + j] = __float2bfloat16_rn(v[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (d0 + j < D) {
                    if (V) V[p * D + d0 + j] = v[j];
                    if (Vb) Vb[p * ldb + d0 + j] = __float2bfloat16_rn(v[j]);
                }
        }
    }
}

__global__ void k_seeds_paths(ProblemDev pd, const float* __restrict__ X, const float* __restrict__ Y,
                              const float* __restrict__ Z, const float* __restrict__ rbuf,
                              float* __restrict__ alpha, float* __restrict__ V, double* __restrict__ path_loss,
                              double* __restrict__ path_alpha, __nv_bfloat16* __restrict__ Vb, int ldb) {
    const int lane = threadIdx.x & 31;
    const int m = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (m >= pd.M) return;
    const int D = pd.D;
    const bool bsb = pd.kind == FBSDE_BSB;
    const float phi_y = bsb ? pd.r : 0.f;
    double pl = 0.0, pa = 0.0;
    for (int n = lane; n < pd.N; n += 32) {
        const size_t p = (size_t)n * pd.M + m;
        const float r = rbuf[p];
        pl += (double)r * (double)r;
        const float a = (n >= 1 ? 2.f * rbuf[p - pd.M] : 0.f) - 2.f * r * (1.f + phi_y * pd.dt);
        alpha[p] = a;
        pa += (double)a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pl += __shfl_xor_sync(0xffffffffu, pl, o);
        pa += __shfl_xor_sync(0xffffffffu, pa, o);
    }
    const float rprev = pd.N >= 1 ? rbuf[(size_t)(pd.N - 1) * pd.M + m] : 0.f;
    // terminal point n = N
    const size_t p = (size_t)pd.N * pd.M + m;
    const float* x = X + p * D;
    const float* z = Z + p * D;
    float s = 0.f;
    for (int d = lane; d < D; d += 32) s = fmaf(x[d], x[d], s);
    s = warp_sum(s);
    const float g = bsb ? s : logf(0.5f * (1.f + s));
    const float rT = Y[p] - g;
    pl += (double)rT * (double)rT;
    float zt = 0.f;
    for (int d = lane; d < D; d += 32) {
        float v = 0.f;
        if (pd.tgt) {
            const float gg = bsb ? 2.f * x[d] : 2.f * x[d] / (1.f + s);
            const float diff = z[d] - gg;
            v = 2.f * diff;
            zt = fmaf(diff, diff, zt);
        }
        if (V) V[p * D + d] = v;
        if (Vb) Vb[p * ldb + d] = __float2bfloat16_rn(v);
    }
    zt = warp_sum(zt);
    if (pd.tgt) pl += (double)zt;
    if (lane == 0) {
        const float a = (pd.N >= 1 ? 2.f * rprev : 0.f) + 2.f * rT;
        alpha[p] = a;
        path_loss[m] = pl;
        path_alpha[m] = pa + (double)a;
    }
}

fbsde_status launch_seeds(fbsde_ctx* ctx, float* loss_dev, float* y0_dev) {
    ProblemDev pd = ctx->pdev();
    const int wpb = 8;  // warps per block
    const int tok = prof_begin(ctx, PROF_OTHER);
    float* V = ctx->need_V32 ? ctx->V : nullptr;
    const long pts = (long)pd.N * pd.M;
    if (pts > 0) {
        k_resid<<<(unsigned)((pts + wpb - 1) / wpb), 32 * wpb, 0, ctx->stream>>>(
            pd, ctx->X, ctx->dW, ctx->Y, ctx->Z, ctx->rbuf, V, ctx->Vb_op, ctx->ld_op);
        FBSDE_CK_LAUNCH(ctx);
    }
    k_seeds_paths<<<(pd.M + wpb - 1) / wpb, 32 * wpb, 0, ctx->stream>>>(
        pd, ctx->X, ctx->Y, ctx->Z, ctx->rbuf, ctx->alpha, V, ctx->path_loss_d, ctx->path_loss_d + pd.M,
        ctx->Vb_op, ctx->ld_op);
    FBSDE_CK_LAUNCH(ctx);
    k_loss_reduce<<<1, 1024, 0, ctx->stream>>>(ctx->path_loss_d, pd.M, ctx->Y, loss_dev, y0_dev,
                                               ctx->nonfinite, ctx->path_loss_d + pd.M, ctx->alpha_sum);
    prof_end(ctx, PROF_OTHER, tok, 0.0);
    FBSDE_CK_LAUNCH(ctx);
    return FBSDE_OK;
}

}  // namespace fbsde
