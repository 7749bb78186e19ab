// Adam (Kingma & Ba 2015, Algorithm 1) with bias correction, as used by the
// paper with learning rate 1e-3 (Section 4.1).  FP32 moments and parameters.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.cuh"

namespace fbsde {

__global__ void k_adam(size_t n, float* __restrict__ theta, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float inv_bc1, float inv_bc2, float eps) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * inv_bc1) / (sqrtf(vi * inv_bc2) + eps);
}

fbsde_status launch_adam(fbsde_ctx* ctx, float* theta, const float* grad, float* m, float* v,
                         uint64_t step, float lr) {
    const double b1 = 0.9, b2 = 0.999;
    const double bc1 = 1.0 - std::pow(b1, (double)step);
    const double bc2 = 1.0 - std::pow(b2, (double)step);
    const size_t n = ctx->pl.total;
    const int tok = prof_begin(ctx, PROF_OTHER);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
        n, theta, grad, m, v, lr, (float)b1, (float)b2, (float)(1.0 / bc1), (float)(1.0 / bc2), 1e-8f);
    prof_end(ctx, PROF_OTHER, tok, 0.0);
    FBSDE_CK_LAUNCH(ctx);
    return FBSDE_OK;
}

}  // namespace fbsde
