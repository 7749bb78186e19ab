// Adam (Kingma & Ba 2015, Algorithm 1) with bias correction, as used by the
// paper with learning rate 1e-3 (Section 4.1).  FP32 moments and parameters.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.cuh"

namespace fbsde {

// The bias corrections 1 / (1 - beta^step) are formed on the device (FP64,
// once per block of a grid of two blocks per SM) from the step passed by
// value or read from step_dev, so a
// step replayed from a CUDA graph computes exactly what a direct call does.
// The weights 1 - beta of the new gradient are formed in FP64 before rounding
// (1 - (float)0.999 would be 1.3e-5 away from 1e-3).
// b^k by binary exponentiation (FP64 multiplies: a library pow in FP64 is
// slow on this part, and each block needs the value before its first element).
__device__ __forceinline__ double pow_int(double b, uint64_t k) {
    double p = 1.0;
    while (k) {
        if (k & 1) p *= b;
        b *= b;
        k >>= 1;
    }
    return p;
}

__global__ void k_adam(size_t n, float* __restrict__ theta, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, double b1d, double b2d,
                       uint64_t step_host, const uint64_t* __restrict__ step_dev, float eps) {
    __shared__ float inv_bc[2];
    const float b1 = (float)b1d, b2 = (float)b2d;
    const float c1 = (float)(1.0 - b1d), c2 = (float)(1.0 - b2d);
    if (threadIdx.x == 0) {
        const uint64_t step = step_dev ? *step_dev : step_host;
        inv_bc[0] = (float)(1.0 / (1.0 - pow_int(b1d, step)));
        inv_bc[1] = (float)(1.0 / (1.0 - pow_int(b2d, step)));
    }
    __syncthreads();
    const float inv_bc1 = inv_bc[0], inv_bc2 = inv_bc[1];
    // a few blocks per SM, each over a strided range of the parameters
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + c1 * gi;
        const float vi = b2 * v[i] + c2 * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi * inv_bc1) / (sqrtf(vi * inv_bc2) + eps);
    }
}

fbsde_status launch_adam(fbsde_ctx* ctx, float* theta, const float* grad, float* m, float* v,
                         uint64_t step, float lr) {
    const size_t n = ctx->pl.total;
    const int tok = prof_begin(ctx, PROF_OTHER);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (n + 255) / 256, cap = (size_t)(sms > 0 ? sms : 1) * 2;
    k_adam<<<(unsigned)(want < cap ? want : cap), 256, 0, ctx->stream>>>(n, theta, grad, m, v, lr, 0.9, 0.999, step,
                                                                          ctx->step_dev, 1e-8f);
    prof_end(ctx, PROF_OTHER, tok, 0.0);
    FBSDE_CK_LAUNCH(ctx);
    return FBSDE_OK;
}

__global__ void k_step_advance(uint64_t* step) { *step += 1; }

fbsde_status launch_step_advance(fbsde_ctx* ctx, uint64_t* step) {
    k_step_advance<<<1, 1, 0, ctx->stream>>>(step);
    FBSDE_CK_LAUNCH(ctx);
    return FBSDE_OK;
}

}  // namespace fbsde
