// fbsde_residual_loss_noalloc: the residual / loss-seed / loss step for
// callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc at all: a host application whose own
// memory pool owns every byte of device memory (a direct cudaMalloc would
// escape its accounting and can fail once the pool has reserved the device),
// or a latency-critical loop where an allocation's implicit device
// synchronisation is not acceptable.  Such a caller already holds the paths,
// the network values and the output buffers; what the step still needs is a
// per-path scratch for the FP64 loss terms before their fixed-order sum.  Here
// that scratch is a file-scope device array of a fixed size, reserved on every
// GPU that loads the library for as long as the process lives.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace fbsde {

// Largest number of paths M the array serves: 65536 FP64 terms = 512 KiB.
constexpr int kNoAllocMaxPaths = 65536;

static __device__ __align__(256) double g_noalloc_path_loss[kNoAllocMaxPaths];

// The per-path residual and seed kernel of the allocating path (paths.cu).
__global__ void k_seeds(ProblemDev pd, const float* __restrict__ X, const float* __restrict__ dW,
                        const float* __restrict__ Y, const float* __restrict__ Z, float* __restrict__ alpha,
                        float* __restrict__ V, double* __restrict__ path_loss, __nv_bfloat16* __restrict__ Vb,
                        int ldb);

// Fixed-order sum of the M per-path terms held in the array (one block), and
// Y_0 = Y[0].  Every term read here was written by this call's k_seeds.
__global__ void k_noalloc_loss_reduce(const double* __restrict__ path_loss, int M, const float* __restrict__ Y,
                                      float* __restrict__ loss_out, float* __restrict__ y0_out) {
    __shared__ double sh[1024];
    double acc = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) acc += path_loss[m];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *loss_out = (float)sh[0];
        *y0_out = Y[0];
    }
}

// Device address of the array, looked up once per device (with that device
// current) and cached.
static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[64] = {};

static cudaError_t noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_path_loss);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace fbsde

using namespace fbsde;

extern "C" fbsde_status fbsde_residual_loss_noalloc(const fbsde_problem* problem, const float* X_dev,
                                                    const float* dW_dev, const float* Y_dev, const float* Z_dev,
                                                    float* alpha_dev, float* V_dev, float* loss_dev, float* y0_dev,
                                                    void* cuda_stream, char* err_msg_host) {
    auto fail = [&](fbsde_status s, const std::string& m) {
        if (err_msg_host) {
            std::strncpy(err_msg_host, m.c_str(), 255);
            err_msg_host[255] = 0;
        }
        return s;
    };
    if (!problem) return fail(FBSDE_ERR_INVALID, "problem must be non-NULL");
    if (problem->kind != FBSDE_BSB && problem->kind != FBSDE_HJB)
        return fail(FBSDE_ERR_INVALID, "problem.kind must be FBSDE_BSB or FBSDE_HJB");
    if (problem->D < 1 || problem->N < 1 || problem->M < 1)
        return fail(FBSDE_ERR_INVALID, "problem.D, problem.N and problem.M must be >= 1");
    if (problem->M > kNoAllocMaxPaths)
        return fail(FBSDE_ERR_INVALID, "problem.M = " + std::to_string(problem->M) +
                                           " exceeds the no-allocation limit of " +
                                           std::to_string(kNoAllocMaxPaths) + " paths");
    if (!(problem->T > 0) || !std::isfinite(problem->T)) return fail(FBSDE_ERR_INVALID, "problem.T must be > 0");
    if (!X_dev || !dW_dev || !Y_dev || !Z_dev || !alpha_dev || !V_dev || !loss_dev || !y0_dev)
        return fail(FBSDE_ERR_INVALID, "every buffer must be non-NULL");

    double* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return fail(FBSDE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

    ProblemDev pd;
    pd.kind = problem->kind; pd.D = problem->D; pd.N = problem->N; pd.M = problem->M;
    pd.dt = (float)(problem->T / problem->N);
    pd.sqrt_dt = (float)std::sqrt(problem->T / problem->N);
    pd.r = (float)problem->r; pd.sigma = (float)problem->sigma; pd.tgt = problem->terminal_grad_term;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int wpb = 8;
    k_seeds<<<(pd.M + wpb - 1) / wpb, 32 * wpb, 0, st>>>(pd, X_dev, dW_dev, Y_dev, Z_dev, alpha_dev, V_dev, scratch,
                                                         nullptr, 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_noalloc_loss_reduce<<<1, 1024, 0, st>>>(scratch, pd.M, Y_dev, loss_dev, y0_dev);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? FBSDE_OK : fail(FBSDE_ERR_CUDA, cudaGetErrorString(e));
}
