// Internal definitions shared by the translation units of libfbsde.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/fbsde.h"

namespace fbsde {

constexpr int kMaxDepth = 16;
constexpr int kMaxWidth = 512;

// Offsets of each tensor inside the flat FP32 parameter vector (the order is
// documented in fbsde.h).  For NAIS, W[l] is R_l, b[l] is C_l, B[l] is B_l.
struct ParamLayout {
    size_t Win = 0, bin = 0, wo = 0, bo = 0, total = 0;
    size_t W[kMaxDepth + 1] = {}, b[kMaxDepth + 1] = {}, B[kMaxDepth + 1] = {};
};

ParamLayout make_layout(int D, int w, int L, int arch_kind);

// Device-side description of one evaluation, passed by value to kernels.
struct ProblemDev {
    int kind;     // FBSDE_BSB / FBSDE_HJB
    int D, N, M;  // current level N
    float dt, sqrt_dt, r, sigma;
    int tgt;      // terminal gradient term
};

// Per-form workspace: FP32 form (CUDA-core FP32 GEMMs).
struct Fp32Work {
    float* A[kMaxDepth + 1];   // pre-activations a_l          [P, w]
    float* H[kMaxDepth + 1];   // layer outputs h_l            [P, w]
    float* E[kMaxDepth + 1];   // e_l = c act'(a_l) g_l        [P, w]
    float* G[kMaxDepth + 1];   // g_l = d y / d h_l            [P, w]
    float* HD[kMaxDepth + 1];  // tangent h'_l                 [P, w]
    float* S[kMaxDepth + 1];   // c act''(a_l) a'_l g_l        [P, w]
    float* AB[kMaxDepth + 1];  // adjoint abar_l               [P, w]
    float* HB[kMaxDepth + 1];  // adjoint hbar_l               [P, w]
};

struct Bf16Work;  // tensor-core form, defined in tc_path.cu

// Kernel-class timing (fbsde_profile_*): CUDA events around launches.
constexpr int kProfClasses = 3;
enum { PROF_POINTS = 0, PROF_WGRAD = 1, PROF_OTHER = 2 };
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;       // events, reused across reads
    size_t used = 0;
    std::vector<std::pair<int, int>> spans[kProfClasses];
    double flops[kProfClasses] = {};
    uint64_t launches[kProfClasses] = {};
};

}  // namespace fbsde

struct fbsde_ctx {
    // problem
    int kind = 0, D = 0, N = 0, N_max = 0, M = 0, tgt = 0;
    double T = 1, r = 0, sigma = 0;
    std::vector<double> x0;
    // architecture
    int akind = 0, w = 0, L = 0, act = 0, prec = 0;
    double h = 1, eps = 0.01, delta = 1;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    // When set, the iteration / Adam step number is read from this device
    // word by the kernels (a step captured in a CUDA graph) instead of being
    // passed by value.
    const uint64_t* step_dev = nullptr;
    // Upper bound on the CTAs of the fused per-tile kernels (0: one per SM);
    // set by fbsde_set_grid_cap / the group autotuner so that the instances
    // of a group share the SMs.
    int grid_cap = 0;
    fbsde::ParamLayout pl;
    std::string err;

    // workspace (one device allocation, carved into the buffers below)
    void* arena = nullptr;
    size_t arena_bytes = 0;
    float* x0_dev = nullptr;
    float* X = nullptr;        // paths X_n            [(N_max+1) M, D]
    float* dW = nullptr;       // increments           [N_max M, D]
    float* Y = nullptr;        // network values       [(N_max+1) M]
    float* Z = nullptr;        // input gradients      [(N_max+1) M, D]
    float* alpha = nullptr;    // d loss / d Y_n       [(N_max+1) M]
    float* V = nullptr;        // d loss / d Z_n       [(N_max+1) M, D]
    float* ones_t = nullptr;   // (1, t_n) per point   [(N_max+1) M, 2]
    double* path_loss_d = nullptr;  // per-path loss [M], then per-path sum of alpha [M]
    float* rbuf = nullptr;     // Y-residuals r_n      [N_max M]
    bool need_V32 = true;      // FP32 v_n consumed (FP32 form, layered BF16 sweeps)
    float* Amat[fbsde::kMaxDepth + 1] = {};  // NAIS A_l = -R^T R - eps I [w, w]
    float* gA[fbsde::kMaxDepth + 1] = {};    // NAIS d loss / d A_l       [w, w]
    float* part = nullptr;     // split-K partial sums
    size_t part_floats = 0;
    float* alpha_sum = nullptr;  // sum of alpha over all points (the gradient in b_o)
    float* fscal = nullptr;    // device float scalars (projection scales)
    int* nonfinite = nullptr;  // set when a loss/gradient entry is NaN/Inf
    float* gradbuf = nullptr;  // gradient of fbsde_train_step [num_params]
    // BF16 operand copies of X and V written by the path and seed kernels for
    // the fused tensor-core kernels (rows of ld_op; NULL in the other forms)
    __nv_bfloat16* Xb_op = nullptr;
    __nv_bfloat16* Vb_op = nullptr;
    int ld_op = 0;
    fbsde::Fp32Work f32{};
    fbsde::Profiler prof;
    uint64_t n_launch = 0;     // kernels launched by this context
    fbsde::Bf16Work* bf = nullptr;

    size_t P() const { return (size_t)M * (size_t)(N + 1); }
    size_t Pmax() const { return (size_t)M * (size_t)(N_max + 1); }
    fbsde::ProblemDev pdev() const {
        fbsde::ProblemDev p;
        p.kind = kind; p.D = D; p.N = N; p.M = M;
        p.dt = (float)(T / N); p.sqrt_dt = (float)std::sqrt(T / N);
        p.r = (float)r; p.sigma = (float)sigma; p.tgt = tgt;
        return p;
    }
};

// An instantiated CUDA graph of training steps (fbsde_graph_capture,
// fbsde_group_capture), replayed on `stream`.
struct fbsde_graph {
    fbsde_ctx* ctx = nullptr;  // error reporting (NULL for a group)
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace fbsde {

// Error plumbing: every CUDA call in host code goes through CK(), which
// records the failing call in ctx->err and returns FBSDE_ERR_CUDA.
fbsde_status set_err(fbsde_ctx* ctx, fbsde_status s, const std::string& msg);

#define FBSDE_CK(ctx, call)                                                             \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::fbsde::set_err((ctx), FBSDE_ERR_CUDA,                              \
                                    std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define FBSDE_CK_LAUNCH(ctx)                  \
    do {                                      \
        ++(ctx)->n_launch;                    \
        FBSDE_CK((ctx), cudaGetLastError());  \
    } while (0)

// Bracket a launch with profiler events: int t = prof_begin(ctx, cls); launch;
// prof_end(ctx, cls, t, flops).  No-ops while profiling is off.
int prof_begin(fbsde_ctx* ctx, int cls);
void prof_end(fbsde_ctx* ctx, int cls, int tok, double flops);

#define FBSDE_TRY(expr)                     \
    do {                                    \
        fbsde_status s_ = (expr);           \
        if (s_ != FBSDE_OK) return s_;      \
    } while (0)

// Shared device steps (paths.cu).
fbsde_status launch_paths(fbsde_ctx* ctx, uint64_t iter);
fbsde_status launch_seeds(fbsde_ctx* ctx, float* loss_dev, float* y0_dev);
fbsde_status launch_init(fbsde_ctx* ctx, float* theta);

// FP32 form (fp32_path.cu).
size_t fp32_workspace_floats(const fbsde_ctx* ctx);
void fp32_carve(fbsde_ctx* ctx, float*& cursor);
fbsde_status fp32_prepare_weights(fbsde_ctx* ctx, const float* theta);
fbsde_status fp32_forward(fbsde_ctx* ctx, const float* theta);
fbsde_status fp32_backward(fbsde_ctx* ctx, const float* theta, float* grad);
fbsde_status nais_project(fbsde_ctx* ctx, float* theta);

// BF16 tensor-core form (tc_path.cu).
fbsde_status bf16_create(fbsde_ctx* ctx);
// Device flag the tensor-core kernels raise when a bounded wait runs out (NULL: no BF16 workspace).
int* bf16_error_flag(fbsde_ctx* ctx);
// Arms the test hook of the pipelined kernels (fbsde_test_timeout_once).
fbsde_status arm_timeout_test(fbsde_ctx* c);
void bf16_destroy(fbsde_ctx* ctx);
fbsde_status bf16_prepare_weights(fbsde_ctx* ctx, const float* theta);
fbsde_status bf16_forward(fbsde_ctx* ctx, const float* theta, bool for_grad);
fbsde_status bf16_backward(fbsde_ctx* ctx, const float* theta, float* grad);

// Helpers of the FP32 form reused by the BF16 form.
fbsde_status launch_rowdot(fbsde_ctx* c, const float* h, const float* theta, float* y);
fbsde_status nais_chain_R(fbsde_ctx* c, const float* theta, float* grad);
fbsde_status launch_check_finite(fbsde_ctx* c, const float* x, size_t n);

// Skip s and scale c of layer l in h_l = s h_{l-1} + c act(a_l): (0, 1) for
// the lift and FC layers, (1, 1) for ResNet blocks, (1, h) for NAIS blocks.
inline float layer_skip(const fbsde_ctx* c, int l) {
    return (l == 0 || c->akind == FBSDE_FC) ? 0.f : 1.f;
}
inline float layer_scale(const fbsde_ctx* c, int l) {
    return (l > 0 && c->akind == FBSDE_NAIS) ? (float)c->h : 1.f;
}

// Adam (adam.cu).
// ++*step on the device (end of a device-numbered training step).
fbsde_status launch_step_advance(fbsde_ctx* ctx, uint64_t* step);
fbsde_status launch_adam(fbsde_ctx* ctx, float* theta, const float* grad, float* m, float* v,
                         uint64_t step, float lr);

// Activation and its first two derivatives (FP32 form: accurate library
// functions, no fast-math).  act = 0: sin, 1: tanh.
struct Act3 { float f, d1, d2; };
__device__ __forceinline__ Act3 act3_accurate(int act, float a) {
    Act3 r;
    if (act == FBSDE_SIN) {
        float s, c;
        sincosf(a, &s, &c);
        r.f = s; r.d1 = c; r.d2 = -s;
    } else {
        // tanh' = sech^2 computed from cosh to keep relative accuracy where
        // tanh saturates (1 - tanh^2 would cancel there).
        float t = tanhf(a);
        float ch = coshf(a);
        float d1 = 1.0f / (ch * ch);
        r.f = t; r.d1 = d1; r.d2 = -2.0f * t * d1;
    }
    return r;
}

}  // namespace fbsde
