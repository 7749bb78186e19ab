// C ABI of libfbsde (declared in include/fbsde.h): specification checks,
// workspace ownership, and the order of the device steps of one evaluation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.cuh"

namespace fbsde {

fbsde_status copy_path_loss(fbsde_ctx* ctx, float* out);
cudaError_t philox_blocks(const uint32_t* ctr, uint32_t k0, uint32_t k1, size_t count,
                          uint32_t* out, cudaStream_t st);

fbsde_status set_err(fbsde_ctx* ctx, fbsde_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}

// ---- profiler: CUDA events bracketing launches on the context stream
int prof_begin(fbsde_ctx* c, int cls) {
    if (!c->prof.on || cls < 0 || cls >= kProfClasses) return -1;
    Profiler& p = c->prof;
    while (p.pool.size() < p.used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        p.pool.push_back(e);
    }
    const int tok = (int)p.used;
    p.used += 2;
    cudaEventRecord(p.pool[tok], c->stream);
    return tok;
}

void prof_end(fbsde_ctx* c, int cls, int tok, double flops) {
    if (tok < 0) return;
    Profiler& p = c->prof;
    cudaEventRecord(p.pool[tok + 1], c->stream);
    p.spans[cls].push_back({tok, tok + 1});
    p.flops[cls] += flops;
    p.launches[cls] += 1;
}

ParamLayout make_layout(int D, int w, int L, int arch_kind) {
    ParamLayout p;
    const size_t Din = (size_t)D + 1;
    size_t off = 0;
    p.Win = off; off += (size_t)w * Din;
    p.bin = off; off += w;
    for (int l = 1; l <= L; ++l) {
        p.W[l] = off; off += (size_t)w * w;
        p.b[l] = off; off += w;
        if (arch_kind == FBSDE_NAIS) { p.B[l] = off; off += (size_t)w * Din; }
    }
    p.wo = off; off += w;
    p.bo = off; off += 1;
    p.total = off;
    return p;
}

static std::string validate(const fbsde_problem* pb, const fbsde_arch* ar, int N_max) {
    if (!pb || !ar) return "problem and arch must be non-NULL";
    if (pb->kind != FBSDE_BSB && pb->kind != FBSDE_HJB) return "problem.kind must be FBSDE_BSB or FBSDE_HJB";
    if (pb->D < 1 || pb->D > 4096) return "problem.D must be in [1, 4096]";
    if (pb->N < 1 || pb->N > 4096) return "problem.N must be in [1, 4096]";
    if (pb->M < 1) return "problem.M must be >= 1";
    if (!(pb->T > 0) || !std::isfinite(pb->T)) return "problem.T must be finite and > 0";
    if (pb->kind == FBSDE_BSB && (!std::isfinite(pb->r) || !std::isfinite(pb->sigma) || pb->sigma < 0))
        return "problem.r must be finite and problem.sigma finite and >= 0";
    if (!pb->x0_host) return "problem.x0_host must be non-NULL";
    for (int i = 0; i < pb->D; ++i)
        if (!std::isfinite(pb->x0_host[i])) return "problem.x0_host must be finite";
    if (pb->terminal_grad_term != 0 && pb->terminal_grad_term != 1) return "problem.terminal_grad_term must be 0 or 1";
    if (ar->kind != FBSDE_FC && ar->kind != FBSDE_RESNET && ar->kind != FBSDE_NAIS)
        return "arch.kind must be FBSDE_FC, FBSDE_RESNET or FBSDE_NAIS";
    if (ar->width < 16 || ar->width > kMaxWidth || ar->width % 16 != 0)
        return "arch.width must be a multiple of 16 in [16, 512]";
    if (ar->depth < 0 || ar->depth > kMaxDepth) return "arch.depth must be in [0, 16]";
    if (ar->act != FBSDE_SIN && ar->act != FBSDE_TANH) return "arch.act must be FBSDE_SIN or FBSDE_TANH";
    if (ar->kind == FBSDE_NAIS) {
        if (!(ar->h > 0) || !std::isfinite(ar->h)) return "arch.h must be finite and > 0 for NAIS";
        if (!(ar->eps > 0) || !std::isfinite(ar->eps)) return "arch.eps must be finite and > 0 for NAIS";
        if (!std::isfinite(ar->proj_delta)) return "arch.proj_delta must be finite";
    }
    if (ar->prec != FBSDE_FP32 && ar->prec != FBSDE_BF16 && ar->prec != FBSDE_FP8_HIDDEN)
        return "arch.prec must be FBSDE_FP32, FBSDE_BF16 or FBSDE_FP8_HIDDEN";
    if (N_max != 0 && N_max < pb->N) return "N_max must be 0 or >= problem.N";
    const long long nm = N_max ? N_max : pb->N;
    if ((long long)pb->M * (nm + 1) >= (1LL << 31)) return "M * (N_max + 1) must be < 2^31";
    return "";
}

}  // namespace fbsde

using namespace fbsde;

extern "C" {

const char* fbsde_status_string(fbsde_status s) {
    switch (s) {
        case FBSDE_OK: return "ok";
        case FBSDE_ERR_INVALID: return "invalid argument";
        case FBSDE_ERR_UNSUPPORTED: return "unsupported";
        case FBSDE_ERR_CUDA: return "CUDA error";
        case FBSDE_ERR_NONFINITE: return "non-finite loss or gradient";
        case FBSDE_ERR_TIMEOUT: return "device wait timed out";
        case FBSDE_ERR_OOM: return "out of device memory";
    }
    return "unknown status";
}

const char* fbsde_last_error(const fbsde_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

size_t fbsde_param_count(const fbsde_problem* problem, const fbsde_arch* arch) {
    if (!validate(problem, arch, 0).empty()) return 0;
    return make_layout(problem->D, arch->width, arch->depth, arch->kind).total;
}

fbsde_status fbsde_create(const fbsde_problem* problem, const fbsde_arch* arch, uint64_t seed,
                          void* cuda_stream, int N_max, fbsde_ctx** out, char* err_msg_host) {
    auto fail = [&](fbsde_status s, const std::string& m) {
        if (err_msg_host) {
            std::strncpy(err_msg_host, m.c_str(), 255);
            err_msg_host[255] = 0;
        }
        return s;
    };
    if (!out) return fail(FBSDE_ERR_INVALID, "out must be non-NULL");
    *out = nullptr;
    std::string why = validate(problem, arch, N_max);
    if (!why.empty()) return fail(FBSDE_ERR_INVALID, why);

    fbsde_ctx* c = new (std::nothrow) fbsde_ctx();
    if (!c) return fail(FBSDE_ERR_OOM, "host allocation failed");
    c->kind = problem->kind; c->D = problem->D; c->N = problem->N;
    c->N_max = N_max ? N_max : problem->N; c->M = problem->M;
    c->T = problem->T; c->r = problem->r; c->sigma = problem->sigma;
    c->tgt = problem->terminal_grad_term;
    c->x0.assign(problem->x0_host, problem->x0_host + problem->D);
    c->akind = arch->kind; c->w = arch->width; c->L = arch->depth; c->act = arch->act;
    c->prec = arch->prec; c->h = arch->h; c->eps = arch->eps;
    c->delta = arch->proj_delta > 0 ? arch->proj_delta : 0.99 * (2.0 / arch->h - arch->eps);
    if (arch->kind != FBSDE_NAIS) { c->h = 1.0; }
    c->seed = seed;
    c->stream = (cudaStream_t)cuda_stream;
    c->pl = make_layout(c->D, c->w, c->L, c->akind);

    // workspace layout (floats, each buffer 256-byte aligned)
    const size_t Pm = c->Pmax(), D = c->D, w = c->w, L = c->L;
    const size_t maxc = std::max<size_t>(std::max<size_t>(w, D), 2);
    c->part_floats = (size_t)256 * w * maxc;
    size_t total = 0;
    auto add = [&](size_t n) { total += (n + 63) / 64 * 64; };
    add(D);                    // x0
    add((c->N_max + 1) * (size_t)c->M * D);  // X
    add((size_t)c->N_max * c->M * D);        // dW
    add(Pm); add(Pm * D); add(Pm); add(Pm * D); add(2 * Pm);  // Y Z alpha V ones_t
    add(Pm);                   // residuals r_n
    add(4 * (size_t)c->M);     // per-path loss and alpha sums (double)
    if (c->akind == FBSDE_NAIS) { add(2 * L * w * w); }
    add(c->part_floats);
    add(16); add(kMaxDepth + 1); add(16); // alpha_sum, fscal, nonfinite
    add(c->pl.total);          // gradient buffer of train_step
    if (c->prec == FBSDE_FP32) add(fp32_workspace_floats(c));
    c->arena_bytes = total * sizeof(float);

    cudaError_t e = cudaMalloc(&c->arena, c->arena_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(e == cudaErrorMemoryAllocation ? FBSDE_ERR_OOM : FBSDE_ERR_CUDA,
                    std::string("cudaMalloc workspace (") + std::to_string(total * 4 >> 20) +
                        " MiB): " + cudaGetErrorString(e));
    }
    float* cur = (float*)c->arena;
    auto take = [&](size_t n) { float* p = cur; cur += (n + 63) / 64 * 64; return p; };
    c->x0_dev = take(D);
    c->X = take((c->N_max + 1) * (size_t)c->M * D);
    c->dW = take((size_t)c->N_max * c->M * D);
    c->Y = take(Pm); c->Z = take(Pm * D); c->alpha = take(Pm); c->V = take(Pm * D);
    c->ones_t = take(2 * Pm);
    c->rbuf = take(Pm);
    c->path_loss_d = (double*)take(4 * (size_t)c->M);
    if (c->akind == FBSDE_NAIS)
        for (int l = 1; l <= c->L; ++l) { c->Amat[l] = take(w * w); c->gA[l] = take(w * w); }
    c->part = take(c->part_floats);
    c->alpha_sum = take(16);
    c->fscal = take(kMaxDepth + 1);
    c->nonfinite = (int*)take(16);
    c->gradbuf = take(c->pl.total);
    if (c->prec == FBSDE_FP32) fp32_carve(c, cur);

    std::vector<float> x0f(c->D);
    for (int i = 0; i < c->D; ++i) x0f[i] = (float)c->x0[i];
    e = cudaMemcpy(c->x0_dev, x0f.data(), D * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->nonfinite, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(c->arena);
        delete c;
        return fail(FBSDE_ERR_CUDA, std::string("workspace setup: ") + cudaGetErrorString(e));
    }
    if (c->prec != FBSDE_FP32) {
        fbsde_status s = bf16_create(c);
        if (s != FBSDE_OK) {
            std::string m = c->err;
            bf16_destroy(c);
            cudaFree(c->arena);
            delete c;
            return fail(s, m);
        }
    }
    *out = c;
    return FBSDE_OK;
}

fbsde_status fbsde_destroy(fbsde_ctx* ctx) {
    if (!ctx) return FBSDE_OK;
    cudaStreamSynchronize(ctx->stream);
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    if (ctx->bf) bf16_destroy(ctx);
    cudaError_t e = cudaFree(ctx->arena);
    delete ctx;
    return e == cudaSuccess ? FBSDE_OK : FBSDE_ERR_CUDA;
}

size_t fbsde_num_params(const fbsde_ctx* ctx) { return ctx ? ctx->pl.total : 0; }

fbsde_status fbsde_init_params(fbsde_ctx* ctx, float* theta_dev) {
    if (!ctx || !theta_dev) return set_err(ctx, FBSDE_ERR_INVALID, "ctx and theta_dev must be non-NULL");
    return launch_init(ctx, theta_dev);
}

}  // extern "C"

namespace fbsde {

// paths -> network values and Z -> residuals, seeds, loss
static fbsde_status evaluate(fbsde_ctx* c, const float* theta, uint64_t iter, float* loss, float* y0,
                             bool for_grad = false) {
    FBSDE_TRY(launch_paths(c, iter));
    if (c->prec == FBSDE_FP32) {
        FBSDE_TRY(fp32_prepare_weights(c, theta));
        FBSDE_TRY(fp32_forward(c, theta));
    } else {
        FBSDE_TRY(bf16_prepare_weights(c, theta));
        FBSDE_TRY(bf16_forward(c, theta, for_grad));
    }
    return launch_seeds(c, loss, y0);
}

static fbsde_status gradient(fbsde_ctx* c, const float* theta, float* grad) {
    if (c->prec == FBSDE_FP32) return fp32_backward(c, theta, grad);
    return bf16_backward(c, theta, grad);
}

}  // namespace fbsde

extern "C" {

fbsde_status fbsde_rollout_loss(fbsde_ctx* ctx, const float* theta_dev, uint64_t iter,
                                float* loss_dev, float* y0_dev) {
    if (!ctx || !theta_dev) return set_err(ctx, FBSDE_ERR_INVALID, "ctx and theta_dev must be non-NULL");
    return evaluate(ctx, theta_dev, iter, loss_dev, y0_dev);
}

fbsde_status fbsde_rollout_grad(fbsde_ctx* ctx, const float* theta_dev, uint64_t iter,
                                float* loss_dev, float* y0_dev, float* grad_dev) {
    if (!ctx || !theta_dev || !grad_dev)
        return set_err(ctx, FBSDE_ERR_INVALID, "ctx, theta_dev and grad_dev must be non-NULL");
    FBSDE_TRY(evaluate(ctx, theta_dev, iter, loss_dev, y0_dev, true));
    return gradient(ctx, theta_dev, grad_dev);
}

fbsde_status fbsde_train_step(fbsde_ctx* ctx, float* theta_dev, float* adam_m_dev, float* adam_v_dev,
                              uint64_t step, float lr, float* loss_dev, float* y0_dev) {
    if (!ctx || !theta_dev || !adam_m_dev || !adam_v_dev)
        return set_err(ctx, FBSDE_ERR_INVALID, "ctx, theta_dev, adam_m_dev, adam_v_dev must be non-NULL");
    if (step < 1) return set_err(ctx, FBSDE_ERR_INVALID, "step counts Adam steps from 1");
    if (!(lr > 0) || !std::isfinite(lr)) return set_err(ctx, FBSDE_ERR_INVALID, "lr must be finite and > 0");
    float* grad = ctx->gradbuf;
    FBSDE_TRY(evaluate(ctx, theta_dev, step, loss_dev, y0_dev, true));
    FBSDE_TRY(gradient(ctx, theta_dev, grad));
    FBSDE_TRY(launch_adam(ctx, theta_dev, grad, adam_m_dev, adam_v_dev, step, lr));
    if (ctx->akind == FBSDE_NAIS) FBSDE_TRY(nais_project(ctx, theta_dev));
    return FBSDE_OK;
}

fbsde_status fbsde_train_step_dev(fbsde_ctx* ctx, float* theta_dev, float* adam_m_dev, float* adam_v_dev,
                                  uint64_t* step_dev, float lr, float* loss_dev, float* y0_dev) {
    if (!ctx || !theta_dev || !adam_m_dev || !adam_v_dev || !step_dev)
        return set_err(ctx, FBSDE_ERR_INVALID, "ctx, theta_dev, adam_m_dev, adam_v_dev, step_dev must be non-NULL");
    if (!(lr > 0) || !std::isfinite(lr)) return set_err(ctx, FBSDE_ERR_INVALID, "lr must be finite and > 0");
    ctx->step_dev = step_dev;
    // the host step value is unused while step_dev is set; 1 passes the checks
    fbsde_status st = fbsde_train_step(ctx, theta_dev, adam_m_dev, adam_v_dev, 1, lr, loss_dev, y0_dev);
    ctx->step_dev = nullptr;
    if (st != FBSDE_OK) return st;
    return launch_step_advance(ctx, step_dev);
}


fbsde_status fbsde_graph_capture(fbsde_ctx* ctx, float* theta_dev, float* adam_m_dev, float* adam_v_dev,
                                 uint64_t* step_dev, float lr, float* loss_dev, float* y0_dev, int steps,
                                 fbsde_graph** out) {
    if (!ctx || !out) return set_err(ctx, FBSDE_ERR_INVALID, "ctx and out must be non-NULL");
    *out = nullptr;
    if (steps < 1) return set_err(ctx, FBSDE_ERR_INVALID, "steps must be >= 1");
    if (!ctx->stream)
        return set_err(ctx, FBSDE_ERR_UNSUPPORTED, "graph capture needs a context created on a non-default stream");
    if (ctx->prof.on) return set_err(ctx, FBSDE_ERR_INVALID, "disable profiling before capturing a graph");
    if (!theta_dev || !adam_m_dev || !adam_v_dev || !step_dev)
        return set_err(ctx, FBSDE_ERR_INVALID, "theta_dev, adam_m_dev, adam_v_dev, step_dev must be non-NULL");
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return set_err(ctx, FBSDE_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    fbsde_status st = FBSDE_OK;
    for (int k = 0; k < steps && st == FBSDE_OK; ++k)
        st = fbsde_train_step_dev(ctx, theta_dev, adam_m_dev, adam_v_dev, step_dev, lr, loss_dev, y0_dev);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != FBSDE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return set_err(ctx, FBSDE_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_err(ctx, FBSDE_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    fbsde_graph* g = new (std::nothrow) fbsde_graph();
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return set_err(ctx, FBSDE_ERR_OOM, "host allocation failed");
    }
    g->ctx = ctx; g->stream = ctx->stream; g->graph = graph; g->exec = exec;
    *out = g;
    return FBSDE_OK;
}

fbsde_status fbsde_graph_launch(fbsde_graph* graph) {
    if (!graph) return FBSDE_ERR_INVALID;
    cudaError_t e = cudaGraphLaunch(graph->exec, graph->stream);
    if (e != cudaSuccess) return set_err(graph->ctx, FBSDE_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return FBSDE_OK;
}

fbsde_status fbsde_graph_destroy(fbsde_graph* graph) {
    if (!graph) return FBSDE_OK;
    cudaError_t e1 = cudaGraphExecDestroy(graph->exec);
    cudaError_t e2 = cudaGraphDestroy(graph->graph);
    delete graph;
    return (e1 == cudaSuccess && e2 == cudaSuccess) ? FBSDE_OK : FBSDE_ERR_CUDA;
}

fbsde_status fbsde_rollout_detail(fbsde_ctx* ctx, const float* theta_dev, uint64_t iter, float* Y_dev,
                                  float* Z_dev, float* path_loss_dev) {
    if (!ctx || !theta_dev) return set_err(ctx, FBSDE_ERR_INVALID, "ctx and theta_dev must be non-NULL");
    FBSDE_TRY(evaluate(ctx, theta_dev, iter, nullptr, nullptr));
    const size_t P = ctx->P();
    if (Y_dev)
        FBSDE_CK(ctx, cudaMemcpyAsync(Y_dev, ctx->Y, P * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    if (Z_dev)
        FBSDE_CK(ctx, cudaMemcpyAsync(Z_dev, ctx->Z, P * ctx->D * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    if (path_loss_dev) FBSDE_TRY(copy_path_loss(ctx, path_loss_dev));
    return FBSDE_OK;
}

fbsde_status fbsde_sample_paths(fbsde_ctx* ctx, uint64_t iter, float* dW_dev, float* X_dev) {
    if (!ctx) return FBSDE_ERR_INVALID;
    FBSDE_TRY(launch_paths(ctx, iter));
    const size_t MD = (size_t)ctx->M * ctx->D;
    if (dW_dev)
        FBSDE_CK(ctx, cudaMemcpyAsync(dW_dev, ctx->dW, (size_t)ctx->N * MD * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    if (X_dev)
        FBSDE_CK(ctx, cudaMemcpyAsync(X_dev, ctx->X, (size_t)(ctx->N + 1) * MD * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    return FBSDE_OK;
}

fbsde_status fbsde_philox4x32_10(const uint32_t* ctr_dev, uint32_t key0, uint32_t key1, size_t count,
                                 uint32_t* out_dev, void* cuda_stream) {
    if (count > 0 && (!ctr_dev || !out_dev)) return FBSDE_ERR_INVALID;
    return philox_blocks(ctr_dev, key0, key1, count, out_dev, (cudaStream_t)cuda_stream) == cudaSuccess
               ? FBSDE_OK : FBSDE_ERR_CUDA;
}

fbsde_status fbsde_set_level(fbsde_ctx* ctx, int N_level) {
    if (!ctx) return FBSDE_ERR_INVALID;
    if (N_level < 1 || N_level > ctx->N_max)
        return set_err(ctx, FBSDE_ERR_INVALID, "N_level must be in [1, N_max]");
    ctx->N = N_level;
    return FBSDE_OK;
}

fbsde_status fbsde_train_schedule(fbsde_ctx* ctx, float* theta_dev, float* adam_m_dev, float* adam_v_dev,
                                  const int* N_levels_host, const int* steps_per_level_host, int n_levels,
                                  uint64_t first_step, float lr, float* loss_trace_dev,
                                  float* y0_trace_dev) {
    if (!ctx) return FBSDE_ERR_INVALID;
    if (!N_levels_host || !steps_per_level_host || n_levels < 1)
        return set_err(ctx, FBSDE_ERR_INVALID, "N_levels_host and steps_per_level_host must hold n_levels >= 1 ints");
    for (int i = 0; i < n_levels; ++i) {
        if (N_levels_host[i] < 1 || N_levels_host[i] > ctx->N_max)
            return set_err(ctx, FBSDE_ERR_INVALID, "level " + std::to_string(i) + ": N must be in [1, N_max]");
        if (steps_per_level_host[i] < 0)
            return set_err(ctx, FBSDE_ERR_INVALID, "level " + std::to_string(i) + ": step count must be >= 0");
    }
    if (first_step < 1) return set_err(ctx, FBSDE_ERR_INVALID, "step counts Adam steps from 1");
    uint64_t step = first_step;
    size_t k = 0;
    for (int i = 0; i < n_levels; ++i) {
        FBSDE_TRY(fbsde_set_level(ctx, N_levels_host[i]));
        for (int s = 0; s < steps_per_level_host[i]; ++s, ++step, ++k)
            FBSDE_TRY(fbsde_train_step(ctx, theta_dev, adam_m_dev, adam_v_dev, step, lr,
                                       loss_trace_dev ? loss_trace_dev + k : nullptr,
                                       y0_trace_dev ? y0_trace_dev + k : nullptr));
    }
    return FBSDE_OK;
}

fbsde_status fbsde_set_x0(fbsde_ctx* ctx, const double* x0_host) {
    if (!ctx || !x0_host) return set_err(ctx, FBSDE_ERR_INVALID, "ctx and x0_host must be non-NULL");
    for (int i = 0; i < ctx->D; ++i)
        if (!std::isfinite(x0_host[i])) return set_err(ctx, FBSDE_ERR_INVALID, "x0 must be finite");
    ctx->x0.assign(x0_host, x0_host + ctx->D);
    std::vector<float> x0f(ctx->D);
    for (int i = 0; i < ctx->D; ++i) x0f[i] = (float)x0_host[i];
    // pageable source: the copy is staged before the call returns, so the
    // caller's buffer may be reused immediately
    FBSDE_CK(ctx, cudaMemcpyAsync(ctx->x0_dev, x0f.data(), ctx->D * sizeof(float),
                                  cudaMemcpyHostToDevice, ctx->stream));
    FBSDE_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return FBSDE_OK;
}

fbsde_status fbsde_set_x0_device(fbsde_ctx* ctx, const float* x0_dev) {
    if (!ctx || !x0_dev) return set_err(ctx, FBSDE_ERR_INVALID, "ctx and x0_dev must be non-NULL");
    FBSDE_CK(ctx, cudaMemcpyAsync(ctx->x0_dev, x0_dev, ctx->D * sizeof(float), cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    return FBSDE_OK;
}

fbsde_status fbsde_profile_enable(fbsde_ctx* ctx, int on) {
    if (!ctx) return FBSDE_ERR_INVALID;
    FBSDE_CK(ctx, cudaStreamSynchronize(ctx->stream));
    Profiler& p = ctx->prof;
    p.on = on != 0;
    p.used = 0;
    for (int k = 0; k < kProfClasses; ++k) { p.spans[k].clear(); p.flops[k] = 0; p.launches[k] = 0; }
    return FBSDE_OK;
}

fbsde_status fbsde_profile_read(fbsde_ctx* ctx, int cls, double* ms_total, uint64_t* launches,
                                double* flops) {
    if (!ctx || cls < 0 || cls >= kProfClasses)
        return set_err(ctx, FBSDE_ERR_INVALID, "cls must be 0, 1 or 2");
    FBSDE_CK(ctx, cudaStreamSynchronize(ctx->stream));
    const Profiler& p = ctx->prof;
    double ms = 0;
    for (const auto& sp : p.spans[cls]) {
        float t = 0;
        FBSDE_CK(ctx, cudaEventElapsedTime(&t, p.pool[sp.first], p.pool[sp.second]));
        ms += t;
    }
    if (ms_total) *ms_total = ms;
    if (launches) *launches = p.launches[cls];
    if (flops) *flops = p.flops[cls];
    return FBSDE_OK;
}

uint64_t fbsde_launch_count(const fbsde_ctx* ctx) { return ctx ? ctx->n_launch : 0; }

fbsde_status fbsde_test_timeout_once(fbsde_ctx* ctx) {
    if (!ctx) return FBSDE_ERR_INVALID;
    return arm_timeout_test(ctx);
}

fbsde_status fbsde_check_finite(fbsde_ctx* ctx) {
    if (!ctx) return FBSDE_ERR_INVALID;
    int flag = 0, timeout = 0;
    int* terr = bf16_error_flag(ctx);
    FBSDE_CK(ctx, cudaMemcpyAsync(&flag, ctx->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (terr) FBSDE_CK(ctx, cudaMemcpyAsync(&timeout, terr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    FBSDE_CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (timeout) {
        FBSDE_CK(ctx, cudaMemsetAsync(terr, 0, sizeof(int), ctx->stream));
        if (flag) FBSDE_CK(ctx, cudaMemsetAsync(ctx->nonfinite, 0, sizeof(int), ctx->stream));
        return set_err(ctx, FBSDE_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait; results are invalid");
    }
    if (flag) {
        FBSDE_CK(ctx, cudaMemsetAsync(ctx->nonfinite, 0, sizeof(int), ctx->stream));
        return set_err(ctx, FBSDE_ERR_NONFINITE, "a loss or gradient entry was NaN or Inf");
    }
    return FBSDE_OK;
}

}  // extern "C"
