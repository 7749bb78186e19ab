// Groups of independent FBSDE instances trained together (many problems of
// uneven D, N, M and width at once).  Each instance keeps its own context,
// stream and workspace; the group step can be captured as one CUDA graph and
// replayed with a single launch.  Two ways to run a step:
//
//   * grouped launches (default): the instances served by the fused BF16
//     kernels with a common kernel variant and at most two tiles per SM
//     (larger ones fill the GPU alone) run their forward kernels as ONE
//     persistent launch and their backward kernels as one more (CTA ranges
//     per instance, each walking its own tiles); the per-instance steps
//     around them (paths, weights, residuals, weight gradients, Adam) run on
//     the instances' streams between fork and join events.  Other instances
//     run whole steps on their own streams alongside.
//   * streams: every instance's whole step on its own stream, concurrently.
//
// The fused kernels of an instance alone take every SM; in a group the
// instances share them.  The autotuner times candidate splits (each
// instance's CTA count) on scratch copies of the training state and keeps
// the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"
#include "bf16_work.cuh"

using namespace fbsde;

struct fbsde_group {
    std::vector<fbsde_ctx*> ctx;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, fork2 = nullptr, fork3 = nullptr;
    std::vector<cudaEvent_t> join;
    int sms = 0;
    int mode = FBSDE_GROUP_GROUPED;
    FusedGroupBuf buf;
};

namespace {

#define GCK(call)                                              \
    do {                                                       \
        if ((call) != cudaSuccess) return FBSDE_ERR_CUDA;      \
    } while (0)

// An instance with more tiles than this many per SM fills the GPU by itself:
// it runs its whole step on its own stream, where its weight gradients (bound
// by HBM) can overlap other instances' point contractions, instead of joining
// the grouped launches.  (On the 32-instance batch: 95.7 ms per round with
// every fused instance grouped, 92.1 with this rule, 92.0 in streams mode.)
constexpr long kGroupedTilesPerSM = 2;

// instances whose fused kernels go into the grouped launches: fused BF16
// instances of at most kGroupedTilesPerSM x SMs tiles, of the first such
// instance's kernel variant (at least two)
std::vector<int> grouped_members(const fbsde_group* g) {
    std::vector<int> gi;
    int variant = -1;
    for (size_t i = 0; i < g->ctx.size(); ++i) {
        const fbsde_ctx* c = g->ctx[i];
        if (!fused_groupable(c)) continue;
        if ((long)((c->P() + 127) / 128) > kGroupedTilesPerSM * g->sms) continue;
        if (variant < 0) variant = fused_variant(c);
        if (fused_variant(c) == variant) gi.push_back((int)i);
    }
    if (g->mode != FBSDE_GROUP_GROUPED || gi.size() < 2) gi.clear();
    return gi;
}

// the arguments of the grouped launches, uploaded when they changed
fbsde_status group_prepare(fbsde_group* g, const std::vector<int>& gi, float* const* theta) {
    if (gi.empty()) return FBSDE_OK;
    std::vector<fbsde_ctx*> gc;
    std::vector<const float*> gt;
    for (int i : gi) {
        gc.push_back(g->ctx[i]);
        gt.push_back(theta[i]);
    }
    if (g->buf.cap < (int)gi.size()) FBSDE_TRY(fused_group_alloc(&g->buf, (int)g->ctx.size()));
    return fused_group_prepare(gc.data(), gt.data(), (int)gi.size(), &g->buf, g->stream);
}

fbsde_status group_enqueue(fbsde_group* g, float* const* theta, float* const* m, float* const* v,
                           uint64_t* step_dev, float lr, float* loss_dev, float* y0_dev) {
    const int n = (int)g->ctx.size();
    const std::vector<int> gi = grouped_members(g);
    std::vector<char> in_group(n, 0);
    for (int i : gi) in_group[i] = 1;
    FBSDE_TRY(group_prepare(g, gi, theta));
    GCK(cudaEventRecord(g->fork, g->stream));
    // whole steps on the instances' own streams
    for (int i = 0; i < n; ++i) {
        if (in_group[i]) continue;
        fbsde_ctx* c = g->ctx[i];
        GCK(cudaStreamWaitEvent(c->stream, g->fork, 0));
        FBSDE_TRY(fbsde_train_step_dev(c, theta[i], m[i], v[i], step_dev + i, lr,
                                       loss_dev ? loss_dev + i : nullptr, y0_dev ? y0_dev + i : nullptr));
        GCK(cudaEventRecord(g->join[i], c->stream));
    }
    if (!gi.empty()) {
        std::vector<fbsde_ctx*> gc;
        for (int i : gi) gc.push_back(g->ctx[i]);
        const int ng = (int)gi.size();
        // each stage runs per instance on its stream between fork and join
        // events around the grouped launches on the group's stream
        auto stage = [&](cudaEvent_t after, auto&& body) -> fbsde_status {
            for (int i : gi) {
                fbsde_ctx* c = g->ctx[i];
                GCK(cudaStreamWaitEvent(c->stream, after, 0));
                c->step_dev = step_dev + i;
                const fbsde_status st = body(i, c);
                c->step_dev = nullptr;
                FBSDE_TRY(st);
                GCK(cudaEventRecord(g->join[i], c->stream));
                GCK(cudaStreamWaitEvent(g->stream, g->join[i], 0));
            }
            return FBSDE_OK;
        };
        // paths and BF16 weights; then every forward kernel in one launch
        FBSDE_TRY(stage(g->fork, [&](int i, fbsde_ctx* c) -> fbsde_status {
            FBSDE_TRY(launch_paths(c, 1));
            return bf16_prepare_weights(c, theta[i]);
        }));
        FBSDE_TRY(fused_group_forward(gc.data(), ng, &g->buf, g->stream));
        GCK(cudaEventRecord(g->fork2, g->stream));
        // residuals, loss and seeds, the backward's parameter table; then
        // every backward kernel in one launch
        FBSDE_TRY(stage(g->fork2, [&](int i, fbsde_ctx* c) -> fbsde_status {
            FBSDE_TRY(launch_seeds(c, loss_dev ? loss_dev + i : nullptr, y0_dev ? y0_dev + i : nullptr));
            return fused_group_stage_pvec(c, theta[i], c->stream);
        }));
        FBSDE_TRY(fused_group_backward(gc.data(), ng, &g->buf, g->stream));
        GCK(cudaEventRecord(g->fork3, g->stream));
        // weight gradients, Adam (device step), NAIS-Net projection, next step
        FBSDE_TRY(stage(g->fork3, [&](int i, fbsde_ctx* c) -> fbsde_status {
            FBSDE_TRY(bf16_wgrad_tail(c, theta[i], c->gradbuf));
            FBSDE_TRY(launch_adam(c, theta[i], c->gradbuf, m[i], v[i], 1, lr));
            if (c->akind == FBSDE_NAIS) FBSDE_TRY(nais_project(c, theta[i]));
            return FBSDE_OK;
        }));
        for (int i : gi) {
            fbsde_ctx* c = g->ctx[i];
            FBSDE_TRY(launch_step_advance(c, step_dev + i));
            GCK(cudaEventRecord(g->join[i], c->stream));
        }
    }
    for (int i = 0; i < n; ++i) GCK(cudaStreamWaitEvent(g->stream, g->join[i], 0));
    return FBSDE_OK;
}

}  // namespace

extern "C" {

fbsde_status fbsde_stream_create(void** out) {
    if (!out) return FBSDE_ERR_INVALID;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return FBSDE_ERR_CUDA;
    *out = st;
    return FBSDE_OK;
}

fbsde_status fbsde_stream_destroy(void* stream) {
    if (!stream) return FBSDE_OK;
    return cudaStreamDestroy((cudaStream_t)stream) == cudaSuccess ? FBSDE_OK : FBSDE_ERR_CUDA;
}

fbsde_status fbsde_set_grid_cap(fbsde_ctx* ctx, int ctas) {
    if (!ctx) return FBSDE_ERR_INVALID;
    if (ctas < 0) return set_err(ctx, FBSDE_ERR_INVALID, "ctas must be >= 0 (0: one CTA per SM)");
    ctx->grid_cap = ctas;
    return FBSDE_OK;
}

fbsde_status fbsde_group_create(fbsde_ctx* const* ctxs, int n, void* cuda_stream, fbsde_group** out) {
    if (!out) return FBSDE_ERR_INVALID;
    *out = nullptr;
    if (!ctxs || n < 1 || !cuda_stream) return FBSDE_ERR_INVALID;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !ctxs[i]->stream) return FBSDE_ERR_INVALID;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return FBSDE_ERR_INVALID;
    }
    fbsde_group* g = new (std::nothrow) fbsde_group();
    if (!g) return FBSDE_ERR_OOM;
    g->ctx.assign(ctxs, ctxs + n);
    g->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    bool ok = cudaGetDevice(&dev) == cudaSuccess &&
              cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->fork2, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->fork3, cudaEventDisableTiming) == cudaSuccess;
    g->join.assign(n, nullptr);
    for (int i = 0; ok && i < n; ++i) ok = cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        fbsde_group_destroy(g);
        return FBSDE_ERR_CUDA;
    }
    *out = g;
    return FBSDE_OK;
}

fbsde_status fbsde_group_destroy(fbsde_group* g) {
    if (!g) return FBSDE_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    fused_group_free(&g->buf);
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->fork2) cudaEventDestroy(g->fork2);
    if (g->fork3) cudaEventDestroy(g->fork3);
    for (cudaEvent_t e : g->join)
        if (e) cudaEventDestroy(e);
    delete g;
    return FBSDE_OK;
}

fbsde_status fbsde_group_set_mode(fbsde_group* g, int mode) {
    if (!g || (mode != FBSDE_GROUP_STREAMS && mode != FBSDE_GROUP_GROUPED)) return FBSDE_ERR_INVALID;
    g->mode = mode;
    return FBSDE_OK;
}

fbsde_status fbsde_group_train_step(fbsde_group* g, float* const* theta, float* const* m, float* const* v,
                                    uint64_t* step_dev, float lr, float* loss_dev, float* y0_dev) {
    if (!g || !theta || !m || !v || !step_dev) return FBSDE_ERR_INVALID;
    return group_enqueue(g, theta, m, v, step_dev, lr, loss_dev, y0_dev);
}

fbsde_status fbsde_group_capture(fbsde_group* g, float* const* theta, float* const* m, float* const* v,
                                 uint64_t* step_dev, float lr, float* loss_dev, float* y0_dev, int steps,
                                 fbsde_graph** out) {
    if (!out) return FBSDE_ERR_INVALID;
    *out = nullptr;
    if (!g || !theta || !m || !v || !step_dev || steps < 1) return FBSDE_ERR_INVALID;
    for (fbsde_ctx* c : g->ctx)
        if (c->prof.on) return set_err(c, FBSDE_ERR_INVALID, "disable profiling before capturing a graph");
    // the grouped launches' arguments go to the device before the capture
    FBSDE_TRY(group_prepare(g, grouped_members(g), theta));
    if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FBSDE_ERR_CUDA;
    fbsde_status st = FBSDE_OK;
    for (int k = 0; k < steps && st == FBSDE_OK; ++k) st = group_enqueue(g, theta, m, v, step_dev, lr, loss_dev, y0_dev);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
    if (st != FBSDE_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != FBSDE_OK ? st : FBSDE_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return FBSDE_ERR_CUDA;
    }
    fbsde_graph* gr = new (std::nothrow) fbsde_graph();
    if (!gr) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return FBSDE_ERR_OOM;
    }
    gr->ctx = nullptr; gr->stream = g->stream; gr->graph = graph; gr->exec = exec;
    *out = gr;
    return FBSDE_OK;
}

fbsde_status fbsde_group_autotune(fbsde_group* g, const float* const* theta, float lr, int trial_steps,
                                  int* caps_out, float* ms_out) {
    if (!g || !theta || !caps_out || trial_steps < 1) return FBSDE_ERR_INVALID;
    const int n = (int)g->ctx.size();
    // scratch copies of the state: the trials must not move the caller's training
    std::vector<float*> th(n, nullptr), mm(n, nullptr), vv(n, nullptr);
    uint64_t* steps = nullptr;
    float* junk = nullptr;
    auto release = [&]() {
        for (int i = 0; i < n; ++i) {
            if (th[i]) cudaFree(th[i]);
            if (mm[i]) cudaFree(mm[i]);
            if (vv[i]) cudaFree(vv[i]);
        }
        if (steps) cudaFree(steps);
        if (junk) cudaFree(junk);
    };
    bool ok = cudaMalloc(&steps, n * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&junk, 2 * n * sizeof(float)) == cudaSuccess;
    for (int i = 0; ok && i < n; ++i) {
        const size_t bytes = g->ctx[i]->pl.total * sizeof(float);
        ok = cudaMalloc(&th[i], bytes) == cudaSuccess && cudaMalloc(&mm[i], bytes) == cudaSuccess &&
             cudaMalloc(&vv[i], bytes) == cudaSuccess;
    }
    if (!ok) {
        release();
        return FBSDE_ERR_OOM;
    }
    // candidate splits: every instance on all SMs; SMs in proportion to each
    // instance's points x width^2 (its share of the contraction work), and
    // twice that; half and a quarter of the SMs each
    std::vector<double> work(n);
    double total = 0;
    for (int i = 0; i < n; ++i) {
        const fbsde_ctx* c = g->ctx[i];
        work[i] = (double)c->P() * c->w * c->w * (c->L + 1);
        total += work[i];
    }
    std::vector<std::vector<int>> cands;
    cands.push_back(std::vector<int>(n, 0));
    std::vector<int> prop(n);
    for (int i = 0; i < n; ++i) prop[i] = std::max(8, (int)std::lround(g->sms * work[i] / total));
    cands.push_back(prop);
    cands.push_back(std::vector<int>(n, std::max(1, g->sms / 2)));
    cands.push_back(std::vector<int>(n, std::max(1, g->sms / 4)));
    std::vector<int> prop2(n);
    for (int i = 0; i < n; ++i) prop2[i] = std::min(g->sms, 2 * prop[i]);
    cands.push_back(prop2);
    std::vector<int> saved(n);
    for (int i = 0; i < n; ++i) saved[i] = g->ctx[i]->grid_cap;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    float best = -1.f;
    size_t best_k = 0;
    fbsde_status st = ok ? FBSDE_OK : FBSDE_ERR_CUDA;
    std::vector<uint64_t> ones(n, 1);
    for (size_t k = 0; k < cands.size() && st == FBSDE_OK; ++k) {
        for (int i = 0; i < n; ++i) {
            g->ctx[i]->grid_cap = cands[k][i];
            const size_t bytes = g->ctx[i]->pl.total * sizeof(float);
            if (cudaMemcpyAsync(th[i], theta[i], bytes, cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess ||
                cudaMemsetAsync(mm[i], 0, bytes, g->stream) != cudaSuccess ||
                cudaMemsetAsync(vv[i], 0, bytes, g->stream) != cudaSuccess)
                st = FBSDE_ERR_CUDA;
        }
        if (st != FBSDE_OK ||
            cudaMemcpyAsync(steps, ones.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice, g->stream) != cudaSuccess) {
            st = FBSDE_ERR_CUDA;
            break;
        }
        st = group_enqueue(g, th.data(), mm.data(), vv.data(), steps, lr, junk, junk + n);  // warm-up
        if (st == FBSDE_OK && cudaEventRecord(e0, g->stream) != cudaSuccess) st = FBSDE_ERR_CUDA;
        for (int s = 0; s < trial_steps && st == FBSDE_OK; ++s)
            st = group_enqueue(g, th.data(), mm.data(), vv.data(), steps, lr, junk, junk + n);
        if (st == FBSDE_OK && (cudaEventRecord(e1, g->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            st = FBSDE_ERR_CUDA;
        float ms = 0.f;
        if (st == FBSDE_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = FBSDE_ERR_CUDA;
        if (st == FBSDE_OK && (best < 0 || ms < best)) {
            best = ms;
            best_k = k;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(g->stream);
    release();
    if (st != FBSDE_OK) {
        for (int i = 0; i < n; ++i) g->ctx[i]->grid_cap = saved[i];
        return st;
    }
    for (int i = 0; i < n; ++i) {
        g->ctx[i]->grid_cap = cands[best_k][i];
        caps_out[i] = cands[best_k][i];
    }
    if (ms_out) *ms_out = best / (float)trial_steps;
    return FBSDE_OK;
}

}  // extern "C"
