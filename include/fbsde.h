/*
 * fbsde.h -- C ABI of libfbsde, the GB300 (sm_103a) hot path of the deep
 * FBSDE solver of Guler, Laignelet and Parpas, "Towards Robust and Stable Deep
 * Learning Algorithms for Forward Backward Stochastic Differential Equations"
 * (arXiv 1910.11623).
 *
 * What one call computes, for M sample paths over N uniform Euler steps:
 *   - Brownian increments Delta W_n ~ N(0, Delta t) (Section 2.2, Eq. "disc
 *     equations", first line) from a counter-based Philox4x32-10 stream;
 *   - the forward Euler-Maruyama path X_{n+1} = X_n + sigma(X_n) Delta W_n
 *     (Eq. "disc equations", second line; mu = 0 for every supported problem);
 *   - Y_n = u(t_n, X_n; Theta) and Z_n = grad_x u(t_n, X_n; Theta) for one
 *     network shared by all time points (Section 2.2), in the architectures of
 *     Section 3.1 (fully connected, ResNet, NAIS-Net);
 *   - the loss of Eq. "loss": the squared Y-residual
 *     Y_{n+1} - Y_n - phi Delta t - Z_n^T sigma Delta W_n summed over paths and
 *     steps, plus the squared terminal mismatch Y_N - g(X_N), plus (optional,
 *     the term suggested right after Eq. "loss") |Z_N - grad g(X_N)|^2;
 *   - its gradient in Theta, including the mixed second derivative that Z
 *     brings in; and an Adam step (Section 4.1, learning rate 1e-3).
 *
 * Conventions shared by every entry point:
 *   - Pointers named *_dev are CUDA device pointers; *_host are host pointers.
 *     The caller owns every buffer it passes; the context owns its workspace
 *     (allocated in fbsde_create, freed in fbsde_destroy).
 *   - All device work is enqueued on the stream given to fbsde_create, with no
 *     host synchronisation inside compute calls: results are ready once that
 *     stream reaches them.
 *   - Nothing throws across the ABI.  Every call returns an fbsde_status; on
 *     failure a one-line reason is kept per context (fbsde_last_error).
 *   - Parameter vector Theta: FP32, contiguous, in this order
 *       W_in [w x (D+1)] row-major (column 0 multiplies t), b_in [w];
 *       per layer l = 1..L:  FC / ResNet: W_l [w x w], b_l [w]
 *                            NAIS:        R_l [w x w], C_l [w], B_l [w x (D+1)]
 *       w_o [w], b_o [1].
 *     NAIS uses A_l = -R_l^T R_l - eps I (Section 3.1); the context forms A_l.
 *   - Noise: Philox4x32-10 (Salmon et al., SC'11) with key (seed mod 2^32,
 *     seed >> 32); the increment of step n, path m, dimensions 4q..4q+3 of
 *     iteration `iter` uses counter (q, n, m, iter mod 2^32); word pairs
 *     (w0,w1), (w2,w3) give two Box-Muller pairs with u = (k + 1/2) 2^-32.
 */
#ifndef FBSDE_H
#define FBSDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FBSDE_OK = 0,
    FBSDE_ERR_INVALID = 1,     /* bad argument or specification            */
    FBSDE_ERR_UNSUPPORTED = 2, /* valid request this library does not serve */
    FBSDE_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed          */
    FBSDE_ERR_NONFINITE = 4,   /* loss or gradient not finite (checked by fbsde_check_finite) */
    FBSDE_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up         */
    FBSDE_ERR_OOM = 6          /* device allocation failed                   */
} fbsde_status;

/* Benchmark problems of Section 4. */
typedef enum {
    FBSDE_BSB = 0, /* Black-Scholes-Barenblatt: sigma(x) = sigma diag(x),
                      phi = r (y - z^T x), g(x) = ||x||^2                       */
    FBSDE_HJB = 1  /* Hamilton-Jacobi-Bellman: sigma = sqrt(2) I, phi = ||z||^2,
                      g(x) = ln(0.5 (1 + ||x||^2))                              */
} fbsde_kind;

/* Network architectures of Section 3.1 / Section 4.1.  Every architecture
 * has an input lift h_0 = act(W_in (t, x) + b_in) and a linear read-out
 * y = w_o^T h_L + b_o. */
typedef enum {
    FBSDE_FC = 0,     /* h_l = act(W_l h_{l-1} + b_l)                           */
    FBSDE_RESNET = 1, /* h_l = h_{l-1} + act(W_l h_{l-1} + b_l)  (Euler, h = 1)  */
    FBSDE_NAIS = 2    /* h_l = h_{l-1} + h act(A_l h_{l-1} + B_l (t,x) + C_l)    */
} fbsde_arch_kind;

typedef enum { FBSDE_SIN = 0, FBSDE_TANH = 1 } fbsde_act;

/* Arithmetic of the network GEMMs.  FBSDE_FP32: CUDA-core FP32 throughout.
 * FBSDE_BF16: BF16 operands on the tcgen05 tensor cores with FP32
 * accumulation; X, Y, residuals, reductions and Adam stay FP32. */
/* Arithmetic forms.  FBSDE_FP8_HIDDEN: the BF16 form with the forward
 * contractions of the hidden layers (W_l h_{l-1}, l = 1..L, in the rollout
 * that gives Y, Z and the loss) in FP8 E4M3 with per-tensor scales and FP32
 * accumulation; the lift, the Z pass, the gradient sweeps and the weight
 * gradients stay BF16.  Needs an FC or ResNet network served by the fused
 * kernels (depth <= 8, width <= 256 and a multiple of 32, D <= 256), else
 * FBSDE_ERR_UNSUPPORTED at create. */
typedef enum { FBSDE_FP32 = 0, FBSDE_BF16 = 1, FBSDE_FP8_HIDDEN = 2 } fbsde_prec;

/* Problem specification (Section 2.1 Eq. "coupled" with mu = 0, Section 4). */
typedef struct {
    int kind;               /* fbsde_kind                                       */
    int D;                  /* space dimension d >= 1                           */
    int N;                  /* Euler steps, Delta t = T / N, N >= 1             */
    int M;                  /* paths (batch size of Eq. "loss"), M >= 1         */
    double T;               /* horizon > 0                                      */
    double r;               /* BSB rate r (ignored for HJB)                     */
    double sigma;           /* BSB volatility sigma (ignored for HJB)           */
    const double* x0_host;  /* X_0 = x0, D values, copied at create             */
    int terminal_grad_term; /* 1: add sum_m |Z_N - grad g(X_N)|^2 to the loss   */
} fbsde_problem;

/* Architecture specification (Section 3.1). */
typedef struct {
    int kind;          /* fbsde_arch_kind                                       */
    int width;         /* w, multiple of 16, 16 <= w <= 512 (the fused kernels  */
                       /* serve w <= 256; wider layers run layered)          */
    int depth;         /* L hidden layers / blocks, 0 <= L <= 16                */
    int act;           /* fbsde_act                                             */
    double h;          /* NAIS step h > 0 (Section 3.1); ignored otherwise      */
    double eps;        /* NAIS eps > 0 in A = -R^T R - eps I (paper: 0.01)      */
    double proj_delta; /* NAIS bound on ||R^T R||_F; <= 0 selects 0.99 (2/h - eps) */
    int prec;          /* fbsde_prec                                            */
} fbsde_arch;

typedef struct fbsde_ctx fbsde_ctx;

/* Create a context for one problem and architecture.  Validates both specs
 * before touching the GPU (FBSDE_ERR_INVALID on a bad value, with the reason
 * in *err_msg_host if non-NULL: up to 255 chars + NUL), then allocates the
 * workspace on the current CUDA device.  `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream).  N_max >= N sizes the workspace for later
 * fbsde_set_level calls (pass 0 for N_max = N).  On success *out owns the
 * context. */
fbsde_status fbsde_create(const fbsde_problem* problem, const fbsde_arch* arch,
                          uint64_t seed, void* cuda_stream, int N_max,
                          fbsde_ctx** out, char* err_msg_host);

/* Free the workspace and the context (NULL is accepted). */
fbsde_status fbsde_destroy(fbsde_ctx* ctx);

/* Number of FP32 entries of Theta for this context's problem/architecture. */
size_t fbsde_num_params(const fbsde_ctx* ctx);

/* Number of parameters for a specification, without a context or a GPU;
 * 0 if the specification is invalid. */
size_t fbsde_param_count(const fbsde_problem* problem, const fbsde_arch* arch);

/* Theta_0: Xavier-normal weights N(0, 2 / (fan_in + fan_out)) and zero
 * biases; normal number i of the flat vector comes from Philox counter
 * (i >> 2, 0, 0, 0) under key (seed_lo ^ 0x494E4954, seed_hi), Box-Muller
 * slot i & 3.  NAIS R blocks are then projected onto ||R^T R||_F <= delta
 * (Section 3.1).  theta_dev: fbsde_num_params floats. */
fbsde_status fbsde_init_params(fbsde_ctx* ctx, float* theta_dev);

/* Loss of Eq. "loss" and Y_0 = u(0, x0; Theta) for the paths of iteration
 * `iter`.  theta_dev: read-only; loss_dev, y0_dev: one float each. */
fbsde_status fbsde_rollout_loss(fbsde_ctx* ctx, const float* theta_dev, uint64_t iter,
                                float* loss_dev, float* y0_dev);

/* As fbsde_rollout_loss, plus d loss / d Theta into grad_dev (num_params
 * floats, overwritten).  The gradient includes the mixed derivative
 * d Z / d Theta (Section 2.2: Z by automatic differentiation). */
fbsde_status fbsde_rollout_grad(fbsde_ctx* ctx, const float* theta_dev, uint64_t iter,
                                float* loss_dev, float* y0_dev, float* grad_dev);

/* One training iteration (Section 4.1): loss and gradient at Theta for the
 * paths of iteration `step`, then Adam (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected, `step` >= 1 counts Adam steps) on theta_dev with moments
 * adam_m_dev / adam_v_dev (num_params floats each, caller zeroes them before
 * step 1), then the NAIS projection.  loss_dev / y0_dev receive the values at
 * the Theta the step started from. */
fbsde_status fbsde_train_step(fbsde_ctx* ctx, float* theta_dev, float* adam_m_dev,
                              float* adam_v_dev, uint64_t step, float lr,
                              float* loss_dev, float* y0_dev);

/* Per-point detail of one evaluation, for checking and analysis:
 * Y_dev [(N+1) * M] with index n * M + m, Z_dev [(N+1) * M * D] with index
 * (n * M + m) * D + i, path_loss_dev [M] (the per-path terms of Eq. "loss"
 * whose sum is the loss).  Any pointer may be NULL. */
fbsde_status fbsde_rollout_detail(fbsde_ctx* ctx, const float* theta_dev, uint64_t iter,
                                  float* Y_dev, float* Z_dev, float* path_loss_dev);

/* The Brownian increments and paths of iteration `iter` (Eq. "disc
 * equations"): dW_dev [N * M * D] index (n * M + m) * D + i, X_dev
 * [(N+1) * M * D] index (n * M + m) * D + i.  Either may be NULL. */
fbsde_status fbsde_sample_paths(fbsde_ctx* ctx, uint64_t iter, float* dW_dev, float* X_dev);

/* Raw Philox4x32-10 blocks: out_dev[4 j .. 4 j + 3] = Philox(ctr_dev[4 j ..
 * 4 j + 3], key) for j < count, key = (key0, key1).  Device pointers; the
 * work runs on `cuda_stream`.  The generator's definition is Salmon et al.,
 * SC'11; the paper only asks for Delta W_n ~ N(0, Delta t). */
fbsde_status fbsde_philox4x32_10(const uint32_t* ctr_dev, uint32_t key0, uint32_t key1,
                                 size_t count, uint32_t* out_dev, void* cuda_stream);

/* The tensor-core contraction every network layer of the BF16 form is built
 * on (Section 2.2: the same network is evaluated at all M (N+1) points, so each
 * layer is one product over points): C[m][n] = sum_k A(m,k) B(n,k) with BF16
 * operands (raw 16-bit patterns) and FP32 accumulation, on tcgen05.
 *   trans = 0: A [rows x K] row-major (lda), B [N x K] row-major (ldb);
 *   trans = 1: A [K x rows] row-major (lda), B [K x N] row-major (ldb), i.e.
 *              the contraction runs over the leading index (weight gradients).
 * C [rows x N] row-major (ldc), FP32, overwritten.  Requires rows, K >= 1,
 * N a multiple of 16 in [16, 256], lda and ldb multiples of 8, A and B
 * 16-byte aligned.  Runs on `cuda_stream` and waits for completion. */
fbsde_status fbsde_gemm_bf16(const void* A_dev, const void* B_dev, float* C_dev, int rows, int N, int K,
                             int lda, int ldb, int ldc, int trans, void* cuda_stream);

/* Multilevel discretisation (Section 3.2): switch the context to N_level
 * Euler steps (Delta t = T / N_level), 1 <= N_level <= N_max.  Theta and the
 * Adam moments are untouched, so training continues on the finer grid. */
fbsde_status fbsde_set_level(fbsde_ctx* ctx, int N_level);

/* fbsde_train_step with the step number in device memory: *step_dev (one
 * uint64, >= 1) keys the Brownian increments and Adam's bias correction as
 * `step` does, and is incremented by one on the device at the end of the
 * step.  Nothing of the step is then fixed on the host, so it can be captured
 * once in a CUDA graph and replayed (fbsde_graph_capture).  Same outputs and
 * errors as fbsde_train_step; step_dev must be non-NULL. */
fbsde_status fbsde_train_step_dev(fbsde_ctx* ctx, float* theta_dev, float* adam_m_dev, float* adam_v_dev,
                                  uint64_t* step_dev, float lr, float* loss_dev, float* y0_dev);

/* A CUDA graph of `steps` consecutive fbsde_train_step_dev calls (the whole
 * training step: paths, network, Z, loss, seeds, gradient, Adam), captured on
 * the context's stream and instantiated.  Replaying it with
 * fbsde_graph_launch enqueues the steps as one graph launch on that stream;
 * each replay advances *step_dev by `steps`.  The graph bakes in the
 * pointers, lr and the context's current level: capture again after
 * fbsde_set_level or fbsde_set_x0.  Requires a context created on a
 * non-default stream (FBSDE_ERR_UNSUPPORTED otherwise) and profiling off
 * (FBSDE_ERR_INVALID).  *out owns the graph; free it with
 * fbsde_graph_destroy before the context. */
typedef struct fbsde_graph fbsde_graph;
fbsde_status fbsde_graph_capture(fbsde_ctx* ctx, float* theta_dev, float* adam_m_dev, float* adam_v_dev,
                                 uint64_t* step_dev, float lr, float* loss_dev, float* y0_dev, int steps,
                                 fbsde_graph** out);
fbsde_status fbsde_graph_launch(fbsde_graph* graph);
fbsde_status fbsde_graph_destroy(fbsde_graph* graph);

/* Groups of independent instances (many FBSDEs of uneven D, N, M, width
 * trained at once; the paper trains one at a time, this is a batching layer
 * over its training step).
 *
 * fbsde_group_create: a group over n >= 1 distinct contexts, each created on
 * a non-default stream; `cuda_stream` (non-default) is the group's stream,
 * where group steps fork and join.  Instances run concurrently as far as
 * their streams differ (contexts sharing a stream run one after another).
 * The group does not own the contexts; destroy it before them.
 * FBSDE_ERR_INVALID on NULLs or repeated contexts.
 *
 * fbsde_group_train_step: one training step of every instance (as
 * fbsde_train_step_dev): theta, m, v are n device pointers (host array),
 * step_dev a device array of n uint64 step counters, loss_dev / y0_dev NULL
 * or device arrays of n floats (instance i writes index i).  On return the
 * group's stream is ordered after all of them.  In FBSDE_GROUP_GROUPED mode
 * (the default) the instances served by the fused BF16 kernels with the same
 * kernel variant (activation and network kind; FP8 forms excluded) and at
 * most two 128-point tiles per SM (a larger instance fills the GPU alone and
 * runs its whole step on its own stream), when there are at least two, run
 * their forward kernels as one persistent launch
 * and their backward kernels as one more, instance i on its own range of
 * CTAs (its grid cap, one per SM when unset); their other kernels, and every
 * other instance's whole step, run on the instances' streams.  The launch
 * arguments live in device memory owned by the group and are re-uploaded
 * (with a synchronisation of the group's stream) only when they change, e.g.
 * when theta pointers change.  In FBSDE_GROUP_STREAMS mode every instance
 * runs its whole step on its own stream, concurrently.
 *
 * fbsde_group_set_mode: FBSDE_GROUP_GROUPED or FBSDE_GROUP_STREAMS
 * (FBSDE_ERR_INVALID otherwise).
 *
 * fbsde_group_capture: `steps` group steps captured on the group's stream as
 * one CUDA graph (fbsde_graph_launch replays it with a single launch).
 *
 * fbsde_set_grid_cap: at most `ctas` CTAs (0: one per SM) for the context's
 * fused per-tile kernels, so that the instances of a group share the SMs.
 *
 * fbsde_group_autotune: times `trial_steps` group steps (after one warm-up)
 * for each candidate split of the SMs (all SMs for every instance; SMs in
 * proportion to each instance's contraction work, and twice that; half and a
 * quarter of the SMs each) on
 * scratch copies of theta (Adam moments zero, step 1), keeps the fastest
 * split in the contexts and writes each instance's cap to caps_out (n ints)
 * and the step time in ms to *ms_out (may be NULL).  Synchronises the group's
 * stream; the caller's theta is only read. */
typedef struct fbsde_group fbsde_group;
enum { FBSDE_GROUP_STREAMS = 0, FBSDE_GROUP_GROUPED = 1 };
/* A new non-blocking CUDA stream (cudaStream_t in *out), for callers whose
 * framework hands out pooled streams, so that every instance of a group can
 * have one of its own; fbsde_stream_destroy frees it (NULL accepted). */
fbsde_status fbsde_stream_create(void** out);
fbsde_status fbsde_stream_destroy(void* stream);
fbsde_status fbsde_group_create(fbsde_ctx* const* ctxs, int n, void* cuda_stream, fbsde_group** out);
fbsde_status fbsde_group_destroy(fbsde_group* group);
fbsde_status fbsde_group_set_mode(fbsde_group* group, int mode);
fbsde_status fbsde_group_train_step(fbsde_group* group, float* const* theta_dev, float* const* adam_m_dev,
                                    float* const* adam_v_dev, uint64_t* step_dev, float lr, float* loss_dev,
                                    float* y0_dev);
fbsde_status fbsde_group_capture(fbsde_group* group, float* const* theta_dev, float* const* adam_m_dev,
                                 float* const* adam_v_dev, uint64_t* step_dev, float lr, float* loss_dev,
                                 float* y0_dev, int steps, fbsde_graph** out);
fbsde_status fbsde_set_grid_cap(fbsde_ctx* ctx, int ctas);
fbsde_status fbsde_group_autotune(fbsde_group* group, const float* const* theta_dev, float lr, int trial_steps,
                                  int* caps_out, float* ms_out);

/* Multilevel training (Section 3.2: coarse grids first, the number of Euler
 * steps growing geometrically, e.g. 2, 4, 8, 16, 32 in Section 4.3): for
 * level i = 0 .. n_levels-1, switch to N_levels[i] steps (as
 * fbsde_set_level) and run steps_per_level[i] Adam steps (as
 * fbsde_train_step) numbered first_step, first_step + 1, ... across all
 * levels, so every step draws fresh Brownian increments.  Theta and the Adam
 * moments carry over from level to level.
 *   N_levels_host, steps_per_level_host: n_levels host ints (each level in
 *     [1, N_max], each count >= 0); n_levels >= 1.
 *   loss_trace_dev, y0_trace_dev: NULL or device arrays of
 *     sum(steps_per_level) floats; step k of the schedule writes its loss and
 *     Y_0 at index k.
 * The context stays at the last level.  Enqueued on the context's stream with
 * no host synchronisation; the arguments are checked before anything is
 * enqueued (FBSDE_ERR_INVALID). */
fbsde_status fbsde_train_schedule(fbsde_ctx* ctx, float* theta_dev, float* adam_m_dev, float* adam_v_dev,
                                  const int* N_levels_host, const int* steps_per_level_host, int n_levels,
                                  uint64_t first_step, float lr, float* loss_trace_dev,
                                  float* y0_trace_dev);

/* Replace the initial condition X_0 = x0 (D host doubles), e.g. for the
 * generalisation test of Section 4.2 (perturbed X_0, same Theta). */
fbsde_status fbsde_set_x0(fbsde_ctx* ctx, const double* x0_host);

/* Waits for the context's stream, then reports FBSDE_ERR_TIMEOUT if a
 * tensor-core kernel of this context gave up a bounded wait (its tiles were
 * left incomplete and the results since the last check are invalid), else
 * FBSDE_ERR_NONFINITE if the last loss or gradient held a NaN or Inf.  Both
 * flags are cleared by the call. */
fbsde_status fbsde_check_finite(fbsde_ctx* ctx);

/* Test hook for the bounded waits of the tensor-core kernels (not a
 * computation of the paper).  The next launch of the context's pipelined
 * forward kernel and of its pipelined backward kernel (FC and ResNet networks
 * in BF16) each start with a wait on a barrier that nothing completes, with a
 * wait budget of about 10 us: every role of the kernel gives up there, before
 * it issues any copy or contraction, sets the context's device error flag and
 * releases its TMEM, so the launches complete and the context stays usable.
 * The next fbsde_check_finite then returns FBSDE_ERR_TIMEOUT (and clears the
 * flag); the results of those launches are invalid.  The hook disarms itself
 * at the launch it affects.  FBSDE_ERR_UNSUPPORTED for a context whose
 * network is not served by the pipelined kernels (NAIS-Net, FP8, FP32, the
 * layered path). */
fbsde_status fbsde_test_timeout_once(fbsde_ctx* ctx);

/* Replace x0 from a device buffer (D floats), ordered on the context stream:
 * the variant of fbsde_set_x0 for callers that stage x0 in device memory. */
fbsde_status fbsde_set_x0_device(fbsde_ctx* ctx, const float* x0_dev);

/* Kernel-class timing.  Classes: 0 = contractions over the points (network
 * forward, Z-reverse, tangent and adjoint sweeps), 1 = weight-gradient
 * contractions, 2 = everything else (noise and paths, residuals and loss,
 * reductions, Adam).  fbsde_profile_enable(ctx, 1) resets the counters and
 * brackets every later launch with CUDA events on the context stream;
 * fbsde_profile_read waits for the stream and returns, for class `cls`, the
 * summed device time in ms, the number of launches and the algorithmic
 * floating-point operations of those launches (2 per multiply-add of the
 * method; recomputation and padding excluded). */
fbsde_status fbsde_profile_enable(fbsde_ctx* ctx, int on);
fbsde_status fbsde_profile_read(fbsde_ctx* ctx, int cls, double* ms_total, uint64_t* launches,
                                double* flops);

/* Kernels launched by this context since it was created. */
uint64_t fbsde_launch_count(const fbsde_ctx* ctx);

/* The residual, loss-seed and loss step (what fbsde_rollout_loss does after
 * the network pass) for callers that cannot allocate device memory, e.g. an
 * application whose own pool owns all device memory, or a loop that cannot
 * afford an allocation's implicit synchronisation.  The paper has no
 * counterpart: this is a deployment variant of the same step.
 * Inputs, in the layouts of fbsde_sample_paths and fbsde_rollout_detail:
 * X_dev [(N+1) M D], dW_dev [N M D], Y_dev [(N+1) M], Z_dev [(N+1) M D].
 * Outputs: alpha_dev [(N+1) M] = d loss / d Y_n, V_dev [(N+1) M D] =
 * d loss / d Z_n, loss_dev and y0_dev (one float each), as fbsde_rollout_loss.
 * No allocation: the per-path FP64 loss terms go to a fixed device array of
 * 65536 doubles (512 KiB, reserved on every GPU that loads the library until
 * the process exits), so M must be <= 65536 (FBSDE_ERR_INVALID otherwise,
 * with the reason in err_msg_host if non-NULL, 256 bytes).  Each call writes
 * all M terms before summing them, so nothing has to start at zero, but every
 * call on a device uses the same array: calls whose work overlaps on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * The first call on a device looks up the array's device address once (with
 * that device current); make that first call before any stream capture.
 * Work is enqueued on `cuda_stream`; no host synchronisation. */
fbsde_status fbsde_residual_loss_noalloc(const fbsde_problem* problem, const float* X_dev,
                                         const float* dW_dev, const float* Y_dev, const float* Z_dev,
                                         float* alpha_dev, float* V_dev, float* loss_dev, float* y0_dev,
                                         void* cuda_stream, char* err_msg_host);

const char* fbsde_status_string(fbsde_status s);
const char* fbsde_last_error(const fbsde_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FBSDE_H */
