"""ctypes binding of libfbsde (include/fbsde.h): argument marshalling only.

Each ``fbsde_*`` function below has the name, arguments and meaning of the C
entry point it wraps; device pointers are passed as integers (for torch
tensors, ``tensor.data_ptr()``).  Loading fails loudly if the library has not
been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_size_t, c_uint32, c_uint64, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfbsde.so")

FBSDE_OK, FBSDE_ERR_INVALID, FBSDE_ERR_UNSUPPORTED, FBSDE_ERR_CUDA = 0, 1, 2, 3
FBSDE_ERR_NONFINITE, FBSDE_ERR_TIMEOUT, FBSDE_ERR_OOM = 4, 5, 6
FBSDE_BSB, FBSDE_HJB = 0, 1
FBSDE_FC, FBSDE_RESNET, FBSDE_NAIS = 0, 1, 2
FBSDE_SIN, FBSDE_TANH = 0, 1
FBSDE_FP32, FBSDE_BF16, FBSDE_FP8_HIDDEN = 0, 1, 2
FBSDE_GROUP_STREAMS, FBSDE_GROUP_GROUPED = 0, 1


class fbsde_problem(ctypes.Structure):
    _fields_ = [("kind", c_int), ("D", c_int), ("N", c_int), ("M", c_int),
                ("T", c_double), ("r", c_double), ("sigma", c_double),
                ("x0_host", POINTER(c_double)), ("terminal_grad_term", c_int)]


class fbsde_arch(ctypes.Structure):
    _fields_ = [("kind", c_int), ("width", c_int), ("depth", c_int), ("act", c_int),
                ("h", c_double), ("eps", c_double), ("proj_delta", c_double), ("prec", c_int)]


# name -> (restype, argtypes); the same list is checked against include/fbsde.h
SIGNATURES = {
    "fbsde_create": (c_int, [POINTER(fbsde_problem), POINTER(fbsde_arch), c_uint64, c_void_p, c_int,
                             POINTER(c_void_p), c_char_p]),
    "fbsde_destroy": (c_int, [c_void_p]),
    "fbsde_num_params": (c_size_t, [c_void_p]),
    "fbsde_param_count": (c_size_t, [POINTER(fbsde_problem), POINTER(fbsde_arch)]),
    "fbsde_init_params": (c_int, [c_void_p, c_void_p]),
    "fbsde_rollout_loss": (c_int, [c_void_p, c_void_p, c_uint64, c_void_p, c_void_p]),
    "fbsde_rollout_grad": (c_int, [c_void_p, c_void_p, c_uint64, c_void_p, c_void_p, c_void_p]),
    "fbsde_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_uint64, c_float,
                                 c_void_p, c_void_p]),
    "fbsde_rollout_detail": (c_int, [c_void_p, c_void_p, c_uint64, c_void_p, c_void_p, c_void_p]),
    "fbsde_sample_paths": (c_int, [c_void_p, c_uint64, c_void_p, c_void_p]),
    "fbsde_philox4x32_10": (c_int, [c_void_p, c_uint32, c_uint32, c_size_t, c_void_p, c_void_p]),
    "fbsde_gemm_bf16": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int, c_int,
                                c_int, c_void_p]),
    "fbsde_set_level": (c_int, [c_void_p, c_int]),
    "fbsde_train_step_dev": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p,
                                     c_void_p]),
    "fbsde_graph_capture": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_void_p,
                                    c_void_p, c_int, POINTER(c_void_p)]),
    "fbsde_graph_launch": (c_int, [c_void_p]),
    "fbsde_group_create": (c_int, [POINTER(c_void_p), c_int, c_void_p, POINTER(c_void_p)]),
    "fbsde_group_destroy": (c_int, [c_void_p]),
    "fbsde_group_set_mode": (c_int, [c_void_p, c_int]),
    "fbsde_group_train_step": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                                       c_void_p, c_float, c_void_p, c_void_p]),
    "fbsde_group_capture": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                                    c_void_p, c_float, c_void_p, c_void_p, c_int, POINTER(c_void_p)]),
    "fbsde_set_grid_cap": (c_int, [c_void_p, c_int]),
    "fbsde_stream_create": (c_int, [POINTER(c_void_p)]),
    "fbsde_stream_destroy": (c_int, [c_void_p]),
    "fbsde_group_autotune": (c_int, [c_void_p, POINTER(c_void_p), c_float, c_int, POINTER(c_int),
                                     POINTER(c_float)]),
    "fbsde_graph_destroy": (c_int, [c_void_p]),
    "fbsde_train_schedule": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int), POINTER(c_int), c_int,
                                     c_uint64, c_float, c_void_p, c_void_p]),
    "fbsde_set_x0": (c_int, [c_void_p, POINTER(c_double)]),
    "fbsde_check_finite": (c_int, [c_void_p]),
    "fbsde_test_timeout_once": (c_int, [c_void_p]),
    "fbsde_set_x0_device": (c_int, [c_void_p, c_void_p]),
    "fbsde_profile_enable": (c_int, [c_void_p, c_int]),
    "fbsde_profile_read": (c_int, [c_void_p, c_int, POINTER(c_double), POINTER(c_uint64),
                                   POINTER(c_double)]),
    "fbsde_launch_count": (c_uint64, [c_void_p]),
    "fbsde_residual_loss_noalloc": (c_int, [POINTER(fbsde_problem), c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_char_p]),
    "fbsde_status_string": (c_char_p, [c_int]),
    "fbsde_last_error": (c_char_p, [c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfbsde.so and set the prototypes; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"libfbsde.so not found at {path}: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FBSDEError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {status_string(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


def status_string(s: int) -> str:
    return load().fbsde_status_string(s).decode()


def check(status: int, where: str, ctx=None):
    if status != FBSDE_OK:
        detail = load().fbsde_last_error(ctx).decode() if ctx else ""
        raise FBSDEError(status, where, detail)


# ---- entry points, same names as the C ABI ----------------------------------

def fbsde_create(problem: fbsde_problem, arch: fbsde_arch, seed: int, stream: int, N_max: int = 0):
    ctx = c_void_p()
    msg = ctypes.create_string_buffer(256)
    s = load().fbsde_create(ctypes.byref(problem), ctypes.byref(arch), seed & (2**64 - 1),
                            c_void_p(stream or None), N_max, ctypes.byref(ctx), msg)
    if s != FBSDE_OK:
        raise FBSDEError(s, "fbsde_create", msg.value.decode())
    return ctx


def fbsde_destroy(ctx):
    return load().fbsde_destroy(ctx)


def fbsde_num_params(ctx) -> int:
    return int(load().fbsde_num_params(ctx))


def fbsde_param_count(problem: fbsde_problem, arch: fbsde_arch) -> int:
    return int(load().fbsde_param_count(ctypes.byref(problem), ctypes.byref(arch)))


def fbsde_init_params(ctx, theta_ptr: int):
    check(load().fbsde_init_params(ctx, c_void_p(theta_ptr)), "fbsde_init_params", ctx)


def fbsde_rollout_loss(ctx, theta_ptr: int, it: int, loss_ptr: int, y0_ptr: int):
    check(load().fbsde_rollout_loss(ctx, c_void_p(theta_ptr), it, c_void_p(loss_ptr or None),
                                    c_void_p(y0_ptr or None)), "fbsde_rollout_loss", ctx)


def fbsde_rollout_grad(ctx, theta_ptr: int, it: int, loss_ptr: int, y0_ptr: int, grad_ptr: int):
    check(load().fbsde_rollout_grad(ctx, c_void_p(theta_ptr), it, c_void_p(loss_ptr or None),
                                    c_void_p(y0_ptr or None), c_void_p(grad_ptr)),
          "fbsde_rollout_grad", ctx)


def fbsde_train_step(ctx, theta_ptr: int, m_ptr: int, v_ptr: int, step: int, lr: float,
                     loss_ptr: int, y0_ptr: int):
    check(load().fbsde_train_step(ctx, c_void_p(theta_ptr), c_void_p(m_ptr), c_void_p(v_ptr), step,
                                  lr, c_void_p(loss_ptr or None), c_void_p(y0_ptr or None)),
          "fbsde_train_step", ctx)


def fbsde_rollout_detail(ctx, theta_ptr: int, it: int, Y_ptr: int, Z_ptr: int, pl_ptr: int):
    check(load().fbsde_rollout_detail(ctx, c_void_p(theta_ptr), it, c_void_p(Y_ptr or None),
                                      c_void_p(Z_ptr or None), c_void_p(pl_ptr or None)),
          "fbsde_rollout_detail", ctx)


def fbsde_sample_paths(ctx, it: int, dW_ptr: int, X_ptr: int):
    check(load().fbsde_sample_paths(ctx, it, c_void_p(dW_ptr or None), c_void_p(X_ptr or None)),
          "fbsde_sample_paths", ctx)


def fbsde_philox4x32_10(ctr_ptr: int, key0: int, key1: int, count: int, out_ptr: int, stream: int):
    check(load().fbsde_philox4x32_10(c_void_p(ctr_ptr), key0, key1, count, c_void_p(out_ptr),
                                     c_void_p(stream or None)), "fbsde_philox4x32_10")


def fbsde_gemm_bf16(A_ptr: int, B_ptr: int, C_ptr: int, rows: int, N: int, K: int, lda: int, ldb: int,
                    ldc: int, trans: int, stream: int):
    check(load().fbsde_gemm_bf16(c_void_p(A_ptr), c_void_p(B_ptr), c_void_p(C_ptr), rows, N, K, lda, ldb, ldc,
                                 trans, c_void_p(stream or None)), "fbsde_gemm_bf16")


def fbsde_train_step_dev(ctx, theta_ptr: int, m_ptr: int, v_ptr: int, step_ptr: int, lr: float,
                         loss_ptr: int = 0, y0_ptr: int = 0):
    check(load().fbsde_train_step_dev(ctx, c_void_p(theta_ptr), c_void_p(m_ptr), c_void_p(v_ptr),
                                      c_void_p(step_ptr), lr, c_void_p(loss_ptr or None),
                                      c_void_p(y0_ptr or None)),
          "fbsde_train_step_dev", ctx)


def fbsde_graph_capture(ctx, theta_ptr: int, m_ptr: int, v_ptr: int, step_ptr: int, lr: float,
                        loss_ptr: int, y0_ptr: int, steps: int):
    out = c_void_p()
    check(load().fbsde_graph_capture(ctx, c_void_p(theta_ptr), c_void_p(m_ptr), c_void_p(v_ptr),
                                     c_void_p(step_ptr), lr, c_void_p(loss_ptr or None),
                                     c_void_p(y0_ptr or None), steps, ctypes.byref(out)),
          "fbsde_graph_capture", ctx)
    return out


def fbsde_graph_launch(graph, ctx=None):
    check(load().fbsde_graph_launch(graph), "fbsde_graph_launch", ctx)


def fbsde_graph_destroy(graph):
    load().fbsde_graph_destroy(graph)


def _ptr_array(ptrs):
    return (c_void_p * max(len(ptrs), 1))(*[c_void_p(p) for p in ptrs])


def fbsde_group_create(ctxs, stream: int):
    arr = (c_void_p * len(ctxs))(*ctxs)
    out = c_void_p()
    check(load().fbsde_group_create(arr, len(ctxs), c_void_p(stream or None), ctypes.byref(out)),
          "fbsde_group_create")
    return out


def fbsde_group_destroy(group):
    load().fbsde_group_destroy(group)


def fbsde_group_set_mode(group, mode: int):
    check(load().fbsde_group_set_mode(group, mode), "fbsde_group_set_mode")


def fbsde_group_train_step(group, theta_ptrs, m_ptrs, v_ptrs, step_ptr: int, lr: float, loss_ptr: int = 0,
                           y0_ptr: int = 0):
    check(load().fbsde_group_train_step(group, _ptr_array(theta_ptrs), _ptr_array(m_ptrs), _ptr_array(v_ptrs),
                                        c_void_p(step_ptr), lr, c_void_p(loss_ptr or None),
                                        c_void_p(y0_ptr or None)),
          "fbsde_group_train_step")


def fbsde_group_capture(group, theta_ptrs, m_ptrs, v_ptrs, step_ptr: int, lr: float, loss_ptr: int,
                        y0_ptr: int, steps: int):
    out = c_void_p()
    check(load().fbsde_group_capture(group, _ptr_array(theta_ptrs), _ptr_array(m_ptrs), _ptr_array(v_ptrs),
                                     c_void_p(step_ptr), lr, c_void_p(loss_ptr or None),
                                     c_void_p(y0_ptr or None), steps, ctypes.byref(out)),
          "fbsde_group_capture")
    return out


def fbsde_stream_create() -> int:
    out = c_void_p()
    check(load().fbsde_stream_create(ctypes.byref(out)), "fbsde_stream_create")
    return int(out.value)


def fbsde_stream_destroy(stream: int):
    load().fbsde_stream_destroy(c_void_p(stream or None))


def fbsde_set_grid_cap(ctx, ctas: int):
    check(load().fbsde_set_grid_cap(ctx, ctas), "fbsde_set_grid_cap", ctx)


def fbsde_group_autotune(group, theta_ptrs, lr: float, trial_steps: int):
    n = len(theta_ptrs)
    caps = (c_int * n)()
    ms = c_float()
    check(load().fbsde_group_autotune(group, _ptr_array(theta_ptrs), lr, trial_steps, caps, ctypes.byref(ms)),
          "fbsde_group_autotune")
    return list(caps), float(ms.value)


def fbsde_set_level(ctx, N: int):
    check(load().fbsde_set_level(ctx, N), "fbsde_set_level", ctx)


def fbsde_train_schedule(ctx, theta_ptr: int, m_ptr: int, v_ptr: int, levels, steps, first_step: int,
                         lr: float, loss_trace_ptr: int = 0, y0_trace_ptr: int = 0):
    n = len(levels)
    if len(steps) != n:
        raise ValueError("levels and steps must have the same length")
    lv = (c_int * max(n, 1))(*levels)
    st = (c_int * max(n, 1))(*steps)
    check(load().fbsde_train_schedule(ctx, c_void_p(theta_ptr), c_void_p(m_ptr), c_void_p(v_ptr), lv, st, n,
                                      first_step, lr, c_void_p(loss_trace_ptr or None),
                                      c_void_p(y0_trace_ptr or None)),
          "fbsde_train_schedule", ctx)


def fbsde_set_x0(ctx, x0):
    arr = (c_double * len(x0))(*[float(v) for v in x0])
    check(load().fbsde_set_x0(ctx, arr), "fbsde_set_x0", ctx)


def fbsde_check_finite(ctx):
    check(load().fbsde_check_finite(ctx), "fbsde_check_finite", ctx)


def fbsde_test_timeout_once(ctx):
    check(load().fbsde_test_timeout_once(ctx), "fbsde_test_timeout_once", ctx)


def fbsde_set_x0_device(ctx, x0_ptr: int):
    check(load().fbsde_set_x0_device(ctx, c_void_p(x0_ptr)), "fbsde_set_x0_device", ctx)


def fbsde_profile_enable(ctx, on: bool):
    check(load().fbsde_profile_enable(ctx, int(bool(on))), "fbsde_profile_enable", ctx)


def fbsde_profile_read(ctx, cls: int):
    """-> (ms_total, launches, flops) of kernel class `cls`."""
    ms, n, fl = c_double(), c_uint64(), c_double()
    check(load().fbsde_profile_read(ctx, cls, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)),
          "fbsde_profile_read", ctx)
    return ms.value, int(n.value), fl.value


def fbsde_launch_count(ctx) -> int:
    return int(load().fbsde_launch_count(ctx))


def fbsde_residual_loss_noalloc(problem: fbsde_problem, X_ptr: int, dW_ptr: int, Y_ptr: int, Z_ptr: int,
                                alpha_ptr: int, V_ptr: int, loss_ptr: int, y0_ptr: int, stream: int):
    """Residuals, seeds and loss from caller-held paths and network values,
    without any device allocation (scratch in a fixed device array, M <= 65536)."""
    msg = ctypes.create_string_buffer(256)
    s = load().fbsde_residual_loss_noalloc(ctypes.byref(problem), c_void_p(X_ptr), c_void_p(dW_ptr),
                                           c_void_p(Y_ptr), c_void_p(Z_ptr), c_void_p(alpha_ptr),
                                           c_void_p(V_ptr), c_void_p(loss_ptr), c_void_p(y0_ptr),
                                           c_void_p(stream or None), msg)
    if s != FBSDE_OK:
        raise FBSDEError(s, "fbsde_residual_loss_noalloc", msg.value.decode())


def fbsde_status_string(s: int) -> str:
    return status_string(s)


def fbsde_last_error(ctx) -> str:
    return load().fbsde_last_error(ctx).decode()
