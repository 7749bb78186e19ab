"""Torch-facing wrapper of libfbsde: tensor ownership and the current stream.

PyTorch only allocates the caller-owned buffers (Theta, gradient, Adam
moments, output scalars) and supplies the CUDA stream; every step of the
method runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

_KIND = {"bsb": L.FBSDE_BSB, "hjb": L.FBSDE_HJB}
_ARCH = {"fc": L.FBSDE_FC, "resnet": L.FBSDE_RESNET, "nais": L.FBSDE_NAIS}
_ACT = {"sin": L.FBSDE_SIN, "tanh": L.FBSDE_TANH}
_PREC = {"fp32": L.FBSDE_FP32, "bf16": L.FBSDE_BF16, "fp8": L.FBSDE_FP8_HIDDEN}


@dataclass
class ProblemSpec:
    """FBSDE of Section 4 (mu = 0).  kind 'bsb' or 'hjb'."""
    kind: str
    D: int
    N: int
    M: int
    x0: Sequence[float]
    T: float = 1.0
    r: float = 0.05
    sigma: float = 0.4
    terminal_grad_term: bool = False

    def to_c(self):
        x0 = np.ascontiguousarray(np.asarray(self.x0, dtype=np.float64))
        if x0.shape != (self.D,):
            raise ValueError(f"x0 must have {self.D} entries")
        st = L.fbsde_problem(kind=_KIND[self.kind], D=self.D, N=self.N, M=self.M, T=self.T,
                             r=self.r, sigma=self.sigma,
                             x0_host=x0.ctypes.data_as(L.POINTER(L.c_double)),
                             terminal_grad_term=int(bool(self.terminal_grad_term)))
        return st, x0  # keep x0 alive while the struct is in use


@dataclass
class ArchSpec:
    """Network of Section 3.1: kind 'fc' | 'resnet' | 'nais'; act 'sin' | 'tanh';
    prec 'fp32' (CUDA-core form) | 'bf16' (tcgen05 tensor-core form) | 'fp8' (the BF16 form with
    the hidden-layer forward contractions in E4M3)."""
    kind: str
    width: int
    depth: int
    act: str
    prec: str = "fp32"
    h: float = 1.0
    eps: float = 0.01
    proj_delta: float = 0.0

    def to_c(self):
        return L.fbsde_arch(kind=_ARCH[self.kind], width=self.width, depth=self.depth,
                            act=_ACT[self.act], h=self.h, eps=self.eps,
                            proj_delta=self.proj_delta, prec=_PREC[self.prec])


def param_count(problem: ProblemSpec, arch: ArchSpec) -> int:
    p, _keep = problem.to_c()
    return L.fbsde_param_count(p, arch.to_c())


class Solver:
    """One libfbsde context on the current CUDA device and stream."""

    def __init__(self, problem: ProblemSpec, arch: ArchSpec, seed: int = 0,
                 stream: Optional[torch.cuda.Stream] = None, N_max: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("libfbsde needs a CUDA device")
        self.problem, self.arch, self.seed = problem, arch, seed
        self.stream = stream or torch.cuda.current_stream()
        p, self._x0 = problem.to_c()
        self.ctx = L.fbsde_create(p, arch.to_c(), seed, self.stream.cuda_stream, N_max)
        self.n_params = L.fbsde_num_params(self.ctx)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self._loss = torch.zeros(1, device=dev)
        self._y0 = torch.zeros(1, device=dev)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            L.fbsde_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_theta(self, t: torch.Tensor):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.numel() != self.n_params:
            raise ValueError(f"expected a contiguous CUDA float32 tensor of {self.n_params} entries")

    def init_params(self) -> torch.Tensor:
        """Theta_0 (Xavier; NAIS-Net blocks projected), written on the solver's
        stream; the caller's current stream is ordered after it, so the tensor
        can be used (or copied) there at once.  The other methods enqueue on
        the solver's stream only: run them under torch.cuda.stream(solver.stream)
        or order the streams yourself."""
        cur = torch.cuda.current_stream(self.device)
        theta = torch.empty(self.n_params, device=self.device)
        self.stream.wait_stream(cur)
        L.fbsde_init_params(self.ctx, theta.data_ptr())
        cur.wait_stream(self.stream)
        return theta

    def rollout_loss(self, theta: torch.Tensor, iteration: int):
        self._check_theta(theta)
        loss = torch.empty(1, device=self.device)
        y0 = torch.empty(1, device=self.device)
        L.fbsde_rollout_loss(self.ctx, theta.data_ptr(), iteration, loss.data_ptr(), y0.data_ptr())
        return loss, y0

    def rollout_grad(self, theta: torch.Tensor, iteration: int, grad: Optional[torch.Tensor] = None):
        self._check_theta(theta)
        loss = torch.empty(1, device=self.device)
        y0 = torch.empty(1, device=self.device)
        if grad is None:
            grad = torch.empty(self.n_params, device=self.device)
        L.fbsde_rollout_grad(self.ctx, theta.data_ptr(), iteration, loss.data_ptr(), y0.data_ptr(),
                             grad.data_ptr())
        return loss, y0, grad

    def train_step(self, theta, m, v, step: int, lr: float = 1e-3, loss=None, y0=None):
        for t in (theta, m, v):
            self._check_theta(t)
        loss = self._loss if loss is None else loss
        y0 = self._y0 if y0 is None else y0
        L.fbsde_train_step(self.ctx, theta.data_ptr(), m.data_ptr(), v.data_ptr(), step, lr,
                           loss.data_ptr(), y0.data_ptr())
        return loss, y0

    def rollout_detail(self, theta: torch.Tensor, iteration: int):
        self._check_theta(theta)
        P = self.problem.M * (self.problem_N + 1)
        Y = torch.empty(P, device=self.device)
        Z = torch.empty(P * self.problem.D, device=self.device)
        pl = torch.empty(self.problem.M, device=self.device)
        L.fbsde_rollout_detail(self.ctx, theta.data_ptr(), iteration, Y.data_ptr(), Z.data_ptr(),
                               pl.data_ptr())
        N1 = self.problem_N + 1
        return Y.view(N1, self.problem.M), Z.view(N1, self.problem.M, self.problem.D), pl

    def sample_paths(self, iteration: int):
        M, D, N = self.problem.M, self.problem.D, self.problem_N
        dW = torch.empty(N, M, D, device=self.device)
        X = torch.empty(N + 1, M, D, device=self.device)
        L.fbsde_sample_paths(self.ctx, iteration, dW.data_ptr(), X.data_ptr())
        return dW, X

    @property
    def problem_N(self) -> int:
        return getattr(self, "_level", self.problem.N)

    def set_level(self, N: int):
        L.fbsde_set_level(self.ctx, N)
        self._level = N

    def set_x0(self, x0):
        L.fbsde_set_x0(self.ctx, list(x0))

    def train_step_dev(self, theta, m, v, step_dev, lr: float = 1e-3, loss=None, y0=None):
        """One training step numbered by the device word step_dev (int64
        tensor of one element), which the step advances by one."""
        loss = loss if loss is not None else torch.empty(1, device=self.device)
        y0 = y0 if y0 is not None else torch.empty(1, device=self.device)
        L.fbsde_train_step_dev(self.ctx, theta.data_ptr(), m.data_ptr(), v.data_ptr(), step_dev.data_ptr(), lr,
                               loss.data_ptr(), y0.data_ptr())
        return loss, y0

    def capture_train_steps(self, theta, m, v, step_dev, lr: float = 1e-3, steps: int = 1):
        """CUDA graph of `steps` training steps (see TrainGraph)."""
        return TrainGraph(self, theta, m, v, step_dev, lr, steps)

    def train_schedule(self, theta, m, v, levels, steps, first_step: int, lr: float):
        """Multilevel training (Section 3.2): steps[i] Adam steps on a grid of
        levels[i] Euler steps, Theta and the moments carried across levels.
        Returns the per-step loss and Y_0 traces (device tensors)."""
        total = int(sum(steps))
        loss = torch.empty(max(total, 1), device=self.device)
        y0 = torch.empty(max(total, 1), device=self.device)
        L.fbsde_train_schedule(self.ctx, theta.data_ptr(), m.data_ptr(), v.data_ptr(), list(levels),
                               list(steps), first_step, lr, loss.data_ptr(), y0.data_ptr())
        self._level = int(levels[-1])
        return loss[:total], y0[:total]

    def generalisation(self, theta, x0s, iteration: int = 7 * 10**6):
        """Y_0 = u(0, x0') of a trained Theta at other initial conditions
        (Section 4.2: the parameters are not re-optimised).  Restores x0."""
        out = []
        try:
            for k, x0 in enumerate(x0s):
                self.set_x0(x0)
                _, y0 = self.rollout_loss(theta, iteration + k)
                out.append(float(y0.item()))
        finally:
            self.set_x0(self.problem.x0)
        return out

    def check_finite(self):
        L.fbsde_check_finite(self.ctx)


class TrainGraph:
    """A captured, instantiated CUDA graph of consecutive training steps of a
    Solver (fbsde_graph_capture); launch() replays them on the solver's
    stream and advances the device step counter.  The loss and Y_0 of the
    last replayed step are in .loss and .y0."""

    def __init__(self, solver: "Solver", theta, m, v, step_dev, lr: float, steps: int):
        self.solver, self.steps = solver, steps
        self._keep = (theta, m, v, step_dev)
        self.loss = torch.empty(1, device=solver.device)
        self.y0 = torch.empty(1, device=solver.device)
        self.handle = L.fbsde_graph_capture(solver.ctx, theta.data_ptr(), m.data_ptr(), v.data_ptr(),
                                            step_dev.data_ptr(), lr, self.loss.data_ptr(), self.y0.data_ptr(),
                                            steps)

    def launch(self):
        L.fbsde_graph_launch(self.handle, self.solver.ctx)

    def close(self):
        if self.handle:
            L.fbsde_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Independent instances (each a Solver on its own stream) trained
    together: one group step trains every instance (the fused BF16 ones of a
    common kernel variant and at most two tiles per SM through one grouped
    forward and one grouped backward launch, mode "grouped"; or every step on
    its own stream, mode
    "streams"), capture() makes it one CUDA graph, autotune() splits the SMs
    between the instances (cached per set of shapes in a JSON file)."""

    def __init__(self, solvers, stream: Optional[torch.cuda.Stream] = None):
        self.solvers = list(solvers)
        self.stream = stream or torch.cuda.Stream()
        self.handle = L.fbsde_group_create([s.ctx for s in self.solvers], self.stream.cuda_stream)
        n = len(self.solvers)
        self.loss = torch.empty(n, device="cuda")
        self.y0 = torch.empty(n, device="cuda")

    def _ptrs(self, ts):
        return [t.data_ptr() for t in ts]

    def set_mode(self, mode: str):
        """"grouped" (default) or "streams"."""
        L.fbsde_group_set_mode(self.handle, {"streams": L.FBSDE_GROUP_STREAMS,
                                             "grouped": L.FBSDE_GROUP_GROUPED}[mode])

    def train_step(self, thetas, ms, vs, step_dev, lr: float = 1e-3):
        L.fbsde_group_train_step(self.handle, self._ptrs(thetas), self._ptrs(ms), self._ptrs(vs),
                                 step_dev.data_ptr(), lr, self.loss.data_ptr(), self.y0.data_ptr())
        return self.loss, self.y0

    def capture(self, thetas, ms, vs, step_dev, lr: float = 1e-3, steps: int = 1):
        g = L.fbsde_group_capture(self.handle, self._ptrs(thetas), self._ptrs(ms), self._ptrs(vs),
                                  step_dev.data_ptr(), lr, self.loss.data_ptr(), self.y0.data_ptr(), steps)
        return _GraphHandle(g, (thetas, ms, vs, step_dev))

    def shapes_key(self) -> str:
        import json
        return json.dumps([[s.problem.kind, s.problem.D, s.problem_N, s.problem.M, s.arch.kind, s.arch.width,
                            s.arch.depth, s.arch.act, s.arch.prec] for s in self.solvers])

    def autotune(self, thetas, lr: float = 1e-3, trial_steps: int = 2, cache_path: Optional[str] = None):
        """Per-instance caps on the fused kernels' CTAs; read from / written
        to cache_path keyed by the instances' shapes."""
        import json, os
        key = self.shapes_key()
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        if key in cache:
            caps = cache[key]["caps"]
            for s, c in zip(self.solvers, caps):
                L.fbsde_set_grid_cap(s.ctx, int(c))
            return caps, cache[key].get("ms_per_step"), True
        caps, ms = L.fbsde_group_autotune(self.handle, self._ptrs(thetas), lr, trial_steps)
        if cache_path:
            cache[key] = {"caps": caps, "ms_per_step": ms}
            with open(cache_path, "w") as f:
                json.dump(cache, f)
        return caps, ms, False

    def close(self):
        if self.handle:
            L.fbsde_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _GraphHandle:
    def __init__(self, handle, keep):
        self.handle, self._keep = handle, keep

    def launch(self):
        L.fbsde_graph_launch(self.handle)

    def close(self):
        if self.handle:
            L.fbsde_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox4x32_10(ctr: torch.Tensor, key0: int, key1: int) -> torch.Tensor:
    """Raw Philox4x32-10 blocks on the GPU: ctr int32 [n, 4] (bit patterns) -> [n, 4]."""
    assert ctr.is_cuda and ctr.dtype == torch.int32 and ctr.is_contiguous() and ctr.shape[-1] == 4
    out = torch.empty_like(ctr)
    L.fbsde_philox4x32_10(ctr.data_ptr(), key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF, ctr.shape[0],
                          out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return out


class RolloutLoss(torch.autograd.Function):
    """loss(Theta) of Eq. (loss) as an autograd node: forward runs the rollout
    and the hand-written adjoint in one library call; backward scales the
    stored gradient by the incoming scalar."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, solver: Solver, iteration: int):
        loss, y0, grad = solver.rollout_grad(theta.detach().contiguous(), iteration)
        ctx.save_for_backward(grad)
        ctx.mark_non_differentiable(y0)
        return loss[0], y0[0]

    @staticmethod
    def backward(ctx, gloss, gy0):
        grad, = ctx.saved_tensors
        return gloss * grad, None, None
