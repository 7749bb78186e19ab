"""FP64 CPU oracle of the deep FBSDE solver's training step (test infrastructure).

This is the reference the CUDA path is checked against: plain NumPy in FP64,
one statement per step of the method, no blocking or fusion.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it;
the library (``paper_1910_11623_gb300``) never does, and this package imports
nothing from the library.

Method (Guler, Laignelet, Parpas, "Towards Robust and Stable Deep Learning
Algorithms for FBSDEs", arXiv 1910.11623):

* Section 2.1, Eq. "coupled": dX = mu dt + sigma dW, dY = phi dt + Z^T sigma dW,
  Y_T = g(X_T); Y_t = u(t, X_t), Z_t = grad u(t, X_t).
* Section 2.2, Eq. "disc equations": Euler--Maruyama for X and Y with
  Delta W_n ~ N(0, Delta t_n).
* Section 2.2: one network u(t, x; Theta) shared by all t_n, Z by automatic
  differentiation (here: the reverse pass written out by hand).
* Section 2.2, Eq. "loss": sum over paths m and steps n of the squared
  Y-residual plus the squared terminal mismatch; the optional term
  sum_m |Z_N - grad g(X_N)|^2 mentioned right after it.
* Section 3.1: ResNet x(k+1) = x(k) + f(x(k), theta(k)) (forward Euler, h = 1)
  and NAIS-Net x(k+1) = x(k) + h sigma(A x(k) + B u + C), A = -R^T R - eps I,
  eps = 0.01, with a projection on ||R^T R||_F.
* Section 4: Black--Scholes--Barenblatt (BSB) and HJB benchmark problems;
  Section 4.1: Adam with learning rate 1e-3.

Readings where the paper is silent or garbled (each is stated where it is used):
HJB PDE uses ||Du||^2 (printed ||D^2u||^2) and W_{T-t} (printed W_{t-t});
loss is a plain sum; input lift h0 = act(W_in (t,x) + b_in) before the blocks;
ResNet f = act(W x + b); NAIS step h and projection bound delta are parameters
(default h = 1, delta = 0.99 (2/h - eps)); Adam beta1 = 0.9, beta2 = 0.999,
eps = 1e-8 with bias correction; uniform Delta t = T/N.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

from . import philox

# ---------------------------------------------------------------------------
# Specifications
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Problem:
    """A decoupled FBSDE (mu = 0, sigma = sigma(x)) from Section 4.

    kind 'bsb': sigma(x) = sigma diag(x), phi = r (y - z^T x), g = ||x||^2.
    kind 'hjb': sigma(x) = sqrt(2) I,    phi = ||z||^2,       g = ln(0.5 (1 + ||x||^2)).
    """
    kind: str
    D: int
    N: int
    M: int
    x0: np.ndarray
    T: float = 1.0
    r: float = 0.05
    sigma: float = 0.4
    terminal_grad_term: bool = False

    @property
    def dt(self) -> float:
        return self.T / self.N


@dataclass(frozen=True)
class Arch:
    """Network u(t, x; Theta): lift, `depth` hidden layers/blocks, linear output.

    kind 'fc'    : h_l = act(W_l h_{l-1} + b_l)                 (Section 4.1)
    kind 'resnet': h_l = h_{l-1} + act(W_l h_{l-1} + b_l)       (Section 3.1, h = 1)
    kind 'nais'  : h_l = h_{l-1} + h act(A_l h_{l-1} + B_l u + C_l),
                   A_l = -R_l^T R_l - eps I                      (Section 3.1)
    The lift is h_0 = act(W_in u + b_in) with u = (t, x); y = w_o^T h_L + b_o.
    """
    kind: str
    width: int
    depth: int
    act: str
    h: float = 1.0
    eps: float = 0.01
    proj_delta: Optional[float] = None

    @property
    def delta(self) -> float:
        """Projection bound on ||R^T R||_F (paper: unspecified; reading: keep
        the explicit Euler step I + h act' A contractive for act' <= 1, i.e.
        ||R^T R|| < 2/h - eps, with a 1% margin)."""
        if self.proj_delta is not None:
            return float(self.proj_delta)
        return 0.99 * (2.0 / self.h - self.eps)


def param_layout(problem: Problem, arch: Arch):
    """Flat parameter order: list of (name, shape, fan_in, fan_out, is_weight).

    W_in [w, D+1], b_in [w]; per layer l = 1..L: FC/ResNet W_l [w, w], b_l [w];
    NAIS R_l [w, w], C_l [w], B_l [w, D+1]; then w_o [w], b_o [1].
    """
    w, Din = arch.width, problem.D + 1
    out = [("W_in", (w, Din), Din, w, True), ("b_in", (w,), Din, w, False)]
    for l in range(1, arch.depth + 1):
        if arch.kind == "nais":
            out += [(f"R_{l}", (w, w), w, w, True), (f"C_{l}", (w,), w, w, False),
                    (f"B_{l}", (w, Din), Din, w, True)]
        else:
            out += [(f"W_{l}", (w, w), w, w, True), (f"b_{l}", (w,), w, w, False)]
    out += [("w_o", (w,), w, 1, True), ("b_o", (1,), w, 1, False)]
    return out


def num_params(problem: Problem, arch: Arch) -> int:
    return int(sum(np.prod(s) for _, s, _, _, _ in param_layout(problem, arch)))


def unpack(theta: np.ndarray, problem: Problem, arch: Arch) -> dict:
    """Views of the flat parameter vector, keyed by name."""
    out, off = {}, 0
    for name, shape, _, _, _ in param_layout(problem, arch):
        n = int(np.prod(shape))
        out[name] = theta[off:off + n].reshape(shape)
        off += n
    assert off == theta.size
    return out


# ---------------------------------------------------------------------------
# Initialisation and NAIS constraint
# ---------------------------------------------------------------------------


def init_params(problem: Problem, arch: Arch, seed: int) -> np.ndarray:
    """Xavier-normal weights N(0, 2/(fan_in + fan_out)), zero biases.

    The normals come from Philox under the init key (see philox.init_normals),
    indexed by the flat parameter index.  NAIS R blocks are projected onto the
    feasible set right away (Section 3.1: the projection keeps the weights
    feasible)."""
    P = num_params(problem, arch)
    z = philox.init_normals(seed, P)
    theta = np.zeros(P)
    off = 0
    for _, shape, fi, fo, is_w in param_layout(problem, arch):
        n = int(np.prod(shape))
        if is_w:
            theta[off:off + n] = z[off:off + n] * np.sqrt(2.0 / (fi + fo))
        off += n
    if arch.kind == "nais":
        theta = nais_project(theta, problem, arch)
    return theta


def nais_A(R: np.ndarray, eps: float) -> np.ndarray:
    """A = -R^T R - eps I (Section 3.1)."""
    return -R.T @ R - eps * np.eye(R.shape[0])


def nais_project(theta: np.ndarray, problem: Problem, arch: Arch) -> np.ndarray:
    """Projection on ||R^T R||_F <= delta (Section 3.1).  Reading: if the norm
    exceeds delta, scale R by sqrt(delta / ||R^T R||_F), which maps R^T R onto
    the sphere of radius delta along its own ray."""
    theta = theta.copy()
    p = unpack(theta, problem, arch)
    for l in range(1, arch.depth + 1):
        R = p[f"R_{l}"]
        nrm = np.linalg.norm(R.T @ R, "fro")
        if nrm > arch.delta:
            R *= np.sqrt(arch.delta / nrm)
    return theta


# ---------------------------------------------------------------------------
# Problem data (Section 4) and the forward SDE (Eq. disc equations)
# ---------------------------------------------------------------------------


def sigma_dW(problem: Problem, X: np.ndarray, dW: np.ndarray) -> np.ndarray:
    """sigma(t_n, X_n) Delta W_n.  BSB: sigma diag(X) dW; HJB: sqrt(2) dW."""
    if problem.kind == "bsb":
        return problem.sigma * X * dW
    return np.sqrt(2.0) * dW


def driver(problem: Problem, X, Y, Z):
    """phi(t, x, y, z) and its partials (d phi/dy scalar, d phi/dz vector).

    BSB (Section 4, Black--Scholes): u_t = -1/2 Tr[sigma^2 diag(x^2) D^2u]
    + r (u - Du^T x) with f = phi - mu^T z - 1/2 Tr[sigma sigma^T gamma]
    (Section 2.1) gives phi = r (y - z^T x).
    HJB (Section 4): u_t = -Tr[D^2u] + ||Du||^2 with sigma = sqrt(2) I gives
    phi = ||z||^2 (reading: the printed ||D^2u||^2 is taken as ||Du||^2, the
    only form the printed closed-form solution satisfies)."""
    if problem.kind == "bsb":
        zx = np.sum(Z * X, axis=-1)
        phi = problem.r * (Y - zx)
        phi_y = np.full_like(Y, problem.r)
        phi_z = -problem.r * X
    else:
        phi = np.sum(Z * Z, axis=-1)
        phi_y = np.zeros_like(Y)
        phi_z = 2.0 * Z
    return phi, phi_y, phi_z


def terminal(problem: Problem, X):
    """g(x) and grad g(x).  BSB: ||x||^2; HJB: ln(0.5 (1 + ||x||^2))."""
    s = np.sum(X * X, axis=-1)
    if problem.kind == "bsb":
        return s, 2.0 * X
    return np.log(0.5 * (1.0 + s)), 2.0 * X / (1.0 + s)[..., None]


def forward_sde(problem: Problem, dW: np.ndarray) -> np.ndarray:
    """X_{n+1} = X_n + mu Delta t + sigma(X_n) Delta W_n with mu = 0 and
    X_0 = x0 for every path (Eq. disc equations, second line).
    dW: [N, M, D]  ->  X: [N+1, M, D]."""
    N, M, D = dW.shape
    X = np.empty((N + 1, M, D))
    X[0] = problem.x0[None, :]
    for n in range(N):
        X[n + 1] = X[n] + sigma_dW(problem, X[n], dW[n])
    return X


def sample_paths(problem: Problem, seed: int, iteration: int, paths=None):
    """Brownian increments and forward paths of one iteration.

    paths: optional array of path indices (a subset of 0..M-1); the noise of a
    path depends only on (seed, iteration, path, step, dimension)."""
    dW = philox.brownian_increments(seed, iteration, problem.M, problem.N,
                                    problem.D, problem.T, paths)
    return dW, forward_sde(problem, dW)


def network_inputs(problem: Problem, X: np.ndarray) -> np.ndarray:
    """u = (t_n, X_n) for every point, t first: [N+1, M, D+1] (Fig. "neural":
    the network at time t_n receives (t_n, X_n))."""
    Np1, M, D = X.shape
    t = (np.arange(Np1) * problem.dt)[:, None, None] * np.ones((1, M, 1))
    return np.concatenate([t, X], axis=-1)


# ---------------------------------------------------------------------------
# Network, its input gradient Z, and the adjoint of the loss
# ---------------------------------------------------------------------------


def act(kind, a):
    return np.sin(a) if kind == "sin" else np.tanh(a)


def act_d1(kind, a):
    if kind == "sin":
        return np.cos(a)
    t = np.tanh(a)
    return 1.0 - t * t


def act_d2(kind, a):
    if kind == "sin":
        return -np.sin(a)
    t = np.tanh(a)
    return -2.0 * t * (1.0 - t * t)


def _layers(problem: Problem, arch: Arch, p: dict):
    """Per hidden layer l = 1..L: (matrix acting on h, bias, input-injection
    matrix or None, skip s, scale c) with h_l = s h_{l-1} + c act(a_l)."""
    out = []
    for l in range(1, arch.depth + 1):
        if arch.kind == "nais":
            out.append((nais_A(p[f"R_{l}"], arch.eps), p[f"C_{l}"], p[f"B_{l}"], 1.0, arch.h))
        elif arch.kind == "resnet":
            out.append((p[f"W_{l}"], p[f"b_{l}"], None, 1.0, 1.0))
        else:
            out.append((p[f"W_{l}"], p[f"b_{l}"], None, 0.0, 1.0))
    return out


def net_forward(problem: Problem, arch: Arch, theta: np.ndarray, U: np.ndarray):
    """y = u(t, x; Theta) for points U [P, D+1].  Returns y [P] and the cache
    (pre-activations a_l and outputs h_l, l = 0..L)."""
    p = unpack(theta, problem, arch)
    a = [U @ p["W_in"].T + p["b_in"]]
    h = [act(arch.act, a[0])]
    for (W, b, B, s, c) in _layers(problem, arch, p):
        al = h[-1] @ W.T + b
        if B is not None:
            al = al + U @ B.T
        a.append(al)
        h.append(s * h[-1] + c * act(arch.act, al))
    y = h[-1] @ p["w_o"] + p["b_o"][0]
    return y, {"a": a, "h": h}


def net_input_grad(problem: Problem, arch: Arch, theta: np.ndarray, U: np.ndarray, cache):
    """Z = grad_x u(t, x; Theta) by reverse-mode differentiation of net_forward
    (Section 2.2: Z from automatic differentiation).

    g_L = w_o; e_l = c act'(a_l) g_l; g_{l-1} = s g_l + W_l^T e_l; the
    input receives W_in^T e_0 plus (NAIS) B_l^T e_l from every block.
    Returns Z [P, D] and the per-layer (g_l, e_l), l = 0..L."""
    p = unpack(theta, problem, arch)
    layers = _layers(problem, arch, p)
    L = arch.depth
    g = [None] * (L + 1)
    e = [None] * (L + 1)
    g[L] = np.broadcast_to(p["w_o"], cache["h"][L].shape).copy()
    gu = np.zeros_like(U)
    for l in range(L, 0, -1):
        W, _, B, s, c = layers[l - 1]
        e[l] = c * act_d1(arch.act, cache["a"][l]) * g[l]
        g[l - 1] = s * g[l] + e[l] @ W
        if B is not None:
            gu += e[l] @ B
    e[0] = act_d1(arch.act, cache["a"][0]) * g[0]
    gu += e[0] @ p["W_in"]
    return gu[:, 1:], {"g": g, "e": e}


def net_param_grad(problem: Problem, arch: Arch, theta: np.ndarray, U: np.ndarray,
                   cache, zcache, alpha: np.ndarray, v: np.ndarray) -> np.ndarray:
    """d/dTheta of sum_points [alpha * y + v^T Z] (the chain rule of the loss
    through Y_n = u(t_n, X_n; Theta) and Z_n = grad u(t_n, X_n; Theta)).

    v^T Z is the derivative of y along the input direction u' = (0, v), so the
    sum is differentiated as a forward tangent pass followed by a reverse pass
    over both the primal and the tangent:
      tangent: a'_0 = W_in u', h'_0 = act'(a_0) a'_0,
               a'_l = W_l h'_{l-1} (+ B_l u'), h'_l = s h'_{l-1} + c act'(a_l) a'_l;
      adjoint of the tangent is (g_l, e_l) of net_input_grad;
      adjoint: hbar_L = alpha w_o,
               abar_l = c (act'(a_l) hbar_l + act''(a_l) a'_l g_l),
               hbar_{l-1} = s hbar_l + W_l^T abar_l;
      grads:   dW_l = abar_l h_{l-1}^T + e_l h'_{l-1}^T, db_l = abar_l,
               (NAIS) dB_l = abar_l u^T + e_l u'^T, dW_in = abar_0 u^T + e_0 u'^T,
               dw_o = alpha h_L + h'_L, db_o = alpha; all summed over points.
    NAIS: the gradient with respect to A_l is chained to R_l through
    A = -R^T R - eps I, i.e. dR = -R (dA + dA^T)."""
    p = unpack(theta, problem, arch)
    layers = _layers(problem, arch, p)
    L = arch.depth
    a, h = cache["a"], cache["h"]
    g, e = zcache["g"], zcache["e"]
    Ud = np.concatenate([np.zeros((U.shape[0], 1)), v], axis=1)  # u' = (0, v)

    # tangent sweep (upward)
    ad = [Ud @ p["W_in"].T]
    hd = [act_d1(arch.act, a[0]) * ad[0]]
    for l in range(1, L + 1):
        W, _, B, s, c = layers[l - 1]
        adl = hd[-1] @ W.T
        if B is not None:
            adl = adl + Ud @ B.T
        ad.append(adl)
        hd.append(s * hd[-1] + c * act_d1(arch.act, a[l]) * adl)

    grad = {name: np.zeros(shape) for name, shape, _, _, _ in param_layout(problem, arch)}
    grad["w_o"] = alpha @ h[L] + hd[L].sum(axis=0)
    grad["b_o"] = np.array([alpha.sum()])

    # adjoint sweep (downward)
    hbar = alpha[:, None] * p["w_o"][None, :]
    for l in range(L, 0, -1):
        W, _, B, s, c = layers[l - 1]
        abar = c * (act_d1(arch.act, a[l]) * hbar + act_d2(arch.act, a[l]) * ad[l] * g[l])
        gW = abar.T @ h[l - 1] + e[l].T @ hd[l - 1]
        if arch.kind == "nais":
            R = p[f"R_{l}"]
            grad[f"R_{l}"] = -R @ (gW + gW.T)
            grad[f"C_{l}"] = abar.sum(axis=0)
            grad[f"B_{l}"] = abar.T @ U + e[l].T @ Ud
        else:
            grad[f"W_{l}"] = gW
            grad[f"b_{l}"] = abar.sum(axis=0)
        hbar = s * hbar + abar @ W
    abar0 = act_d1(arch.act, a[0]) * hbar + act_d2(arch.act, a[0]) * ad[0] * g[0]
    grad["W_in"] = abar0.T @ U + e[0].T @ Ud
    grad["b_in"] = abar0.sum(axis=0)
    return np.concatenate([grad[name].reshape(-1) for name, *_ in param_layout(problem, arch)])


# ---------------------------------------------------------------------------
# Loss (Eq. loss) and its seeds
# ---------------------------------------------------------------------------


@dataclass
class Rollout:
    """Everything one loss evaluation produces (arrays over steps and paths)."""
    loss: float
    y0: float
    X: np.ndarray        # [N+1, M, D]
    dW: np.ndarray       # [N, M, D]
    Y: np.ndarray        # [N+1, M]
    Z: np.ndarray        # [N+1, M, D]
    r: np.ndarray        # [N, M]    Y-residuals
    rT: np.ndarray       # [M]       Y_N - g(X_N)
    path_loss: np.ndarray  # [M]     per-path contribution to the loss
    extras: dict = field(default_factory=dict)


def evaluate_network(problem: Problem, arch: Arch, theta: np.ndarray, X: np.ndarray):
    """Y_n = u(t_n, X_n; Theta), Z_n = grad u(t_n, X_n; Theta) at every point
    (Section 2.2, the same parameters for all time points)."""
    Np1, M, D = X.shape
    U = network_inputs(problem, X).reshape(-1, D + 1)
    y, cache = net_forward(problem, arch, theta, U)
    Z, zcache = net_input_grad(problem, arch, theta, U, cache)
    return y.reshape(Np1, M), Z.reshape(Np1, M, D), U, cache, zcache


def residuals(problem: Problem, X, dW, Y, Z):
    """r_n = Y_{n+1} - Y_n - phi(t_n, X_n, Y_n, Z_n) Dt - Z_n^T sigma(X_n) DW_n
    for n < N, and r_T = Y_N - g(X_N) (Eq. loss)."""
    N = problem.N
    phi, _, _ = driver(problem, X[:N], Y[:N], Z[:N])
    zsdw = np.sum(Z[:N] * sigma_dW(problem, X[:N], dW), axis=-1)
    r = Y[1:] - Y[:N] - phi * problem.dt - zsdw
    gT, gradT = terminal(problem, X[N])
    rT = Y[N] - gT
    return r, rT, gradT


def rollout_loss(problem: Problem, arch: Arch, theta: np.ndarray, seed: int,
                 iteration: int, paths=None) -> Rollout:
    """Loss of Eq. (loss) for one iteration's Brownian paths.

    loss = sum_m sum_{n<N} r_n^2 + sum_m r_T^2 [+ sum_m ||Z_N - grad g(X_N)||^2
    when problem.terminal_grad_term].  y0 = u(0, x0; Theta).
    With `paths`, only those paths are simulated and summed."""
    dW, X = sample_paths(problem, seed, iteration, paths)
    Y, Z, U, cache, zcache = evaluate_network(problem, arch, theta, X)
    r, rT, gradT = residuals(problem, X, dW, Y, Z)
    path_loss = np.sum(r * r, axis=0) + rT * rT
    if problem.terminal_grad_term:
        path_loss = path_loss + np.sum((Z[-1] - gradT) ** 2, axis=-1)
    u0 = np.concatenate([[0.0], problem.x0])[None, :]
    y0, _ = net_forward(problem, arch, theta, u0)
    ro = Rollout(loss=float(path_loss.sum()), y0=float(y0[0]), X=X, dW=dW, Y=Y, Z=Z,
                 r=r, rT=rT, path_loss=path_loss)
    ro.extras = {"U": U, "cache": cache, "zcache": zcache, "gradT": gradT}
    return ro


def loss_seeds(problem: Problem, ro: Rollout):
    """alpha_n = dLoss/dY_n and v_n = dLoss/dZ_n from Eq. (loss):
      alpha_n = 2 r_{n-1} [n>=1] - 2 r_n (1 + phi_y Dt) [n<N] + 2 r_T [n=N]
      v_n     = -2 r_n (phi_z Dt + sigma(X_n) DW_n) [n<N]
                + 2 (Z_N - grad g(X_N)) [n=N, optional term].
    X does not depend on Theta (mu = 0, sigma = sigma(x)), so no other path
    carries a derivative."""
    N = problem.N
    X, dW, Y, Z, r, rT = ro.X, ro.dW, ro.Y, ro.Z, ro.r, ro.rT
    _, phi_y, phi_z = driver(problem, X[:N], Y[:N], Z[:N])
    alpha = np.zeros_like(Y)
    v = np.zeros_like(Z)
    alpha[1:] += 2.0 * r
    alpha[:N] += -2.0 * r * (1.0 + phi_y * problem.dt)
    alpha[N] += 2.0 * rT
    v[:N] = -2.0 * r[..., None] * (phi_z * problem.dt + sigma_dW(problem, X[:N], dW))
    if problem.terminal_grad_term:
        v[N] += 2.0 * (Z[N] - ro.extras["gradT"])
    return alpha, v


def rollout_grad(problem: Problem, arch: Arch, theta: np.ndarray, seed: int,
                 iteration: int, paths=None):
    """(Rollout, dLoss/dTheta) for one iteration."""
    ro = rollout_loss(problem, arch, theta, seed, iteration, paths)
    alpha, v = loss_seeds(problem, ro)
    grad = net_param_grad(problem, arch, theta, ro.extras["U"], ro.extras["cache"],
                          ro.extras["zcache"], alpha.reshape(-1),
                          v.reshape(-1, problem.D))
    ro.extras["alpha"], ro.extras["v"] = alpha, v
    return ro, grad


# ---------------------------------------------------------------------------
# Optimiser (Section 4.1: Adam, learning rate 1e-3)
# ---------------------------------------------------------------------------

ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_update(theta, grad, m, v, step: int, lr: float):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) with bias correction;
    `step` counts from 1.  Returns new (theta, m, v)."""
    m = ADAM_BETA1 * m + (1.0 - ADAM_BETA1) * grad
    v = ADAM_BETA2 * v + (1.0 - ADAM_BETA2) * grad * grad
    mhat = m / (1.0 - ADAM_BETA1 ** step)
    vhat = v / (1.0 - ADAM_BETA2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v


def train_step(problem: Problem, arch: Arch, theta, m, v, seed: int, step: int, lr: float):
    """One training iteration: paths of iteration `step`, loss and gradient at
    the current Theta, Adam update, then (NAIS) the projection.
    Returns (loss, y0, theta, m, v)."""
    ro, grad = rollout_grad(problem, arch, theta, seed, step)
    theta, m, v = adam_update(theta, grad, m, v, step, lr)
    if arch.kind == "nais":
        theta = nais_project(theta, problem, arch)
    return ro.loss, ro.y0, theta, m, v


def train_schedule(problem: Problem, arch: Arch, theta, m, v, seed: int, levels, steps,
                   first_step: int, lr: float):
    """Multilevel training (Section 3.2): the discretisation starts coarse and
    is refined geometrically (Section 4.3 uses 2, 4, 8, 16 and 32 steps); at
    level i the problem is solved on N = levels[i] Euler steps of
    Delta t = T / N for steps[i] Adam iterations, and Theta and the Adam
    moments carry over to the next level.  Step numbers continue across
    levels (each iteration draws its own increments).  Returns
    (losses, y0s, theta, m, v) with one loss and Y_0 per iteration."""
    losses, y0s = [], []
    step = first_step
    for N, count in zip(levels, steps):
        level = replace(problem, N=int(N))
        for _ in range(int(count)):
            loss, y0, theta, m, v = train_step(level, arch, theta, m, v, seed, step, lr)
            losses.append(loss)
            y0s.append(y0)
            step += 1
    return np.array(losses), np.array(y0s), theta, m, v

