"""Pins of the oracle's forward SDE, network, input gradient Z, loss, seeds,
parameter gradient, Adam and NAIS constraint -- each against something other
than the oracle itself (statistics of the exact SDE law, closed-form PDE
solutions, finite differences, torch autograd in FP64, torch.optim.Adam)."""
import numpy as np
import pytest
import torch

from oracle import fbsde as F
from oracle import philox


def bsb(D=3, N=4, M=5, **kw):
    x0 = np.array([1.0 if i % 2 == 0 else 0.5 for i in range(D)])
    return F.Problem(kind="bsb", D=D, N=N, M=M, x0=x0, **kw)


def hjb(D=3, N=4, M=5, **kw):
    return F.Problem(kind="hjb", D=D, N=N, M=M, x0=np.zeros(D), **kw)


def perturbed_theta(problem, arch, seed=7, scale=0.3):
    th = F.init_params(problem, arch, seed)
    return th + scale * np.random.default_rng(seed).standard_normal(th.size)


# ---------------------------------------------------------------- forward SDE

def test_bsb_sde_moments():
    # mu = 0: E[X_N] = x0; E[X_N^2] = x0^2 (1 + sigma^2 dt)^N exactly for the
    # Euler product X_N = x0 prod(1 + sigma dW_n).
    p = bsb(D=4, N=8, M=40000)
    _, X = F.sample_paths(p, seed=1, iteration=0)
    XN = X[-1]
    m1 = XN.mean(axis=0)
    se1 = XN.std(axis=0) / np.sqrt(p.M)
    assert np.all(np.abs(m1 - p.x0) < 5 * se1)
    m2 = (XN ** 2).mean(axis=0)
    se2 = (XN ** 2).std(axis=0) / np.sqrt(p.M)
    want = p.x0 ** 2 * (1 + p.sigma ** 2 * p.dt) ** p.N
    assert np.all(np.abs(m2 - want) < 5 * se2)


def test_hjb_sde_law():
    # X_N = x0 + sqrt(2) W_T ~ N(x0, 2T I).
    p = hjb(D=5, N=6, M=30000, T=1.5)
    _, X = F.sample_paths(p, seed=2, iteration=3)
    XN = X[-1].reshape(-1)
    assert abs(XN.mean()) < 5 * np.sqrt(2 * p.T / XN.size)
    assert abs(XN.var() / (2 * p.T) - 1.0) < 5 * np.sqrt(2.0 / XN.size)


def test_path_subset_matches_full():
    p = bsb(D=3, N=4, M=9)
    dW, X = F.sample_paths(p, 5, 2)
    dWs, Xs = F.sample_paths(p, 5, 2, paths=[2, 7])
    assert np.array_equal(dWs, dW[:, [2, 7]]) and np.array_equal(Xs, X[:, [2, 7]])


# ---------------------------------------------------------------- network

def _torch_fc(problem, arch, theta):
    """The FC network as a torch.nn.Sequential of Linear layers."""
    p = F.unpack(theta, problem, arch)
    actm = {"sin": None, "tanh": torch.nn.Tanh()}[arch.act]
    layers = []
    lin = torch.nn.Linear(problem.D + 1, arch.width).double()
    lin.weight.data = torch.tensor(p["W_in"]); lin.bias.data = torch.tensor(p["b_in"])
    layers.append(lin)
    for l in range(1, arch.depth + 1):
        layers.append(actm)
        lin = torch.nn.Linear(arch.width, arch.width).double()
        lin.weight.data = torch.tensor(p[f"W_{l}"]); lin.bias.data = torch.tensor(p[f"b_{l}"])
        layers.append(lin)
    layers.append(actm)
    lin = torch.nn.Linear(arch.width, 1).double()
    lin.weight.data = torch.tensor(p["w_o"][None, :]); lin.bias.data = torch.tensor(p["b_o"])
    layers.append(lin)
    return torch.nn.Sequential(*layers)


def test_fc_forward_matches_torch_nn():
    p = bsb(D=6)
    arch = F.Arch(kind="fc", width=16, depth=3, act="tanh")
    th = perturbed_theta(p, arch)
    U = np.random.default_rng(0).standard_normal((11, p.D + 1))
    y, _ = F.net_forward(p, arch, th, U)
    yt = _torch_fc(p, arch, th)(torch.tensor(U)).detach().numpy()[:, 0]
    np.testing.assert_allclose(y, yt, rtol=1e-12, atol=1e-12)


def test_resnet_with_zero_blocks_is_the_lift():
    # act(0) = 0 for sin and tanh, so zero blocks leave h_0 unchanged.
    for a in ["sin", "tanh"]:
        p = bsb(D=4)
        res = F.Arch(kind="resnet", width=8, depth=3, act=a)
        fc0 = F.Arch(kind="fc", width=8, depth=0, act=a)
        th = perturbed_theta(p, res)
        pr = F.unpack(th, p, res)
        for l in range(1, 4):
            pr[f"W_{l}"][:] = 0.0
            pr[f"b_{l}"][:] = 0.0
        th0 = np.concatenate([pr["W_in"].ravel(), pr["b_in"], pr["w_o"], pr["b_o"]])
        U = np.random.default_rng(1).standard_normal((7, p.D + 1))
        np.testing.assert_allclose(F.net_forward(p, res, th, U)[0],
                                   F.net_forward(p, fc0, th0, U)[0], rtol=1e-14)


def test_nais_with_zero_R_is_a_scalar_recursion():
    # R = 0, B = 0, C = 0 -> A = -eps I, so each unit follows
    # x <- x + h act(-eps x) independently.
    p = bsb(D=3)
    arch = F.Arch(kind="nais", width=5, depth=4, act="tanh", h=0.7, eps=0.3)
    th = perturbed_theta(p, arch)
    pr = F.unpack(th, p, arch)
    for l in range(1, 5):
        pr[f"R_{l}"][:] = 0.0; pr[f"B_{l}"][:] = 0.0; pr[f"C_{l}"][:] = 0.0
    U = np.random.default_rng(2).standard_normal((4, p.D + 1))
    y, cache = F.net_forward(p, arch, th, U)
    x = np.tanh(U @ pr["W_in"].T + pr["b_in"])
    for _ in range(4):
        x = x + 0.7 * np.tanh(-0.3 * x)
    np.testing.assert_allclose(y, x @ pr["w_o"] + pr["b_o"][0], rtol=1e-13)


@pytest.mark.parametrize("kind", ["fc", "resnet", "nais"])
@pytest.mark.parametrize("act", ["sin", "tanh"])
def test_Z_matches_finite_differences_in_x(kind, act):
    p = bsb(D=5)
    arch = F.Arch(kind=kind, width=12, depth=3, act=act)
    th = perturbed_theta(p, arch)
    U = np.random.default_rng(3).standard_normal((6, p.D + 1))
    y, cache = F.net_forward(p, arch, th, U)
    Z, _ = F.net_input_grad(p, arch, th, U, cache)
    h = 1e-5
    for i in range(p.D):
        Up, Um = U.copy(), U.copy()
        Up[:, 1 + i] += h; Um[:, 1 + i] -= h
        fd = (F.net_forward(p, arch, th, Up)[0] - F.net_forward(p, arch, th, Um)[0]) / (2 * h)
        np.testing.assert_allclose(Z[:, i], fd, rtol=1e-7, atol=1e-8)


# ---------------------------------------------------------------- loss

def _exact_bsb(p, t, X):
    s = np.exp((p.r + p.sigma ** 2) * (p.T - t))
    return s * np.sum(X * X, axis=-1), 2.0 * s[..., None] * X


def _exact_loss_per_path(p, seed, u_exact):
    dW, X = F.sample_paths(p, seed, 0)
    t = (np.arange(p.N + 1) * p.dt)[:, None] * np.ones((1, p.M))
    Y, Z = u_exact(p, t, X)
    r, rT, _ = F.residuals(p, X, dW, Y, Z)
    return np.mean(np.sum(r * r, axis=0)), np.max(np.abs(rT))


def test_bsb_exact_solution_makes_the_residuals_vanish_with_dt():
    # With the closed form u of Section 4 in place of the network, the terminal
    # mismatch is exactly zero and the summed squared Y-residual is a pure
    # Euler-Maruyama discretisation error: O(dt), so it halves as N doubles.
    # A wrong sign in phi or a missing Z^T sigma dW term makes it O(1).
    vals = []
    for N in [16, 32, 64]:
        p = bsb(D=4, N=N, M=4000)
        mean_r2, maxrT = _exact_loss_per_path(p, 11, _exact_bsb)
        assert maxrT < 1e-12
        vals.append(mean_r2)
    assert 1.6 < vals[0] / vals[1] < 2.5 and 1.6 < vals[1] / vals[2] < 2.5


def _exact_hjb_1d(p, t, X):
    # D = 1: u(t,x) = -ln E[2 / (1 + (x + sqrt(2) W_{T-t})^2)] by Gauss-Hermite
    # quadrature; Z = d u / d x.
    z, wq = np.polynomial.hermite_e.hermegauss(200)
    wq = wq / wq.sum()
    tau = (p.T - t)[..., None]
    x = X[..., 0][..., None]
    yv = x + np.sqrt(2 * tau) * z
    v = np.sum(wq * 2.0 / (1.0 + yv ** 2), axis=-1)
    dv = np.sum(wq * (-4.0 * yv) / (1.0 + yv ** 2) ** 2, axis=-1)
    return -np.log(v), (-dv / v)[..., None]


def test_hjb_exact_solution_makes_the_residuals_vanish_with_dt():
    # Cole-Hopf: u = -ln E[exp(-g(x + sqrt(2) W_{T-t}))] solves
    # u_t = -Tr D^2u + ||Du||^2, whose driver is phi = ||z||^2.
    vals = []
    for N in [16, 32, 64]:
        p = F.Problem(kind="hjb", D=1, N=N, M=4000, x0=np.array([0.3]))
        mean_r2, maxrT = _exact_loss_per_path(p, 12, _exact_hjb_1d)
        assert maxrT < 1e-10
        vals.append(mean_r2)
    assert 1.6 < vals[0] / vals[1] < 2.5 and 1.6 < vals[1] / vals[2] < 2.5


@pytest.mark.parametrize("pk", ["bsb", "hjb"])
@pytest.mark.parametrize("tgt", [False, True])
def test_loss_seeds_match_finite_differences(pk, tgt):
    # alpha = dLoss/dY_n and v = dLoss/dZ_n, checked by perturbing Y and Z.
    p = (bsb if pk == "bsb" else hjb)(D=3, N=4, M=3, terminal_grad_term=tgt)
    arch = F.Arch(kind="fc", width=6, depth=1, act="tanh")
    ro = F.rollout_loss(p, arch, perturbed_theta(p, arch), 2, 1)
    alpha, v = F.loss_seeds(p, ro)

    def loss_of(Y, Z):
        r, rT, gT = F.residuals(p, ro.X, ro.dW, Y, Z)
        out = np.sum(r * r) + np.sum(rT * rT)
        if tgt:
            out += np.sum((Z[-1] - gT) ** 2)
        return out

    h = 1e-6
    for (n, m) in [(0, 0), (2, 1), (p.N, 2)]:
        Yp, Ym = ro.Y.copy(), ro.Y.copy()
        Yp[n, m] += h; Ym[n, m] -= h
        assert abs((loss_of(Yp, ro.Z) - loss_of(Ym, ro.Z)) / (2 * h) - alpha[n, m]) < 1e-6 * (1 + abs(alpha[n, m]))
        for i in range(p.D):
            Zp, Zm = ro.Z.copy(), ro.Z.copy()
            Zp[n, m, i] += h; Zm[n, m, i] -= h
            fd = (loss_of(ro.Y, Zp) - loss_of(ro.Y, Zm)) / (2 * h)
            assert abs(fd - v[n, m, i]) < 1e-6 * (1 + abs(v[n, m, i]))


# ---------------------------------------------------------------- gradient

@pytest.mark.parametrize("kind", ["fc", "resnet", "nais"])
@pytest.mark.parametrize("pk", ["bsb", "hjb"])
def test_param_gradient_matches_finite_differences(kind, pk):
    p = (bsb if pk == "bsb" else hjb)(D=3, N=4, M=4, terminal_grad_term=(kind == "resnet"))
    arch = F.Arch(kind=kind, width=8, depth=2, act="sin" if kind == "fc" else "tanh")
    th = perturbed_theta(p, arch)
    _, g = F.rollout_grad(p, arch, th, 3, 11)
    h = 1e-6
    fd = np.empty_like(th)
    for i in range(th.size):
        tp, tm = th.copy(), th.copy()
        tp[i] += h; tm[i] -= h
        fd[i] = (F.rollout_loss(p, arch, tp, 3, 11).loss - F.rollout_loss(p, arch, tm, 3, 11).loss) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * np.max(np.abs(g))


def _torch_loss(p, arch, theta_t, X, dW):
    """Eq. (loss) with the network in torch ops, Z by torch.autograd.grad with
    create_graph=True: an independent route to d loss / d theta."""
    shapes = F.param_layout(p, arch)
    parts, off = {}, 0
    for name, shape, *_ in shapes:
        n = int(np.prod(shape))
        parts[name] = theta_t[off:off + n].reshape(shape)
        off += n
    act = torch.sin if arch.act == "sin" else torch.tanh
    Np1, M, D = X.shape
    t = torch.arange(Np1, dtype=torch.float64)[:, None, None].expand(Np1, M, 1) * p.dt
    x = torch.tensor(X).requires_grad_(True)
    u = torch.cat([t, x], dim=-1)
    h = act(u @ parts["W_in"].T + parts["b_in"])
    for l in range(1, arch.depth + 1):
        if arch.kind == "nais":
            R = parts[f"R_{l}"]
            A = -R.T @ R - arch.eps * torch.eye(arch.width, dtype=torch.float64)
            h = h + arch.h * act(h @ A.T + u @ parts[f"B_{l}"].T + parts[f"C_{l}"])
        elif arch.kind == "resnet":
            h = h + act(h @ parts[f"W_{l}"].T + parts[f"b_{l}"])
        else:
            h = act(h @ parts[f"W_{l}"].T + parts[f"b_{l}"])
    Y = h @ parts["w_o"] + parts["b_o"][0]
    Z, = torch.autograd.grad(Y.sum(), x, create_graph=True)
    dWt = torch.tensor(dW)
    Xn = x.detach()
    if p.kind == "bsb":
        phi = p.r * (Y[:-1] - (Z[:-1] * Xn[:-1]).sum(-1))
        zs = (Z[:-1] * p.sigma * Xn[:-1] * dWt).sum(-1)
        g = (Xn[-1] ** 2).sum(-1)
    else:
        phi = (Z[:-1] ** 2).sum(-1)
        zs = (Z[:-1] * np.sqrt(2.0) * dWt).sum(-1)
        g = torch.log(0.5 * (1 + (Xn[-1] ** 2).sum(-1)))
    r = Y[1:] - Y[:-1] - phi * p.dt - zs
    return (r ** 2).sum() + ((Y[-1] - g) ** 2).sum()


@pytest.mark.parametrize("kind", ["fc", "resnet", "nais"])
def test_param_gradient_matches_torch_double_backward(kind):
    p = bsb(D=10, N=8, M=16) if kind != "nais" else hjb(D=6, N=8, M=16)
    arch = F.Arch(kind=kind, width=32, depth=3, act="sin" if kind == "fc" else "tanh")
    th = perturbed_theta(p, arch, scale=0.1)
    ro, g = F.rollout_grad(p, arch, th, 0, 4)
    tt = torch.tensor(th, requires_grad=True)
    loss = _torch_loss(p, arch, tt, ro.X, ro.dW)
    gt, = torch.autograd.grad(loss, tt)
    assert abs(loss.item() - ro.loss) <= 1e-12 * abs(ro.loss)
    assert np.max(np.abs(gt.numpy() - g)) <= 1e-10 * np.max(np.abs(g))


# ---------------------------------------------------------------- optimiser / NAIS / init

def test_adam_matches_torch_optim_adam():
    rng = np.random.default_rng(0)
    th = rng.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    tt = torch.tensor(th.copy(), requires_grad=True)
    opt = torch.optim.Adam([tt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 8):
        g = rng.standard_normal(50) * (10.0 ** rng.integers(-3, 3))
        th, m, v = F.adam_update(th, g, m, v, step, 1e-3)
        tt.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(th, tt.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_adam_first_step_is_lr_times_sign():
    # m_hat = g, v_hat = g^2 at step 1, so the step is lr g / (|g| + eps).
    g = np.array([2.0, -3.0, 1e-3])
    th, _, _ = F.adam_update(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 1e-3)
    np.testing.assert_allclose(th, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-14)


def test_nais_projection_and_A_definiteness():
    p = hjb(D=4)
    arch = F.Arch(kind="nais", width=16, depth=2, act="tanh", h=1.0, eps=0.01)
    th = F.init_params(p, arch, 3)
    th = th + np.random.default_rng(3).standard_normal(th.size)
    thp = F.nais_project(th, p, arch)
    for l in (1, 2):
        R = F.unpack(thp, p, arch)[f"R_{l}"]
        assert abs(np.linalg.norm(R.T @ R, "fro") - arch.delta) < 1e-10
        ev = np.linalg.eigvalsh(F.nais_A(R, arch.eps))
        assert ev.max() <= -arch.eps + 1e-12          # symmetric negative definite
        assert ev.min() >= -(arch.delta + arch.eps) - 1e-9
        # explicit Euler step I + h act' A is a contraction for act' in [0, 1]
        assert np.all(np.abs(1 + arch.h * ev) < 1)
    # projecting twice changes nothing beyond rounding, and strictly inside
    # the bound the projection is the identity
    np.testing.assert_allclose(F.nais_project(thp, p, arch), thp, rtol=1e-14)
    inner = F.init_params(p, arch, 4)
    pi = F.unpack(inner, p, arch)
    for l in (1, 2):
        pi[f"R_{l}"] *= 0.5
    np.testing.assert_array_equal(F.nais_project(inner, p, arch), inner)


def test_xavier_init_statistics():
    p = bsb(D=100)
    arch = F.Arch(kind="resnet", width=256, depth=5, act="tanh")
    th = F.init_params(p, arch, 0)
    parts = F.unpack(th, p, arch)
    for name, shape, fi, fo, is_w in F.param_layout(p, arch):
        x = parts[name].ravel()
        if not is_w:
            assert np.all(x == 0)
        elif x.size > 1000:
            assert abs(x.std() / np.sqrt(2.0 / (fi + fo)) - 1) < 0.05
    assert F.num_params(p, arch) == 256 * 101 + 256 + 5 * (256 * 256 + 256) + 256 + 1
    # the same seed reproduces theta, another seed does not
    np.testing.assert_array_equal(th, F.init_params(p, arch, 0))
    assert not np.allclose(th, F.init_params(p, arch, 1))


def test_init_uses_the_init_key():
    p = bsb(D=2)
    arch = F.Arch(kind="fc", width=4, depth=1, act="sin")
    th = F.init_params(p, arch, 9)
    z = philox.init_normals(9, th.size)
    assert th[0] == z[0] * np.sqrt(2.0 / (3 + 4))


def test_train_schedule_is_levels_of_train_steps():
    # Section 3.2: a multilevel schedule is plain training on successively
    # finer grids, Theta and the Adam moments carried across; its first level
    # must agree with single-level training on that grid, and the levels must
    # really change Delta t (the losses on the coarse and the fine grid differ)
    p = F.Problem(kind="bsb", D=3, N=8, M=4, x0=np.array([1.0, 0.5, 1.0]))
    a = F.Arch(kind="fc", width=8, depth=1, act="tanh")
    th0 = F.init_params(p, a, 3)
    z = np.zeros_like(th0)
    losses, y0s, th, m, v = F.train_schedule(p, a, th0, z, z, 3, [2, 4], [2, 1], 1, 1e-3)
    assert losses.shape == (3,) and y0s.shape == (3,)
    th_r, m_r, v_r = th0, z, z
    want = []
    for N, step in [(2, 1), (2, 2), (4, 3)]:
        from dataclasses import replace
        lo, _, th_r, m_r, v_r = F.train_step(replace(p, N=N), a, th_r, m_r, v_r, 3, step, 1e-3)
        want.append(lo)
    np.testing.assert_allclose(losses, want, rtol=0, atol=0)
    np.testing.assert_array_equal(th, th_r)
    # same Theta, same iteration, different grids: different losses
    l2 = F.rollout_loss(replace(p, N=2), a, th0, 3, 9).loss
    l4 = F.rollout_loss(replace(p, N=4), a, th0, 3, 9).loss
    assert abs(l2 - l4) > 1e-6 * max(abs(l2), abs(l4))
