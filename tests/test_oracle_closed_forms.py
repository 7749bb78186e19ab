"""Closed-form anchors of the two benchmark problems (Section 4), checked
through the oracle's problem data (x0, g, noise scale)."""
import os

import numpy as np
from scipy import integrate, stats

from oracle import fbsde as F
from oracle import philox


def _paper_values(golden_dir):
    out = {}
    with open(os.path.join(golden_dir, "paper_values.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, val, tol, *_ = line.split()
                out[name] = (float(val), float(tol))
    return out


def bsb_closed_form(p, t, x):
    """u(x, t) = exp((r + sigma^2)(T - t)) ||x||^2 (Section 4)."""
    return np.exp((p.r + p.sigma ** 2) * (p.T - t)) * np.sum(x * x, axis=-1)


def test_bsb_y0_matches_the_value_printed_in_the_paper(golden_dir):
    want, tol = _paper_values(golden_dir)["bsb_y0_d100"]
    D = 100
    x0 = np.array([1.0 if i % 2 == 0 else 0.5 for i in range(D)])
    p = F.Problem(kind="bsb", D=D, N=64, M=1, x0=x0)
    y0 = bsb_closed_form(p, 0.0, x0)
    assert abs(y0 - want) < tol
    assert abs(y0 - 62.5 * np.exp(0.21)) < 1e-12
    # and the oracle's terminal condition is the closed form at t = T
    g, _ = F.terminal(p, x0[None, :])
    assert abs(g[0] - bsb_closed_form(p, p.T, x0)) < 1e-12


def test_paper_hyperparameters(golden_dir):
    vals = _paper_values(golden_dir)
    arch = F.Arch(kind="nais", width=8, depth=1, act="tanh")
    assert arch.eps == vals["nais_eps"][0]
    assert vals["adam_lr"][0] == 1e-3


def hjb_u00_quadrature(D=100, T=1.0):
    """u(0, 0) = -ln E[exp(-g(sqrt(2) W_T))] = -ln E[2 / (1 + 2 T Q)],
    Q ~ chi^2_D (Cole-Hopf form of the Section 4 HJB solution, read with
    W_{T-t}), by 1-D quadrature over the chi-square density."""
    f = lambda q: 2.0 / (1.0 + 2.0 * T * q) * stats.chi2.pdf(q, D)
    val, _ = integrate.quad(f, 0, np.inf, limit=500)
    return -np.log(val)


def test_hjb_u00_quadrature_agrees_with_monte_carlo_through_the_oracle():
    # u(0, x0=0) for D=100, T=1 by quadrature, against a Monte Carlo estimate
    # that uses the oracle's own increments (one Euler step: X_N = sqrt(2) W_T)
    # and the oracle's terminal function g.
    u_quad = hjb_u00_quadrature()
    assert abs(u_quad - 4.590162) < 1e-5
    D, M = 100, 100000
    p = F.Problem(kind="hjb", D=D, N=1, M=M, x0=np.zeros(D))
    dW = philox.brownian_increments(21, 0, M, 1, D, p.T)
    XN = F.forward_sde(p, dW)[-1]
    g, _ = F.terminal(p, XN)
    w = np.exp(-g)
    u_mc = -np.log(w.mean())
    se = w.std() / np.sqrt(M) / w.mean()
    assert abs(u_mc - u_quad) < 5 * se
