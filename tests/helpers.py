"""Shared test helpers: build matching oracle and library specifications from
one description, and the error measures used by the parity tests."""
import numpy as np

from oracle import fbsde as F


def oracle_specs(problem, arch):
    """Library ProblemSpec/ArchSpec -> oracle Problem/Arch."""
    p = F.Problem(kind=problem.kind, D=problem.D, N=problem.N, M=problem.M,
                  x0=np.asarray(problem.x0, dtype=np.float64), T=problem.T, r=problem.r,
                  sigma=problem.sigma, terminal_grad_term=bool(problem.terminal_grad_term))
    a = F.Arch(kind=arch.kind, width=arch.width, depth=arch.depth, act=arch.act, h=arch.h,
               eps=arch.eps, proj_delta=(arch.proj_delta if arch.proj_delta > 0 else None))
    return p, a


def rel_max(got, want):
    """max |got - want| / max |want| (scale-aware elementwise error)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.max(np.abs(want))
    return float(np.max(np.abs(got - want)) / (scale if scale > 0 else 1.0))


def rel(got, want):
    return abs(float(got) - float(want)) / max(abs(float(want)), 1e-300)
