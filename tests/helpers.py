"""Shared test helpers: build matching oracle and library specifications from
one description, and the error measures used by the parity tests."""
import numpy as np

from oracle import fbsde as F

# Absolute floor of the per-block gradient error, as a fraction of the largest
# gradient entry: a block is measured against its own largest entry, or
# against this fraction of the whole gradient's largest entry when that is
# larger (a block that is exactly zero, or 1000x below the rest, is not
# measured against rounding noise alone).
GRAD_FLOOR = 1e-3


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


def block_errors(got, want, problem, arch, floor=GRAD_FLOOR):
    """Error of a flat parameter-sized vector per parameter block (W_in, b_in,
    W_l or R_l, b_l or C_l, B_l, w_o, b_o): max |got - want| over the block
    divided by max(max |want| over the block, floor * max |want| overall).
    `problem` and `arch` are the oracle's Problem and Arch."""
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    want = np.asarray(want, dtype=np.float64).reshape(-1)
    big = float(np.max(np.abs(want))) if want.size else 0.0
    out, off = {}, 0
    for name, shape, *_ in F.param_layout(problem, arch):
        n = int(np.prod(shape))
        g, o = got[off:off + n], want[off:off + n]
        scale = max(float(np.max(np.abs(o))), floor * big)
        out[name] = float(np.max(np.abs(g - o)) / (scale if scale > 0 else 1.0))
        off += n
    assert off == want.size
    return out
