"""Host-side workload definitions: the named workloads are valid specifications
for the library, the seeded batch of uneven instances has the advertised
shape mix and fits its memory budget, and the closed-form anchors follow
from the BSB solution of Section 4.1."""
import math
import os

import pytest

from oracle import fbsde as F
from tests.helpers import oracle_specs


@pytest.fixture(scope="module")
def P():
    import paper_1910_11623_gb300 as P
    from paper_1910_11623_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1910_11623_gb300 import build
        build.build()
    _lib.load()
    return P


def test_named_workloads_are_valid_specs(P):
    from paper_1910_11623_gb300 import _lib as L
    for name, w in P.workloads.WORKLOADS.items():
        assert name == w.name
        pc, _keep = w.problem.to_c()
        n = L.fbsde_param_count(pc, w.arch.to_c())
        op, oa = oracle_specs(w.problem, w.arch)
        assert n == F.num_params(op, oa) > 0, name


def test_bsb_anchor_is_the_closed_form(P):
    # u(0, x0) = exp((r + sigma^2) T) ||x0||^2 with x0 = (1, 0.5, ...): 62.5 e^0.21 at D = 100
    x0 = P.workloads.bsb_x0(100)
    assert P.workloads.bsb_y0(x0) == pytest.approx(62.5 * math.exp(0.21), rel=1e-15)
    assert P.workloads.BSB_Y0_D100 == pytest.approx(P.workloads.bsb_y0(x0), rel=1e-9)
    assert P.workloads.BSB_Y0_D10 == pytest.approx(P.workloads.bsb_y0(P.workloads.bsb_x0(10)), rel=1e-9)


def test_multilevel_levels_double_up_to_the_target_grid(P):
    lv = P.workloads.MULTILEVEL_LEVELS
    assert all(b == 2 * a for a, b in zip(lv, lv[1:]))
    assert lv[-1] == P.workloads.WORKLOADS["bsb_d100_n64_m4096_resnet5x256_tanh"].problem.N


def test_batched_instances_mix_and_budget(P):
    ws = P.workloads.batched_instances(0)
    again = P.workloads.batched_instances(0)
    assert [w.name for w in ws] == [w.name for w in again]  # seeded
    assert len(ws) == 32
    assert sum(w.problem.kind == "bsb" for w in ws) == 16
    for w in ws:
        p, a = w.problem, w.arch
        assert p.D in (10, 20, 50, 100, 200) and p.N in (16, 32, 64, 128)
        assert p.M in (1024, 4096, 16384) or (p.M < 16384 and 16384 % p.M == 0)
        assert a.kind == "resnet" and a.width in (128, 256, 512) and a.prec == "bf16"
        assert len(p.x0) == p.D
    assert {w.arch.width for w in ws} == {128, 256, 512}
    # a smaller budget halves the largest instances until the estimate fits
    small = P.workloads.batched_instances(0, budget_gb=20.0)
    assert sum(w.problem.M for w in small) < sum(w.problem.M for w in ws)
