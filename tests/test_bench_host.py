"""Host logic of bench.py that decides reported numbers, checked on the CPU:
the held-accuracy criterion (Y0 within 1 % of the closed form at a run of
consecutive checks) and the algorithmic byte count the HBM view of the
roofline divides by."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_held_needs_a_full_run_inside_the_band(bench):
    target = 100.0
    h = bench.Held(target, tol=0.01, hold=3)
    # touches the band at step 50, leaves it, then stays from step 200 on
    seq = [(0, 90.0), (50, 99.5), (100, 102.0), (150, 98.0), (200, 100.4), (250, 99.2), (300, 100.9),
           (350, 100.1)]
    got = [h.check(step, step / 100.0, y0) for step, y0 in seq]
    assert h.first == (50, 0.5)
    # the held run starts at the first of three consecutive checks inside
    assert h.held == (200, 2.0)
    assert got == [False, False, False, False, False, False, True, True]
    # the recorded errors are relative to the target
    assert h.checks[1] == (50, pytest.approx(0.005))


def test_held_boundary_is_inclusive_and_runs_reset(bench):
    h = bench.Held(10.0, tol=0.1, hold=2)
    assert not h.check(1, 0.0, 11.0)       # exactly on the band's edge: inside
    assert h.first == (1, 0.0)
    assert not h.check(2, 0.0, 11.5)       # outside resets the run
    assert not h.check(3, 0.0, 9.0)        # inside again (edge)
    assert h.check(4, 0.0, 10.2)           # second consecutive: held from step 3
    assert h.held == (3, 0.0)
    assert h.check(5, 0.0, 20.0)           # leaving later does not undo it
    assert h.held == (3, 0.0)


def test_algorithmic_bytes_of_the_pipelined_kernels(bench):
    import paper_1910_11623_gb300 as P
    w = P.workloads.WORKLOADS["bsb_d100_n64_m4096_resnet5x256_tanh"].with_prec("bf16")
    P_ = 4096 * 65
    stack = P_ * 256 * 2            # one BF16 operand block of the whole batch
    rows = P_ * 128 * 2             # BF16 X (or v) rows, D = 100 padded to 128
    L = 5
    # forward: e_l (L + 1) and g_l (L) written, Z (FP32) and Y written, X rows read
    fwd = (2 * L + 1) * stack + rows + P_ * 100 * 4 + P_ * 4
    # backward: h_l, h'_l (l < L) and abar_l (l <= L) written, g_l read, X and v rows read,
    # the read-out gradient's partial sums (tiles x 4 row groups x w) written
    bwd = (3 * L + 1) * stack + L * stack + 2 * rows + (P_ // 128) * 4 * 256 * 4
    assert bench.fused_algorithmic_bytes(w) == pytest.approx((fwd + bwd) / 2)
    # NAIS-Net runs on the general kernels, which also store h_L and h'_L
    wn = P.workloads.WORKLOADS["hjb_d100_n64_m8192_nais6x256_tanh"].with_prec("bf16")
    Pn = 8192 * 65
    sn, rn, Ln = Pn * 256 * 2, Pn * 128 * 2, 6
    fwdn = (2 * Ln + 1) * sn + rn + Pn * 100 * 4 + Pn * 4
    bwdn = 3 * (Ln + 1) * sn + Ln * sn + 2 * rn
    assert bench.fused_algorithmic_bytes(wn) == pytest.approx((fwdn + bwdn) / 2)
    # outside the fused kernels' limits there is no such figure
    assert bench.fused_algorithmic_bytes(w.with_prec("fp32")) is None


def test_traffic_figure_only_for_the_sources_it_was_taken_on(bench, monkeypatch):
    import json
    wl = "bsb_d100_n64_m4096_resnet5x256_tanh"
    with open(os.path.join(bench.ROOT, "profiles", f"traffic_bf16_{wl}.json")) as f:
        d = json.load(f)
    # the figure is reported while the sources it names hash as at its capture
    monkeypatch.setattr(bench, "source_hash", lambda files=bench.KERNEL_SOURCES: d["source_hash"])
    assert bench.ncu_traffic("bf16", wl) == d["dram_bytes_per_launch"]
    # any change to those sources withdraws it
    monkeypatch.setattr(bench, "source_hash", lambda files=bench.KERNEL_SOURCES: "0" * 16)
    assert bench.ncu_traffic("bf16", wl) is None
    # and no figure exists for a workload never captured
    assert bench.ncu_traffic("bf16", "no_such_workload") is None
