"""The C ABI: every entry point declared in include/fbsde.h is exported by
libfbsde.so and bound by the Python layer under the same name, and invalid
specifications are rejected on the host before any CUDA call."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fbsde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fbsde_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_1910_11623_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1910_11623_gb300 import build
        build.build()
    _lib.load()
    return _lib


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ["fbsde_create", "fbsde_destroy", "fbsde_num_params", "fbsde_init_params",
                 "fbsde_rollout_loss", "fbsde_rollout_grad", "fbsde_train_step",
                 "fbsde_set_level", "fbsde_status_string", "fbsde_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(L):
    lib = L.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(L):
    assert sorted(L.SIGNATURES) == _declared()
    for name in _declared():
        assert callable(getattr(L, name)), name


def test_no_torch_types_in_the_header():
    src = open(os.path.join(ROOT, "include", "fbsde.h")).read()
    assert "torch" not in src.lower().replace("pytorch", "") and "at::" not in src


def _specs(**kw):
    import paper_1910_11623_gb300 as P
    p = dict(kind="bsb", D=4, N=3, M=5, x0=[1.0, 0.5, 1.0, 0.5])
    a = dict(kind="fc", width=16, depth=2, act="tanh")
    for k, v in kw.items():
        (a if k.startswith("a_") else p)[k[2:] if k.startswith("a_") else k] = v
    return P.ProblemSpec(**p), P.ArchSpec(**a)


@pytest.mark.parametrize("bad,needle", [
    (dict(D=0, x0=[]), "problem.D"),
    (dict(N=0), "problem.N"),
    (dict(M=0), "problem.M"),
    (dict(T=-1.0), "problem.T"),
    (dict(sigma=-0.1), "sigma"),
    (dict(a_width=20), "arch.width"),
    (dict(a_width=528), "arch.width"),
    (dict(a_depth=17), "arch.depth"),
    (dict(a_kind="nais", a_eps=0.0), "arch.eps"),
    (dict(a_kind="nais", a_h=0.0), "arch.h"),
])
def test_create_rejects_invalid_specs_without_a_gpu(L, bad, needle):
    p, a = _specs(**bad)
    pc, _keep = p.to_c()
    with pytest.raises(L.FBSDEError) as ei:
        L.fbsde_create(pc, a.to_c(), 0, 0, 0)
    assert ei.value.status == L.FBSDE_ERR_INVALID
    assert needle in str(ei.value)
    assert L.fbsde_param_count(pc, a.to_c()) == 0


def test_create_rejects_small_N_max(L):
    p, a = _specs()
    pc, _keep = p.to_c()
    with pytest.raises(L.FBSDEError) as ei:
        L.fbsde_create(pc, a.to_c(), 0, 0, 2)
    assert "N_max" in str(ei.value)


def test_param_count_matches_the_oracle_layout(L):
    import numpy as np
    from oracle import fbsde as F
    from tests.helpers import oracle_specs
    for kind in ["fc", "resnet", "nais"]:
        p, a = _specs(a_kind=kind, D=7, x0=[0.0] * 7, a_width=32, a_depth=3)
        pc, _keep = p.to_c()
        op, oa = oracle_specs(p, a)
        assert L.fbsde_param_count(pc, a.to_c()) == F.num_params(op, oa)


def test_status_strings(L):
    for s in range(7):
        assert L.fbsde_status_string(s)


def test_schedule_rejects_a_null_context_without_a_gpu(L):
    lib = L.load()
    lv = (L.c_int * 2)(2, 4)
    st = (L.c_int * 2)(1, 1)
    rc = lib.fbsde_train_schedule(None, None, None, None, lv, st, 2, 1, 1e-3, None, None)
    assert rc == L.FBSDE_ERR_INVALID


def test_graph_entry_points_reject_null_arguments_without_a_gpu(L):
    lib = L.load()
    out = L.c_void_p()
    assert lib.fbsde_graph_capture(None, None, None, None, None, 1e-3, None, None, 1,
                                   L.ctypes.byref(out)) == L.FBSDE_ERR_INVALID
    assert lib.fbsde_graph_launch(None) == L.FBSDE_ERR_INVALID
    assert lib.fbsde_graph_destroy(None) == L.FBSDE_OK
    assert lib.fbsde_train_step_dev(None, None, None, None, None, 1e-3, None, None) == L.FBSDE_ERR_INVALID


def test_group_entry_points_reject_bad_arguments_without_a_gpu(L):
    lib = L.load()
    out = L.c_void_p()
    assert lib.fbsde_group_create(None, 0, None, L.ctypes.byref(out)) == L.FBSDE_ERR_INVALID
    assert lib.fbsde_group_destroy(None) == L.FBSDE_OK
    assert lib.fbsde_group_train_step(None, None, None, None, None, 1e-3, None, None) == L.FBSDE_ERR_INVALID
    assert lib.fbsde_set_grid_cap(None, 0) == L.FBSDE_ERR_INVALID
    assert lib.fbsde_group_set_mode(None, L.FBSDE_GROUP_GROUPED) == L.FBSDE_ERR_INVALID
