"""fbsde_residual_loss_noalloc: the residual / loss step for callers that may
not allocate device memory (their own pool owns it, or they cannot take an
allocation's synchronisation).  It must give what the allocating path gives
from the same paths and network values, call after call, although every call
reuses one fixed device array for its per-path scratch.

The calls alternate between a larger and a smaller problem (other D, N, M and
other paths), so that terms a previous call left in the shared array would
show in the loss; the loss seeds alpha and V are compared with the oracle's
seeds computed in FP64 from the same X, dW, Y and Z."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fbsde as F
from tests.helpers import oracle_specs, rel_max

pytestmark = pytest.mark.gpu


def _oracle_seeds(problem, arch, X, dW, Y, Z):
    """alpha, V of Eq. "loss" from the given arrays (time-major point order)."""
    op, _ = oracle_specs(problem, arch)
    N, M, D = op.N, op.M, op.D
    X = X.cpu().numpy().astype(np.float64).reshape(N + 1, M, D)
    dW = dW.cpu().numpy().astype(np.float64).reshape(N, M, D)
    Y = Y.cpu().numpy().astype(np.float64).reshape(N + 1, M)
    Z = Z.cpu().numpy().astype(np.float64).reshape(N + 1, M, D)
    r, rT, gradT = F.residuals(op, X, dW, Y, Z)
    ro = F.Rollout(loss=0.0, y0=0.0, X=X, dW=dW, Y=Y, Z=Z, r=r, rT=rT, path_loss=None)
    ro.extras = {"gradT": gradT}
    return F.loss_seeds(op, ro)


def test_noalloc_loss_matches_the_allocating_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_11623_gb300 as P
    from paper_1910_11623_gb300 import _lib as L

    w = P.workloads.WORKLOADS["bsb_d10_n8_m64_fc4x64_sin"]
    cases = [(w.problem, 3),
             (P.ProblemSpec(kind="hjb", D=13, N=5, M=37, x0=[0.0] * 13, terminal_grad_term=True), 4)]
    prepared = []
    for problem, it in cases:
        s = P.Solver(problem, w.arch, seed=1)
        theta = s.init_params()
        dW, X = s.sample_paths(it)
        Y, Z, _ = s.rollout_detail(theta, it)
        loss_ref, y0_ref = s.rollout_loss(theta, it)
        torch.cuda.synchronize()
        a_ref, v_ref = _oracle_seeds(problem, w.arch, X, dW, Y, Z)
        prepared.append((problem, X, dW, Y, Z, loss_ref.item(), y0_ref.item(), a_ref, v_ref))
        s.close()
    st = torch.cuda.current_stream().cuda_stream
    # larger, smaller, larger again: each call after the first finds the
    # previous call's terms in the shared array
    for k in (0, 1, 0, 1):
        problem, X, dW, Y, Z, loss_ref, y0_ref, a_ref, v_ref = prepared[k]
        pc, _keep = problem.to_c()
        P1, D = problem.M * (problem.N + 1), problem.D
        alpha = torch.full((P1,), float("nan"), device="cuda")
        V = torch.full((P1 * D,), float("nan"), device="cuda")
        loss = torch.full((1,), float("nan"), device="cuda")
        y0 = torch.full((1,), float("nan"), device="cuda")
        L.fbsde_residual_loss_noalloc(pc, X.data_ptr(), dW.data_ptr(), Y.data_ptr(), Z.data_ptr(),
                                      alpha.data_ptr(), V.data_ptr(), loss.data_ptr(), y0.data_ptr(), st)
        torch.cuda.synchronize()
        assert abs(loss.item() - loss_ref) <= 1e-5 * abs(loss_ref), (k, loss.item(), loss_ref)
        assert abs(y0.item() - y0_ref) <= 1e-5 * abs(y0_ref), (k, y0.item(), y0_ref)
        ea = rel_max(alpha.cpu().numpy().reshape(a_ref.shape), a_ref)
        ev = rel_max(V.cpu().numpy().reshape(v_ref.shape), v_ref)
        assert ea < 1e-5 and ev < 1e-5, (k, ea, ev)


def test_noalloc_rejects_more_paths_than_its_array_holds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_11623_gb300 as P
    from paper_1910_11623_gb300 import _lib as L
    problem = P.ProblemSpec(kind="bsb", D=4, N=2, M=65537, x0=[1.0] * 4)
    pc, _keep = problem.to_c()
    buf = torch.zeros(16, device="cuda")
    with pytest.raises(L.FBSDEError) as ei:
        L.fbsde_residual_loss_noalloc(pc, *([buf.data_ptr()] * 8), torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == L.FBSDE_ERR_INVALID
    assert "65536" in str(ei.value)
