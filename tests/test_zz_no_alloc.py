"""fbsde_residual_loss_noalloc: the residual / loss step for callers that may
not allocate device memory (their own pool owns it, or they cannot take an
allocation's synchronisation).  It must give what the allocating path gives
from the same paths and network values, call after call, although every call
reuses one fixed device array for its per-path scratch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_loss_matches_the_allocating_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_11623_gb300 as P
    from paper_1910_11623_gb300 import _lib as L

    w = P.workloads.WORKLOADS["bsb_d10_n8_m64_fc4x64_sin"]
    for problem, it in [(w.problem, 3), (P.ProblemSpec(kind="hjb", D=13, N=5, M=37, x0=[0.0] * 13,
                                                         terminal_grad_term=True), 4)]:
        s = P.Solver(problem, w.arch, seed=1)
        theta = s.init_params()
        dW, X = s.sample_paths(it)
        Y, Z, _ = s.rollout_detail(theta, it)
        loss_ref, y0_ref = s.rollout_loss(theta, it)
        pc, _keep = problem.to_c()
        P1, D = problem.M * (problem.N + 1), problem.D
        st = torch.cuda.current_stream().cuda_stream
        for _ in range(2):  # the shared scratch keeps the previous call's terms
            alpha = torch.full((P1,), float("nan"), device="cuda")
            V = torch.full((P1 * D,), float("nan"), device="cuda")
            loss = torch.full((1,), float("nan"), device="cuda")
            y0 = torch.full((1,), float("nan"), device="cuda")
            L.fbsde_residual_loss_noalloc(pc, X.data_ptr(), dW.data_ptr(), Y.data_ptr(), Z.data_ptr(),
                                          alpha.data_ptr(), V.data_ptr(), loss.data_ptr(), y0.data_ptr(), st)
            torch.cuda.synchronize()
            assert abs(loss.item() - loss_ref.item()) <= 1e-5 * abs(loss_ref.item())
            assert abs(y0.item() - y0_ref.item()) <= 1e-5 * abs(y0_ref.item())
            assert torch.isfinite(alpha).all() and torch.isfinite(V).all()
        s.close()


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
