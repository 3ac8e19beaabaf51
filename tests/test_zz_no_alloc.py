"""mrs_velocity_noalloc: the pair sum for callers that cannot allocate device memory.

Collected last on purpose (file name): it checks, through the C ABI, that two calls in a row of
the no-allocation entry point agree with mrs_velocity, the entry point that builds its own
scratch, within the float32 tolerance of the other pair-sum tests, and that sizes beyond the
fixed scratch are rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def rel_l2(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_mrs_velocity_two_calls():
    from paper_2604_12083_gb300 import build as B, mrs, workloads as W
    B.build()
    ctx = mrs.Context(0)
    try:
        # two calls in a row with different sizes: stale scratch from the first must not leak
        for p in (W.single_system(), W.single_system(seed=80, n_fil=3, M=1000)):
            X, f, n = (torch.from_numpy(a).cuda() for a in (p.X, p.f, p.n))
            eps = float(p.eps[0])
            u_ref = torch.empty_like(X)
            w_ref = torch.empty_like(X)
            mrs.mrs_velocity(ctx, p.offsets, X, f, n, u_ref, w_ref, p.mu, eps,
                             precision=mrs.MRS_F32_COMP)
            u = torch.full_like(X, float("nan"))
            w = torch.full_like(X, float("nan"))
            mrs.mrs_velocity_noalloc(p.n_points, X, f, n, u, w, p.mu, eps)
            torch.cuda.synchronize()
            assert torch.isfinite(u).all() and torch.isfinite(w).all()
            assert rel_l2(u, u_ref) < TOL32 and rel_l2(w, w_ref) < TOL32
    finally:
        ctx.close()


def test_noalloc_rejects_oversize_and_accepts_empty():
    from paper_2604_12083_gb300 import build as B, mrs
    B.build()
    X = torch.zeros((8, 3), device="cuda")
    u = torch.zeros_like(X)
    w = torch.zeros_like(X)
    with pytest.raises(mrs.MrsError) as e:
        mrs.mrs_velocity_noalloc((1 << 20) + 1, X, X, X, u, w, 1.0, 0.01)
    assert e.value.status == mrs.MRS_EINVAL and "at most" in str(e.value)
    with pytest.raises(mrs.MrsError):
        mrs.mrs_velocity_noalloc(8, X, X, X, u, w, 1.0, 0.0)
    mrs.mrs_velocity_noalloc(0, X, X, X, u, w, 1.0, 0.01)
