"""mrs_velocity_noalloc: the pair sum for callers that cannot allocate device memory.

Collected last on purpose (file name), so that a run stopping at the first failure has run
every other test before it.  Through the C ABI it checks two calls in a row of the
no-allocation entry point against the FP64 CPU oracle (the parity bar of the other float32
pair-sum tests) and against mrs_velocity, the entry point that builds its own scratch; and that
sizes beyond the fixed scratch, aliased outputs and misaligned pointers are rejected before any
launch.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_oracle_and_mrs_velocity_two_calls():
    import oracle
    from paper_2604_12083_gb300 import build as B, mrs, workloads as W
    B.build()
    oracle.build()
    ctx = mrs.Context(0)
    try:
        # two calls in a row with different sizes (a ragged last tile in both): stale scratch
        # from the first call must not leak into the second
        for p in (W.single_system(seed=81, n_fil=5, M=1000), W.single_system(seed=80, n_fil=3, M=700)):
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
            un, wn = u.cpu().numpy(), w.cpu().numpy()
            assert np.isfinite(un).all() and np.isfinite(wn).all()
            uo, wo = oracle.mrs_velocity(p.X, p.f, p.n, eps, p.mu)
            assert rel_l2(un, uo) < TOL32 and rel_l2(wn, wo) < TOL32
            assert rel_l2(un, u_ref.cpu().numpy()) < TOL32
            assert rel_l2(wn, w_ref.cpu().numpy()) < TOL32
    finally:
        ctx.close()


def test_noalloc_rejects_bad_arguments_and_accepts_empty():
    from paper_2604_12083_gb300 import build as B, mrs
    B.build()
    X = torch.zeros((8, 3), device="cuda")
    u = torch.zeros_like(X)
    w = torch.zeros_like(X)
    with pytest.raises(mrs.MrsError) as e:
        mrs.mrs_velocity_noalloc((1 << 20) + 1, X, X, X, u, w, 1.0, 0.01)
    assert e.value.status == mrs.MRS_EINVAL and "at most" in str(e.value)
    bad = [
        lambda: mrs.mrs_velocity_noalloc(8, X, X, X, u, w, 1.0, 0.0),     # eps = 0
        lambda: mrs.mrs_velocity_noalloc(8, X, X, X, X, w, 1.0, 0.01),    # u aliases X
        lambda: mrs.mrs_velocity_noalloc(8, X, X, X, u, u, 1.0, 0.01),    # w aliases u
    ]
    for call in bad:
        with pytest.raises(mrs.MrsError) as e:
            call()
        assert e.value.status == mrs.MRS_EINVAL
    # outputs overlapping an input by part of a row, and a source pointer that is not
    # float-aligned, through the C entry point directly (rejected before any launch)
    big = torch.zeros((16, 3), device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = ctypes.c_void_p
    st = mrs.lib().mrs_velocity_noalloc(8, vp(big.data_ptr()), vp(X.data_ptr()), vp(X.data_ptr()),
                                        vp(big.data_ptr() + 4 * 20), vp(w.data_ptr()), 1.0, 0.01, s)
    assert st == mrs.MRS_EINVAL
    st = mrs.lib().mrs_velocity_noalloc(4, vp(big.data_ptr() + 2), vp(X.data_ptr()),
                                        vp(X.data_ptr()), vp(u.data_ptr()), vp(w.data_ptr()),
                                        1.0, 0.01, s)
    assert st == mrs.MRS_EINVAL
    mrs.mrs_velocity_noalloc(0, X, X, X, u, w, 1.0, 0.01)
