"""GPU parity of the rod path (rotation square root, rod forces, Euler/RK2 steps, Parareal)
against the FP64 CPU oracle.

Bars: float64 kernels (rotation sqrt, forces) to ~1e-12 relative; time stepping with the
float32 pair sum <= 1e-4 relative on positions AND on the displacement X(T) - X(0) after the
stated number of steps; with the float64 pair sum, 1e-9 on the displacement.
"""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_rotation_sqrt.json")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_12083_gb300 import build as B, mrs
    B.build()
    c = mrs.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def params(W_cfg, eps, mu=1.0):
    from paper_2604_12083_gb300 import mrs
    import oracle
    g = mrs.RodParams.make(W_cfg["L"], W_cfg["a"], W_cfg["b"], W_cfg["wave_A"], W_cfg["wave_k"],
                           W_cfg["wave_f"], mu, eps)
    o = oracle.RodParams.make(W_cfg["L"], W_cfg["a"], W_cfg["b"], W_cfg["wave_A"], W_cfg["wave_k"],
                              W_cfg["wave_f"])
    return g, o


def test_rotation_sqrt_paper_sweep(ctx, orc):
    """Table 2's sweep (100 angles in [-0.1, pi+0.1], random axes) on the GPU routine."""
    from scipy.spatial.transform import Rotation
    from paper_2604_12083_gb300 import mrs
    g = json.load(open(GOLDEN))
    rng = np.random.default_rng(70)
    Rs = []
    for _ in range(20):
        ax = rng.standard_normal(3)
        ax /= np.linalg.norm(ax)
        for th in np.linspace(-0.1, math.pi + 0.1, 100):
            Rs.append(Rotation.from_rotvec(ax * th).as_matrix())
    R = np.array(Rs)
    Rd = torch.from_numpy(R).cuda()
    Sd = torch.empty_like(Rd)
    mrs.rot_sqrt_batch(ctx, Rd, Sd)
    torch.cuda.synchronize()
    S = Sd.cpu().numpy()
    err = np.linalg.norm(S @ S - R, axis=(1, 2))
    assert err.max() < 1e-13
    assert err.mean() <= g["cuda_error"]["mean"]
    orth = np.abs(np.einsum("nij,nkj->nik", S, S) - np.eye(3)).max()
    assert orth < 1e-14
    for i in range(0, len(R), 7):
        np.testing.assert_allclose(S[i], orc.rot_sqrt(R[i]), atol=1e-13)


def perturbed(seed, n_rods, M, amp=0.02):
    from scipy.spatial.transform import Rotation
    from paper_2604_12083_gb300 import workloads as W
    rs = W.rod_system(seed, n_rods, M, box=3.0)
    rng = np.random.default_rng(seed)
    X = rs.X + amp * rng.standard_normal(rs.X.shape) / M
    Rr = Rotation.from_rotvec(amp * rng.standard_normal((len(X), 3))).as_matrix()
    D = np.einsum("krc,kic->kir", Rr, rs.D)
    return rs, X, D


def test_rod_forces_match_oracle(ctx, orc):
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs, X, D = perturbed(71, 1, 17)
    # three rods of different lengths, including the 2-node minimum
    rs2, X2, D2 = perturbed(72, 1, 1024)
    X = np.concatenate([X, np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.01]]), X2])
    D = np.concatenate([D, np.tile(np.eye(3), (2, 1, 1)), D2])
    off = np.array([0, 17, 19, 19 + 1024], np.int64)
    gp, op = params(dict(W.ROD_PLAIN), 0.01)
    for t in (0.0, 0.37):
        Xd, Dd = torch.from_numpy(X).cuda(), torch.from_numpy(D).cuda()
        g = torch.empty_like(Xd)
        m = torch.empty_like(Xd)
        mrs.rod_forces(ctx, off, gp, Xd, Dd, t, g, m)
        torch.cuda.synchronize()
        go, mo = orc.rod_forces(off, X, D, op, t)
        gg, mm = g.cpu().numpy(), m.cpu().numpy()
        assert np.abs(gg - go).max() <= 1e-11 * np.abs(go).max()
        assert np.abs(mm - mo).max() <= 1e-11 * np.abs(mo).max()


@pytest.mark.parametrize("mode", [1, 2])
def test_rod_force_kernels_match_oracle(ctx, orc, mode):
    """Both force kernels -- one thread per segment (mode 1) and warp-cooperative (mode 2) -- on
    rods of 2, 3, 8, 9, 16, 17, 51 and 300 nodes (around the warp kernel's chunks of 8 nodes
    and the thread kernel's of 127), once with frames near their neighbours' (the quaternion
    branch of the trace) and once with independent random frames (relative rotations of any
    angle below pi: every branch of the rotation square root), at two times: against the
    oracle to 1e-11 of the largest entry."""
    from scipy.spatial.transform import Rotation
    from paper_2604_12083_gb300 import mrs, workloads as W
    sizes = [2, 3, 8, 9, 16, 17, 51, 300]
    rng = np.random.default_rng(91)
    Xs, Ds = [], []
    for M in sizes:
        X, D = W.sinusoid_filament(M)
        Xs.append(X + rng.uniform(0.0, 2.0, 3))
        Ds.append(D)
    X = np.concatenate(Xs)
    D0 = np.concatenate(Ds)
    Drand = Rotation.random(len(X), random_state=92).as_matrix()   # rows: the directors
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    gp, op = params(dict(W.ROD_PLAIN), 0.01)
    ctx.set_rod_force_kernel(mode)
    try:
        for D in (D0, Drand):
            for t in (0.0, 0.37):
                Xd, Dd = torch.from_numpy(X).cuda(), torch.from_numpy(D).cuda()
                g, m = torch.empty_like(Xd), torch.empty_like(Xd)
                mrs.rod_forces(ctx, off, gp, Xd, Dd, t, g, m)
                torch.cuda.synchronize()
                go, mo = orc.rod_forces(off, X, D, op, t)
                gg, mm = g.cpu().numpy(), m.cpu().numpy()
                assert np.abs(gg - go).max() <= 1e-11 * np.abs(go).max(), (mode, t)
                assert np.abs(mm - mo).max() <= 1e-11 * np.abs(mo).max(), (mode, t)
    finally:
        ctx.set_rod_force_kernel(0)


@pytest.mark.parametrize("scheme", [0, 1])
def test_rod_force_kernels_agree_in_stepping(ctx, orc, scheme):
    """200 steps of 4 rods of 51 points (a paper size) on the kernel graphs with each force
    kernel: both match the oracle's steps (float32 pair sum: 1e-4 on the displacement) and each
    other to float32 rounding of the packed forces."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs, X, D = perturbed(93, 4, 51)
    cfg = dict(W.ROD_PLAIN)
    eps = 4.0 / 50
    gp, op = params(cfg, eps)
    dt = cfg["dt"]
    Xo, _ = orc.rod_step(rs.rod_off, X, D, op, eps, 1.0, 0.0, dt, 200, scheme)
    out = {}
    try:
        ctx.set_fused_steps(0)
        for mode in (1, 2):
            ctx.set_rod_force_kernel(mode)
            Xs_, Ds_ = torch.from_numpy(X.copy()).cuda(), torch.from_numpy(D.copy()).cuda()
            mrs.rod_step(ctx, rs.rod_off, gp, Xs_, Ds_, 0.0, dt, 200, scheme)
            torch.cuda.synchronize()
            out[mode] = Xs_.cpu().numpy()
            assert rel(out[mode] - X, Xo - X) < 1e-4, mode
    finally:
        ctx.set_rod_force_kernel(0)
        ctx.set_fused_steps(1)
    assert rel(out[2] - X, out[1] - X) < 1e-6


@pytest.mark.parametrize("scheme", [0, 1])
def test_plain_rod_200_steps(ctx, orc, scheme):
    """One rod of 128 nodes, 200 steps at dt = 1e-6 (the plain-method configuration)."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(1, 1, 128)
    cfg = dict(W.ROD_PLAIN)
    gp, op = params(cfg, rs.eps)
    Xo, Do = orc.rod_step(rs.rod_off, rs.X, rs.D, op, rs.eps, 1.0, 0.0, cfg["dt"], 200, scheme)
    for prec, tol in ((mrs.MRS_F32_COMP, 1e-4), (mrs.MRS_F64, 1e-9)):
        Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
        mrs.rod_step(ctx, rs.rod_off, gp, Xd, Dd, 0.0, cfg["dt"], 200, scheme, precision=prec)
        torch.cuda.synchronize()
        Xg, Dg = Xd.cpu().numpy(), Dd.cpu().numpy()
        assert rel(Xg, Xo) < 1e-4
        assert rel(Xg - rs.X, Xo - rs.X) < tol, (prec, rel(Xg - rs.X, Xo - rs.X))
        assert rel(Dg - rs.D, Do - rs.D) < 10 * tol
        assert np.abs(np.einsum("kir,kjr->kij", Dg, Dg) - np.eye(3)).max() < 1e-12


def test_multi_rod_rk2_and_resume(ctx, orc):
    """Four interacting rods; 37 steps in one call equal 20 + 17 steps in two calls."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(73, 4, 64, box=2.0)
    cfg = dict(W.ROD_PLAIN, a=(2e-3,) * 3, b=(20.0,) * 3)
    gp, op = params(cfg, rs.eps)
    dt = 2e-6
    Xo, _ = orc.rod_step(rs.rod_off, rs.X, rs.D, op, rs.eps, 1.0, 0.1, dt, 37, orc.RK2)
    Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    mrs.rod_step(ctx, rs.rod_off, gp, Xd, Dd, 0.1, dt, 37, mrs.MRS_RK2)
    Xa = Xd.cpu().numpy()
    Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    mrs.rod_step(ctx, rs.rod_off, gp, Xd, Dd, 0.1, dt, 20, mrs.MRS_RK2)
    mrs.rod_step(ctx, rs.rod_off, gp, Xd, Dd, 0.1 + 20 * dt, dt, 17, mrs.MRS_RK2)
    Xb = Xd.cpu().numpy()
    assert rel(Xa - rs.X, Xo - rs.X) < 1e-4
    assert rel(Xb - rs.X, Xo - rs.X) < 1e-4


def test_parareal_matches_oracle_and_serial_fine(ctx, orc):
    from oracle import parareal as PR
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(74, 2, 24, box=1.5)
    cfg = dict(W.WAVE, a=(2e-3,) * 3, b=(0.3,) * 3)
    gp, op = params(cfg, rs.eps)
    Ns, dt, r = 6, 5e-5, 4
    T1 = Ns * 16 * dt
    tol = 1e-10
    states, incr = PR.rod_parareal(rs.rod_off, rs.X, rs.D, op, rs.eps, 1.0, 0.0, T1, Ns, dt, r,
                                   Ns, tol)
    Xo, _ = PR.unpack_rod_state(states[-1][-1])
    Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    st = mrs.parareal_run(ctx, rs.rod_off, gp, Xd, Dd, 0.0, T1, Ns, dt, r, Ns, tol)
    Xg = Xd.cpu().numpy()
    assert rel(Xg - rs.X, Xo - rs.X) < 1e-4
    assert abs(st.iterations - len(incr)) <= 1
    # the first increments follow the oracle's (before either reaches float32 round-off)
    assert abs(st.incr[0] - incr[0]) <= 1e-3 * incr[0]
    # converged Parareal equals serial fine stepping
    Xs, Ds = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    mrs.rod_step(ctx, rs.rod_off, gp, Xs, Ds, 0.0, dt, Ns * 16, mrs.MRS_RK2)
    assert rel(Xg - rs.X, Xs.cpu().numpy() - rs.X) < 1e-5
    assert st.fine_steps > 0 and st.coarse_steps > 0


def test_rod_invalid_arguments(ctx):
    from paper_2604_12083_gb300 import mrs, workloads as W
    X = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    D = torch.zeros((4, 3, 3), dtype=torch.float64, device="cuda")
    gp, _ = params(dict(W.ROD_PLAIN), 0.01)
    with pytest.raises(mrs.MrsError):
        mrs.rod_step(ctx, [0, 1, 4], gp, X, D, 0.0, 1e-6, 1, 0)      # 1-node rod
    with pytest.raises(mrs.MrsError):
        ctx.set_fused_steps(3)                                        # modes are 0, 1, 2
    for bad in (-1, 3):
        with pytest.raises(mrs.MrsError):
            ctx.set_rod_force_kernel(bad)                             # modes are 0, 1, 2
    cfg = dict(W.ROD_PLAIN)
    zero_L = mrs.RodParams.make(0.0, cfg["a"], cfg["b"], cfg["wave_A"], cfg["wave_k"], cfg["wave_f"], 1.0, 0.01)
    nan_a = mrs.RodParams.make(1.0, (float("nan"),) * 3, cfg["b"], cfg["wave_A"], cfg["wave_k"],
                               cfg["wave_f"], 1.0, 0.01)
    g = torch.zeros_like(X)
    bad = [
        lambda: mrs.rod_forces(ctx, [0, 4], zero_L, X, D, 0.0, g, g.clone()),        # L = 0
        lambda: mrs.rod_forces(ctx, [0, 4], nan_a, X, D, 0.0, g, g.clone()),         # moduli
        lambda: mrs.rod_step(ctx, [0, 4], gp, X, D, 0.0, 1e-6, 1, 2),                # scheme
        lambda: mrs.rod_step(ctx, [0, 4], gp, X, D, 0.0, 1e-6, 1, 0, precision=9),
        lambda: mrs.rod_step(ctx, [0, 4], gp, X, D, float("inf"), 1e-6, 1, 0),       # t0
        lambda: mrs.parareal_run(ctx, [0, 4], gp, X, D, 0.0, 65e-6, 65, 1e-6, 1, 3, 1e-9),   # slices
        lambda: mrs.parareal_run(ctx, [0, 4], gp, X, D, 0.0, 3e-5, 3, 1e-6, 3, 3, 1e-9),     # 10 % 3
    ]
    for call in bad:
        with pytest.raises(mrs.MrsError) as e:
            call()
        assert e.value.status == mrs.MRS_EINVAL
    with pytest.raises(mrs.MrsError):
        mrs.rod_step(ctx, [0, 4], gp, X, D, 0.0, -1.0, 1, 0)          # dt < 0
    with pytest.raises(mrs.MrsError):
        mrs.parareal_run(ctx, [0, 4], gp, X, D, 0.0, 1e-3, 3, 1e-4, 4, 3, 1e-9)  # ragged slices


@pytest.mark.parametrize("group_size", [1, 2, 4])
def test_pipelined_parareal_equals_regular(ctx, group_size):
    """Same iteration, different schedule: the pipelined run reaches the regular run's result
    (up to float32 rounding of the pair sums, whose batches are cut differently) in the same
    number of iterations."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(75, 2, 24, box=1.5)
    cfg = dict(W.WAVE, a=(2e-3,) * 3, b=(0.3,) * 3)
    gp, _ = params(cfg, rs.eps)
    Ns, dt, r = 8, 5e-5, 4
    T1 = Ns * 16 * dt
    res = {}
    for gs in (0, group_size):
        Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
        st = mrs.parareal_run(ctx, rs.rod_off, gp, Xd, Dd, 0.0, T1, Ns, dt, r, Ns, 1e-10,
                              group_size=gs)
        res[gs] = (Xd.cpu().numpy(), Dd.cpu().numpy(), st)
    (Xa, Da, sa), (Xb, Db, sb) = res[0], res[group_size]
    assert rel(Xb - rs.X, Xa - rs.X) < 1e-5
    assert np.abs(np.einsum("kir,kjr->kij", Db, Db) - np.eye(3)).max() < 1e-12
    assert abs(sa.iterations - sb.iterations) <= 1
    assert abs(sa.incr[0] - sb.incr[0]) <= 1e-3 * sa.incr[0]


def test_rod_forces_with_lj_match_oracle(ctx, orc):
    """Two rods crossing within the Lennard-Jones cut-off: g = elastic + LJ force (Section IV-A)."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    M = 40
    X1, D1 = W.sinusoid_filament(M)
    X2, D2 = W.sinusoid_filament(M)
    Q = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])   # rod 2 rotated and shifted
    X2 = X2 @ Q.T + np.array([0.5, 0.0, 0.004])
    D2 = np.einsum("rc,kic->kir", Q, D2)
    X = np.concatenate([X1, X2])
    D = np.concatenate([D1, D2])
    off = np.array([0, M, 2 * M], np.int64)
    eps = 1.5 / (M - 1)
    cfg = dict(W.ROD_PLAIN)
    gp = mrs.RodParams.make(cfg["L"], cfg["a"], cfg["b"], cfg["wave_A"], cfg["wave_k"],
                            cfg["wave_f"], 1.0, eps, lj_eps=0.05)
    op = orc.RodParams.make(cfg["L"], cfg["a"], cfg["b"], cfg["wave_A"], cfg["wave_k"], cfg["wave_f"])
    Xd, Dd = torch.from_numpy(X).cuda(), torch.from_numpy(D).cuda()
    g = torch.empty_like(Xd)
    m = torch.empty_like(Xd)
    mrs.rod_forces(ctx, off, gp, Xd, Dd, 0.2, g, m)
    torch.cuda.synchronize()
    go, mo = orc.rod_forces(off, X, D, op, 0.2)
    rid = np.repeat([0, 1], M)
    lj = orc.lj_forces(X, rid, 3.0 * eps, 0.05)     # the library's default sigma = 3 eps
    assert np.abs(lj).max() > 1e-3 * np.abs(go).max()       # the rods do touch
    ref = go + lj
    assert np.abs(g.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(m.cpu().numpy() - mo).max() <= 1e-11 * np.abs(mo).max()


def test_rod_advance_matches_oracle(ctx, orc):
    """Eqs. newx/newD with given velocities, float32 and float64 velocity inputs."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(76, 3, 50)
    rng = np.random.default_rng(76)
    u = rng.standard_normal(rs.X.shape)
    w = rng.standard_normal(rs.X.shape) * 30.0
    w[5] = 0.0
    dt = 1e-3
    for dtype in (torch.float32, torch.float64):
        uu = torch.from_numpy(u).to(dtype).cuda()
        ww = torch.from_numpy(w).to(dtype).cuda()
        Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
        mrs.rod_advance(ctx, Xd, Dd, uu, ww, dt)
        torch.cuda.synchronize()
        ug = uu.double().cpu().numpy()
        wg = ww.double().cpu().numpy()
        np.testing.assert_allclose(Xd.cpu().numpy(), rs.X + ug * dt, rtol=0, atol=1e-15)
        np.testing.assert_allclose(Dd.cpu().numpy(), orc.rodrigues_update(rs.D, wg, dt), rtol=0, atol=1e-14)


def test_checkpoint_resume_is_exact(ctx, tmp_path):
    """Stepping 30 steps, or 12 steps + checkpoint + restore into fresh buffers + 18 steps, gives
    bit-identical states; corrupted or mismatched checkpoints are rejected."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(77, 2, 48, box=2.0)
    cfg = dict(W.ROD_PLAIN)
    gp, _ = params(cfg, rs.eps)
    dt = 1e-6
    Xa, Da = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    mrs.rod_step(ctx, rs.rod_off, gp, Xa, Da, 0.0, dt, 30, mrs.MRS_RK2)
    Xb, Db = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    mrs.rod_step(ctx, rs.rod_off, gp, Xb, Db, 0.0, dt, 12, mrs.MRS_RK2)
    path = str(tmp_path / "rods.ckpt")
    mrs.rod_checkpoint_save(path, rs.rod_off, Xb, Db, 12 * dt)
    Xc, Dc = torch.zeros_like(Xb), torch.zeros_like(Db)
    t = mrs.rod_checkpoint_load(path, rs.rod_off, Xc, Dc)
    assert t == 12 * dt
    mrs.rod_step(ctx, rs.rod_off, gp, Xc, Dc, t, dt, 18, mrs.MRS_RK2)
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xc) and torch.equal(Da, Dc)
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(mrs.MrsError):
        mrs.rod_checkpoint_load(bad, rs.rod_off, Xc, Dc)
    with pytest.raises(mrs.MrsError):
        mrs.rod_checkpoint_load(path, [0, 48], Xc[:48], Dc[:48])


def test_parareal_reports_non_convergence(ctx):
    """Too few iterations for the tolerance, and an unstable coarse step, both give MRS_ENOCONV
    (the state then holds the last iterate)."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(78, 2, 24, box=1.5)
    cfg = dict(W.WAVE, a=(2e-3,) * 3, b=(0.3,) * 3)
    gp, _ = params(cfg, rs.eps)
    Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    with pytest.raises(mrs.MrsError) as e:
        mrs.parareal_run(ctx, rs.rod_off, gp, Xd, Dd, 0.0, 8 * 16 * 5e-5, 8, 5e-5, 4, 1, 1e-30)
    assert e.value.status == mrs.MRS_ENOCONV
    stiff = dict(W.WAVE, a=(5.0,) * 3, b=(500.0,) * 3)
    gs, _ = params(stiff, rs.eps)
    Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    st = mrs.parareal_run(ctx, rs.rod_off, gs, Xd, Dd, 0.0, 4 * 64 * 1e-4, 4, 1e-4, 64, 4, 1e-10,
                          raise_on_noconv=False)
    assert not (st.final_incr < 1e-10)


@pytest.mark.parametrize("scheme", [0, 1])
def test_fused_and_graph_stepping_agree(ctx, orc, scheme):
    """The fused path (one launch per call, state in shared memory; the default for small
    instances in large batches) and the per-step kernel graphs compute the same steps: 200 steps of the
    128-node rod and of four interacting 64-node rods agree to float32 rounding of the pair
    sum, and both match the oracle."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    cases = [(W.rod_system(1, 1, 128), dict(W.ROD_PLAIN), 0.0, W.ROD_PLAIN["dt"]),
             (W.rod_system(73, 4, 64, box=2.0), dict(W.ROD_PLAIN, a=(2e-3,) * 3, b=(20.0,) * 3),
              0.1, 2e-6)]
    for rs, cfg, t0, dt in cases:
        gp, op = params(cfg, rs.eps)
        out = []
        try:
            for mode in (2, 0):       # fused (one launch per call), per-step graphs
                ctx.set_fused_steps(mode)
                Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
                mrs.rod_step(ctx, rs.rod_off, gp, Xd, Dd, t0, dt, 200, scheme)
                torch.cuda.synchronize()
                out.append((Xd.cpu().numpy(), Dd.cpu().numpy()))
        finally:
            ctx.set_fused_steps(1)
        Xo, _ = orc.rod_step(rs.rod_off, rs.X, rs.D, op, rs.eps, 1.0, t0, dt, 200, scheme)
        Xg, Dg = out[1]
        for Xf, Df in out[:1]:
            assert rel(Xf - rs.X, Xg - rs.X) < 1e-5
            assert rel(Df - rs.D, Dg - rs.D) < 1e-4
            assert rel(Xf - rs.X, Xo - rs.X) < 1e-4


@pytest.mark.parametrize("n_rods,M", [(1, 2), (1, 16), (1, 31), (2, 10), (1, 33)])
def test_fused_stepping_short_instances(ctx, orc, n_rods, M):
    """Instances of fewer than 32 nodes (and one just above) take the fused path's split pair
    sum, whose split point is rounded to whole 32-source chunks: the first half of the CTA must
    then cover every source and read nothing past the instance.  Fused, graph and oracle
    stepping agree over 50 Euler and 50 RK2 steps."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(90 + M, n_rods, M, box=2.0)
    cfg = dict(W.ROD_PLAIN)
    gp, op = params(cfg, rs.eps)
    for scheme in (mrs.MRS_EULER, mrs.MRS_RK2):
        out = []
        try:
            for mode in (2, 0):
                ctx.set_fused_steps(mode)
                Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
                mrs.rod_step(ctx, rs.rod_off, gp, Xd, Dd, 0.0, cfg["dt"], 50, scheme)
                torch.cuda.synchronize()
                out.append(Xd.cpu().numpy())
        finally:
            ctx.set_fused_steps(1)
        Xo, _ = orc.rod_step(rs.rod_off, rs.X, rs.D, op, rs.eps, 1.0, 0.0, cfg["dt"], 50, scheme)
        assert np.isfinite(out[0]).all()
        assert rel(out[0] - rs.X, out[1] - rs.X) < 1e-5
        assert rel(out[0] - rs.X, Xo - rs.X) < 1e-4


def test_parareal_fused_and_graph_fine_solves_agree(ctx):
    """Parareal whose fine and coarse solves run fused (one launch per solve, one CTA per
    slice) reaches the same state as with the per-step kernel graphs."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(74, 2, 24, box=1.5)
    cfg = dict(W.WAVE, a=(2e-3,) * 3, b=(0.3,) * 3)
    gp, _ = params(cfg, rs.eps)
    Ns, dt, r = 6, 5e-5, 4
    T1 = Ns * 16 * dt
    res = []
    try:
        for mode in (2, 0):
            ctx.set_fused_steps(mode)
            Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
            st = mrs.parareal_run(ctx, rs.rod_off, gp, Xd, Dd, 0.0, T1, Ns, dt, r, Ns, 1e-10)
            res.append((Xd.cpu().numpy(), st.iterations))
    finally:
        ctx.set_fused_steps(1)
    assert rel(res[0][0] - rs.X, res[1][0] - rs.X) < 1e-5
    assert abs(res[0][1] - res[1][1]) <= 1


def test_fused_and_graph_stepping_agree_with_lj(ctx):
    """Two parallel rods 0.12 apart, inside the Lennard-Jones cut-off 2^(1/6) sigma = 0.129,
    60 RK2 steps: the fused path (the repulsion evaluated inside the one-launch solve) and the
    kernel graphs (rod_lj_kernel, pinned to the oracle by test_rod_forces_with_lj_match_oracle)
    reach the same state, and the repulsion changes the motion."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    M = 40
    X1, D1 = W.sinusoid_filament(M)
    X = np.concatenate([X1, X1 + np.array([0.0, 0.0, 0.12])])
    D = np.concatenate([D1, D1])
    off = np.array([0, M, 2 * M], np.int64)
    eps = 1.5 / (M - 1)                                     # sigma = 3 eps = 0.115
    cfg = dict(W.ROD_PLAIN, a=(2e-3,) * 3, b=(20.0,) * 3)
    out = {}
    try:
        for lj in (0.0, 0.05):
            gp = mrs.RodParams.make(cfg["L"], cfg["a"], cfg["b"], cfg["wave_A"], cfg["wave_k"],
                                    cfg["wave_f"], 1.0, eps, lj_eps=lj)
            for fused in (2, 0):
                ctx.set_fused_steps(fused)
                Xd, Dd = torch.from_numpy(X.copy()).cuda(), torch.from_numpy(D.copy()).cuda()
                mrs.rod_step(ctx, off, gp, Xd, Dd, 0.0, 2e-6, 60, mrs.MRS_RK2)
                torch.cuda.synchronize()
                out[(lj, fused)] = Xd.cpu().numpy()
    finally:
        ctx.set_fused_steps(1)
    assert np.isfinite(out[(0.05, 2)]).all()
    assert rel(out[(0.05, 2)] - X, out[(0.05, 0)] - X) < 1e-5
    assert rel(out[(0.0, 2)] - X, out[(0.0, 0)] - X) < 1e-5
    assert rel(out[(0.05, 0)] - X, out[(0.0, 0)] - X) > 1e-3      # the repulsion acts


@pytest.mark.parametrize("r", [4, 16])
@pytest.mark.parametrize("group_size", [0, 8])
def test_parareal_full_size_workload(ctx, orc, group_size, r):
    """The Parareal workload at full size and in the launch configuration the benchmark times:
    8 filaments x 512 nodes, 64 slices x 16 fine RK2 steps (dt = 1e-6), coarse Euler r dt
    (r = 4, and 16 as the configuration names), tol 1e-11, regular and pipelined schedules.  Too large for the oracle's Parareal, so:
    converged Parareal equals serial fine stepping on the GPU (a property at any size), the
    increments fall monotonically, and one step of the full system matches the oracle.

    The pair sum sees the float64 state rounded to float32, relative to a reference point c,
    the mean of the middle nodes of the 8 rods; with |X - c| up to ~6 against a node spacing of
    2e-3 that rounding alone moves the oracle's own velocities by 3.5e-5, relative L2 (1.3e-4
    if rounded without c).  So the velocities of one Euler step, u = (X1 - X) / dt, are compared at 1e-5
    with the oracle pair sum on the same rounded positions, and the RK2 step with the exact
    oracle at 1e-4."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(4, 8, 512)
    gp, op = params(dict(W.ROD_PARAREAL), rs.eps)
    dt = W.ROD_PARAREAL["dt"]
    Ns, nf = 64, 16
    T1 = Ns * nf * dt
    fresh = lambda: (torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda())
    # one Euler step (all 4096 points): its velocities against the oracle's on the rounded state
    X1, D1 = fresh()
    mrs.rod_step(ctx, rs.rod_off, gp, X1, D1, 0.0, dt, 1, mrs.MRS_EULER)
    g, m = orc.rod_forces(rs.rod_off, rs.X, rs.D, op, 0.0)
    mid = [rs.rod_off[r] + (rs.rod_off[r + 1] - rs.rod_off[r] - 1) // 2 for r in range(8)]
    c = rs.X[mid].sum(axis=0) * (1.0 / 8)
    Xr = (rs.X - c).astype(np.float32).astype(np.float64)
    ur, _ = orc.mrs_velocity(Xr, g, m, rs.eps, 1.0)
    assert rel((X1.cpu().numpy() - rs.X) / dt, ur) < 1e-5
    # one fine RK2 step against the exact oracle
    X1, D1 = fresh()
    mrs.rod_step(ctx, rs.rod_off, gp, X1, D1, 0.0, dt, 1, mrs.MRS_RK2)
    Xo, _ = orc.rod_step(rs.rod_off, rs.X, rs.D, op, rs.eps, 1.0, 0.0, dt, 1, mrs.MRS_RK2)
    assert rel(X1.cpu().numpy() - rs.X, Xo - rs.X) < 1e-4
    # serial fine stepping over the whole horizon
    Xs, Ds = fresh()
    mrs.rod_step(ctx, rs.rod_off, gp, Xs, Ds, 0.0, dt, Ns * nf, mrs.MRS_RK2)
    disp_s = Xs.cpu().numpy() - rs.X
    Xp, Dp = fresh()
    st = mrs.parareal_run(ctx, rs.rod_off, gp, Xp, Dp, 0.0, T1, Ns, dt, r, 12, 1e-11,
                          group_size=group_size)
    assert st.final_incr < 1e-11 and 2 <= st.iterations <= 12
    inc = [st.incr[i] for i in range(st.iterations)]
    assert all(b < a for a, b in zip(inc, inc[1:])), inc
    assert rel(Xp.cpu().numpy() - rs.X, disp_s) < 1e-5
    # frames stay orthonormal after the corrections
    Dn = Dp.cpu().numpy()
    eye = np.einsum("kij,klj->kil", Dn, Dn)
    assert np.abs(eye - np.eye(3)).max() < 1e-10


def test_ragged_rod_batch(ctx, orc):
    """Unit rods of 2, 3, 5, 127, 128, 129, 255 and 300 nodes in one call (node spacings from 1
    to 1/299, around the fused force kernel's chunks of 127 nodes): rod_forces against the
    oracle, and 30 RK2 steps against the oracle's (949 nodes exceed the fused propagator's
    shared memory, so even mode 2 takes the kernel graphs)."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    sizes = [2, 3, 5, 127, 128, 129, 255, 300]
    rng = np.random.default_rng(86)
    Xs, Ds = [], []
    for M in sizes:
        X, D = W.sinusoid_filament(M)
        Q = np.linalg.qr(rng.standard_normal((3, 3)))[0]
        Q *= np.sign(np.linalg.det(Q))
        Xs.append(X @ Q.T + rng.uniform(0.0, 2.0, 3))
        Ds.append(np.einsum("rc,kic->kir", Q, D))
    X = np.concatenate(Xs)
    D = np.concatenate(Ds)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eps = 1.5 / 299.0
    cfg = dict(W.ROD_PLAIN, a=(2e-3,) * 3, b=(20.0,) * 3)
    gp, op = params(cfg, eps)
    Xd, Dd = torch.from_numpy(X).cuda(), torch.from_numpy(D).cuda()
    g, m = torch.empty_like(Xd), torch.empty_like(Xd)
    mrs.rod_forces(ctx, off, gp, Xd, Dd, 0.3, g, m)
    go, mo = orc.rod_forces(off, X, D, op, 0.3)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-11 * np.abs(go).max()
    assert np.abs(m.cpu().numpy() - mo).max() <= 1e-11 * np.abs(mo).max()
    dt = 2e-7                               # resolves the stiffest mode of the 300-node rod
    Xo, _ = orc.rod_step(off, X, D, op, eps, 1.0, 0.0, dt, 30, mrs.MRS_RK2)
    try:
        for fused in (2, 0):
            ctx.set_fused_steps(fused)
            Xs_, Ds_ = torch.from_numpy(X.copy()).cuda(), torch.from_numpy(D.copy()).cuda()
            mrs.rod_step(ctx, off, gp, Xs_, Ds_, 0.0, dt, 30, mrs.MRS_RK2)
            torch.cuda.synchronize()
            assert rel(Xs_.cpu().numpy() - X, Xo - X) < 1e-4, fused
    finally:
        ctx.set_fused_steps(1)


def test_rod_far_from_the_origin(ctx, orc):
    """The plain 128-node rod moved to (1000, -500, 250): packing float32 positions relative to
    the rod's middle node keeps the pair sum as accurate as at the origin (rounded as they
    are, positions near 1000 would move near-neighbour separations by 1000 2^-24 / ds ~ 8e-3
    relative).  200 RK2 steps on both stepping paths against the oracle, and against the same
    rod stepped at the origin."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(1, 1, 128)
    shift = np.array([1000.0, -500.0, 250.0])
    gp, op = params(dict(W.ROD_PLAIN), rs.eps)
    dt = W.ROD_PLAIN["dt"]
    Xo, _ = orc.rod_step(rs.rod_off, rs.X + shift, rs.D, op, rs.eps, 1.0, 0.0, dt, 200, mrs.MRS_RK2)
    disp_o = Xo - (rs.X + shift)
    try:
        for fused in (2, 0):
            ctx.set_fused_steps(fused)
            out = []
            for sh in (shift, np.zeros(3)):
                Xd = torch.from_numpy(rs.X + sh).cuda()
                Dd = torch.from_numpy(rs.D.copy()).cuda()
                mrs.rod_step(ctx, rs.rod_off, gp, Xd, Dd, 0.0, dt, 200, mrs.MRS_RK2)
                torch.cuda.synchronize()
                out.append(Xd.cpu().numpy() - (rs.X + sh))
            assert rel(out[0], disp_o) < 1e-4, fused
            assert rel(out[0], out[1]) < 1e-5, fused
    finally:
        ctx.set_fused_steps(1)
