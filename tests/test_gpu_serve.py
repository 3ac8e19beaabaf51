"""Serving (continuous batching) on the GPU: every job's result is the same alone and in the
mix, within the float32 tolerance; admission respects slots and the memory pool; results match
the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_12083_gb300 import build as B, mrs
    B.build()
    c = mrs.Context(0)
    yield c
    c.close()


def velocity_job(seed, n_fil, M=256):
    from paper_2604_12083_gb300 import workloads as W
    return W.single_system(seed=seed, n_fil=n_fil, M=M, box=4.0)


def rod_job(seed, n_rods, M=64):
    from paper_2604_12083_gb300 import workloads as W
    return W.rod_system(seed, n_rods, M, box=3.0)


def rod_params(eps):
    from paper_2604_12083_gb300 import mrs, workloads as W
    c = dict(W.ROD_PLAIN, a=(2e-3,) * 3, b=(20.0,) * 3)
    return mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"], 1.0, eps)


def run_velocity(srv, p):
    X, f, n = (torch.from_numpy(a).cuda() for a in (p.X, p.f, p.n))
    u = torch.full_like(X, float("nan"))
    w = torch.full_like(X, float("nan"))
    t = srv.submit_velocity(X, f, n, u, w, p.mu, float(p.eps[0]))
    return t, (X, f, n, u, w)


def run_rod(srv, rs, nsteps=12, scheme=1):
    X = torch.from_numpy(rs.X.copy()).cuda()
    D = torch.from_numpy(rs.D.copy()).cuda()
    t = srv.submit_rod(rs.rod_off, X, D, rod_params(rs.eps), 0.0, 2e-6, nsteps, scheme, 1.0, rs.eps)
    return t, (X, D)


def test_results_same_alone_and_in_mix(ctx):
    from paper_2604_12083_gb300 import mrs
    import oracle
    oracle.build()
    srv = mrs.Server(ctx, 1 << 30, 64)
    try:
        pv = velocity_job(90, 5)             # 1280 points
        pr = rod_job(91, 3)                  # 3 rods x 64 nodes
        # alone
        tv, bv = run_velocity(srv, pv)
        srv.drain()
        it0 = srv.stats()["iterations"]
        tr, br = run_rod(srv, pr)
        srv.drain()
        # alone, the rod job's 24 RK2 stages run several per iteration (at most 16 each: the
        # server's cap), not one iteration per stage
        assert 2 <= srv.stats()["iterations"] - it0 <= 3
        u_alone, w_alone = bv[3].cpu().numpy(), bv[4].cpu().numpy()
        X_alone = br[0].cpu().numpy()
        assert srv.poll(tv)[0] and srv.poll(tr)[0]
        # in a mix of 24 other jobs of different sizes, all inputs prepared first and then
        # submitted in one burst so that they are on the GPU together
        vjobs = [velocity_job(100 + i, 1 + (i % 7)) for i in range(12)]
        rjobs = [rod_job(200 + i, 1 + (i % 3)) for i in range(12)]
        torch.cuda.synchronize()
        others = []
        for i in range(12):
            others.append(run_velocity(srv, vjobs[i])[1])
            # long enough (40+ steps) to be still running when the measured jobs join
            others.append(run_rod(srv, rjobs[i], nsteps=40 + i % 5)[1])
        tv2, bv2 = run_velocity(srv, pv)
        tr2, br2 = run_rod(srv, pr)
        srv.drain()
        st = srv.stats()
        assert st["peak_active"] >= 6
        # with 1 GiB the scratch holds these iterations' partials: the batched launches ran
        # the symmetric kernel (each unordered pair once)
        assert st["symmetric_iterations"] >= 1
        assert rel(bv2[3].cpu().numpy(), u_alone) < TOL32 and rel(bv2[4].cpu().numpy(), w_alone) < TOL32
        assert rel(br2[0].cpu().numpy() - pr.X, X_alone - pr.X) < 1e-4
        # and the velocity job matches the FP64 oracle
        ur, wr = oracle.mrs_velocity(pv.X, pv.f, pv.n, pv.eps[0], pv.mu)
        assert rel(u_alone, ur) < TOL32 and rel(w_alone, wr) < TOL32
        # the rod job matches the oracle's RK2 integration
        op = oracle.RodParams.make(1.0, [2e-3] * 3, [20.0] * 3, 0.05, 2 * np.pi, 2 * np.pi)
        Xo, _ = oracle.rod_step(pr.rod_off, pr.X, pr.D, op, pr.eps, 1.0, 0.0, 2e-6, 12, oracle.RK2)
        assert rel(X_alone - pr.X, Xo - pr.X) < 1e-4
        for b in others:
            assert all(torch.isfinite(x).all() for x in b[:2])
        lat = [srv.poll(t)[1] for t in (tv2, tr2)]
        assert all(l is not None and l > 0 for l in lat)
    finally:
        srv.close()


def test_admission_by_pool_budget(ctx):
    """A pool that holds only a few jobs at once: every job still completes, never more
    admitted than fit.  Its symmetric scratch (3 % of 4 MiB) is too small for these jobs'
    partial sums, so every batched launch takes the ordered kernel; results match the oracle."""
    from paper_2604_12083_gb300 import mrs
    import oracle
    oracle.build()
    srv = mrs.Server(ctx, 4 << 20, 64)    # 4 MiB: ~18k point slots
    try:
        bufs = []
        tickets = []
        jobs = [velocity_job(300 + i, 16) for i in range(16)]   # 4096 points each
        for i in range(16):
            t, b = run_velocity(srv, jobs[i])
            tickets.append(t)
            bufs.append(b)
        srv.drain()
        st = srv.stats()
        assert st["completed"] == 16
        assert st["peak_active"] <= 5
        assert st["peak_pool_bytes"] <= 4 << 20
        assert st["symmetric_iterations"] == 0
        for b in bufs:
            assert torch.isfinite(b[3]).all() and torch.isfinite(b[4]).all()
        p = jobs[3]
        ur, wr = oracle.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
        assert rel(bufs[3][3].cpu().numpy(), ur) < TOL32 and rel(bufs[3][4].cpu().numpy(), wr) < TOL32
    finally:
        srv.close()


def test_invalid_and_oversize_jobs(ctx):
    from paper_2604_12083_gb300 import mrs
    srv = mrs.Server(ctx, 2 << 20, 4)
    try:
        p = velocity_job(400, 64)       # 16384 points: more than a 2 MiB pool holds
        with pytest.raises(mrs.MrsError) as e:
            run_velocity(srv, p)
        assert e.value.status == mrs.MRS_EBUSY
        X = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
        D = torch.zeros((4, 3, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(mrs.MrsError) as e:
            srv.submit_rod([0, 1, 4], X, D, rod_params(0.01), 0.0, 1e-6, 2, 0, 1.0, 0.01)
        assert e.value.status == mrs.MRS_EINVAL
    finally:
        srv.close()


def test_cancel_waiting_job(ctx):
    """With one slot, a second job waits behind a long rod job and can be cancelled; a running
    job cannot; the cancelled job's outputs are never written."""
    from paper_2604_12083_gb300 import mrs
    srv = mrs.Server(ctx, 1 << 28, 1)
    try:
        pw = velocity_job(501, 4)
        t_long, _ = run_rod(srv, rod_job(500, 4, M=256), nsteps=1500, scheme=0)
        # the scheduler thread admits the long job asynchronously: wait until it has run an
        # iteration (1500 Euler steps take far longer than this wait)
        import time
        t0 = time.time()
        while srv.stats()["iterations"] < 1 and time.time() - t0 < 10.0:
            time.sleep(1e-4)
        assert srv.stats()["iterations"] >= 1
        t_wait, bw = run_velocity(srv, pw)
        srv.cancel(t_wait)
        with pytest.raises(mrs.MrsError) as e:
            srv.cancel(t_long)
        assert e.value.status in (mrs.MRS_EBUSY, mrs.MRS_EINVAL)
        srv.drain()
        with pytest.raises(mrs.MrsError) as e:
            srv.poll(t_wait)
        assert e.value.status == mrs.MRS_ECANCELED
        assert torch.isnan(bw[3]).all()          # never written
        assert srv.poll(t_long)[0]
    finally:
        srv.close()


def test_served_rod_job_with_lennard_jones(ctx):
    """A served rod job with the Lennard-Jones repulsion (two parallel rods 0.12 apart, inside
    the cut-off) reaches the state rod_step reaches (the fused one-launch solve and the per-step
    kernel graphs), and the repulsion changes its motion."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    M = 40
    X1, D1 = W.sinusoid_filament(M)
    X = np.concatenate([X1, X1 + np.array([0.0, 0.0, 0.12])])
    D = np.concatenate([D1, D1])
    off = np.array([0, M, 2 * M], np.int64)
    eps = 1.5 / (M - 1)
    c = dict(W.ROD_PLAIN, a=(2e-3,) * 3, b=(20.0,) * 3)
    out = {}
    for lj in (0.0, 0.05):
        prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"],
                                 1.0, eps, lj_eps=lj)
        srv = mrs.Server(ctx, 1 << 28, 8)
        try:
            Xs, Ds = torch.from_numpy(X.copy()).cuda(), torch.from_numpy(D.copy()).cuda()
            t = srv.submit_rod(off, Xs, Ds, prm, 0.0, 2e-6, 60, mrs.MRS_RK2, 1.0, eps)
            srv.drain()
            assert srv.poll(t)[0]
            out[(lj, "serve")] = Xs.cpu().numpy()
        finally:
            srv.close()
        try:
            for fused in (2, 0):
                ctx.set_fused_steps(fused)
                Xd, Dd = torch.from_numpy(X.copy()).cuda(), torch.from_numpy(D.copy()).cuda()
                mrs.rod_step(ctx, off, prm, Xd, Dd, 0.0, 2e-6, 60, mrs.MRS_RK2)
                torch.cuda.synchronize()
                out[(lj, fused)] = Xd.cpu().numpy()
        finally:
            ctx.set_fused_steps(1)
    for lj in (0.0, 0.05):
        ref = out[(lj, 0)] - X
        assert rel(out[(lj, "serve")] - X, ref) < 1e-5
        assert rel(out[(lj, 2)] - X, ref) < 1e-5
    assert rel(out[(0.05, "serve")] - X, out[(0.0, "serve")] - X) > 1e-3


def test_full_size_serving_mix(ctx):
    """The serving workload at full size: the first 10 ms of the nominal Poisson trace (2000
    jobs/s, 70 % single pair sums, 30 % 100-step Euler rod integrations, N log-uniform in
    [1k, 64k], filaments of 256 nodes in a 10^3 box), all submitted before the server drains
    them together.  Velocity jobs match the oracle on 128 sampled targets each; rod jobs equal
    rod_step run alone, and the smallest one matches the oracle's 100 steps."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    import oracle
    oracle.build()
    c = W.ROD_SERVE
    trace = W.serve_trace(seed=5, rate_hz=2000.0, window_s=0.01)
    assert len(trace) >= 10 and max(N for _, _, N in trace) > 16384
    rng = np.random.default_rng(5)
    jobs = []
    for (_, kind, N) in trace:
        X, D = W.place_filaments(rng, N // 256, 256, box=10.0)
        eps = float(np.float32(W.EPS_OVER_DS / 255))
        if kind == 0:
            f = rng.standard_normal((N, 3)).astype(np.float32)
            n = rng.standard_normal((N, 3)).astype(np.float32)
            jobs.append((kind, N, eps, (X.astype(np.float32), f, n)))
        else:
            jobs.append((kind, N, eps, (X, D, np.arange(0, N + 1, 256, dtype=np.int64))))
    srv = mrs.Server(ctx, 32 << 30, 256)
    bufs = []
    try:
        for kind, N, eps, h in jobs:
            if kind == 0:
                b = [torch.from_numpy(a).cuda() for a in h]
                b += [torch.full_like(b[0], float("nan")), torch.full_like(b[0], float("nan"))]
                t = srv.submit_velocity(b[0], b[1], b[2], b[3], b[4], 1.0, eps)
            else:
                b = [torch.from_numpy(h[0].copy()).cuda(), torch.from_numpy(h[1].copy()).cuda()]
                prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"],
                                         c["wave_f"], 1.0, eps)
                t = srv.submit_rod(h[2], b[0], b[1], prm, 0.0, c["dt"], 100, mrs.MRS_EULER, 1.0, eps)
            bufs.append((t, b))
        srv.drain(600.0)
        assert srv.stats()["symmetric_iterations"] >= 1
        assert all(srv.poll(t)[0] for t, _ in bufs)
    finally:
        srv.close()
    smallest_rod = min((j for j in range(len(jobs)) if jobs[j][0] == 1), key=lambda j: jobs[j][1])
    for j, ((kind, N, eps, h), (_, b)) in enumerate(zip(jobs, bufs)):
        if kind == 0:
            idx = np.random.default_rng(j).choice(N, 128, replace=False)
            ur, wr = oracle.mrs_velocity(h[0], h[1], h[2], eps, 1.0, xt=h[0][idx])
            assert rel(b[3].cpu().numpy()[idx], ur) < TOL32 and rel(b[4].cpu().numpy()[idx], wr) < TOL32, (j, N)
        else:
            prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"],
                                     1.0, eps)
            Xa, Da = torch.from_numpy(h[0].copy()).cuda(), torch.from_numpy(h[1].copy()).cuda()
            mrs.rod_step(ctx, h[2], prm, Xa, Da, 0.0, c["dt"], 100, mrs.MRS_EULER)
            torch.cuda.synchronize()
            disp = b[0].cpu().numpy() - h[0]
            assert np.isfinite(disp).all()
            assert rel(disp, Xa.cpu().numpy() - h[0]) < 1e-5, (j, N)
            if j == smallest_rod:
                op = oracle.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"])
                Xo, _ = oracle.rod_step(h[2], h[0], h[1], op, eps, 1.0, 0.0, c["dt"], 100, oracle.EULER)
                assert rel(disp, Xo - h[0]) < 1e-4, (j, N)


def test_big_jobs_in_order_small_jobs_alongside(ctx):
    """serve_set_policy: with a threshold that makes two long rod jobs "big", the second one
    advances only after the first has finished (admission order, as one request per launch
    would run them), velocity jobs submitted after both still finish before the first big one
    (small jobs never wait behind a big one), and every result equals the job run alone."""
    from paper_2604_12083_gb300 import mrs
    srv = mrs.Server(ctx, 1 << 30, 64)
    try:
        srv.set_policy(big_job_pairs=1e7, max_big_jobs=1)
        ra, rb = rod_job(301, 4), rod_job(302, 4)          # 256 nodes, 300 RK2 steps: 3.9e7 pairs
        vs = [velocity_job(303 + i, 5) for i in range(3)]   # 1280 points: 1.6e6 pairs
        alone = []
        for rs in (ra, rb):
            t, b = run_rod(srv, rs, nsteps=300)
            srv.drain()
            alone.append(b[0].cpu().numpy())
        v_alone = []
        for p in vs:
            t, b = run_velocity(srv, p)
            srv.drain()
            v_alone.append((b[3].cpu().numpy(), b[4].cpu().numpy()))
        torch.cuda.synchronize()
        ta, ba = run_rod(srv, ra, nsteps=300)
        tb, bb = run_rod(srv, rb, nsteps=300)
        tv = [run_velocity(srv, p) for p in vs]
        srv.drain()
        lat = {t: srv.poll(t)[1] for t in [ta, tb] + [t for t, _ in tv]}
        # completion times relative to the first submission (submissions are microseconds apart)
        done_a, done_b = lat[ta], lat[tb]
        assert done_b - done_a > 0.5 * done_a, (done_a, done_b)      # b waited for a
        assert all(lat[t] < done_a for t, _ in tv), (lat, done_a)
        assert rel(ba[0].cpu().numpy() - ra.X, alone[0] - ra.X) < 1e-4
        assert rel(bb[0].cpu().numpy() - rb.X, alone[1] - rb.X) < 1e-4
        for (t, b), (u0, w0) in zip(tv, v_alone):
            assert rel(b[3].cpu().numpy(), u0) < TOL32 and rel(b[4].cpu().numpy(), w0) < TOL32
        # every job small again: both rod jobs advance together and finish close together
        srv.set_policy(big_job_pairs=0.0)
        ta, ba = run_rod(srv, ra, nsteps=300)
        tb, bb = run_rod(srv, rb, nsteps=300)
        srv.drain()
        la, lb = srv.poll(ta)[1], srv.poll(tb)[1]
        assert abs(lb - la) < 0.5 * la, (la, lb)
        with pytest.raises(mrs.MrsError):
            srv.set_policy(1e9, 0)
    finally:
        srv.close()


def test_injected_allocation_failure(ctx):
    """A job whose admission fails (allocation failure injected on the host) finishes with
    MRS_ENOMEM, its buffers untouched; the jobs before and after it complete and match the
    oracle."""
    from paper_2604_12083_gb300 import mrs
    import oracle
    oracle.build()
    srv = mrs.Server(ctx, 1 << 30, 1)     # one slot: the velocity jobs wait for the rod job
    try:
        rs = rod_job(310, 4)
        ta, ba = run_rod(srv, rs, nsteps=600)              # ~1200 stages: tens of ms
        vs = [velocity_job(311 + i, 3) for i in range(3)]
        tv = [run_velocity(srv, p) for p in vs]
        srv.inject_alloc_failure(tv[1][0])
        srv.drain()
        with pytest.raises(mrs.MrsError) as e:
            srv.poll(tv[1][0])
        assert e.value.status == mrs.MRS_ENOMEM and "allocation" in str(e.value)
        assert torch.isnan(tv[1][1][3]).all() and torch.isnan(tv[1][1][4]).all()
        for i in (0, 2):
            p, b = vs[i], tv[i][1]
            assert srv.poll(tv[i][0])[0]
            ur, wr = oracle.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
            assert rel(b[3].cpu().numpy(), ur) < TOL32 and rel(b[4].cpu().numpy(), wr) < TOL32
        assert srv.poll(ta)[0] and torch.isfinite(ba[0]).all()
        # a job that is no longer waiting cannot be failed
        with pytest.raises(mrs.MrsError) as e:
            srv.inject_alloc_failure(ta)
        assert e.value.status == mrs.MRS_EBUSY
    finally:
        srv.close()
