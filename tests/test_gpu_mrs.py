"""GPU parity of the pair sum (mrs_velocity / plans) against the FP64 CPU oracle.

Bar (per velocity field, over the compared targets): relative L2 error <= 1e-5 for the float32
paths, <= 1e-12 for the float64 path.  Inputs are float32-representable (see
paper_2604_12083_gb300.workloads), so both sides see identical positions, forces and torques.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def run(ctx, p, precision, config=None, Xt=None):
    from paper_2604_12083_gb300 import mrs
    dt = torch.float64 if precision == mrs.MRS_F64 else torch.float32
    X, f, n = dev(p.X, dt), dev(p.f, dt), dev(p.n, dt)
    xt = None if Xt is None else dev(Xt, dt)
    u = torch.full_like(X, float("nan"))
    w = torch.full_like(X, float("nan"))
    if config is None:
        mrs.mrs_velocity(ctx, p.offsets, X, f, n, u, w, p.mu, 0.0, eps_per_sys=p.eps,
                         precision=precision, Xt=xt)
    else:
        pl = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=precision,
                      config=config)
        pl.execute(X, f, n, u, w, Xt=xt)
        torch.cuda.synchronize()
        pl.close()
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64), w.cpu().numpy().astype(np.float64)


def test_plain_rod_float64(ctx, orc):
    """One rod of 128 nodes, one FP64 call (the plain-method configuration)."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.plain_rod()
    u, w = run(ctx, p, mrs.MRS_F64)
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
    assert rel_l2(u, ur) < TOL64 and rel_l2(w, wr) < TOL64


@pytest.mark.parametrize("precision", [1, 2])
def test_plain_rod_float32(ctx, orc, precision):
    from paper_2604_12083_gb300 import workloads as W
    p = W.plain_rod()
    u, w = run(ctx, p, precision)
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
    assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32


def ragged_batch():
    """Systems of awkward sizes (empty, 1, around the 32-source unit, around 256/512-target
    tiles, a ragged 4097), placed like the batched workload."""
    from paper_2604_12083_gb300 import workloads as W
    rng = np.random.default_rng(60)
    sizes = [0, 1, 2, 31, 32, 33, 255, 256, 257, 511, 513, 1000, 4097, 0, 3]
    Xs, fs, ns = [], [], []
    for s in sizes:
        X = rng.uniform(0.0, 2.0, (s, 3))
        Xs.append(X)
        fs.append(rng.standard_normal((s, 3)))
        ns.append(rng.standard_normal((s, 3)))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eps = np.array([float(np.float32(0.01 + 0.002 * i)) for i in range(len(sizes))])
    f32 = lambda a: np.concatenate(a).astype(np.float32)
    return W.MRSProblem("ragged", off, f32(Xs), f32(fs), f32(ns), eps, 1.3)


N_CONFIGS = 29          # ordered 0..16, symmetric (pair-reuse) 17..26, ordered cluster 27..28
SYM_CONFIGS = list(range(17, 27))
CLUSTER_CONFIGS = [27, 28]
CLUSTER_TM = {27: 32, 28: 64}   # 256 threads as 32 targets x 8 and 64 x 4 source groups


@pytest.mark.parametrize("config", list(range(N_CONFIGS)))
@pytest.mark.parametrize("precision", [1, 2])
def test_ragged_batch_every_config(ctx, orc, config, precision):
    p = ragged_batch()
    u, w = run(ctx, p, precision, config=config)
    ur, wr = orc.mrs_velocity_batch(p.offsets, p.X, p.f, p.n, 0.0, p.mu, eps_per_sys=p.eps)
    for s in range(len(p.offsets) - 1):
        a, b = p.offsets[s], p.offsets[s + 1]
        if a == b:
            continue
        assert rel_l2(u[a:b], ur[a:b]) < TOL32, (s, b - a)
        assert rel_l2(w[a:b], wr[a:b]) < TOL32, (s, b - a)


@pytest.fixture(scope="module")
def mid_system(orc):
    """One system of 20 filaments x 1000 nodes (20000 points) and its oracle velocities: large
    enough that every persistent CTA of every configuration sweeps several 32-source units and
    several 128-source chunks of a tile row, which the ragged batch's small systems never do."""
    from paper_2604_12083_gb300 import workloads as W
    p = W.single_system(seed=66, n_fil=20, M=1000)
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
    return p, ur, wr


@pytest.mark.parametrize("config", list(range(N_CONFIGS)))
@pytest.mark.parametrize("precision", [1, 2])
def test_mid_system_every_config(ctx, mid_system, config, precision):
    p, ur, wr = mid_system
    u, w = run(ctx, p, precision, config=config)
    assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32
    assert per_target_max(u, ur) < PER_TARGET and per_target_max(w, wr) < PER_TARGET


def test_ragged_batch_float64(ctx, orc):
    from paper_2604_12083_gb300 import mrs
    p = ragged_batch()
    u, w = run(ctx, p, mrs.MRS_F64)
    ur, wr = orc.mrs_velocity_batch(p.offsets, p.X, p.f, p.n, 0.0, p.mu, eps_per_sys=p.eps)
    for s in range(len(p.offsets) - 1):
        a, b = p.offsets[s], p.offsets[s + 1]
        if a < b:
            assert rel_l2(u[a:b], ur[a:b]) < TOL64 and rel_l2(w[a:b], wr[a:b]) < TOL64


def test_separate_targets(ctx, orc):
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.single_system(seed=61, n_fil=3, M=700)
    rng = np.random.default_rng(61)
    Xt = (p.X + rng.normal(0, 0.01, p.X.shape)).astype(np.float32)
    u, w = run(ctx, p, mrs.MRS_F32_COMP, Xt=Xt)
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu, xt=Xt)
    assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32


@pytest.mark.parametrize("config", [None] + SYM_CONFIGS)
def test_multi_tile_single_system(ctx, orc, config):
    """A few thousand points: several tiles, every tile split over many CTAs (fix-up path;
    for the symmetric configurations, rows split over many CTAs and many column partials)."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.single_system(seed=62, n_fil=3, M=1000)      # 3000 points, ragged last tile
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
    for prec in (mrs.MRS_F32, mrs.MRS_F32_COMP):
        u, w = run(ctx, p, prec, config=config)
        assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32


@pytest.mark.parametrize("config", [None, 8, 9, 13, 14])
def test_small_system_split_cap(ctx, orc, config):
    """Single systems of 1024, 2048 and 4113 points (few tiles): where the full grid would give
    each CTA fewer than 4 work units, an ordered plan cuts each tile over at most 16 CTAs (the
    CTA that completes a tile reads at most 16 partial slots); otherwise it keeps the full grid.
    The result matches the oracle either way."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    for M in (1024, 2048, 4113):
        p = W.single_system(seed=M, n_fil=1, M=M)
        pl = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32_COMP,
                      config=-1 if config is None else config)
        info = pl.info()
        pl.close()
        if not mrs.plan_config_symmetric(info["config"]):
            ci = mrs.plan_config_info(ctx, info["config"])
            TM = CLUSTER_TM.get(info["config"], ci["threads"] * ci["targets_per_thread"])
            tiles = -(-M // TM)
            assert info["grid"] >= 1
            assert info["grid"] <= 16 * tiles or info["work_units"] >= 4 * info["grid"], (M, info)
            if M <= 2048:                       # a few units per CTA at most: the cap binds
                assert info["grid"] <= 16 * tiles, (M, info)
        ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
        u, w = run(ctx, p, mrs.MRS_F32_COMP, config=config)
        assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32, M


@pytest.mark.parametrize("config", SYM_CONFIGS)
def test_symmetric_plan_with_targets(ctx, orc, config):
    """A symmetric plan given targets equal to the sources (the same buffer) takes the
    symmetric path; given other targets it takes the ordered path.  Both match the oracle."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.single_system(seed=69, n_fil=2, M=900)
    dt = torch.float32
    X, f, n = dev(p.X, dt), dev(p.f, dt), dev(p.n, dt)
    pl = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32_COMP,
                  config=config)
    assert pl.info()["config"] == config
    u, w = torch.full_like(X, float("nan")), torch.full_like(X, float("nan"))
    pl.execute(X, f, n, u, w, Xt=X)
    torch.cuda.synchronize()
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
    assert rel_l2(u.cpu().numpy(), ur) < TOL32 and rel_l2(w.cpu().numpy(), wr) < TOL32
    rng = np.random.default_rng(69)
    Xt = (p.X + rng.normal(0, 0.01, p.X.shape)).astype(np.float32)
    u2, w2 = torch.full_like(X, float("nan")), torch.full_like(X, float("nan"))
    pl.execute(X, f, n, u2, w2, Xt=dev(Xt, dt))
    torch.cuda.synchronize()
    pl.close()
    ur2, wr2 = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu, xt=Xt)
    assert rel_l2(u2.cpu().numpy(), ur2) < TOL32 and rel_l2(w2.cpu().numpy(), wr2) < TOL32


@pytest.mark.parametrize("config", [None, 17, 25])
def test_deterministic(ctx, config):
    """Bit-identical results on repeated calls: fixed summation orders, no float atomics."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.single_system(seed=63, n_fil=4, M=1024)
    a = run(ctx, p, mrs.MRS_F32_COMP, config=config)
    b = run(ctx, p, mrs.MRS_F32_COMP, config=config)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def per_target_max(a, b):
    """Largest per-target error norm over the field's RMS per-target norm: a bound that a
    localized error (a wrong tile edge touching a few targets) cannot hide under."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.linalg.norm(a - b, axis=1)) / np.sqrt(np.mean(np.sum(b * b, axis=1))))


PER_TARGET = 1e-4


@pytest.mark.parametrize("config", [None, 17])
def test_full_size_single_system_all_targets(ctx, orc, config):
    """32 filaments x 1024 nodes, the benchmark's launch (cached plan, default config; and the
    symmetric configuration): every one of the 32768 targets against all sources, by the
    oracle.  Relative L2 per field <= 1e-5, and every target's error <= 1e-4 of the field's
    RMS."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.single_system()
    u, w = run(ctx, p, mrs.MRS_F32_COMP, config=config)
    assert np.isfinite(u).all() and np.isfinite(w).all()
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
    assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32
    assert per_target_max(u, ur) < PER_TARGET and per_target_max(w, wr) < PER_TARGET


@pytest.mark.parametrize("config", [None, 17])
def test_full_size_batch_sampled(ctx, orc, config):
    """512 systems of 256..16384 points in one persistent launch: per system its first and
    last target (system and tile edges) and 62 sampled ones against all sources of their own
    system; relative L2 over the samples <= 1e-5 and every sampled target within 1e-4 of its
    system's RMS (float32 accumulation without compensation in this configuration)."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.batch_systems()
    u, w = run(ctx, p, mrs.MRS_F32, config=config)
    assert np.isfinite(u).all() and np.isfinite(w).all()
    rng = np.random.default_rng(65)
    eu_n = eu_d = ew_n = ew_d = 0.0
    worst = 0.0
    for s in range(len(p.offsets) - 1):
        a, b = int(p.offsets[s]), int(p.offsets[s + 1])
        idx = np.unique(np.concatenate([[0, b - a - 1], rng.choice(b - a, 62, replace=False)]))
        ur, wr = orc.mrs_velocity(p.X[a:b], p.f[a:b], p.n[a:b], p.eps[s], p.mu, xt=p.X[a:b][idx])
        eu_n += np.sum((u[a:b][idx] - ur) ** 2)
        eu_d += np.sum(ur ** 2)
        ew_n += np.sum((w[a:b][idx] - wr) ** 2)
        ew_d += np.sum(wr ** 2)
        worst = max(worst, per_target_max(u[a:b][idx], ur), per_target_max(w[a:b][idx], wr))
    assert np.sqrt(eu_n / eu_d) < TOL32 and np.sqrt(ew_n / ew_d) < TOL32
    assert worst < PER_TARGET


def test_invalid_arguments_rejected(ctx):
    from paper_2604_12083_gb300 import mrs
    X = torch.zeros((4, 3), device="cuda")
    u = torch.zeros_like(X)
    w = torch.zeros_like(X)
    with pytest.raises(mrs.MrsError) as e:
        mrs.mrs_velocity(ctx, [0, 4], X, X, X, u, w, 1.0, -1.0)
    assert e.value.status == mrs.MRS_EINVAL
    with pytest.raises(mrs.MrsError):
        mrs.mrs_velocity(ctx, [0, 3, 2], X, X, X, u, w, 1.0, 0.1)
    with pytest.raises(mrs.MrsError):
        mrs.mrs_velocity(ctx, [0, 4], X, X, X, u, u, 1.0, 0.1)   # overlapping outputs
    with pytest.raises(mrs.MrsError):
        mrs.mrs_velocity(ctx, [0, 4], X, X, X, u, w, 0.0, 0.1)   # mu = 0
    bad = [
        lambda: mrs.mrs_velocity(ctx, [0, 4], X, X, X, X, w, 1.0, 0.1),         # u aliases X
        lambda: mrs.mrs_velocity(ctx, [0, 4], X, X, X, u, w, 1.0, 0.1, precision=7),
        lambda: mrs.mrs_velocity(ctx, [0, 2, 4], X, X, X, u, w, 1.0, 0.1, eps_per_sys=[0.1, 0.0]),
        lambda: mrs.mrs_velocity(ctx, [1, 4], X, X, X, u, w, 1.0, 0.1),         # offsets[0] != 0
        lambda: mrs.mrs_velocity(ctx, [0, 4], X, X, X, u, w, 1.0, float("nan")),
        lambda: mrs.mrs_velocity(ctx, [0, 4], X, X, X, u, w, float("inf"), 0.1),
    ]
    for call in bad:
        with pytest.raises(mrs.MrsError) as e:
            call()
        assert e.value.status == mrs.MRS_EINVAL
    # a source pointer that is not float-aligned, through the C entry point directly
    import ctypes
    Xb = torch.zeros((8, 3), device="cuda")
    off = np.array([0, 4], np.int64)
    st = mrs.lib().mrs_velocity(ctx.handle, 1, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                ctypes.c_void_p(Xb.data_ptr() + 2), ctypes.c_void_p(X.data_ptr()),
                                ctypes.c_void_p(X.data_ptr()), None, ctypes.c_void_p(u.data_ptr()),
                                ctypes.c_void_p(w.data_ptr()), 1.0, 0.1, None, mrs.MRS_F32_COMP,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == mrs.MRS_EINVAL
    # empty problem: a no-op
    mrs.mrs_velocity(ctx, [0, 0], X, X, X, u, w, 1.0, 0.1)


def test_autotune_picks_a_config_used_by_plans(ctx, orc, tmp_path):
    """The autotuner times every configuration on the batch shape; a default plan built
    afterwards uses the winner, the table round-trips through its JSON file, and the tuned
    plan still matches the oracle."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.batch_systems(seed=66, n_sys=24, lo_exp=8, hi_exp=12)
    best, ms = mrs.autotune(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32,
                            reps=2)
    assert 0 <= best < mrs.plan_config_count() and ms > 0
    pl = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32)
    assert pl.info()["config"] == best
    pl.close()
    path = str(tmp_path / "tune.json")
    mrs.autotune_save(ctx, path)
    c2 = mrs.Context(0)
    mrs.autotune_load(c2, path)
    pl = mrs.Plan(c2, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32)
    assert pl.info()["config"] == best
    pl.close()
    c2.close()
    u, w = run(ctx, p, mrs.MRS_F32)
    ur, wr = orc.mrs_velocity_batch(p.offsets, p.X, p.f, p.n, 0.0, p.mu, eps_per_sys=p.eps)
    assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32


def test_config_table_size(ctx):
    """Every compiled configuration is covered by the ragged-batch parity test above."""
    from paper_2604_12083_gb300 import mrs
    assert mrs.plan_config_count() == N_CONFIGS
    for c in range(N_CONFIGS):
        info = mrs.plan_config_info(ctx, c)
        assert info["ctas_per_sm"] >= 1
        assert mrs.plan_config_symmetric(c) == (c in SYM_CONFIGS)


@pytest.mark.parametrize("config", CLUSTER_CONFIGS)
@pytest.mark.parametrize("shape", [(1, 51), (4, 51), (12, 51), (25, 51), (1, 4099)])
@pytest.mark.parametrize("precision", [1, 2])
def test_cluster_small_systems(ctx, orc, config, shape, precision):
    """The cluster kernel on single systems of the paper's sizes (1, 4, 12, 25 rods of 51
    points) and a ragged 4099-point one: every target against the oracle (field L2 and
    per-target bounds), a second call bit-identical (the cluster sums its CTAs' partials in a
    fixed order), no scratch slots, one cluster of at most 16 CTAs per tile."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    n_fil, M = shape
    p = W.single_system(seed=70 + n_fil, n_fil=n_fil, M=M, box=3.0)
    N = n_fil * M
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
    X, f, n = dev(p.X), dev(p.f), dev(p.n)
    pl = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=precision, config=config)
    outs = []
    for _ in range(2):
        u, w = torch.full_like(X, float("nan")), torch.full_like(X, float("nan"))
        pl.execute(X, f, n, u, w)
        torch.cuda.synchronize()
        outs.append((u.cpu().numpy(), w.cpu().numpy()))
    info = pl.info()
    sc = pl.scratch()
    pl.close()
    (u0, w0), (u1, w1) = outs
    assert np.array_equal(u0, u1) and np.array_equal(w0, w1)
    u, w = u0.astype(np.float64), w0.astype(np.float64)
    assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32, (rel_l2(u, ur), rel_l2(w, wr))
    assert per_target_max(u, ur) < PER_TARGET and per_target_max(w, wr) < PER_TARGET
    TM = CLUSTER_TM[config]
    tiles = -(-N // TM)
    assert info["grid"] % tiles == 0 and 1 <= info["grid"] // tiles <= 16, (info, tiles)
    assert sc["passes"] == 1 and sc["bytes"] == 0


@pytest.mark.parametrize("config", CLUSTER_CONFIGS)
def test_cluster_separate_targets(ctx, orc, config):
    """The cluster kernel with targets apart from the sources (a shifted copy of the points)."""
    from paper_2604_12083_gb300 import workloads as W
    p = W.single_system(seed=75, n_fil=12, M=51, box=3.0)
    Xt = (p.X + np.float32(0.013)).astype(np.float32)
    u, w = run(ctx, p, 2, config=config, Xt=Xt)
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu, xt=Xt)
    assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32
    assert per_target_max(u, ur) < PER_TARGET and per_target_max(w, wr) < PER_TARGET


def test_default_configuration_by_size(ctx):
    """The library's choice for one system, as measured on GB300: the cluster kernel up to
    2560 points (32-target tiles up to 1536), the ordered 256 x 1 kernel up to 8192, the
    symmetric kernel as one wave of CTAs from ~12 work units per resident CTA (12288, 16384)
    and as four waves beyond (32768, the bench system)."""
    from paper_2604_12083_gb300 import mrs
    for N, expect in ((1000, 27), (2048, 28), (4096, 14), (8192, 14), (12288, 23), (16384, 23),
                      (32768, 25)):
        pl = mrs.Plan(ctx, np.array([0, N], np.int64), 1.0, 0.01, precision=mrs.MRS_F32_COMP)
        got = pl.info()["config"]
        pl.close()
        assert got == expect, (N, got, expect)


def test_nonfinite_inputs_raise_the_device_flag(ctx):
    """A NaN force makes non-finite velocities; the context's device flag reports it once."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.single_system(seed=67, n_fil=2, M=600)
    assert ctx.device_status() == 0
    for prec in (mrs.MRS_F32_COMP, mrs.MRS_F64):
        dt = torch.float64 if prec == mrs.MRS_F64 else torch.float32
        X, f, n = (torch.from_numpy(a).to(dt).cuda() for a in (p.X, p.f, p.n))
        u, w = torch.empty_like(X), torch.empty_like(X)
        mrs.mrs_velocity(ctx, p.offsets, X, f, n, u, w, p.mu, float(p.eps[0]), precision=prec)
        assert ctx.device_status() == 0
        f[17, 1] = float("nan")
        mrs.mrs_velocity(ctx, p.offsets, X, f, n, u, w, p.mu, float(p.eps[0]), precision=prec)
        assert ctx.device_status() & mrs.MRS_FLAG_NONFINITE
        assert ctx.device_status() == 0


@pytest.mark.parametrize("config", [-1, 8])
def test_large_ragged_single_system_sampled(ctx, orc, config):
    """2^18 + 17 points (6.9e10 pairs, a ragged last tile): the library's choice -- the
    symmetric kernel, its column partials (2.1 GB in one pass) split into passes so that the
    plan's scratch stays under 256 MB -- and an
    ordered configuration; 256 sampled targets (incl. the last tile) against all sources,
    computed one by one by the oracle."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    rng = np.random.default_rng(68)
    N = (1 << 18) + 17
    X = rng.uniform(0.0, 40.0, (N, 3)).astype(np.float32)
    f = rng.standard_normal((N, 3)).astype(np.float32)
    n = rng.standard_normal((N, 3)).astype(np.float32)
    p = W.MRSProblem("large", np.array([0, N], np.int64), X, f, n, np.array([0.02]), 1.0)
    pl = mrs.Plan(ctx, p.offsets, p.mu, 0.02, precision=mrs.MRS_F32_COMP, config=config)
    sc = pl.scratch()
    if config == -1:
        assert mrs.plan_config_symmetric(pl.info()["config"])
        assert sc["passes"] > 1 and sc["bytes"] <= 256e6, sc
    Xd, fd, nd = dev(p.X), dev(p.f), dev(p.n)
    ud, wd = torch.full_like(Xd, float("nan")), torch.full_like(Xd, float("nan"))
    pl.execute(Xd, fd, nd, ud, wd)
    torch.cuda.synchronize()
    pl.close()
    u, w = ud.double().cpu().numpy(), wd.double().cpu().numpy()
    assert np.isfinite(u).all() and np.isfinite(w).all()
    idx = np.concatenate([rng.choice(N, 250, replace=False), np.arange(N - 6, N)])
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, 0.02, 1.0, xt=p.X[idx])
    assert rel_l2(u[idx], ur) < TOL32 and rel_l2(w[idx], wr) < TOL32
    assert per_target_max(u[idx], ur) < PER_TARGET and per_target_max(w[idx], wr) < PER_TARGET


def run_with_pass_bytes(ctx, p, precision, config, nbytes):
    """Plan built with a column-partial buffer of nbytes per pass; returns (u, w, passes)."""
    from paper_2604_12083_gb300 import mrs
    ctx.set_sym_pass_bytes(nbytes)
    try:
        pl = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=precision,
                      config=config)
    finally:
        ctx.set_sym_pass_bytes(192 << 20)
    X, f, n = dev(p.X), dev(p.f), dev(p.n)
    out = []
    for _ in range(2):
        u, w = torch.full_like(X, float("nan")), torch.full_like(X, float("nan"))
        pl.execute(X, f, n, u, w)
        torch.cuda.synchronize()
        out.append((u.double().cpu().numpy(), w.double().cpu().numpy()))
    npass = pl.scratch()["passes"]
    pl.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    return out[0][0], out[0][1], npass


@pytest.mark.parametrize("config", [17, 20, 25, 26])
@pytest.mark.parametrize("precision", [1, 2])
def test_symmetric_passes_match_oracle(ctx, mid_system, config, precision):
    """A symmetric plan of the 20000-point system split into passes (a 256 KiB column-partial
    buffer: dozens of passes, cut inside the system) gives the oracle's result, as one pass
    does, bit-identically on repeated calls."""
    p, ur, wr = mid_system
    u1, w1, n1 = run_with_pass_bytes(ctx, p, precision, config, 192 << 20)
    u, w, npass = run_with_pass_bytes(ctx, p, precision, config, 256 << 10)
    assert n1 == 1 and npass > 10, (n1, npass)
    assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32
    assert per_target_max(u, ur) < PER_TARGET and per_target_max(w, wr) < PER_TARGET
    assert rel_l2(u, u1) < TOL32 and rel_l2(w, w1) < TOL32


@pytest.mark.parametrize("config", SYM_CONFIGS)
def test_symmetric_passes_ragged_batch(ctx, orc, config):
    """The ragged batch with passes of three work units: passes end inside systems, span
    several small systems and hold single tiles; every system matches the oracle."""
    from paper_2604_12083_gb300 import mrs
    p = ragged_batch()
    u, w, npass = run_with_pass_bytes(ctx, p, mrs.MRS_F32_COMP, config, 3 * 768)
    assert npass >= 10, npass
    ur, wr = orc.mrs_velocity_batch(p.offsets, p.X, p.f, p.n, 0.0, p.mu, eps_per_sys=p.eps)
    for s in range(len(p.offsets) - 1):
        a, b = p.offsets[s], p.offsets[s + 1]
        if a < b:
            assert rel_l2(u[a:b], ur[a:b]) < TOL32, (s, b - a)
            assert rel_l2(w[a:b], wr[a:b]) < TOL32, (s, b - a)


@pytest.mark.parametrize("config", [8, 25, 26])
def test_plan_replays_in_cuda_graph(ctx, orc, config):
    """A plan's execution (one persistent launch, plus the reduction kernel for symmetric
    configurations) captured in a CUDA graph and replayed gives the eager result bit for bit,
    and the oracle's on a ragged batch; replays after the inputs change pick up the new inputs."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.batch_systems(seed=70, n_sys=12, lo_exp=8, hi_exp=13)
    X, f, n = dev(p.X), dev(p.f), dev(p.n)
    pl = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32_COMP,
                  config=config)
    ue, we = torch.empty_like(X), torch.empty_like(X)
    pl.execute(X, f, n, ue, we)
    torch.cuda.synchronize()
    u, w = torch.full_like(X, float("nan")), torch.full_like(X, float("nan"))
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            pl.execute(X, f, n, u, w, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u, ue) and torch.equal(w, we)
    ur, wr = orc.mrs_velocity_batch(p.offsets, p.X, p.f, p.n, 0.0, p.mu, eps_per_sys=p.eps)
    assert rel_l2(u.cpu().numpy(), ur) < TOL32 and rel_l2(w.cpu().numpy(), wr) < TOL32
    f.mul_(-2.0)                      # linear in the forces and torques
    n.mul_(-2.0)
    g.replay()
    torch.cuda.synchronize()
    assert rel_l2(u.cpu().numpy(), -2.0 * ur) < TOL32 and rel_l2(w.cpu().numpy(), -2.0 * wr) < TOL32
    pl.close()


def test_nonfinite_inputs_raise_the_flag_through_the_symmetric_path(ctx):
    """A NaN torque in a symmetric plan's system spreads to every point through the column
    partials; the reduction kernel raises the device flag once."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.single_system(seed=71, n_fil=3, M=700)
    X, f, n = dev(p.X), dev(p.f), dev(p.n)
    u, w = torch.empty_like(X), torch.empty_like(X)
    pl = mrs.Plan(ctx, p.offsets, p.mu, float(p.eps[0]), precision=mrs.MRS_F32_COMP, config=25)
    assert ctx.device_status() == 0
    pl.execute(X, f, n, u, w)
    assert ctx.device_status() == 0
    n[1500, 2] = float("nan")
    pl.execute(X, f, n, u, w)
    assert ctx.device_status() & mrs.MRS_FLAG_NONFINITE
    assert ctx.device_status() == 0
    assert not torch.isfinite(u).all()
    pl.close()


def test_reserve_makes_mrs_velocity_allocation_free(ctx, orc):
    """mrs_reserve builds the cached plan of a shape (its scratch shows up as device memory
    taken); mrs_velocity on that shape then takes no device memory and can be captured in a
    CUDA graph in global capture mode (which rejects allocation), and the replay matches the
    eager call bit for bit and the oracle."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.single_system(seed=81, n_fil=4, M=1024)       # 4096 points: several MB of scratch
    mu, eps = 1.7, float(p.eps[0])                      # a shape no other test caches
    X, f, n = dev(p.X), dev(p.f), dev(p.n)
    ue, we = torch.empty_like(X), torch.empty_like(X)
    u, w = torch.full_like(X, float("nan")), torch.full_like(X, float("nan"))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    mrs.mrs_reserve(ctx, p.offsets, mu, eps)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 < free0
    mrs.mrs_velocity(ctx, p.offsets, X, f, n, ue, we, mu, eps)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="global"):
            mrs.mrs_velocity(ctx, p.offsets, X, f, n, u, w, mu, eps, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u, ue) and torch.equal(w, we)
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, eps, mu)
    assert rel_l2(u.cpu().numpy(), ur) < TOL32 and rel_l2(w.cpu().numpy(), wr) < TOL32
    mrs.mrs_reserve(ctx, p.offsets, mu, eps)             # already cached: nothing new
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1


def degenerate_system():
    """One system with the method's degenerate geometries: points repeated exactly (r = 0
    between distinct points), a cluster within 1e-3 eps, and clusters 1e4 eps apart."""
    from paper_2604_12083_gb300 import workloads as W
    rng = np.random.default_rng(84)
    eps = float(np.float32(0.01))
    base = rng.uniform(0.0, 1.0, (300, 3))
    dup = base[:100].copy()                                  # exact repeats
    tight = base[200] + rng.uniform(-1e-5, 1e-5, (60, 3))    # within 1e-3 eps
    far = rng.uniform(0.0, 1.0, (77, 3)) + 100.0             # 1e4 eps away
    X = np.concatenate([base, dup, tight, far]).astype(np.float32)
    f = rng.standard_normal(X.shape).astype(np.float32)
    n = rng.standard_normal(X.shape).astype(np.float32)
    off = np.array([0, X.shape[0]], np.int64)
    return W.MRSProblem("degenerate", off, X, f, n, np.array([eps]), 1.0)


@pytest.mark.parametrize("config", [None, 8, 14, 25])
def test_degenerate_geometries(ctx, orc, config):
    from paper_2604_12083_gb300 import mrs
    p = degenerate_system()
    ur, wr = orc.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu)
    for prec in (mrs.MRS_F32, mrs.MRS_F32_COMP):
        u, w = run(ctx, p, prec, config=config)
        assert np.isfinite(u).all() and np.isfinite(w).all()
        assert rel_l2(u, ur) < TOL32 and rel_l2(w, wr) < TOL32
    u, w = run(ctx, p, mrs.MRS_F64)
    assert rel_l2(u, ur) < TOL64 and rel_l2(w, wr) < TOL64


def test_single_point_closed_form_and_zero_sources(ctx):
    """A lone point: u = f / (4 pi mu eps), omega = 5 n / (16 pi mu eps^3) (the r = 0 values of
    H1 and H4), in every precision; zero forces and torques give exactly zero."""
    from paper_2604_12083_gb300 import mrs, workloads as W
    eps, mu = 0.05, 1.3
    f = np.array([[0.5, -1.0, 2.0]])
    n = np.array([[1.5, 0.25, -0.75]])
    X = np.array([[3.0, -2.0, 1.0]])
    p = W.MRSProblem("lone", np.array([0, 1], np.int64), X.astype(np.float32),
                     f.astype(np.float32), n.astype(np.float32), np.array([eps]), mu)
    u_ref = f / (4 * np.pi * mu * eps)
    w_ref = 5 * n / (16 * np.pi * mu * eps**3)
    for prec, tol in ((mrs.MRS_F32, 1e-6), (mrs.MRS_F32_COMP, 1e-6), (mrs.MRS_F64, 1e-14)):
        u, w = run(ctx, p, prec)
        assert rel_l2(u, u_ref) < tol and rel_l2(w, w_ref) < tol
    z = W.MRSProblem("zero", np.array([0, 700], np.int64),
                     np.random.default_rng(85).uniform(0, 1, (700, 3)).astype(np.float32),
                     np.zeros((700, 3), np.float32), np.zeros((700, 3), np.float32),
                     np.array([eps]), mu)
    for config in (None, 8, 25):
        u, w = run(ctx, z, mrs.MRS_F32_COMP, config=config)
        assert not u.any() and not w.any()


def test_fma_probe_reports_pipe_throughput(ctx):
    """mrs_fma_probe runs each instruction stream and reports a throughput between a tenth of
    and slightly above the nominal FP32 peak (2 x 128 lanes x SMs x 2.07 GHz)."""
    from paper_2604_12083_gb300 import mrs
    nominal = 2 * 128 * ctx.num_sms * 2.07e9 / 1e12
    for kind in (0, 1, 2):
        tf, ms = mrs.fma_probe(0, kind, 1 << 14)
        assert ms > 0 and 0.1 * nominal < tf < 1.1 * nominal, (kind, tf, nominal)
    tf, ms = mrs.fma_probe(0, 3, 1 << 10)        # float64: a small fraction of the FP32 rate
    assert ms > 0 and 0.0 < tf < 0.2 * nominal, tf
    tf1, ms1 = mrs.fma_probe(0, 4, 1 << 10)      # float64 on one lane per warp: counts 1/32
    assert ms1 > 0 and 0.0 < tf1 < tf, (tf1, tf)  # of the lanes, so never above all 32 lanes
    tf2, _ = mrs.fma_probe(0, 1, 1 << 12, 2)     # 2 warps per scheduler, as the pair kernel
    assert 0.1 * nominal < tf2 < 1.1 * nominal, tf2
    with pytest.raises(mrs.MrsError):
        mrs.fma_probe(0, 5, 16)
    with pytest.raises(mrs.MrsError):
        mrs.fma_probe(0, 1, 16, 17)
