"""Benchmark of the regularized-Stokeslet pair sum on GB300 (one JSON line on stdout).

Workload (one "step"): one mrs_velocity call, float32 with compensated accumulation, on the
single-system configuration -- 32 filaments x 1024 nodes = 32768 points in a 10^3 box with
random orientations, eps = 1.5 ds, mu = 1, Gaussian forces and torques (seeded, synthetic).
Metric: pair interactions per second (N^2 ordered pairs, self included), with the fraction of
the FP32 (non-tensor) peak and the relative L2 error of a sampled set of targets against the
FP64 oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

--impl reference times the FP64 CPU oracle (the only reference there is) on the same workload,
each step a bounded sample of targets.  For N > 1 (torchrun), every rank runs its own replica
(replicas only: the path needs no exchange between GPUs), and value = all ranks' pairs / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_PAIR = 92          # canonical algorithmic flop count of one ordered pair
METRIC = ("MRS pair-interactions/s (frac of FP32 peak) at 1e-5 rel err; "
          "p50/p99 solve latency")
UNIT = "pairs/s"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


def measured_traffic(kernel):
    """DRAM bytes per launch of the pair-sum kernel from the committed ncu capture, or None when
    the capture is of another kernel or the kernel source has changed since it was taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "mrs_traffic.json")))
        if not rec["kernel"].startswith("mrs::" + kernel.split()[0]):
            return None
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
            return None
        return int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"])
    except Exception:
        return None


def fp32_peak_tflops(n_sms, peaks):
    """2 flops (FMA) x 128 FP32 lanes per SM x SMs x the maximum SM clock."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return 2.0 * 128 * n_sms * mhz * 1e6 / 1e12, mhz


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.gpu_id = gpu_id
        self.path = os.path.join("/tmp", "mrs_clocks_%d_%d.csv" % (os.getpid(), int(time.time())))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    """Rank layout from the torchrun environment; NCCL when a GPU is present, else gloo.  The
    process group is used only for the timing barrier and the max/sum of two numbers (no
    data-path collective: every rank runs an independent replica)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg, dev):
    import torch
    if dev.type == "cuda":
        torch.cuda.synchronize()
    if pg is not None:
        if dev.type == "cuda":
            pg.barrier(device_ids=[dev.index])
        else:
            pg.barrier()
    if dev.type == "cuda":
        torch.cuda.synchronize()


def max_over_ranks(pg, value, dev):
    import torch
    if pg is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, value, dev):
    import torch
    if pg is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def aggregate(pg, dev, step_ms, pairs_per_step, steps):
    """Whole-job throughput: all ranks' pairs over the slowest rank's timed region."""
    t_max = max_over_ranks(pg, float(sum(step_ms)), dev)
    pairs_all = sum_over_ranks(pg, float(pairs_per_step) * steps, dev)
    return pairs_all / (t_max * 1e-3), t_max / steps


def oracle_rate(p, seconds_target, seed=0):
    """Pairs/s of the FP64 oracle on a sample of targets of problem p (all sources)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    N = p.n_points
    # calibrate on 64 targets, then size the sample to ~seconds_target
    idx = rng.choice(N, 64, replace=False)
    t0 = time.perf_counter()
    oracle.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu, xt=p.X[idx])
    dt = max(time.perf_counter() - t0, 1e-6)
    rate = 64 * N / dt
    nt = int(min(N, max(64, seconds_target * rate / N)))
    return nt, rate


def plain_rod_times(ctx, dev):
    """The plain-method configuration timed on both sides: one 128-node rod, one float64
    mrs_velocity with Gaussian forces and torques, then 200 RK2 rod_step steps (dt = 1e-6):
    the FP64 oracle on the host cores and the library on the GPU (CUDA events), with the
    agreement of the two results."""
    import torch
    import oracle
    from paper_2604_12083_gb300 import mrs, workloads as W
    pr = W.plain_rod()
    rs = W.rod_system(1, 1, 128)
    c = W.ROD_PLAIN
    op = oracle.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"])
    t0 = time.perf_counter()
    ur, wr = oracle.mrs_velocity(pr.X, pr.f, pr.n, pr.eps[0], pr.mu)
    Xo, _ = oracle.rod_step(rs.rod_off, rs.X, rs.D, op, rs.eps, 1.0, 0.0, c["dt"], 200, oracle.RK2)
    t_oracle = time.perf_counter() - t0
    prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"], 1.0, rs.eps)
    X64, f64, n64 = (torch.from_numpy(a.astype(np.float64)).to(dev) for a in (pr.X, pr.f, pr.n))
    u64, w64 = torch.empty_like(X64), torch.empty_like(X64)
    Xg, Dg = torch.from_numpy(rs.X.copy()).to(dev), torch.from_numpy(rs.D.copy()).to(dev)
    mrs.rod_step(ctx, rs.rod_off, prm, Xg, Dg, 0.0, c["dt"], 4, mrs.MRS_RK2)   # set-up
    mrs.mrs_velocity(ctx, pr.offsets, X64, f64, n64, u64, w64, pr.mu, float(pr.eps[0]),
                     precision=mrs.MRS_F64)                                   # plan built
    Xg.copy_(torch.from_numpy(rs.X))
    Dg.copy_(torch.from_numpy(rs.D))
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    mrs.mrs_velocity(ctx, pr.offsets, X64, f64, n64, u64, w64, pr.mu, float(pr.eps[0]),
                     precision=mrs.MRS_F64)
    mrs.rod_step(ctx, rs.rod_off, prm, Xg, Dg, 0.0, c["dt"], 200, mrs.MRS_RK2)
    b.record(stream)
    torch.cuda.synchronize()
    disp_o = Xo - rs.X
    return {"workload": "one 128-node rod: one FP64 mrs_velocity + 200 RK2 rod_step steps "
                        "(dt = 1e-6)",
            "oracle_s": t_oracle, "gpu_s": a.elapsed_time(b) * 1e-3,
            "rel_err_u_fp64": float(np.linalg.norm(u64.cpu().numpy() - ur) / np.linalg.norm(ur)),
            "rel_err_displacement_200_steps": float(np.linalg.norm(Xg.cpu().numpy() - rs.X - disp_o)
                                                    / np.linalg.norm(disp_o))}


def run_reference(args, world, rank):
    """The oracle arm: FP64 CPU oracle on the same workload, bounded sample per step."""
    if rank != 0:
        return
    import oracle
    from paper_2604_12083_gb300 import workloads as W
    p = W.single_system()
    budget = 150.0 / max(1, args.steps + args.warmup)     # whole run within a few minutes
    nt, _ = oracle_rate(p, budget)
    rng = np.random.default_rng(5)
    times = []
    for it in range(args.warmup + args.steps):
        idx = rng.choice(p.n_points, nt, replace=False)
        t0 = time.perf_counter()
        oracle.mrs_velocity(p.X, p.f, p.n, p.eps[0], p.mu, xt=p.X[idx])
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    pairs = nt * p.n_points
    value = pairs * len(times) / sum(times)
    cores = oracle.num_threads()
    sample = "%d sampled targets x %d sources per step (FP64, OpenMP over targets)" % (nt, p.n_points)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": p.name, "n_points": p.n_points, "eps": float(p.eps[0]), "mu": p.mu,
                   "parallelism": "none (host cores)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_events(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def extra_batch(ctx, dev):
    """512 systems (256..16384 points): one persistent launch (CUDA graph) vs one launch per
    system, float32 accumulation (accuracy against the oracle: the GPU tests)."""
    import torch
    from paper_2604_12083_gb300 import mrs, workloads as W
    p = W.batch_systems()
    X, f, n = (torch.from_numpy(a).to(dev) for a in (p.X, p.f, p.n))
    u = torch.empty_like(X)
    w = torch.empty_like(X)
    stream = torch.cuda.current_stream(dev)
    tuned_cfg, tuned_ms = mrs.autotune(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps,
                                       precision=mrs.MRS_F32, reps=2)
    plan = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32)
    plan.execute(X, f, n, u, w)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            plan.execute(X, f, n, u, w, stream=side)
    stream.wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    ms_graph = _time_events(g.replay, 5, stream)
    plans = []
    for s in range(len(p.offsets) - 1):
        a, b = int(p.offsets[s]), int(p.offsets[s + 1])
        plans.append((a, b, mrs.Plan(ctx, [0, b - a], p.mu, float(p.eps[s]), precision=mrs.MRS_F32)))
    views = [(X[a:b], f[a:b], n[a:b], u[a:b], w[a:b], pl) for a, b, pl in plans]

    def loop():
        for xx, ff, nn, uu, ww, pl in views:
            pl.execute(xx, ff, nn, uu, ww)

    loop()
    torch.cuda.synchronize()
    ms_loop = _time_events(loop, 3, stream)
    for _, _, pl in plans:
        pl.close()
    info = plan.info()
    plan.close()
    return {"workload": p.name + " (N_s log-uniform in [256,16384], filaments of 256 nodes)",
            "pairs": p.pairs, "persistent_graph_ms": ms_graph,
            "persistent_pairs_per_s": p.pairs / (ms_graph * 1e-3),
            "one_launch_per_system_ms": ms_loop,
            "one_launch_per_system_pairs_per_s": p.pairs / (ms_loop * 1e-3),
            "speedup": ms_loop / ms_graph, "plan": info,
            "autotuned_config": tuned_cfg, "autotune_best_ms": tuned_ms}


def extra_rod_step(ctx, dev):
    """One rod of 128 nodes: 200 Euler and 200 RK2 steps at dt = 1e-6 (graph replays)."""
    import torch
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(1, 1, 128)
    c = W.ROD_PLAIN
    prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"], 1.0, rs.eps)
    out = {"workload": "one rod, 128 nodes, 200 steps, dt=1e-6"}
    stream = torch.cuda.current_stream(dev)
    for name, sch in (("euler", mrs.MRS_EULER), ("rk2", mrs.MRS_RK2)):
        Xd, Dd = torch.from_numpy(rs.X.copy()).to(dev), torch.from_numpy(rs.D.copy()).to(dev)
        mrs.rod_step(ctx, rs.rod_off, prm, Xd, Dd, 0.0, c["dt"], 200, sch)
        torch.cuda.synchronize()
        ms = _time_events(lambda: mrs.rod_step(ctx, rs.rod_off, prm, Xd, Dd, 0.0, c["dt"], 200, sch),
                          3, stream)
        out[name + "_us_per_step"] = 1e3 * ms / 200
    return out


def extra_parareal(ctx, dev):
    """8 filaments x 512 nodes, 64 slices, fine RK2 dt = 1e-6 (16 fine steps per slice, a
    shortened horizon), coarse Euler r dt: serial fine RK2 on the GPU, the regular Parareal
    schedule and the pipelined one (groups of 8 slices), for r = 4, 8, 16 -- the one-GPU
    analogue of the paper's regular/pipelined comparison and of its gap-versus-1/r plot."""
    import torch
    from paper_2604_12083_gb300 import mrs, workloads as W
    rs = W.rod_system(4, 8, 512)
    c = W.ROD_PARAREAL
    prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"], 1.0, rs.eps)
    Ns, nf, dt = 64, 16, c["dt"]
    T1 = Ns * nf * dt
    fresh = lambda: (torch.from_numpy(rs.X.copy()).to(dev), torch.from_numpy(rs.D.copy()).to(dev))
    Xs, Ds = fresh()
    mrs.rod_step(ctx, rs.rod_off, prm, Xs, Ds, 0.0, dt, 16, mrs.MRS_RK2)   # capture / warm-up
    Xs, Ds = fresh()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mrs.rod_step(ctx, rs.rod_off, prm, Xs, Ds, 0.0, dt, Ns * nf, mrs.MRS_RK2)
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t0
    disp_s = Xs.cpu().numpy() - rs.X
    out = {"workload": "8 filaments x 512 nodes, 64 slices x 16 fine RK2 steps (dt=1e-6), "
                       "coarse Euler r*dt, tol 1e-11",
           "serial_fine_s": t_serial, "serial_fine_steps": Ns * nf, "runs": []}
    for r in (4, 8, 16):
        for gs in (0, 8):
            for rep in range(2):          # first run sets up workspaces and graphs
                Xp, Dp = fresh()
                st = mrs.parareal_run(ctx, rs.rod_off, prm, Xp, Dp, 0.0, T1, Ns, dt, r, 8, 1e-11,
                                      raise_on_noconv=False, group_size=gs)
            disp_p = Xp.cpu().numpy() - rs.X
            out["runs"].append({
                "r": r, "schedule": "pipelined (groups of 8)" if gs else "regular",
                "iterations": st.iterations, "seconds": st.seconds,
                "converged": bool(st.final_incr < 1e-11),
                "increments": [st.incr[i] for i in range(st.iterations)],
                "fine_steps_executed": st.fine_steps,
                "rel_diff_vs_serial_displacement": float(np.linalg.norm(disp_p - disp_s) /
                                                         np.linalg.norm(disp_s))})
    # a small, launch-bound system: one 128-node rod, where batching the 64 slices of each
    # iteration into one launch per stage uses the GPU far better than serial stepping
    rs1 = W.rod_system(1, 1, 128)
    c1 = W.ROD_PARAREAL_128
    prm1 = mrs.RodParams.make(c1["L"], c1["a"], c1["b"], c1["wave_A"], c1["wave_k"], c1["wave_f"],
                              1.0, rs1.eps)
    nf1 = 256
    T1s = Ns * nf1 * dt
    fresh1 = lambda: (torch.from_numpy(rs1.X.copy()).to(dev), torch.from_numpy(rs1.D.copy()).to(dev))
    Xs, Ds = fresh1()
    mrs.rod_step(ctx, rs1.rod_off, prm1, Xs, Ds, 0.0, dt, 16, mrs.MRS_RK2)
    Xs, Ds = fresh1()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mrs.rod_step(ctx, rs1.rod_off, prm1, Xs, Ds, 0.0, dt, Ns * nf1, mrs.MRS_RK2)
    torch.cuda.synchronize()
    t_serial1 = time.perf_counter() - t0
    # the float32 pair sum puts a floor of ~1e-8 on the relative increment for this system (a
    # rounding flip of a packed position moves the velocities at the 1e-7 level; measured
    # increments after the third iteration stall between 0.8e-8 and 1.5e-8): tol well above it
    tol1 = 3e-8
    small = {"workload": "one rod, 128 nodes, 64 slices x 256 fine RK2 steps (dt=1e-6), coarse 16 dt",
             "tol": tol1, "serial_fine_s": t_serial1, "runs": []}
    for gs in (0, 8):
        for rep in range(2):
            Xp, Dp = fresh1()
            st = mrs.parareal_run(ctx, rs1.rod_off, prm1, Xp, Dp, 0.0, T1s, Ns, dt, 16, 8, tol1,
                                  raise_on_noconv=False, group_size=gs)
        dp = Xp.cpu().numpy() - rs1.X
        ds_ = Xs.cpu().numpy() - rs1.X
        ok = bool(st.final_incr < tol1)
        small["runs"].append({"schedule": "pipelined (groups of 8)" if gs else "regular",
                              "iterations": st.iterations, "seconds": st.seconds,
                              "converged": ok, "final_increment": st.final_incr,
                              "increments": [st.incr[i] for i in range(st.iterations)],
                              "fine_steps_executed": st.fine_steps,
                              "speedup_vs_serial_fine": t_serial1 / st.seconds if ok else None,
                              "rel_diff_vs_serial_displacement":
                                  float(np.linalg.norm(dp - ds_) / np.linalg.norm(ds_))})
    out["small_system"] = small
    return out


def run_large_system(args):
    """One system of 2^18 + 17 points (uniform in a 40^3 box, Gaussian f and n, eps = 0.02; the
    large-system parity test's input): the symmetric pair sum in the library's default plan (its
    column partials split into passes of at most 192 MiB) and in one pass, with the plan's
    passes and scratch, timed with CUDA events (inputs far larger than L2 are not needed: the
    kernel is ALU-bound; 92 flops per ordered pair against the FP32 peak)."""
    import torch
    from paper_2604_12083_gb300 import build as B, mrs, workloads as W
    B.build()
    ctx = mrs.Context(0)
    rng = np.random.default_rng(68)
    N = (1 << 18) + 17
    X = rng.uniform(0.0, 40.0, (N, 3)).astype(np.float32)
    f = rng.standard_normal((N, 3)).astype(np.float32)
    n = rng.standard_normal((N, 3)).astype(np.float32)
    off = np.array([0, N], np.int64)
    Xd, fd, nd = (torch.from_numpy(a).cuda() for a in (X, f, n))
    u, w = torch.empty_like(Xd), torch.empty_like(Xd)
    peak, _ = fp32_peak_tflops(ctx.num_sms, load_peaks())
    clk = ClockSampler(0)
    clk.start()
    out = {"case": "large_system", "workload": "one system of 2^18 + 17 points", "pairs": N * N,
           "runs": []}
    for pass_bytes, label in ((192 << 20, "default (passes of 192 MiB)"), (4 << 30, "one pass")):
        ctx.set_sym_pass_bytes(pass_bytes)
        pl = mrs.Plan(ctx, off, 1.0, 0.02, precision=mrs.MRS_F32_COMP, config=-1)
        ctx.set_sym_pass_bytes(192 << 20)
        pl.execute(Xd, fd, nd, u, w)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            pl.execute(Xd, fd, nd, u, w)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = min(ts)
        tf = 92.0 * N * N / (ms * 1e-3) / 1e12
        out["runs"].append({"plan": label, "config": pl.info()["config"], **pl.scratch(),
                            "ms": ms, "tflops": tf, "frac_of_fp32_peak": tf / peak})
        pl.close()
    out["clocks"] = clk.stop()
    out["peak_tflops"] = peak
    print(json.dumps(out), flush=True)
    ctx.close()


def run_fp32_peak(args):
    """The FP32 FMA pipe's throughput on this GPU (mrs_fma_probe): scalar FFMA, packed FFMA2 and
    the two interleaved, against the nominal 2 x 128 lanes x SMs x maximum SM clock, with the SM
    clock sampled during the runs; and the FP64 pipe's, with all lanes of each warp active and
    with one."""
    import torch
    from paper_2604_12083_gb300 import build as B, mrs
    B.build()
    torch.cuda.init()
    clk = ClockSampler(0)
    clk.start()
    res = {}
    for kind, name in ((0, "ffma"), (1, "ffma2"), (2, "ffma_ffma2_interleaved"), (3, "dfma_fp64"),
                       (4, "dfma_fp64_one_lane_per_warp")):
        best = None
        for _ in range(5):
            tf, ms = mrs.fma_probe(0, kind, (1 << 18) if kind < 3 else (1 << 13))
            if best is None or tf > best[0]:
                best = (tf, ms)
        res[name] = {"tflops": best[0], "ms": best[1]}
    for w in (1, 2, 4):   # the pair-sum kernel runs 2 warps per scheduler
        best = None
        for _ in range(3):
            tf, ms = mrs.fma_probe(0, 1, 1 << 16, w)
            best = tf if best is None or tf > best else best
        res["ffma2_%d_warps_per_scheduler" % w] = {"tflops": best}
    clocks = clk.stop()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = 2 * 128 * sms * float(load_peaks().get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    for k, v in res.items():
        if not k.startswith("dfma"):
            v["frac_of_nominal"] = v["tflops"] / peak
    # a DFMA costs the same whatever the active mask when this ratio is near 32
    res["dfma_all_lanes_over_one_lane"] = (res["dfma_fp64"]["tflops"]
                                           / res["dfma_fp64_one_lane_per_warp"]["tflops"])
    print(json.dumps({"case": "fp32_peak", "nominal_tflops": peak, "sms": sms,
                      "nominal_basis": "2 x 128 FP32 lanes x SMs x max SM clock", **res,
                      "clocks": clocks}), flush=True)


def run_parareal_horizon(args):
    """The Parareal configuration at its configured horizon: 8 filaments x 512 nodes (seed 4),
    64 slices over T = 1/horizon of a beat period (the wave frequency f = 2 pi makes one
    period one time unit), fine RK2 at dt = 1e-6, coarse Euler at 16 dt.  A slice holds a whole
    number of coarse steps, so T = 64 x floor(10^6 / (64 horizon) / 16) x 16 dt (1/16 period:
    976 fine steps per slice, T = 0.062464, 0.9994 of it).  Serial fine RK2 over [0, T] on the
    same GPU is the reference: reported are its wall time, and for the regular and the pipelined
    Parareal schedule the wall time, iterations, the increment series (Eq. true_err's
    increment) and the final state's error against serial fine (Eq. true_err at T)."""
    import torch
    from paper_2604_12083_gb300 import build as B, mrs, workloads as W
    B.build()
    dev = torch.device("cuda", 0)
    ctx = mrs.Context(0)
    rs = W.rod_system(4, 8, 512)
    c = W.ROD_PARAREAL
    prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"], 1.0, rs.eps)
    Ns, r, dt = 64, 16, c["dt"]
    nf = int(1e6 / (Ns * args.horizon) / r) * r
    T1 = Ns * nf * dt
    tol, max_iter = args.tol, args.max_iter
    fresh = lambda: (torch.from_numpy(rs.X.copy()).to(dev), torch.from_numpy(rs.D.copy()).to(dev))
    # warm-up: workspaces, captured graphs and plans of both schedules (a short horizon)
    Xw, Dw = fresh()
    mrs.rod_step(ctx, rs.rod_off, prm, Xw, Dw, 0.0, dt, 2 * r, mrs.MRS_RK2)
    for gs in (0, 8):
        Xw, Dw = fresh()
        mrs.parareal_run(ctx, rs.rod_off, prm, Xw, Dw, 0.0, Ns * r * dt, Ns, dt, r, 2, tol,
                         raise_on_noconv=False, group_size=gs)
    Xs, Ds = fresh()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mrs.rod_step(ctx, rs.rod_off, prm, Xs, Ds, 0.0, dt, Ns * nf, mrs.MRS_RK2)
    torch.cuda.synchronize()
    t_serial = time.perf_counter() - t0
    xs = Xs.cpu().numpy()

    def true_err(x):
        return float(np.max(np.linalg.norm(x - xs, axis=1) / np.linalg.norm(xs, axis=1)))

    out = {"case": "parareal_horizon",
           "workload": "8 filaments x 512 nodes (4096 points), 64 slices x %d fine RK2 steps "
                       "(dt = 1e-6), coarse Euler 16 dt, T = %.6f (1/%g of a beat period)"
                       % (nf, T1, args.horizon),
           "tol": tol, "max_iter": max_iter, "serial_fine_s": t_serial,
           "serial_fine_steps": Ns * nf, "runs": []}
    for gs in (0, 8):
        Xp, Dp = fresh()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = mrs.parareal_run(ctx, rs.rod_off, prm, Xp, Dp, 0.0, T1, Ns, dt, r, max_iter, tol,
                              raise_on_noconv=False, group_size=gs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out["runs"].append({
            "schedule": "pipelined (groups of 8)" if gs else "regular",
            "iterations": st.iterations, "seconds": wall, "converged": bool(st.final_incr < tol),
            "increments": [st.incr[i] for i in range(st.iterations)],
            "fine_steps_executed": st.fine_steps, "coarse_steps_executed": st.coarse_steps,
            "final_state_true_err": true_err(Xp.cpu().numpy()),
            "speedup_vs_serial_fine": t_serial / wall})
    print(json.dumps(out), flush=True)
    ctx.close()


def _serve_jobs(trace, dev, seed):
    """Device buffers for every job of a trace (built before any timing)."""
    import torch
    from paper_2604_12083_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    jobs = []
    for (t, kind, N) in trace:
        n_fil = N // 256
        X, D = W.place_filaments(rng, n_fil, 256, box=10.0)
        eps = float(np.float32(W.EPS_OVER_DS / 255))
        if kind == 0:
            f = rng.standard_normal((N, 3)).astype(np.float32)
            n = rng.standard_normal((N, 3)).astype(np.float32)
            b = [torch.from_numpy(a.astype(np.float32)).to(dev) for a in (X, f, n)]
            b += [torch.empty_like(b[0]), torch.empty_like(b[0])]
        else:
            b = [torch.from_numpy(X).to(dev), torch.from_numpy(D).to(dev),
                 np.arange(0, N + 1, 256, dtype=np.int64)]
        jobs.append((t, kind, N, eps, b))
    return jobs


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


# (label, arrival rate per s, arrival window s, seed): the full measurement (--case serve) runs
# the nominal rate over the configured 2 s window (~4000 jobs, run to drain) and a rate sweep
# with windows long enough for a few hundred jobs; the default bench run the same traces cut
# to about a minute of arrivals in all (the nominal rate to 50 ms: 94 jobs, ~1.6 s of GPU work;
# 20 and 5 jobs/s to half their windows).  With ~100-200 jobs a p99 is still decided by the
# two or three largest jobs.
SERVE_FULL = (("nominal_2000_per_s", 2000.0, 2.0, 5), ("rate_500_per_s", 500.0, 0.4, 8),
              ("rate_100_per_s", 100.0, 2.0, 9), ("rate_20_per_s", 20.0, 20.0, 6),
              ("rate_5_per_s", 5.0, 40.0, 7))
SERVE_SHORT = (("nominal_2000_per_s", 2000.0, 0.05, 5), ("rate_500_per_s", 500.0, 0.4, 8),
               ("rate_100_per_s", 100.0, 2.0, 9), ("rate_20_per_s", 20.0, 10.0, 6),
               ("rate_5_per_s", 5.0, 20.0, 7))


def extra_serve(ctx, dev, full=False):
    """Poisson arrivals of mixed jobs (70 % one pair sum, 30 % 100-step Euler rod integration),
    N log-uniform in [1k, 64k] (filaments of 256 nodes): the continuous-batching server (default
    policy: jobs of at least 1.3e10 pair interactions run in admission order, smaller ones
    alongside) vs the same jobs run one request per launch, both on this GPU."""
    import torch
    from paper_2604_12083_gb300 import mrs, workloads as W
    c = W.ROD_SERVE
    out = {"workload": "Poisson arrivals, 70% mrs_velocity / 30% 100-step Euler rod jobs, "
                       "N log-uniform [1k,64k], HBM budget 150 GB",
           "policy": "big jobs (>= 1.3e10 pairs) one at a time in admission order, small jobs "
                     "batched alongside"}
    for label, rate, window, seed in (SERVE_FULL if full else SERVE_SHORT):
        trace = W.serve_trace(seed=seed, rate_hz=rate, window_s=window)
        jobs = _serve_jobs(trace, dev, seed)
        pairs = sum((N * N) * (1 if k == 0 else 100) for (_, k, N, _, _) in jobs)
        res = {"jobs": len(jobs), "pairs": float(pairs), "rate_per_s": rate, "window_s": window}
        for mode in ("served", "one_request_per_launch"):
            torch.cuda.synchronize()
            lat = []
            if mode == "served":
                srv = mrs.Server(ctx, 150 * 10**9, 256)
                tickets = []
                t0 = time.perf_counter()
                for (ta, kind, N, eps, b) in jobs:
                    while time.perf_counter() - t0 < ta:
                        time.sleep(2e-4)
                    if kind == 0:
                        tickets.append(srv.submit_velocity(b[0], b[1], b[2], b[3], b[4], 1.0, eps))
                    else:
                        prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"],
                                                 c["wave_f"], 1.0, eps)
                        tickets.append(srv.submit_rod(b[2], b[0], b[1], prm, 0.0, c["dt"], 100,
                                                      mrs.MRS_EULER, 1.0, eps))
                srv.drain(900.0)
                makespan = time.perf_counter() - t0
                lat = [srv.poll(t)[1] for t in tickets]
                res["served_stats"] = srv.stats()
                srv.close()
            else:
                s = torch.cuda.current_stream(dev)
                t0 = time.perf_counter()
                for (ta, kind, N, eps, b) in jobs:
                    while time.perf_counter() - t0 < ta:
                        time.sleep(2e-4)
                    if kind == 0:
                        mrs.mrs_velocity(ctx, [0, N], b[0], b[1], b[2], b[3], b[4], 1.0, eps)
                    else:
                        prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"],
                                                 c["wave_f"], 1.0, eps)
                        mrs.rod_step(ctx, b[2], prm, b[0], b[1], 0.0, c["dt"], 100, mrs.MRS_EULER)
                    s.synchronize()
                    lat.append(time.perf_counter() - t0 - ta)
                makespan = time.perf_counter() - t0
            res[mode] = {"makespan_s": makespan, "pairs_per_s": pairs / makespan,
                         "p50_latency_s": _pct(lat, 50), "p99_latency_s": _pct(lat, 99)}
        res["throughput_ratio_served_vs_plain"] = (res["served"]["pairs_per_s"] /
                                                   res["one_request_per_launch"]["pairs_per_s"])
        out[label] = res
        del jobs
        torch.cuda.empty_cache()
    return out


def run_extras(ctx, dev):
    out = {}
    for name, fn in (("batch", extra_batch), ("rod_step", extra_rod_step),
                     ("parareal", extra_parareal), ("serve", extra_serve)):
        try:
            out[name] = fn(ctx, dev)
        except Exception as e:       # reported, never silently replaced by another path
            out[name] = {"error": repr(e)}
    return out


def run_rod_kernels(args):
    """Rod force assembly (segment + node kernels) and the explicit update on 1024 rods x 1024
    nodes (1,048,576 nodes, float64 state): achieved bytes per second against the measured HBM
    copy bandwidth.  Algorithmic bytes per node: forces read X, D (96 B) and write g, m (48 B);
    the update reads X, D and u, w (float32, 24 B) and writes X, D (96 B)."""
    import torch
    from paper_2604_12083_gb300 import build as B, mrs, workloads as W
    B.build()
    dev = torch.device("cuda", 0)
    ctx = mrs.Context(0)
    rs = W.rod_system(21, 1024, 1024, box=60.0)
    c = W.ROD_PLAIN
    prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"], 1.0, rs.eps)
    X = torch.from_numpy(rs.X).to(dev)
    D = torch.from_numpy(rs.D).to(dev)
    g = torch.empty_like(X)
    m = torch.empty_like(X)
    u = (torch.randn(X.shape, device=dev) * 1e-3).float()
    w = (torch.randn(X.shape, device=dev) * 1e-2).float()
    N = X.shape[0]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        tot = 0.0
        for i in range(reps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    reps = max(3, min(args.steps, 50))
    t_f = timed(lambda: mrs.rod_forces(ctx, rs.rod_off, prm, X, D, 0.1, g, m), reps)
    t_a = timed(lambda: mrs.rod_advance(ctx, X, D, u, w, 1e-7), reps)
    peak = float(load_peaks().get("hbm_gbs", 6800.0))
    fb, ab = 144 * N, 216 * N
    line = {"case": "rod_kernels", "workload": "1024 rods x 1024 nodes (1,048,576 nodes), float64",
            "rod_forces": {"ms": t_f, "algorithmic_bytes": fb, "achieved_gbs": fb / (t_f * 1e-3) / 1e9,
                           "frac_of_hbm": fb / (t_f * 1e-3) / 1e9 / peak,
                           "kernels": "rod_forces_fused_kernel"},
            "rod_advance": {"ms": t_a, "algorithmic_bytes": ab, "achieved_gbs": ab / (t_a * 1e-3) / 1e9,
                            "frac_of_hbm": ab / (t_a * 1e-3) / 1e9 / peak, "kernels": "rod_update_kernel"},
            "peak_hbm_gbs": peak, "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_ours(args, world, rank, local, pg):
    import torch
    from paper_2604_12083_gb300 import build as B, mrs, workloads as W
    if rank == 0 or not os.path.exists(mrs.LIB_PATH):
        B.build()
    if pg is not None:
        pg.barrier()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = mrs.Context(local)
    p = W.single_system(seed=2 + rank)      # each rank: its own replica of the workload
    stream = torch.cuda.current_stream(dev)
    X, f, n = (torch.from_numpy(a).to(dev) for a in (p.X, p.f, p.n))
    u = torch.empty_like(X)
    w = torch.empty_like(X)
    eps = float(p.eps[0])

    # the public call (plan cached in the context, the library's choice of configuration), or
    # with --config an explicit plan of that configuration
    forced = None
    if args.config >= 0:
        forced = mrs.Plan(ctx, p.offsets, p.mu, eps, precision=mrs.MRS_F32_COMP, config=args.config)

    def velocity(Xa, fa, na, ua, wa, s=None):
        if forced is not None:
            forced.execute(Xa, fa, na, ua, wa, stream=s)
        else:
            mrs.mrs_velocity(ctx, p.offsets, Xa, fa, na, ua, wa, p.mu, eps,
                             precision=mrs.MRS_F32_COMP, stream=s)

    def step():
        velocity(X, f, n, u, w)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MiB > L2
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # the configuration mrs_velocity chose for this shape (the same library choice as a plan
    # built with config = -1): symmetric ones launch the pair kernel and a reduction kernel
    if forced is not None:
        plan_info = forced.info()
    else:
        probe = mrs.Plan(ctx, p.offsets, p.mu, eps, precision=mrs.MRS_F32_COMP)
        plan_info = probe.info()
        probe.close()
    sym = mrs.plan_config_symmetric(plan_info["config"])
    launches_per_step = 2 if sym else 1
    kernel_name = ("mrs_f32_sym + mrs_sym_reduce (whole step)" if sym else "mrs_f32_persistent")
    # FP32 lane operations per ordered pair: symmetric kernel 85.4 per unordered pair (ncu
    # instruction counters: 83 packed + the scalar fold of each source's share), ordered 50
    lane_ops = 42.7 if sym else 50.0

    # ---- device-timed region: K steps, L2 flushed before each, events around each launch ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(pg, dev)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier(pg, dev)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    value, ms_per_step = aggregate(pg, dev, launch_ms, p.pairs, args.steps)

    # the last timed step's result, for the accuracy figure of the CPU-baseline leg
    u_last = u.cpu().numpy().astype(np.float64)
    w_last = w.cpu().numpy().astype(np.float64)
    rel = None

    # ---- end to end through the public API with host buffers ----
    # Every step copies its inputs from pinned host memory and its result back.  The copies run
    # on a second stream with two device buffer sets, so the inputs of step i+1 travel while
    # step i computes; the pair sums themselves stay on one stream (calls sharing a cached plan
    # must not overlap).
    hX, hf, hn = (torch.from_numpy(a).pin_memory() for a in (p.X, p.f, p.n))
    hu = torch.empty(u.shape, dtype=u.dtype).pin_memory()
    hw = torch.empty(w.shape, dtype=w.dtype).pin_memory()
    bufs = [tuple(torch.empty_like(X) for _ in range(5)) for _ in range(2)]   # X, f, n, u, w
    xs = torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()
    h2d_done, comp_done, d2h_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    for k in range(2):
        comp_done[k].record(stream)
        d2h_done[k].record(stream)

    def h2d(k):
        xs.wait_event(comp_done[k])          # the step that used buffer set k has read it
        with torch.cuda.stream(xs):
            for dst, src in zip(bufs[k][:3], (hX, hf, hn)):
                dst.copy_(src, non_blocking=True)
        h2d_done[k].record(xs)

    def e2e_run(n_steps):
        h2d(0)
        for i in range(n_steps):
            k = i % 2
            stream.wait_event(h2d_done[k])
            stream.wait_event(d2h_done[k])   # the result of step i-2 has been read
            bX, bf, bn, bu, bw = bufs[k]
            velocity(bX, bf, bn, bu, bw, s=stream)
            comp_done[k].record(stream)
            if i + 1 < n_steps:
                h2d((i + 1) % 2)
            xs.wait_event(comp_done[k])
            with torch.cuda.stream(xs):
                hu.copy_(bu, non_blocking=True)
                hw.copy_(bw, non_blocking=True)
            d2h_done[k].record(xs)
        stream.wait_event(d2h_done[(n_steps - 1) % 2])

    e2e_run(3)
    torch.cuda.synchronize()
    e2e_steps = max(10, min(args.steps, 200))
    barrier(pg, dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    xs.wait_event(e0)
    e2e_run(e2e_steps)
    e1.record(stream)
    barrier(pg, dev)
    e_ms = max_over_ranks(pg, e0.elapsed_time(e1), dev)
    e2e_pairs = sum_over_ranks(pg, float(p.pairs) * e2e_steps, dev)
    h2d = int(sum(t.numel() * t.element_size() for t in (hX, hf, hn)))
    d2h = int(sum(t.numel() * t.element_size() for t in (hu, hw)))

    peaks = load_peaks()
    peak, mhz = fp32_peak_tflops(ctx.num_sms, peaks)
    achieved = FLOPS_PER_PAIR * p.pairs / (np.mean(launch_ms) * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": p.name + " (32768 points, eps=1.5ds, mu=1, Gaussian f/n, "
                   "FP32 compensated accumulation)", "n_points": p.n_points,
                   "pairs_per_step": p.pairs, "global_batch": world, "parallelism":
                   "replicas (one independent system per GPU)",
                   "l2": "flushed before every timed step (512 MiB write)"},
        "rel_err": rel,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": measured_traffic(kernel_name),
                     "peak_basis": "2 x 128 FP32 lanes x %d SMs x %.0f MHz (max SM clock)" %
                                   (ctx.num_sms, mhz),
                     "flops_per_pair": FLOPS_PER_PAIR, "kernel": kernel_name,
                     # FP32 lane operations the kernel executes per ordered pair, and the
                     # share of the 128 lanes x SMs x clock they occupy at this rate
                     "lane_ops_per_pair": lane_ops,
                     "fp32_lane_fraction": value / world * lane_ops / (128.0 * ctx.num_sms * mhz * 1e6),
                     "plan": plan_info,
                     "work": ("each unordered pair evaluated once (symmetric reuse); flops counted "
                              "per ordered pair" if sym else "each ordered pair evaluated")},
        "clocks": clocks,
        "e2e": {"value": e2e_pairs / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * launches_per_step,
        "wall_s_timed_region": wall,
    }
    # the CPU baseline and the extras are single-GPU measurements reported at N = 1; with more
    # ranks they would only hold the other GPUs idle
    if world > 1:
        args.cpu_baseline = False
        args.extras = False
    if rank == 0 and args.cpu_baseline:
        # the FP64 oracle on a sample of targets (about 10 s of host work), timed; its values on
        # those targets also give the accuracy of the GPU result (relative L2 per field)
        import oracle
        nt, _ = oracle_rate(p, 10.0)
        idx = np.random.default_rng(11).choice(p.n_points, nt, replace=False)
        t0 = time.perf_counter()
        ur, wr = oracle.mrs_velocity(p.X, p.f, p.n, eps, p.mu, xt=p.X[idx])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nt * p.n_points / dt, "unit": UNIT,
                                "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": "%d sampled targets x %d sources (FP64)" % (nt, p.n_points)}
        line["rel_err"] = {
            "u": float(np.linalg.norm(u_last[idx] - ur) / np.linalg.norm(ur)),
            "w": float(np.linalg.norm(w_last[idx] - wr) / np.linalg.norm(wr)),
            "targets_sampled": int(nt), "against": "the FP64 oracle of the cpu_baseline sample"}
        line["cpu_baseline"]["plain_rod"] = plain_rod_times(ctx, dev)
    line["frac_of_fp32_peak"] = line["roofline"]["frac"]
    if rank == 0 and args.extras:
        line["extras"] = run_extras(ctx, dev)
        nominal = line["extras"].get("serve", {}).get("nominal_2000_per_s", {}).get("served")
        if nominal:
            line["p50_latency_s"] = nominal["p50_latency_s"]
            line["p99_latency_s"] = nominal["p99_latency_s"]
            line["latency_workload"] = ("served jobs, Poisson 2000 req/s, 70 % pair sums / 30 % "
                                        "100-step rod integrations, N log-uniform [1k, 64k]")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if forced is not None:
        forced.close()
    ctx.close()


def run_batch_case(args):
    """The batching workload alone: 512 systems (256..16384 points, filaments of 256 nodes), one
    plan (the autotuned configuration, or --config), 3 warm-up launches and --steps timed ones
    (L2 flushed before each, CUDA events): pairs/s and the fraction of the FP32 peak."""
    import torch
    from paper_2604_12083_gb300 import build as B, mrs, workloads as W
    B.build()
    dev = torch.device("cuda", 0)
    ctx = mrs.Context(0)
    p = W.batch_systems()
    X, f, n = (torch.from_numpy(a).to(dev) for a in (p.X, p.f, p.n))
    u, w = torch.empty_like(X), torch.empty_like(X)
    cfg = args.config
    if cfg < 0:
        cfg, _ = mrs.autotune(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32, reps=2)
    plan = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32, config=cfg)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        plan.execute(X, f, n, u, w)
    torch.cuda.synchronize()
    ms = []
    for i in range(max(1, args.steps)):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.execute(X, f, n, u, w)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    pairs = float(p.pairs)
    peak, mhz = fp32_peak_tflops(ctx.num_sms, load_peaks())
    t = float(np.mean(ms))
    print(json.dumps({"case": "batch", "workload": "batch_512_systems (N_s log-uniform in "
                      "[256,16384], filaments of 256 nodes), MRS_F32", "pairs": pairs,
                      "ms": t, "pairs_per_s": pairs / (t * 1e-3),
                      "frac_of_fp32_peak": FLOPS_PER_PAIR * pairs / (t * 1e-3) / 1e12 / peak,
                      "plan": plan.info(), "steps": len(ms)}), flush=True)
    plan.close()
    ctx.close()


def run_small_systems(args):
    """Latency of one pair sum (the library's default plan, MRS_F32_COMP) on single systems of
    1024 .. 16384 points, the sizes where a call is launch- and latency-bound; 200 back-to-back
    calls per size, CUDA events.  Inputs stay in L2: this is the latency a time step sees."""
    import numpy as np
    import torch
    from paper_2604_12083_gb300 import build as B, mrs
    B.build()
    ctx = mrs.Context(0)
    out = {"case": "small_systems", "unit": "us per call", "precision": "MRS_F32_COMP",
           "sizes": []}
    for N in (1024, 2048, 4096, 8192, 16384):
        rng = np.random.default_rng(N)
        X = torch.from_numpy((rng.random((N, 3)) * 2.0).astype(np.float32)).cuda()
        f = torch.from_numpy(rng.standard_normal((N, 3)).astype(np.float32)).cuda()
        n = torch.from_numpy(rng.standard_normal((N, 3)).astype(np.float32)).cuda()
        u, w = torch.empty_like(X), torch.empty_like(X)
        pl = mrs.Plan(ctx, np.array([0, N], np.int64), 1.0, 0.01, precision=mrs.MRS_F32_COMP)
        for _ in range(10):
            pl.execute(X, f, n, u, w)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(200):
            pl.execute(X, f, n, u, w)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1000.0 / 200
        out["sizes"].append({"points": N, "us_per_call": us, "pairs_per_s": N * N / (us * 1e-6),
                             "plan": pl.info()})
        pl.close()
    print(json.dumps(out), flush=True)
    ctx.close()


# GPU seconds per call that the paper prints for its own sizes (Table 1: rods of 51 points,
# eps = 4 ds, an NVIDIA A100 PCIe with numba.cuda, a wall and Lennard-Jones terms in the model,
# per time step or per solve not stated): MRS velocity computation, force initialisation,
# triad update.  Context for the same calls measured here, not a target.
TABLE1_A100_GPU_S = {1: (0.000389, 0.000683, 0.000230), 4: (0.000381, 0.000680, 0.000229),
                      12: (0.000382, 0.000676, 0.000230), 25: (0.000386, 0.000687, 0.000638)}


def run_paper_sizes(args):
    """The paper's own problem sizes (1, 4, 12, 25 rods of 51 points, eps = 4 ds): per-call
    latency of mrs_velocity, rod_forces and rod_advance, and of one Euler rod_step (forces,
    pack, pair sum, update), 200 back-to-back calls each, CUDA events; mrs_velocity also as
    50 calls replayed from one CUDA graph (the device time of a call without the host path);
    beside the GPU times the paper prints for the first three (Table 1, other hardware:
    context only)."""
    import numpy as np
    import torch
    from paper_2604_12083_gb300 import build as B, mrs, workloads as W
    B.build()
    dev = torch.device("cuda", 0)
    ctx = mrs.Context(0)
    c = W.ROD_PLAIN
    M = 51
    eps = 4.0 / (M - 1)
    stream = torch.cuda.current_stream(dev)

    def per_call_us(fn, reps=200):
        for _ in range(10):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1000.0 / reps

    out = {"case": "paper_sizes", "unit": "us per call",
           "workload": "n rods x 51 points, eps = 4 ds, mu = 1, free space (no wall, no LJ)",
           "paper_context": "GPU times printed in the paper's Table 1 (A100 PCIe, numba.cuda; "
                            "other hardware and model terms): context, not a target",
           "rows": []}
    for n_rods in (1, 4, 12, 25):
        rs = W.rod_system(30 + n_rods, n_rods, M, box=3.0)
        prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"], 1.0, eps)
        N = rs.X.shape[0]
        X = torch.from_numpy(rs.X).to(dev)
        D = torch.from_numpy(rs.D).to(dev)
        rng = np.random.default_rng(n_rods)
        X32 = X.float()
        f32 = torch.from_numpy(rng.standard_normal((N, 3)).astype(np.float32)).to(dev)
        n32 = torch.from_numpy(rng.standard_normal((N, 3)).astype(np.float32)).to(dev)
        u, w = torch.empty_like(X32), torch.empty_like(X32)
        g, m = torch.empty_like(X), torch.empty_like(X)
        off = np.array([0, N], np.int64)
        t_v = per_call_us(lambda: mrs.mrs_velocity(ctx, off, X32, f32, n32, u, w, 1.0, eps))
        # the same call without the host: reserved shape, 50 calls captured in one CUDA graph
        mrs.mrs_reserve(ctx, off, 1.0, eps)
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                for _ in range(50):
                    mrs.mrs_velocity(ctx, off, X32, f32, n32, u, w, 1.0, eps, stream=side)
        stream.wait_stream(side)
        t_vg = per_call_us(graph.replay, reps=20) / 50
        t_f = per_call_us(lambda: mrs.rod_forces(ctx, rs.rod_off, prm, X, D, 0.1, g, m))
        ua, wa = (u * 1e-3).contiguous(), (w * 1e-3).contiguous()
        t_a = per_call_us(lambda: mrs.rod_advance(ctx, X, D, ua, wa, 1e-7))
        Xs, Ds = torch.from_numpy(rs.X.copy()).to(dev), torch.from_numpy(rs.D.copy()).to(dev)
        mrs.rod_step(ctx, rs.rod_off, prm, Xs, Ds, 0.0, c["dt"], 16, mrs.MRS_EULER)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mrs.rod_step(ctx, rs.rod_off, prm, Xs, Ds, 0.0, c["dt"], 200, mrs.MRS_EULER)
        b.record(stream)
        torch.cuda.synchronize()
        t_s = a.elapsed_time(b) * 1000.0 / 200
        pv, pf, pa = TABLE1_A100_GPU_S[n_rods]
        out["rows"].append({
            "rods": n_rods, "points": N,
            "mrs_velocity_us": t_v, "mrs_velocity_graph_us": t_vg,
            "rod_forces_us": t_f, "rod_advance_us": t_a,
            "rod_step_euler_us_per_step": t_s,
            "paper_gpu_us": {"mrs_velocity": pv * 1e6, "forces": pf * 1e6, "update": pa * 1e6},
            "paper_over_ours": {"mrs_velocity": pv * 1e6 / t_v, "mrs_velocity_graph": pv * 1e6 / t_vg,
                                "forces": pf * 1e6 / t_f,
                                "update": pa * 1e6 / t_a}})
    print(json.dumps(out), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--config", type=int, default=-1,
                    help="force this pair-sum plan configuration (default: the library's choice)")
    ap.add_argument("--case", choices=["main", "rod_kernels", "parareal", "small_systems",
                                       "paper_sizes", "batch", "serve", "parareal_horizon", "fp32_peak",
                                       "large_system"],
                    default="main",
                    help="rod_kernels: time the rod force and update kernels on 1M nodes; "
                         "parareal: the Parareal measurements alone; small_systems: latency of "
                         "one pair sum on single systems of 1k..16k points; paper_sizes: "
                         "per-call latency at the paper's own sizes (1..25 rods of 51 points); "
                         "batch: the 512-system batch alone (--config to skip autotuning); "
                         "serve: the serving measurements alone; parareal_horizon: Parareal "
                         "at 1/--horizon of a beat period against serial fine stepping")
    ap.add_argument("--horizon", type=float, default=16.0,
                    help="parareal_horizon: T = 1/horizon of a beat period (1: the full period)")
    ap.add_argument("--tol", type=float, default=1e-11, help="parareal_horizon: increment tolerance")
    ap.add_argument("--max-iter", dest="max_iter", type=int, default=16,
                    help="parareal_horizon: iteration cap")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local, pg = (1, 0, 0, None)
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    if args.case == "rod_kernels":
        run_rod_kernels(args)
        return
    if args.case == "small_systems":
        run_small_systems(args)
        return
    if args.case == "paper_sizes":
        run_paper_sizes(args)
        return
    if args.case == "batch":
        run_batch_case(args)
        return
    if args.case == "parareal_horizon":
        run_parareal_horizon(args)
        return
    if args.case == "fp32_peak":
        run_fp32_peak(args)
        return
    if args.case == "large_system":
        run_large_system(args)
        return
    if args.case == "serve":
        import torch
        from paper_2604_12083_gb300 import build as B, mrs
        B.build()
        ctx = mrs.Context(0)
        print(json.dumps({"case": "serve", **extra_serve(ctx, torch.device("cuda", 0), full=True)}),
              flush=True)
        ctx.close()
        return
    if args.case == "parareal":
        import torch
        from paper_2604_12083_gb300 import build as B, mrs
        B.build()
        ctx = mrs.Context(0)
        print(json.dumps({"case": "parareal", **extra_parareal(ctx, torch.device("cuda", 0))}), flush=True)
        ctx.close()
        return
    world, rank, local, pg = dist_setup()
    run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
