"""The debug build (index checks compiled in, MRS_GB300_DEBUG=1) on the GPU, in a process of its
own: on valid inputs no check fires (mrs_device_status stays clear of MRS_FLAG_BOUNDS) and the
results match the FP64 oracle as the release build's do -- a ragged batch through every kernel
configuration, a symmetric plan in many passes, fused and graph rod stepping (both force
kernels), and a served mix."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import oracle
from paper_2604_12083_gb300 import mrs, workloads as W
from test_gpu_mrs import ragged_batch
assert mrs.LIB_PATH.endswith("libmrs_gb300_debug.so"), mrs.LIB_PATH
oracle.build()
ctx = mrs.Context(0)
rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
worst = 0.0
p = ragged_batch()
ur, wr = oracle.mrs_velocity_batch(p.offsets, p.X, p.f, p.n, 0.0, p.mu, eps_per_sys=p.eps)
X, f, n = (torch.from_numpy(a).cuda() for a in (p.X, p.f, p.n))
nz = [s for s in range(len(p.offsets) - 1) if p.offsets[s] < p.offsets[s + 1]]
for pass_bytes in (192 << 20, 3 * 768):
    ctx.set_sym_pass_bytes(pass_bytes)
    configs = [c for c in range(mrs.plan_config_count()) if pass_bytes > 4096 or mrs.plan_config_symmetric(c)]
    for cfg in configs:
        pl = mrs.Plan(ctx, p.offsets, p.mu, 0.0, eps_per_sys=p.eps, precision=mrs.MRS_F32_COMP, config=cfg)
        u, w = torch.full_like(X, float("nan")), torch.full_like(X, float("nan"))
        pl.execute(X, f, n, u, w)
        torch.cuda.synchronize()
        pl.close()
        uu, ww = u.double().cpu().numpy(), w.double().cpu().numpy()
        for s in nz:
            a, b = p.offsets[s], p.offsets[s + 1]
            worst = max(worst, rel(uu[a:b], ur[a:b]), rel(ww[a:b], wr[a:b]))
ctx.set_sym_pass_bytes(192 << 20)
# rod stepping: the fused path, the graph path with the warp-cooperative kernels (and the pair
# sum applying the update) and with one thread per segment, against the oracle
rs = W.rod_system(95, 3, 40, box=2.0)
cfg = dict(W.ROD_PLAIN, a=(2e-3,) * 3, b=(20.0,) * 3)
gp = mrs.RodParams.make(cfg["L"], cfg["a"], cfg["b"], cfg["wave_A"], cfg["wave_k"], cfg["wave_f"], 1.0, rs.eps)
op = oracle.RodParams.make(cfg["L"], cfg["a"], cfg["b"], cfg["wave_A"], cfg["wave_k"], cfg["wave_f"])
Xo, _ = oracle.rod_step(rs.rod_off, rs.X, rs.D, op, rs.eps, 1.0, 0.0, 2e-6, 20, oracle.RK2)
rod_worst = 0.0
for mode, fk in ((2, 0), (0, 0), (0, 1)):
    ctx.set_fused_steps(mode)
    ctx.set_rod_force_kernel(fk)
    Xd, Dd = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
    mrs.rod_step(ctx, rs.rod_off, gp, Xd, Dd, 0.0, 2e-6, 20, mrs.MRS_RK2)
    torch.cuda.synchronize()
    rod_worst = max(rod_worst, rel(Xd.cpu().numpy() - rs.X, Xo - rs.X))
ctx.set_fused_steps(1)
ctx.set_rod_force_kernel(0)
# a small served mix
srv = mrs.Server(ctx, 1 << 30, 16)
q = W.single_system(seed=96, n_fil=4, M=256, box=4.0)
Xq, fq, nq = (torch.from_numpy(a).cuda() for a in (q.X, q.f, q.n))
uq, wq = torch.empty_like(Xq), torch.empty_like(Xq)
t = srv.submit_velocity(Xq, fq, nq, uq, wq, q.mu, float(q.eps[0]))
Xr, Dr = torch.from_numpy(rs.X.copy()).cuda(), torch.from_numpy(rs.D.copy()).cuda()
t2 = srv.submit_rod(rs.rod_off, Xr, Dr, gp, 0.0, 2e-6, 20, mrs.MRS_RK2, 1.0, rs.eps)
srv.drain()
srv.close()
uo, wo = oracle.mrs_velocity(q.X, q.f, q.n, q.eps[0], q.mu)
serve_worst = max(rel(uq.double().cpu().numpy(), uo), rel(wq.double().cpu().numpy(), wo))
flags = ctx.device_status()
ctx.close()
print(json.dumps({"pair_sum_worst": worst, "rod_worst": rod_worst, "serve_worst": serve_worst,
                  "flags": flags}))
'''


def test_debug_build_parity_and_no_false_alarm():
    from paper_2604_12083_gb300 import build as B
    B.build(debug=True)
    env = dict(os.environ, MRS_GB300_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["flags"] == 0, res
    assert res["pair_sum_worst"] < 1e-5 and res["serve_worst"] < 1e-5, res
    assert res["rod_worst"] < 1e-4, res
