"""Usage example: pair sum, rod stepping, Parareal and serving through the Python binding.

Run from the repository root after building (``python -c "import __graft_entry__ as g;
g.build()"``): ``python examples/usage.py``.  ``run()`` returns the objects it made so that a
test can check them.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def run():
    import torch
    from paper_2604_12083_gb300 import mrs, workloads

    ctx = mrs.Context(0)
    p = workloads.single_system()                        # 32 filaments x 1024 nodes
    X, f, n = (torch.from_numpy(a).cuda() for a in (p.X, p.f, p.n))
    u, w = torch.empty_like(X), torch.empty_like(X)
    mrs.mrs_velocity(ctx, p.offsets, X, f, n, u, w, mu=1.0, eps=float(p.eps[0]),
                     precision=mrs.MRS_F32_COMP)         # u, w: linear and angular velocities

    # Kirchhoff rods coupled through the pair sum: 8 filaments x 512 nodes, 100 RK2 steps
    rs = workloads.rod_system(4, 8, 512)
    c = workloads.ROD_PARAREAL
    prm = mrs.RodParams.make(c["L"], c["a"], c["b"], c["wave_A"], c["wave_k"], c["wave_f"],
                             1.0, rs.eps)                # mu = 1; lj_eps=... adds the LJ repulsion
    Xr, Dr = torch.from_numpy(rs.X).cuda(), torch.from_numpy(rs.D).cuda()
    mrs.rod_step(ctx, rs.rod_off, prm, Xr, Dr, 0.0, c["dt"], 100, mrs.MRS_RK2)

    # Parareal: 64 slices of 16 fine RK2 steps, coarse Euler at 4 dt, pipelined in groups of 8
    st = mrs.parareal_run(ctx, rs.rod_off, prm, Xr, Dr, 0.0, 64 * 16 * c["dt"], 64, c["dt"], 4,
                          8, 1e-11, group_size=8)
    print(st.iterations, st.final_incr)

    # serving: jobs of any size submitted as they arrive, continuously batched on the GPU
    srv = mrs.Server(ctx, 8 << 30, 64)                   # memory budget, slots
    ticket = srv.submit_velocity(X, f, n, u, w, 1.0, float(p.eps[0]))
    srv.drain()
    done, latency_s = srv.poll(ticket)
    srv.close()
    return dict(ctx=ctx, u=u, w=w, Xr=Xr, st=st, done=done, latency_s=latency_s)


if __name__ == "__main__":
    out = run()
    out["ctx"].close()
