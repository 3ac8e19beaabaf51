"""Pins of the oracle's Parareal driver (Section II-D, Eqs. initial, intermediate, serial_correct).

For the linear test equation dx/dt = lambda x with exact-exponential F and one-step Euler G the
Parareal iterates have the closed form (Gander & Vandewalle, 2007)
    X^k_n = sum_{j=0}^{min(k,n)} C(n, j) (F - G)^j G^{n-j} x0,
which the driver must reproduce; after k iterations the first k slices equal the serial fine
solution (a structural property of the iteration); on rods the increments fall to round-off.
"""
import math

import numpy as np
import pytest

from oracle import parareal as PR


@pytest.mark.parametrize("lam,N", [(-1.0, 8), (-7.5, 12), (0.6, 6)])
def test_linear_ode_closed_form(lam, N):
    dT = 0.3
    Fs = math.exp(lam * dT)
    Gs = 1.0 + lam * dT
    x0 = np.array([1.7])
    states, _ = PR.run(x0, lambda n, x: Gs * x, lambda n, x: Fs * x, N, N, -1.0,
                       lambda a, b: 1.0)
    for k, X in enumerate(states):
        for n in range(N + 1):
            terms = [math.comb(n, j) * (Fs - Gs) ** j * Gs ** (n - j) * x0[0]
                     for j in range(0, min(k, n) + 1)]
            ref = sum(terms)
            assert abs(X[n][0] - ref) <= 1e-13 * max(1.0, sum(abs(t) for t in terms))
    # k = N: the serial fine solution everywhere
    for n in range(N + 1):
        assert abs(states[-1][n][0] - Fs**n * x0[0]) <= 1e-13 * max(1.0, Fs**n)


def _small_rods(orc, n_rods=2, M=10):
    from paper_2604_12083_gb300 import workloads as W
    rs = W.rod_system(50, n_rods, M, box=1.5)
    p = orc.RodParams.make(1.0, [2e-3] * 3, [0.3] * 3, 0.05, 2 * math.pi, 2 * math.pi)
    return rs, p


def test_rod_parareal_exact_slices_and_convergence(orc):
    rs, p = _small_rods(orc)
    N, dt, r = 6, 1e-4, 4
    T1 = N * 8 * dt
    states, incr = PR.rod_parareal(rs.rod_off, rs.X, rs.D, p, rs.eps, 1.0, 0.0, T1, N, dt, r,
                                   N, -1.0)
    # serial fine solution at every slice end
    ser = [PR.pack_rod_state(rs.X, rs.D)]
    X, D = rs.X, rs.D
    for n in range(1, N + 1):
        X, D = orc.rod_step(rs.rod_off, X, D, p, rs.eps, 1.0, (n - 1) * T1 / N, dt, 8, orc.RK2)
        ser.append(PR.pack_rod_state(X, D))
    for k in range(1, len(states)):
        for n in range(1, k + 1):
            assert np.abs(states[k][n] - ser[n]).max() < 1e-12
    # the true error eta^k (Eq. true_err) falls with k, the increments too
    eta = [PR.max_rel_point_diff(ser, s) for s in states]
    assert eta[-1] < 1e-12
    assert all(eta[k + 1] <= eta[k] * 1.0001 + 1e-15 for k in range(len(eta) - 1))
    assert incr[0] > incr[2]


def test_stopping_on_increment(orc):
    rs, p = _small_rods(orc)
    states, incr = PR.rod_parareal(rs.rod_off, rs.X, rs.D, p, rs.eps, 1.0, 0.0, 4 * 16 * 1e-4,
                                   4, 1e-4, 4, 10, 1e-9)
    assert incr[-1] < 1e-9
    assert all(i >= 1e-9 for i in incr[:-1])
    # frames of every corrected state are orthonormal
    for s in states[-1]:
        _, D = PR.unpack_rod_state(s)
        assert np.abs(np.einsum("kir,kjr->kij", D, D) - np.eye(3)).max() < 1e-13
