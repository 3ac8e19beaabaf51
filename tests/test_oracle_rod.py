"""Pins of the oracle's rod forces (Sections II-A, II-B) and time stepping (Section III-C-3).

The force pin is exact: g_k = -dE/dX_k for the discrete elastic energy
E = sum_seg ds [ 1/2 sum_j b_j (e.D^j_{k+1/2} - delta_3j)^2 + 1/2 sum_i a_i (kappa_i - Omega_i)^2 ],
which this file builds on its own with scipy.linalg.sqrtm for the mid-segment frame.  The
torque is checked against -dE/d(rotation of one node frame), which the discrete balance
reproduces to first order in the angle between neighbouring frames.
"""
import math

import numpy as np
import pytest
from scipy.linalg import sqrtm
from scipy.spatial.transform import Rotation

from paper_2604_12083_gb300 import workloads as W


def params(orc, a=1.0, b=1.0, A=0.05, f=2 * math.pi, L=1.0):
    return orc.RodParams.make(L, [a, a, a], [b, b, b], A, 2 * math.pi, f)


def energy(X, D, p, t, ds):
    """Discrete elastic energy of one rod (independent of the oracle; sqrtm from scipy)."""
    E = 0.0
    for k in range(X.shape[0] - 1):
        A = sum(np.outer(D[k + 1, j], D[k, j]) for j in range(3))
        S = np.real(sqrtm(A))
        Dh = (S @ D[k].T).T
        e = (X[k + 1] - X[k]) / ds
        s = (k + 0.5) * ds
        Om = np.array([0.0, -p.wave_k**2 * p.wave_A * math.sin(p.wave_k * s + p.wave_f * t), 0.0])
        for j in range(3):
            E += 0.5 * ds * p.b[j] * (e @ Dh[j] - (1.0 if j == 2 else 0.0)) ** 2
        for i in range(3):
            j, l = (i + 1) % 3, (i + 2) % 3
            kap = (D[k + 1, j] - D[k, j]) / ds @ Dh[l]
            E += 0.5 * ds * p.a[i] * (kap - Om[i]) ** 2
    return E


def perturbed_rod(M, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    X, D = W.sinusoid_filament(M)
    X = X + amp * rng.standard_normal(X.shape) / M
    R = Rotation.from_rotvec(amp * rng.standard_normal((M, 3))).as_matrix()
    D = np.einsum("krc,kic->kir", R, D)
    return X, D


def test_force_is_minus_energy_gradient(orc):
    M = 12
    X, D = perturbed_rod(M, 40)
    p = params(orc, a=0.7, b=3.0)
    ds = 1.0 / (M - 1)
    t = 0.3
    g, m = orc.rod_forces([0, M], X, D, p, t)
    h = 1e-6
    for k in range(M):
        for c in range(3):
            Xp = X.copy()
            Xp[k, c] += h
            Xm = X.copy()
            Xm[k, c] -= h
            dE = (energy(Xp, D, p, t, ds) - energy(Xm, D, p, t, ds)) / (2 * h)
            assert abs(-dE - g[k, c]) < 1e-7 * np.abs(g).max()


def test_torque_is_minus_energy_rotation_derivative(orc):
    M = 40
    X, D = perturbed_rod(M, 41, amp=0.01)
    p = params(orc, a=1.0, b=1.0)
    ds = 1.0 / (M - 1)
    g, m = orc.rod_forces([0, M], X, D, p, 0.0)
    h = 1e-6
    err, ref = [], []
    for k in range(1, M - 1):
        for c in range(3):
            a = np.zeros(3)
            a[c] = 1.0
            Dp = D.copy()
            Dm = D.copy()
            Dp[k] = D[k] @ Rotation.from_rotvec(h * a).as_matrix().T
            Dm[k] = D[k] @ Rotation.from_rotvec(-h * a).as_matrix().T
            dE = (energy(X, Dp, p, 0.0, ds) - energy(X, Dm, p, 0.0, ds)) / (2 * h)
            err.append(-dE - m[k, c])
            ref.append(m[k, c])
    err, ref = np.array(err), np.array(ref)
    # first order in the neighbour angle (~ curvature * ds ~ 0.05 here)
    assert np.linalg.norm(err) < 0.1 * np.linalg.norm(ref)


def test_total_force_and_torque_vanish(orc):
    rs = W.rod_system(42, 3, 33)
    X, D = rs.X.copy(), rs.D.copy()
    rng = np.random.default_rng(42)
    X += 1e-3 * rng.standard_normal(X.shape)
    g, m = orc.rod_forces(rs.rod_off, X, D, params(orc, a=0.5, b=7.0), 0.2)
    for r in range(3):
        sl = slice(rs.rod_off[r], rs.rod_off[r + 1])
        scale = np.abs(g[sl]).max() * 10 + np.abs(m[sl]).max()
        assert np.abs(g[sl].sum(axis=0)).max() < 1e-12 * scale
        tot = m[sl].sum(axis=0) + np.cross(X[sl], g[sl]).sum(axis=0)
        assert np.abs(tot).max() < 1e-11 * scale


def test_straight_unstressed_rod_is_force_free(orc):
    M = 17
    X = np.zeros((M, 3))
    X[:, 2] = np.linspace(0.0, 1.0, M)
    D = np.tile(np.eye(3), (M, 1, 1))
    g, m = orc.rod_forces([0, M], X, D, params(orc, A=0.0), 0.0)
    assert np.abs(g).max() < 1e-13 and np.abs(m).max() < 1e-13


def test_initial_sinusoid_forces_vanish_at_second_order(orc):
    """The initial configuration (reading R6): nodes evenly spaced in arclength on the unit
    sinusoid, D3 its tangent.  Shear and stretch then vanish up to the midpoint rule's O(ds^2)
    error, so the point forces g_k = -f_k ds shrink like ds^2 at the free ends and like ds^3
    inside (force densities O(ds^2)) under refinement.  The forces do not depend on the
    preferred curvature, so this holds at any time."""
    p = params(orc, a=0.02, b=140.0)
    g_in, g_all = [], []
    for M in (65, 129, 257):
        X, D = W.sinusoid_filament(M)
        for t in (0.0, 0.1):
            g, _ = orc.rod_forces([0, M], X, D, p, t)
            if t == 0.0:
                g_in.append(np.abs(g[1:-1]).max())
                g_all.append(np.abs(g).max())
            else:
                assert np.array_equal(np.abs(g).max(), g_all[-1])
    for a, b in zip(g_in, g_in[1:]):
        assert math.log2(a / b) > 2.8, g_in
    for a, b in zip(g_all, g_all[1:]):
        assert math.log2(a / b) > 1.8, g_all


def test_objectivity(orc):
    X, D = perturbed_rod(25, 43)
    p = params(orc, a=0.3, b=2.0)
    g, m = orc.rod_forces([0, 25], X, D, p, 0.1)
    Q = W.haar_rotation(np.random.default_rng(43))
    g2, m2 = orc.rod_forces([0, 25], X @ Q.T + 5.0, np.einsum("rc,kic->kir", Q, D), p, 0.1)
    np.testing.assert_allclose(g2, g @ Q.T, atol=1e-11 * np.abs(g).max())
    np.testing.assert_allclose(m2, m @ Q.T, atol=1e-11 * np.abs(m).max())


def test_energy_decreases_under_euler_flow(orc):
    """With a time-independent preferred strain the dynamics are a gradient flow with a PSD
    mobility, so small Euler steps lower the elastic energy (a sign error in g or m raises it)."""
    M = 24
    X, D = perturbed_rod(M, 44, amp=0.05)
    p = params(orc, a=1e-3, b=1.0, f=0.0)
    ds = 1.0 / (M - 1)
    eps = 1.5 * ds
    E0 = energy(X, D, p, 0.0, ds)
    for _ in range(5):
        X, D = orc.rod_step([0, M], X, D, p, eps, 1.0, 0.0, 1e-4, 1, orc.EULER)
        E1 = energy(X, D, p, 0.0, ds)
        assert E1 < E0
        E0 = E1


def test_frames_stay_orthonormal(orc):
    M = 16
    X, D = perturbed_rod(M, 45)
    p = params(orc, a=1e-3, b=0.5)
    X, D = orc.rod_step([0, M], X, D, p, 1.5 / (M - 1), 1.0, 0.0, 1e-5, 10000, orc.RK2)
    err = np.abs(np.einsum("kir,kjr->kij", D, D) - np.eye(3)).max()
    # 10^4 RK2 steps = 2 x 10^4 exact rotations: only rounding drift (below 1e-16 per update;
    # 6.8e-13 here); a scheme that is not an exact rotation would drift by ~(|omega| dt)^2 per
    # update, orders of magnitude more
    assert err < 20000 * 1.25e-16


def test_rodrigues_update_matches_library_rotation(orc):
    """Eq. newD rotates each director by |omega| dt about omega (scipy's rotation-vector map)."""
    rng = np.random.default_rng(47)
    N = 50
    D = np.einsum("krc,kic->kir", Rotation.random(N, random_state=1).as_matrix(),
                  np.tile(np.eye(3), (N, 1, 1)))
    w = rng.standard_normal((N, 3)) * 10.0
    w[3] = 0.0                                   # zero angular velocity: frame unchanged
    dt = 0.037
    out = orc.rodrigues_update(D, w, dt)
    ref = np.einsum("krc,kic->kir", Rotation.from_rotvec(w * dt).as_matrix(), D)
    np.testing.assert_allclose(out, ref, atol=2e-15)
    assert np.array_equal(out[3], D[3])


def test_static_rod_stays_put(orc):
    """A straight unstressed rod with no preferred curvature is force free and does not move."""
    M = 5
    X = np.zeros((M, 3))
    X[:, 0] = np.linspace(0, 1, M)
    D = np.tile(np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]), (M, 1, 1))
    X2, D2 = orc.rod_step([0, M], X, D, params(orc, A=0.0), 0.3, 1.0, 0.0, 1e-3, 3, orc.RK2)
    assert np.array_equal(X2, X) and np.array_equal(D2, D)


@pytest.mark.parametrize("scheme,order", [(0, 1), (1, 2)])
def test_convergence_order(orc, scheme, order):
    M = 12
    X, D = perturbed_rod(M, 46, amp=0.05)
    ds = 1.0 / (M - 1)
    eps = 1.5 * ds
    p = params(orc, a=2e-3, b=0.2)
    T = 2e-3
    Xr, _ = orc.rod_step([0, M], X, D, p, eps, 1.0, 0.0, T / 1024, 1024, orc.RK2)
    errs = []
    for nst in (32, 64, 128):
        Xs, _ = orc.rod_step([0, M], X, D, p, eps, 1.0, 0.0, T / nst, nst, scheme)
        errs.append(np.abs(Xs - Xr).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    target = 2.0**order
    assert abs(r1 - target) < 0.25 * target and abs(r2 - target) < 0.2 * target, (errs, r1, r2)


def _lj_energy(X, rod_id, sigma, e_lj):
    """Total cut LJ energy over pairs of nodes on different rods (independent of the oracle)."""
    rc = 2.0 ** (1.0 / 6.0) * sigma
    E = 0.0
    for i in range(len(X)):
        for j in range(i + 1, len(X)):
            if rod_id[i] == rod_id[j]:
                continue
            r = np.linalg.norm(X[i] - X[j])
            if r < rc:
                E += 4 * e_lj * ((sigma / r) ** 12 - (sigma / r) ** 6) + e_lj   # shifted: 0 at r_c
    return E


def test_lj_force_is_minus_energy_gradient(orc):
    rng = np.random.default_rng(48)
    X = rng.uniform(0, 0.6, (30, 3))
    rid = np.repeat(np.arange(6), 5)
    sigma, e_lj = 0.12, 0.7
    F = orc.lj_forces(X, rid, sigma, e_lj)
    h = 1e-7
    for i in range(len(X)):
        for c in range(3):
            Xp = X.copy()
            Xp[i, c] += h
            Xm = X.copy()
            Xm[i, c] -= h
            dE = (_lj_energy(Xp, rid, sigma, e_lj) - _lj_energy(Xm, rid, sigma, e_lj)) / (2 * h)
            assert abs(-dE - F[i, c]) <= 1e-5 * max(1.0, np.abs(F).max())
    assert np.abs(F.sum(axis=0)).max() <= 1e-10 * np.abs(F).max()          # action = reaction
    assert np.abs(F).max() > 0


def test_lj_cut_and_same_rod_exclusion(orc):
    sigma = 0.1
    rc = 2.0 ** (1.0 / 6.0) * sigma
    X = np.array([[0.0, 0, 0], [rc * (1 + 1e-9), 0, 0], [0.0, 0.5 * sigma, 0]])
    F = orc.lj_forces(X, [0, 1, 0], sigma, 1.0)
    assert np.all(F == 0.0)          # beyond r_c, or on the same rod
    # just inside r_c the force is tiny (continuous at the cut), and repulsive
    X[1, 0] = rc * (1 - 1e-6)
    F = orc.lj_forces(X, [0, 1, 0], sigma, 1.0)
    assert F[1, 0] > 0 and F[1, 0] < 1e-3
