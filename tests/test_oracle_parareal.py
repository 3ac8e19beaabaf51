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


# ---------------------------------------------------------------------------------------------
# Eq. true_err (and the increment of the same form) as the oracle computes it, pinned on a
# worked example.  Reading: the maximum over every point of every slice end T_1..T_N (the
# initial state T_0 is the same in every iterate and is left out), positions only, the norm of
# the difference over the norm of the FIRST argument (x^F for eta, x^k for the increment).
#
# Slice end 0 (left out): point 0 differs by (100, 0, 0).
# Slice end 1: A = (3, 4, 0), (0, 0, 2), (1, 2, 2)       |A| = 5, 2, 3
#              B - A = (0.3, 0.4, 0), (0, 0.6, 0.8), (0.2, 0, 0)
#              ratios 0.5 / 5 = 0.1, 1.0 / 2 = 0.5, 0.2 / 3 = 0.0667
# Slice end 2: A = (6, 8, 0), (0, 2, 0), (2, 1, 2)       |A| = 10, 2, 3
#              B - A = (0, 0, 3), (0, 0.9, 0), (0, 0, 0)
#              ratios 0.3, 0.45, 0
# Frame columns (3..11) differ by 50 everywhere and are not positions.
# eta = 0.5 (slice end 1, point 1).  With |B| as the denominator it would be 1/sqrt(8.2) =
# 0.349; an L2 norm over all points and slice ends (sqrt(sum num^2) / sqrt(sum den^2)) gives
# sqrt(0.25+1+0.04+9+0.81) / sqrt(25+4+9+100+4+9) = 0.271; slice end 0 included, 20.
# ---------------------------------------------------------------------------------------------

def _true_err_example():
    a0 = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 2.0], [1.0, 2.0, 2.0]])
    a1 = a0.copy()
    a2 = np.array([[6.0, 8.0, 0.0], [0.0, 2.0, 0.0], [2.0, 1.0, 2.0]])
    b0 = a0 + np.array([[100.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    b1 = a1 + np.array([[0.3, 0.4, 0.0], [0.0, 0.6, 0.8], [0.2, 0.0, 0.0]])
    b2 = a2 + np.array([[0.0, 0.0, 3.0], [0.0, 0.9, 0.0], [0.0, 0.0, 0.0]])

    def with_frames(x, shift):
        return np.concatenate([x, np.full((3, 9), shift)], axis=1)

    XA = [with_frames(a, 1.0) for a in (a0, a1, a2)]
    XB = [with_frames(b, 51.0) for b in (b0, b1, b2)]
    return XA, XB


def pin_true_err(fn=PR.max_rel_point_diff):
    XA, XB = _true_err_example()
    assert abs(fn(XA, XB) - 0.5) < 1e-15
    # identical iterates: zero
    assert fn(XA, XA) == 0.0


def test_true_err_worked_example():
    pin_true_err()


# ---------------------------------------------------------------------------------------------
# Reading R10: after the additive correction, frames are replaced by their polar factor
# D (D^T D)^{-1/2}, the rotation nearest to D in the Frobenius norm.  Pinned by the uniqueness
# of the polar decomposition (D = Q S with Q a rotation and S symmetric positive-definite gives
# back exactly Q), by R^T D being symmetric positive-definite, and by nearness: no other
# rotation (a QR or Gram-Schmidt factor, small rotations of R) is closer to D.
# ---------------------------------------------------------------------------------------------

def _rot(axis, angle):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def _spd(rng, spread):
    V = _rot(rng.standard_normal(3), rng.uniform(0, math.pi))
    return V @ np.diag(1.0 + spread * rng.uniform(-1, 1, 3)) @ V.T


def _qr_rotation(D):
    Q, R = np.linalg.qr(D)
    return Q * np.sign(np.diag(R))


def pin_polar(fn=PR.polar_orthonormalize):
    rng = np.random.default_rng(11)
    Qs = np.stack([_rot(rng.standard_normal(3), rng.uniform(0.1, 3.0)) for _ in range(16)])
    Ss = np.stack([_spd(rng, s) for s in np.linspace(1e-6, 0.3, 16)])
    D = np.einsum("kij,kjl->kil", Qs, Ss)
    R = fn(D)
    # uniqueness of the polar decomposition: the rotation factor comes back
    assert np.abs(R - Qs).max() < 1e-13
    for k in range(len(D)):
        M = R[k].T @ D[k]
        assert np.abs(M - M.T).max() < 1e-13                      # R^T D symmetric
        assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0.0    # ... and positive-definite
        assert abs(np.linalg.det(R[k]) - 1.0) < 1e-13
        dist = np.linalg.norm(D[k] - R[k])
        assert dist <= np.linalg.norm(D[k] - _qr_rotation(D[k])) + 1e-14
        assert dist <= np.linalg.norm(D[k] - _qr_rotation(D[k].T).T) + 1e-14
        for _ in range(8):
            Rp = R[k] @ _rot(rng.standard_normal(3), 1e-3)
            assert dist < np.linalg.norm(D[k] - Rp)


def test_polar_factor_is_nearest_rotation():
    pin_polar()


def _gram_schmidt_rows(D):
    out = np.empty_like(D)
    for k in range(len(D)):
        e1 = D[k, 0] / np.linalg.norm(D[k, 0])
        v = D[k, 1] - (D[k, 1] @ e1) * e1
        e2 = v / np.linalg.norm(v)
        out[k] = np.stack([e1, e2, np.cross(e1, e2)])
    return out


PARAREAL_HELPER_MUTANTS = {
    # Eq. true_err
    "true_err_includes_slice_0": ("err", lambda XA, XB: max(
        float(np.max(np.linalg.norm(np.asarray(a)[:, :3] - np.asarray(b)[:, :3], axis=1)
                     / np.linalg.norm(np.asarray(a)[:, :3], axis=1))) for a, b in zip(XA, XB))),
    "true_err_l2_over_points": ("err", lambda XA, XB: float(
        np.sqrt(sum(np.sum((np.asarray(a)[:, :3] - np.asarray(b)[:, :3]) ** 2)
                    for a, b in zip(XA[1:], XB[1:])))
        / np.sqrt(sum(np.sum(np.asarray(a)[:, :3] ** 2) for a in XA[1:])))),
    "true_err_other_denominator": ("err", lambda XA, XB: PR.max_rel_point_diff(XB, XA)),
    "true_err_all_columns": ("err", lambda XA, XB: PR.max_rel_point_diff(XA, XB, slice(0, 12))),
    # reading R10
    "polar_by_qr": ("polar", lambda D: np.stack([_qr_rotation(d) for d in D])),
    "polar_by_gram_schmidt": ("polar", _gram_schmidt_rows),
    "polar_transposed": ("polar", lambda D: np.swapaxes(PR.polar_orthonormalize(D), -1, -2)),
    "polar_row_normalise": ("polar", lambda D: D / np.linalg.norm(D, axis=2, keepdims=True)),
}


@pytest.mark.parametrize("name", sorted(PARAREAL_HELPER_MUTANTS))
def test_parareal_helper_mutant_is_caught(name):
    kind, fn = PARAREAL_HELPER_MUTANTS[name]
    pin = pin_true_err if kind == "err" else pin_polar
    with pytest.raises(AssertionError):
        pin(fn)
