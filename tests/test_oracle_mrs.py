"""Pins of the oracle's MRS pair sum (Section II-C) against what the mathematics fixes.

None of these re-types the oracle's H1..H5: the oracle is checked against the Stokes
equations with the paper's blob as forcing, against omega = (1/2) curl u, against the
textbook singular Stokeslet / rotlet / dipole far fields, and against symmetry, positive
semi-definiteness and the equivariances of the mobility operator.
"""
import math

import numpy as np
import pytest
from scipy import integrate

PI = math.pi


def blob(r, eps):
    """phi_eps(r) = 15 eps^4 / (8 pi (r^2 + eps^2)^{7/2})  (Section II-C)."""
    return 15.0 * eps**4 / (8.0 * PI * (r * r + eps * eps) ** 3.5)


def test_blob_integrates_to_one():
    for eps in (0.01, 0.3, 2.0):
        val, _ = integrate.quad(lambda r: 4 * PI * r * r * blob(r, eps), 0, np.inf)
        assert abs(val - 1.0) < 1e-10


def _stencil_points(x0, h):
    """x0 plus +-h, +-2h along each axis (order: centre, then axis a, offsets -2,-1,1,2)."""
    pts = [x0]
    for a in range(3):
        for o in (-2, -1, 1, 2):
            p = x0.copy()
            p[a] += o * h
            pts.append(p)
    return np.array(pts)


def _fd(vals, h):
    """First derivatives J[a] = d/dx_a and second derivatives Q[a] = d^2/dx_a^2 (4th order)."""
    c = vals[0]
    J, Q = [], []
    for a in range(3):
        m2, m1, p1, p2 = vals[1 + 4 * a: 5 + 4 * a]
        J.append((-p2 + 8 * p1 - 8 * m1 + m2) / (12 * h))
        Q.append((-p2 + 16 * p1 - 30 * c + 16 * m1 - m2) / (12 * h * h))
    return np.array(J), np.array(Q)


def _field(orc, x_targets, f, n, eps, mu=1.0):
    X = np.zeros((1, 3))
    return orc.mrs_velocity(X, np.array([f]), np.array([n]), eps, mu, xt=x_targets)


@pytest.mark.parametrize("rfac", [0.0, 0.3, 1.0, 3.0])
def test_stokeslet_solves_regularized_stokes(orc, rfac):
    """u from a point force f at 0 satisfies mu Lap u - grad p + f phi_eps = 0 and div u = 0,
    with the regularized pressure p = (f.x)(2r^2+5eps^2) / (8 pi (r^2+eps^2)^{5/2})."""
    rng = np.random.default_rng(10)
    eps, mu = 0.1, 1.7
    f = rng.standard_normal(3)
    d = rng.standard_normal(3)
    x0 = rfac * eps * d / np.linalg.norm(d)
    h = eps / 320.0          # 4th-order stencil: the residual falls 16x per halving of h
    P = _stencil_points(x0, h)
    u, _ = _field(orc, P, f, np.zeros(3), eps, mu)
    J, Q = _fd(u, h)
    lap = Q.sum(axis=0)

    def pressure(x):
        r2 = x @ x
        return (f @ x) * (2 * r2 + 5 * eps**2) / (8 * PI * (r2 + eps**2) ** 2.5)

    pv = np.array([pressure(p) for p in P])
    Jp, _ = _fd(pv[:, None], h)
    gradp = Jp[:, 0]
    res = mu * lap - gradp + f * blob(np.linalg.norm(x0), eps)
    scale = np.linalg.norm(f) * blob(0.0, eps)
    assert np.linalg.norm(res) < 1e-8 * scale
    div = np.trace(J)
    assert abs(div) < 1e-8 * np.linalg.norm(u[0]) / eps


@pytest.mark.parametrize("rfac", [0.0, 0.5, 1.0, 4.0])
def test_angular_velocity_is_half_curl(orc, rfac):
    """omega = (1/2) curl u for the full field of a point force AND a point torque."""
    rng = np.random.default_rng(11)
    eps = 0.05
    f = rng.standard_normal(3)
    n = rng.standard_normal(3)
    d = rng.standard_normal(3)
    x0 = rfac * eps * d / np.linalg.norm(d)
    h = eps / 320.0
    P = _stencil_points(x0, h)
    u, w = _field(orc, P, f, n, eps)
    J, _ = _fd(u, h)                    # J[a, c] = d u_c / d x_a
    curl = np.array([J[1, 2] - J[2, 1], J[2, 0] - J[0, 2], J[0, 1] - J[1, 0]])
    wscale = np.linalg.norm(w[0])
    assert np.linalg.norm(0.5 * curl - w[0]) < 1e-8 * wscale
    # each half separately: force part and torque part
    for ff, nn in ((f, 0 * n), (0 * f, n)):
        u, w = _field(orc, P, ff, nn, eps)
        J, _ = _fd(u, h)
        curl = np.array([J[1, 2] - J[2, 1], J[2, 0] - J[0, 2], J[0, 1] - J[1, 0]])
        assert np.linalg.norm(0.5 * curl - w[0]) < 1e-8 * wscale


def _singular(x, f, n, mu=1.0):
    """Textbook singular kernels: Stokeslet, rotlet, and omega = (1/2) curl of each."""
    R = np.linalg.norm(x)
    u = (f / R + (f @ x) * x / R**3) / (8 * PI * mu) + np.cross(n, x) / (8 * PI * mu * R**3)
    w = np.cross(f, x) / (8 * PI * mu * R**3) + (-n / R**3 + 3 * (n @ x) * x / R**5) / (16 * PI * mu)
    return u, w


def test_far_field_recovers_singular_kernels(orc):
    """r >> eps: the regularized kernels approach the singular Stokeslet (relative deviation
    ~ (eps/r)^2) and the rotlet and dipole couplings, whose O((eps/r)^2) correction cancels
    (relative deviation ~ (eps/r)^4)."""
    rng = np.random.default_rng(12)
    eps = 0.01
    f = rng.standard_normal(3)
    n = rng.standard_normal(3)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    dev = {}
    for fac in (10.0, 100.0, 1000.0):
        x = fac * eps * d
        u, w = _field(orc, x[None, :], f, 0 * n, eps)
        us, ws = _singular(x, f, 0 * n)
        dev[fac, "stokeslet"] = np.linalg.norm(u[0] - us) / np.linalg.norm(us)
        dev[fac, "f->omega"] = np.linalg.norm(w[0] - ws) / np.linalg.norm(ws)
        u, w = _field(orc, x[None, :], 0 * f, n, eps)
        us, ws = _singular(x, 0 * f, n)
        dev[fac, "rotlet"] = np.linalg.norm(u[0] - us) / np.linalg.norm(us)
        dev[fac, "dipole"] = np.linalg.norm(w[0] - ws) / np.linalg.norm(ws)
    for fac in (10.0, 100.0, 1000.0):
        assert dev[fac, "stokeslet"] < (1 / fac) ** 2
        for k in ("f->omega", "rotlet", "dipole"):
            assert dev[fac, k] < 10 * (1 / fac) ** 4
    assert 70 < dev[10.0, "stokeslet"] / dev[100.0, "stokeslet"] < 130
    for k in ("f->omega", "rotlet", "dipole"):
        assert 7e3 < dev[10.0, k] / dev[100.0, k] < 1.3e4


def test_self_term_closed_form(orc):
    """Single point: u = f/(4 pi mu eps), omega = 5 n /(16 pi mu eps^3) (the r -> 0 limits)."""
    eps, mu = 0.02, 2.0
    f = np.array([0.3, -1.2, 0.7])
    n = np.array([-0.5, 0.25, 1.5])
    u, w = orc.mrs_velocity(np.zeros((1, 3)), f[None], n[None], eps, mu)
    np.testing.assert_allclose(u[0], f / (4 * PI * mu * eps), rtol=1e-14)
    np.testing.assert_allclose(w[0], 5 * n / (16 * PI * mu * eps**3), rtol=1e-14)


def _mobility(orc, X, eps):
    N = X.shape[0]
    M = np.zeros((6 * N, 6 * N))
    z = np.zeros((N, 3))
    for j in range(N):
        for c in range(6):
            f = z.copy()
            n = z.copy()
            (f if c < 3 else n)[j, c % 3] = 1.0
            u, w = orc.mrs_velocity(X, f, n, eps)
            out = np.concatenate([u, w], axis=1).reshape(-1)
            M[:, 6 * j + c] = out
    return M


@pytest.mark.parametrize("kind,ratio", [("rod", 0.3), ("rod", 1.5), ("rod", 4.0), ("random", 1.5)])
def test_mobility_symmetric_psd(orc, kind, ratio):
    from paper_2604_12083_gb300 import workloads as W
    N = 40
    if kind == "rod":
        X, _ = W.sinusoid_filament(N)
        eps = ratio / (N - 1)
    else:
        X = np.random.default_rng(13).uniform(0, 0.5, (N, 3))
        eps = ratio * 0.05
    M = _mobility(orc, X, eps)
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.min() >= -1e-12 * ev.max()
    # Stokeslet block alone: f . u >= 0 for any forces
    S = M.reshape(N, 6, N, 6)[:, :3, :, :3].reshape(3 * N, 3 * N)
    rng = np.random.default_rng(14)
    for _ in range(20):
        f = rng.standard_normal(3 * N)
        assert f @ S @ f >= 0.0


def test_equivariances(orc):
    rng = np.random.default_rng(15)
    N, eps = 64, 0.04
    X = rng.uniform(0, 1, (N, 3))
    f = rng.standard_normal((N, 3))
    n = rng.standard_normal((N, 3))
    u, w = orc.mrs_velocity(X, f, n, eps)
    tol = 1e-11

    def close(a, b):
        return np.abs(a - b).max() <= tol * np.abs(b).max()

    # translation
    u2, w2 = orc.mrs_velocity(X + np.array([3.0, -2.0, 5.0]), f, n, eps)
    assert close(u2, u) and close(w2, w)
    # rotation (proper): every vector and pseudovector rotates
    from paper_2604_12083_gb300.workloads import haar_rotation
    Q = haar_rotation(rng)
    u2, w2 = orc.mrs_velocity(X @ Q.T, f @ Q.T, n @ Q.T, eps)
    assert close(u2, u @ Q.T) and close(w2, w @ Q.T)
    # permutation
    p = rng.permutation(N)
    u2, w2 = orc.mrs_velocity(X[p], f[p], n[p], eps)
    assert close(u2, u[p]) and close(w2, w[p])
    # linearity
    f2 = rng.standard_normal((N, 3))
    n2 = rng.standard_normal((N, 3))
    ua, wa = orc.mrs_velocity(X, f2, n2, eps)
    ub, wb = orc.mrs_velocity(X, 2 * f - 3 * f2, 2 * n - 3 * n2, eps)
    assert close(ub, 2 * u - 3 * ua) and close(wb, 2 * w - 3 * wa)
    # scaling (x, eps, n) -> (lam x, lam eps, lam n): u -> u/lam, omega -> omega/lam^2
    lam = 2.5
    u2, w2 = orc.mrs_velocity(lam * X, f, lam * n, lam * eps)
    assert close(u2, u / lam) and close(w2, w / lam**2)
    # viscosity
    u2, w2 = orc.mrs_velocity(X, f, n, eps, mu=4.0)
    assert close(u2, u / 4.0) and close(w2, w / 4.0)


def test_batch_is_independent_systems(orc):
    from paper_2604_12083_gb300 import workloads as W
    p = W.batch_systems(seed=30, n_sys=5, lo_exp=8, hi_exp=9.5)
    eps = p.eps.copy()
    eps[2] *= 2.0
    u, w = orc.mrs_velocity_batch(p.offsets, p.X, p.f, p.n, 0.0, p.mu, eps_per_sys=eps)
    for s in range(5):
        a, b = p.offsets[s], p.offsets[s + 1]
        us, ws = orc.mrs_velocity(p.X[a:b], p.f[a:b], p.n[a:b], eps[s], p.mu)
        assert np.array_equal(us, u[a:b]) and np.array_equal(ws, w[a:b])


def test_two_point_brute_force_matches_superposition(orc):
    """Superposition (Eq. superposition): the sum over sources equals the sum of one-source fields."""
    rng = np.random.default_rng(16)
    X = rng.uniform(0, 0.2, (7, 3))
    f = rng.standard_normal((7, 3))
    n = rng.standard_normal((7, 3))
    eps = 0.03
    u, w = orc.mrs_velocity(X, f, n, eps)
    us = np.zeros_like(u)
    ws = np.zeros_like(w)
    for j in range(7):
        a, b = orc.mrs_velocity(X[j:j + 1], f[j:j + 1], n[j:j + 1], eps, xt=X)
        us += a
        ws += b
    np.testing.assert_allclose(u, us, rtol=1e-12, atol=1e-12 * np.abs(u).max())
    np.testing.assert_allclose(w, ws, rtol=1e-12, atol=1e-12 * np.abs(w).max())


def _symbolic_fields():
    """The paper's regularized Stokeslet (H1, H2 of its cited source) and blob, Section II-C;
    the other three couplings derived from it: the velocity of a point torque n is
    (1/2) curl of the Stokeslet of n, and omega = (1/2) curl u (Eq. angular_velocity_field).
    Returns the symbols and u_f, omega_f, u_n, omega_n, the Stokes residual and div u."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    e = sp.symbols("epsilon", positive=True)
    f = sp.Matrix(sp.symbols("f1:4", real=True))
    n = sp.Matrix(sp.symbols("n1:4", real=True))
    X = sp.Matrix([x, y, z])
    r2 = x**2 + y**2 + z**2
    d = r2 + e**2
    H1 = (r2 + 2 * e**2) / (8 * sp.pi * d**sp.Rational(3, 2))
    H2 = 1 / (8 * sp.pi * d**sp.Rational(3, 2))
    phi = 15 * e**4 / (8 * sp.pi * d**sp.Rational(7, 2))
    stokeslet = lambda F: F * H1 + F.dot(X) * X * H2
    pressure = lambda F: F.dot(X) * (2 * r2 + 5 * e**2) / (8 * sp.pi * d**sp.Rational(5, 2))
    grad = lambda s: sp.Matrix([sp.diff(s, c) for c in (x, y, z)])
    lap = lambda v: sp.Matrix([sum(sp.diff(v[i], c, 2) for c in (x, y, z)) for i in range(3)])
    curl = lambda v: sp.Matrix([sp.diff(v[2], y) - sp.diff(v[1], z),
                                sp.diff(v[0], z) - sp.diff(v[2], x),
                                sp.diff(v[1], x) - sp.diff(v[0], y)])
    u_f = stokeslet(f)
    resid = lap(u_f) - grad(pressure(f)) + f * phi           # mu = 1
    div = sum(sp.diff(u_f[i], c) for i, c in enumerate((x, y, z)))
    u_n = curl(stokeslet(n)) / 2
    return sp, (x, y, z, e, f, n, d), u_f, curl(u_f) / 2, u_n, curl(u_n) / 2, resid, div


def test_symbolic_stokes_residual_and_divergence():
    """Pin (i): the Stokeslet with the paper's blob as forcing solves the regularized Stokes
    equations mu Lap u - grad p + f phi_eps = 0 and div u = 0 exactly (symbolic algebra)."""
    sp, (x, y, z, e, f, n, d), *_, resid, div = _symbolic_fields()
    for c in resid:
        assert sp.simplify(c * d**sp.Rational(9, 2)) == 0
    assert sp.simplify(div) == 0


@pytest.mark.parametrize("point", [("0", "0", "0"), ("1/3", "1/5", "-1/7"), ("1", "2", "-3"),
                                   ("25/2", "-9", "31/4")])
def test_two_point_case_exact(orc, point):
    """Pin (vii): one source at the origin with rational f, n and eps, one target at a rational
    point (at the source, at a few eps, in the far field), mu = 7/3; the oracle's four
    couplings match the symbolically derived fields evaluated to 30 digits, divided by mu."""
    sp, (x, y, z, e, f, n, d), u_f, w_f, u_n, w_n, *_ = _symbolic_fields()
    eps = sp.Rational(1, 10)
    fv = [sp.Rational(1), sp.Rational(-2), sp.Rational(3, 2)]
    nv = [sp.Rational(-1, 2), sp.Rational(1), sp.Rational(2)]
    pt = [sp.Rational(str(c)) for c in point]
    subs = {x: pt[0], y: pt[1], z: pt[2], e: eps}
    subs.update({f[i]: fv[i] for i in range(3)})
    subs.update({n[i]: nv[i] for i in range(3)})
    exact = lambda v: np.array([float(sp.N(c.subs(subs), 30)) for c in v])
    mu = 7.0 / 3.0
    u_ref = (exact(u_f) + exact(u_n)) / mu
    w_ref = (exact(w_f) + exact(w_n)) / mu
    xt = np.array([[float(c) for c in pt]])
    u, w = orc.mrs_velocity(np.zeros((1, 3)), np.array([[float(c) for c in fv]]),
                            np.array([[float(c) for c in nv]]), 0.1, mu, xt=xt)
    assert np.abs(u[0] - u_ref).max() <= 1e-14 * np.abs(u_ref).max()
    assert np.abs(w[0] - w_ref).max() <= 1e-14 * np.abs(w_ref).max()
