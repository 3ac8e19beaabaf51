"""Parareal (Section II-D, Eqs. initial, intermediate, serial_correct) -- oracle form.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The driver is generic in the
propagators: ``G(n, x)`` and ``F(n, x)`` advance a state from T_{n-1} to T_n.  Iteration k:

  k = 0:   X^0_n = G(X^0_{n-1}) for n = 1..N, X^0_0 = x0  (reading: the garbled start index of
           the loop is taken as n = 1, i.e. the initial coarse sweep covers every slice)
  k >= 1:  X'^k_n = F(X^{k-1}_{n-1})              for n = k..N   (parallel in the paper)
           X^k_n  = X^{k-1}_n                     for n < k
           X^k_k  = X'^k_k
           X^k_n  = X'^k_n + G(X^k_{n-1}) - G(X^{k-1}_{n-1})   for n = k+1..N (serial)

where G(X^{k-1}_{n-1}) is the value the previous iteration computed.  ``post`` is applied to
every corrected state (for rods: re-orthonormalisation of the frames, a reading, since the
paper does not say how an additive correction keeps frames orthonormal).  Iteration stops when
the relative increment of Eq. true_err falls below ``tol`` or after ``max_iter`` iterations.
"""
from __future__ import annotations

import numpy as np


def run(x0, G, F, n_slices, max_iter, tol, incr, post=None):
    """Returns (states, increments): states[k][n] = X^k_n, increments[k-1] = incr(X^k, X^{k-1})."""
    N = n_slices
    X = [np.array(x0, copy=True)]
    for n in range(1, N + 1):
        X.append(G(n, X[n - 1]))
    g_old = [None] + [X[n].copy() for n in range(1, N + 1)]  # G(X^0_{n-1}) = X^0_n
    states = [X]
    increments = []
    for k in range(1, max_iter + 1):
        if k > N:
            break
        Fk = {n: F(n, X[n - 1]) for n in range(k, N + 1)}
        Xn = [X[n] for n in range(0, k)] + [Fk[k]]
        g_new = list(g_old)
        for n in range(k + 1, N + 1):
            g = G(n, Xn[n - 1])
            x = Fk[n] + g - g_old[n]
            if post is not None:
                x = post(x)
            Xn.append(x)
            g_new[n] = g
        g_old = g_new
        increments.append(incr(Xn, X))
        X = Xn
        states.append(X)
        if increments[-1] < tol:
            break
    return states, increments


def polar_orthonormalize(D):
    """Nearest rotation D (D^T D)^{-1/2} of every 3x3 frame in D[..., 3, 3] (SVD form)."""
    U, _, Vt = np.linalg.svd(D)
    return U @ Vt


def max_rel_point_diff(XA, XB, point_slice=slice(0, 3)):
    """Eq. true_err: max over points (and slice ends) of ||x_A - x_B||_2 / ||x_A||_2, positions
    only.  XA, XB are lists of states (one per slice end T_0..T_N); each state is an array whose
    rows are points and whose first three columns are positions."""
    worst = 0.0
    for a, b in zip(XA[1:], XB[1:]):
        pa = np.asarray(a)[:, point_slice]
        pb = np.asarray(b)[:, point_slice]
        num = np.linalg.norm(pa - pb, axis=1)
        den = np.linalg.norm(pa, axis=1)
        worst = max(worst, float(np.max(num / den)))
    return worst


def pack_rod_state(X, D):
    """Rod state as one array: row k = (X_k, D^1_k, D^2_k, D^3_k), 12 numbers per node."""
    return np.concatenate([np.asarray(X), np.asarray(D).reshape(-1, 9)], axis=1)


def unpack_rod_state(x):
    x = np.asarray(x)
    return x[:, :3].copy(), x[:, 3:].reshape(-1, 3, 3).copy()


def rod_parareal(rod_off, X, D, params, eps, mu, T0, T1, n_slices, dt_fine, coarse_ratio,
                 max_iter, tol):
    """Parareal for the rod system: G = explicit Euler with step coarse_ratio * dt_fine,
    F = RK2 with step dt_fine (Section III-B), additive correction on all 12 components of every
    node followed by polar re-orthonormalisation of the frames.  Slice length T/n_slices must
    be a whole number of coarse steps."""
    import oracle
    dT = (T1 - T0) / n_slices
    n_fine = int(round(dT / dt_fine))
    n_coarse = n_fine // coarse_ratio
    assert n_coarse * coarse_ratio == n_fine and abs(n_fine * dt_fine - dT) < 1e-9 * dT
    dt_coarse = dt_fine * coarse_ratio

    def G(n, x):
        Xs, Ds = unpack_rod_state(x)
        Xs, Ds = oracle.rod_step(rod_off, Xs, Ds, params, eps, mu, T0 + (n - 1) * dT,
                                 dt_coarse, n_coarse, oracle.EULER)
        return pack_rod_state(Xs, Ds)

    def F(n, x):
        Xs, Ds = unpack_rod_state(x)
        Xs, Ds = oracle.rod_step(rod_off, Xs, Ds, params, eps, mu, T0 + (n - 1) * dT,
                                 dt_fine, n_fine, oracle.RK2)
        return pack_rod_state(Xs, Ds)

    def post(x):
        Xs, Ds = unpack_rod_state(x)
        return pack_rod_state(Xs, polar_orthonormalize(Ds))

    return run(pack_rod_state(X, D), G, F, n_slices, max_iter, tol, max_rel_point_diff, post)
