"""Seeded synthetic workloads shaped like the paper's swimmer configurations.

This module is the ONLY code shared by the CUDA path's tests/bench and the CPU oracle: it
draws random numbers and lays out filament geometry, and holds none of the method's
arithmetic (no Stokeslet, no rod mechanics, no time stepping).

Geometry (Section IV-A): each filament is a planar sinusoid y = A sin(k x) of arclength L with
k = 2 pi / lambda, nodes evenly spaced in arclength (the arclength is inverted numerically on a
fine grid), frame D^3 = unit tangent, D^2 = e_z (normal of the wave plane), D^1 = D^2 x D^3.
Multi-filament systems rotate each filament by a Haar-random rotation and translate its node
mean to a centre drawn uniformly in a box.  The paper starts from straight rods near a wall;
the sinusoid matches its preferred-curvature wave at t = 0 instead (the wall is not modelled).

Every MRS input set is generated in float64 and rounded to float32; the rounded values are
what both the GPU path and the oracle (promoted back to float64) consume, so both see the
same bits.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

EPS_OVER_DS = 1.5           # regularisation eps = 1.5 ds (the paper uses 4 ds; configs use 1.5)


def sinusoid_filament(M: int, L: float = 1.0, A: float = 0.05, lam: float = 1.0):
    """M nodes evenly spaced in arclength on y = A sin(2 pi x / lam), z = 0.

    Returns X[M,3] (float64) and D[M,3,3] with D[k, i] = director D^{i+1}_k (fresh copies)."""
    X, D = _sinusoid_cached(int(M), float(L), float(A), float(lam))
    return X.copy(), D.copy()


@functools.lru_cache(maxsize=64)
def _sinusoid_cached(M: int, L: float, A: float, lam: float):
    k = 2.0 * math.pi / lam
    # arclength s(x) on a fine grid (composite trapezoid on 2^20 intervals), then invert
    xmax = L * 1.05 + 1e-3
    xs = np.linspace(0.0, xmax, (1 << 20) + 1)
    speed = np.sqrt(1.0 + (A * k * np.cos(k * xs)) ** 2)
    s = np.concatenate([[0.0], np.cumsum(0.5 * (speed[1:] + speed[:-1]) * np.diff(xs))])
    s_nodes = np.linspace(0.0, L, M)
    x = np.interp(s_nodes, s, xs)
    X = np.stack([x, A * np.sin(k * x), np.zeros_like(x)], axis=1)
    t = np.stack([np.ones_like(x), A * k * np.cos(k * x), np.zeros_like(x)], axis=1)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    d2 = np.tile(np.array([0.0, 0.0, 1.0]), (M, 1))
    d1 = np.cross(d2, t)
    D = np.stack([d1, d2, t], axis=1)
    return X, D


def haar_rotation(rng: np.random.Generator) -> np.ndarray:
    """A Haar-distributed rotation (QR of a Gaussian matrix with the sign convention fixed)."""
    Z = rng.standard_normal((3, 3))
    Q, R = np.linalg.qr(Z)
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def place_filaments(rng, n_fil: int, M: int, box: float = 10.0, L: float = 1.0,
                    A: float = 0.05, lam: float = 1.0):
    """n_fil filaments of M nodes, random orientation, node mean uniform in [0, box]^3."""
    X0, D0 = sinusoid_filament(M, L, A, lam)
    X0 = X0 - X0.mean(axis=0)
    Xs, Ds = [], []
    for _ in range(n_fil):
        Q = haar_rotation(rng)
        c = rng.uniform(0.0, box, size=3)
        Xs.append(X0 @ Q.T + c)
        Ds.append(np.einsum("rc,kic->kir", Q, D0))
    return np.concatenate(Xs), np.concatenate(Ds)


@dataclass
class MRSProblem:
    """Inputs of one mrs_velocity call: float32-representable arrays stored as float32."""
    name: str
    offsets: np.ndarray            # int64 [n_sys+1]
    X: np.ndarray                  # float32 [N,3]
    f: np.ndarray                  # float32 [N,3]
    n: np.ndarray                  # float32 [N,3]
    eps: np.ndarray                # float64 [n_sys] (float32-representable)
    mu: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return int(self.offsets[-1])

    @property
    def pairs(self) -> int:
        sz = np.diff(self.offsets)
        return int(np.sum(sz.astype(np.int64) ** 2))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _gauss_fn(rng, N):
    f = rng.standard_normal((N, 3))
    n = rng.standard_normal((N, 3))
    return _f32(f), _f32(n)


def plain_rod(seed: int = 1, M: int = 128) -> MRSProblem:
    """One rod of M = 128 nodes on the unit sinusoid, eps = 1.5 ds, mu = 1, N(0,1) f and n."""
    rng = np.random.default_rng(seed)
    X, _ = sinusoid_filament(M)
    f, n = _gauss_fn(rng, M)
    ds = 1.0 / (M - 1)
    eps = float(np.float32(EPS_OVER_DS * ds))
    return MRSProblem("plain_rod_128", np.array([0, M], np.int64), _f32(X), f, n,
                      np.array([eps]), 1.0, {"M": M})


def single_system(seed: int = 2, n_fil: int = 32, M: int = 1024, box: float = 10.0) -> MRSProblem:
    """32 filaments x 1024 nodes (32768 points) in a 10^3 box, eps = 1.5 ds, Gaussian f, n."""
    rng = np.random.default_rng(seed)
    X, _ = place_filaments(rng, n_fil, M, box)
    f, n = _gauss_fn(rng, X.shape[0])
    eps = float(np.float32(EPS_OVER_DS / (M - 1)))
    return MRSProblem("single_system_%dx%d" % (n_fil, M), np.array([0, X.shape[0]], np.int64),
                      _f32(X), f, n, np.array([eps]), 1.0, {"n_fil": n_fil, "M": M, "box": box})


def batch_sizes(rng, n_sys: int = 512, lo_exp: float = 8.0, hi_exp: float = 14.0, unit: int = 256):
    """N_s = unit * round(2^U(lo,hi) / unit), at least one unit (log-uniform in [256, 16384])."""
    N = unit * np.round(2.0 ** rng.uniform(lo_exp, hi_exp, size=n_sys) / unit)
    return np.maximum(N, unit).astype(np.int64)


def batch_systems(seed: int = 3, n_sys: int = 512, M: int = 256, lo_exp: float = 8.0,
                  hi_exp: float = 14.0, box: float = 10.0) -> MRSProblem:
    """512 independent systems, N_s log-uniform in [256, 16384], filaments of 256 nodes."""
    rng = np.random.default_rng(seed)
    sizes = batch_sizes(rng, n_sys, lo_exp, hi_exp, M)
    Xs = []
    for Ns in sizes:
        Xi, _ = place_filaments(rng, int(Ns) // M, M, box)
        Xs.append(Xi)
    X = np.concatenate(Xs)
    f, n = _gauss_fn(rng, X.shape[0])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    eps = float(np.float32(EPS_OVER_DS / (M - 1)))
    return MRSProblem("batch_%d_systems" % n_sys, off, _f32(X), f, n,
                      np.full(n_sys, eps), 1.0, {"M": M, "sizes": sizes})


def subset(p: MRSProblem, systems) -> MRSProblem:
    """The listed systems of a batch as a new (smaller) batch, same values."""
    systems = list(systems)
    parts = [(int(p.offsets[s]), int(p.offsets[s + 1])) for s in systems]
    idx = np.concatenate([np.arange(a, b) for a, b in parts])
    sizes = np.array([b - a for a, b in parts], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return MRSProblem(p.name + "_subset", off, p.X[idx], p.f[idx], p.n[idx],
                      p.eps[systems], p.mu, dict(p.meta))


@dataclass
class RodSystem:
    """Rod state for rod_forces / rod_step / parareal_run: float64 X[N,3], D[N,3,3]."""
    name: str
    rod_off: np.ndarray            # int64 [n_rods+1]
    X: np.ndarray
    D: np.ndarray
    L: float
    eps: float
    meta: dict = field(default_factory=dict)


def rod_system(seed: int, n_rods: int, M: int, box: float = 10.0) -> RodSystem:
    """n_rods sinusoid filaments of M nodes; n_rods = 1 keeps the unit rod at the origin."""
    rng = np.random.default_rng(seed)
    if n_rods == 1:
        X, D = sinusoid_filament(M)
    else:
        X, D = place_filaments(rng, n_rods, M, box)
    off = np.arange(0, (n_rods + 1) * M, M, dtype=np.int64)
    eps = float(np.float32(EPS_OVER_DS / (M - 1)))
    return RodSystem("rods_%dx%d" % (n_rods, M), off, X, D, 1.0, eps, {"M": M})


def serve_trace(seed: int = 5, rate_hz: float = 2000.0, window_s: float = 2.0,
                frac_mrs: float = 0.7, n_lo: int = 1024, n_hi: int = 65536, unit: int = 256):
    """Poisson arrivals over a fixed window: (t_arrive, kind, N) with kind 0 = one
    mrs_velocity, 1 = a 100-step rod integration; N log-uniform in [1k, 64k] (multiple of 256)."""
    rng = np.random.default_rng(seed)
    t, jobs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= window_s:
            break
        kind = 0 if rng.uniform() < frac_mrs else 1
        N = int(unit * round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))) / unit))
        jobs.append((t, kind, max(N, unit)))
    return jobs


# Physical parameters.  The paper never lists its moduli (it only says they stay fixed);
# these are chosen so that the stated time steps are stable for the stiffest mode of each
# configuration, measured on the oracle's linearised dynamics (lambda_max ~ 1.9e7 a and
# 572 b for 128-node rods, ~ 5.0e9 a and 9.2e3 b for 512-node rods, eps = 1.5 ds, mu = 1),
# with b/a ~ 1/eps^2 as for a slender rod of radius eps.
#   plain rod, dt = 1e-6 (Euler and RK2):  lambda_max dt ~ 0.4
#   Parareal rods, fine dt = 1e-6, coarse 16 dt (Euler): lambda_max * 16 dt ~ 1.2
WAVE = dict(L=1.0, wave_A=0.05, wave_k=2.0 * math.pi, wave_f=2.0 * math.pi)
ROD_PLAIN = dict(WAVE, a=(0.02, 0.02, 0.02), b=(140.0, 140.0, 140.0), dt=1e-6)
ROD_PARAREAL = dict(WAVE, a=(1.5e-5, 1.5e-5, 1.5e-5), b=(1.8, 1.8, 1.8), dt=1e-6)
# serving rod jobs: filaments of 256 nodes, explicit Euler at dt = 1e-6; bending stiffens as
# M^4 and stretching as M^2 (lambda_max ~ 3.1e8 a and 2.3e3 b at 256 nodes), so a = 1e-3,
# b = 20 give lambda_max dt ~ 0.3 (ROD_PLAIN's moduli would give ~6: unstable)
ROD_SERVE = dict(WAVE, a=(1e-3, 1e-3, 1e-3), b=(20.0, 20.0, 20.0), dt=1e-6)
#   Parareal on one 128-node rod, fine dt = 1e-6, coarse 16 dt: lambda_max * 16 dt ~ 1.2
ROD_PARAREAL_128 = dict(WAVE, a=(4e-3, 4e-3, 4e-3), b=(28.0, 28.0, 28.0), dt=1e-6)
