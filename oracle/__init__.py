"""FP64 CPU oracle for the regularized-Stokeslet Kirchhoff-rod method.

TEST INFRASTRUCTURE ONLY.  The product library never imports this package; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.  The numerical
routines live in ``mrs_oracle.c`` (plain double-precision C, one OpenMP loop over targets);
this module compiles it with gcc and wraps it with ctypes.  It shares no code with the CUDA
path: the two meet only through the seeded input generators.

Paper sections implemented (see the C file for each routine's citation):
  * Section II-C, Eqs. velocity_field / angular_velocity_field / superposition -- MRS pair sum
  * Section III-C-1, Eqs. rodrigues / halfangle                               -- rotation sqrt
  * Sections II-A, II-B, Eqs. discrete_f / discrete_n / F_comp / N_comp / mid_triad -- rod forces
  * Section III-C-3, Eqs. newx / newD; Section III-B (Euler coarse, RK2 fine)   -- time step
  * Section II-D, Eqs. initial / intermediate / serial_correct                  -- Parareal
    (``oracle.parareal``, numpy)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle C source into ``oracle/_build/liborc.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class RodParams(ctypes.Structure):
    """Mirror of ``orc_rod_params`` (physical parameters of Sections II-A, II-B, IV-A)."""
    _fields_ = [("L", ctypes.c_double), ("a", ctypes.c_double * 3), ("b", ctypes.c_double * 3),
                ("wave_A", ctypes.c_double), ("wave_k", ctypes.c_double),
                ("wave_f", ctypes.c_double)]

    @classmethod
    def make(cls, L, a, b, wave_A, wave_k, wave_f):
        p = cls()
        p.L = L
        for q in range(3):
            p.a[q] = a[q]
            p.b[q] = b[q]
        p.wave_A, p.wave_k, p.wave_f = wave_A, wave_k, wave_f
        return p


def _bind(L):
    L.orc_mrs_kernels.argtypes = [ctypes.c_double, ctypes.c_double, _dp]
    L.orc_mrs_velocity.argtypes = [ctypes.c_int64, _dp, ctypes.c_int64, _dp, _dp, _dp,
                                   ctypes.c_double, ctypes.c_double, _dp, _dp]
    L.orc_mrs_velocity_batch.argtypes = [ctypes.c_int, _i64p, _dp, _dp, _dp,
                                         ctypes.c_double, _dp, ctypes.c_double, _dp, _dp]
    L.orc_rot_sqrt.argtypes = [_dp, _dp]
    L.orc_rod_forces.argtypes = [ctypes.c_int, _i64p, _dp, _dp,
                                 ctypes.POINTER(RodParams), ctypes.c_double, _dp, _dp]
    L.orc_rod_step.argtypes = [ctypes.c_int, _i64p, _dp, _dp, ctypes.POINTER(RodParams),
                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int, ctypes.c_int]
    L.orc_rodrigues_update.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, _dp]
    L.orc_lj_forces.argtypes = [ctypes.c_int64, _dp, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                ctypes.c_double, _dp]
    L.orc_num_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


class _Variant:
    """The oracle's Python API bound to another compiled copy of the C source."""

    def __init__(self, L):
        self._L = L

    def __getattr__(self, name):
        fn = globals()[name]
        if callable(fn) and not isinstance(fn, type):
            def bound(*a, **k):
                return fn(*a, _L=self._L, **k)
            return bound
        return fn


def variant(substitutions, tag):
    """Compile a copy of mrs_oracle.c with textual substitutions [(old, new), ...] applied and
    return the oracle API bound to it.  Tests use this to plant mistakes and check that the
    pins catch them; every `old` must occur in the source."""
    src = open(_SRC).read()
    for old, new in substitutions:
        if old not in src:
            raise ValueError("substitution target not found: %r" % old)
        src = src.replace(old, new)
    os.makedirs(_BUILD, exist_ok=True)
    cpath = os.path.join(_BUILD, "variant_%s.c" % tag)
    so = os.path.join(_BUILD, "libvariant_%s_%d.so" % (tag, os.getpid()))
    open(cpath, "w").write(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    cpath, "-o", so, "-lm"], check=True)
    return _Variant(_bind(ctypes.CDLL(so)))


def _d(a):
    """A C-contiguous float64 copy/view of ``a`` and its pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_i64p)


def num_threads(_L=None) -> int:
    return int((_L or lib()).orc_num_threads())


def mrs_kernels(r2: float, eps: float, _L=None) -> np.ndarray:
    """H1..H5 of the blob phi_eps at squared distance r2 (Section II-C)."""
    H = np.zeros(5)
    (_L or lib()).orc_mrs_kernels(float(r2), float(eps), H.ctypes.data_as(_dp))
    return H


def mrs_velocity(X, f, n, eps, mu=1.0, xt=None, _L=None):
    """u, omega at targets xt (default: the sources X) from all sources (Eq. superposition)."""
    X, pX = _d(X)
    f, pf = _d(f)
    n, pn = _d(n)
    xt, pt = _d(X if xt is None else xt)
    nt, ns = xt.shape[0], X.shape[0]
    u = np.zeros((nt, 3))
    w = np.zeros((nt, 3))
    (_L or lib()).orc_mrs_velocity(nt, pt, ns, pX, pf, pn, float(eps), float(mu),
                           u.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
    return u, w


def mrs_velocity_batch(offsets, X, f, n, eps, mu=1.0, eps_per_sys=None, _L=None):
    """Independent systems given by CSR point offsets; each system's targets are its sources."""
    off, po = _i64(offsets)
    X, pX = _d(X)
    f, pf = _d(f)
    n, pn = _d(n)
    u = np.zeros_like(X)
    w = np.zeros_like(X)
    if eps_per_sys is None:
        pe = None
    else:
        eps_per_sys, pe = _d(eps_per_sys)
    (_L or lib()).orc_mrs_velocity_batch(len(off) - 1, po, pX, pf, pn, float(eps), pe, float(mu),
                                 u.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
    return u, w


def rot_sqrt(R, _L=None) -> np.ndarray:
    """Principal square root of one 3x3 rotation matrix (Section III-C-1)."""
    R, pR = _d(np.asarray(R).reshape(3, 3))
    S = np.zeros((3, 3))
    (_L or lib()).orc_rot_sqrt(pR, S.ctypes.data_as(_dp))
    return S


def rod_forces(rod_off, X, D, params: RodParams, t: float, _L=None):
    """Point force g and torque m each node applies to the fluid (Eqs. discrete_f/discrete_n)."""
    off, po = _i64(rod_off)
    X, pX = _d(X)
    D, pD = _d(D)
    g = np.zeros_like(X)
    m = np.zeros_like(X)
    (_L or lib()).orc_rod_forces(len(off) - 1, po, pX, pD, ctypes.byref(params), float(t),
                         g.ctypes.data_as(_dp), m.ctypes.data_as(_dp))
    return g, m


def rodrigues_update(D, w, dt, _L=None):
    """Eq. newD: every director of node k rotated by |w_k| dt about w_k / |w_k|."""
    D, pD = _d(D)
    w, pw = _d(w)
    out = np.zeros_like(D)
    (_L or lib()).orc_rodrigues_update(D.shape[0], pD, pw, float(dt), out.ctypes.data_as(_dp))
    return out


def lj_forces(X, rod_id, sigma, e_lj, F=None, _L=None):
    """Section IV-A repulsion between nodes of different rods; returns F + the LJ forces."""
    X, pX = _d(X)
    rid = np.ascontiguousarray(np.asarray(rod_id, dtype=np.int32))
    out = np.zeros_like(X) if F is None else np.array(F, dtype=np.float64, copy=True)
    (_L or lib()).orc_lj_forces(X.shape[0], pX, rid.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                float(sigma), float(e_lj), out.ctypes.data_as(_dp))
    return out


EULER, RK2 = 0, 1


def rod_step(rod_off, X, D, params: RodParams, eps, mu, t0, dt, nsteps, scheme, _L=None):
    """``nsteps`` explicit steps (EULER: Eqs. newx/newD; RK2: midpoint).  Returns new (X, D)."""
    off, po = _i64(rod_off)
    X = np.array(X, dtype=np.float64, order="C", copy=True)
    D = np.array(D, dtype=np.float64, order="C", copy=True)
    (_L or lib()).orc_rod_step(len(off) - 1, po, X.ctypes.data_as(_dp), D.ctypes.data_as(_dp),
                       ctypes.byref(params), float(eps), float(mu), float(t0), float(dt),
                       int(nsteps), int(scheme))
    return X, D
