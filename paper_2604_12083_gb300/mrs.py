"""Thin ctypes binding of the C ABI declared in ``include/mrs_gb300.h``.

Argument marshalling only: every step of the computation runs in the CUDA library
``_build/libmrs_gb300.so``.  Device arrays are passed as torch CUDA tensors (their
``data_ptr()``), host arrays as numpy arrays, streams as ``torch.cuda.Stream`` (or None for
torch's current stream).  There is no CPU fallback: if the library is missing or a call fails,
an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MRS_GB300_DEBUG=1 loads the debug build (index checks that raise MRS_FLAG_BOUNDS instead of
# touching memory through a bad table entry; paper_2604_12083_gb300.build.build(debug=True))
LIB_PATH = os.path.join(HERE, "_build", "libmrs_gb300_debug.so" if os.environ.get("MRS_GB300_DEBUG") == "1"
                        else "libmrs_gb300.so")

MRS_OK, MRS_EINVAL, MRS_ENOMEM, MRS_ECUDA, MRS_ETIMEOUT, MRS_ENOCONV, MRS_EBUSY, MRS_PENDING = range(8)
MRS_ECANCELED = 8
MRS_F64, MRS_F32, MRS_F32_COMP = 0, 1, 2
MRS_EULER, MRS_RK2 = 0, 1
STATUS_NAMES = {0: "MRS_OK", 1: "MRS_EINVAL", 2: "MRS_ENOMEM", 3: "MRS_ECUDA", 4: "MRS_ETIMEOUT",
                5: "MRS_ENOCONV", 6: "MRS_EBUSY", 7: "MRS_PENDING", 8: "MRS_ECANCELED"}

# Every symbol include/mrs_gb300.h declares (kept in sync by tests/test_abi.py).
EXPORTS = [
    "mrs_last_error", "mrs_version", "mrs_ctx_create", "mrs_ctx_destroy", "mrs_ctx_num_sms",
    "mrs_ctx_set_fused_steps", "mrs_ctx_set_rod_force_kernel", "mrs_ctx_set_sym_pass_bytes",
    "mrs_fma_probe",
    "mrs_velocity", "mrs_plan_create", "mrs_plan_execute", "mrs_plan_destroy",
    "mrs_plan_config_count", "mrs_plan_config_symmetric", "mrs_plan_config_info", "mrs_plan_info",
    "mrs_plan_scratch",
    "rod_forces", "rod_step", "rot_sqrt_batch", "parareal_run", "mrs_velocity_noalloc",
    "serve_create", "serve_submit", "serve_poll", "serve_drain", "serve_stats", "serve_destroy",
    "serve_set_policy", "serve_inject_alloc_failure",
    "serve_cancel",
    "mrs_autotune", "mrs_autotune_save", "mrs_autotune_load", "parareal_run_pipelined",
    "rod_advance", "rod_checkpoint_save", "rod_checkpoint_load", "mrs_device_status",
    "mrs_reserve",
]
MRS_FLAG_NONFINITE, MRS_FLAG_BOUNDS = 1, 2
MRS_JOB_VELOCITY, MRS_JOB_ROD = 0, 1

_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class MrsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class RodParams(ctypes.Structure):
    """``mrs_rod_params``."""
    _fields_ = [("L", ctypes.c_double), ("a", ctypes.c_double * 3), ("b", ctypes.c_double * 3),
                ("wave_A", ctypes.c_double), ("wave_k", ctypes.c_double),
                ("wave_f", ctypes.c_double), ("mu", ctypes.c_double), ("eps", ctypes.c_double),
                ("lj_eps", ctypes.c_double), ("lj_sigma", ctypes.c_double)]

    @classmethod
    def make(cls, L, a, b, wave_A, wave_k, wave_f, mu, eps, lj_eps=0.0, lj_sigma=None):
        p = cls()
        p.L = L
        for q in range(3):
            p.a[q] = a[q]
            p.b[q] = b[q]
        p.wave_A, p.wave_k, p.wave_f, p.mu, p.eps = wave_A, wave_k, wave_f, mu, eps
        p.lj_eps = lj_eps
        p.lj_sigma = 0.0 if lj_sigma is None else lj_sigma   # 0: the library's 3 eps
        return p


class PararealStats(ctypes.Structure):
    """``mrs_parareal_stats``."""
    _fields_ = [("iterations", ctypes.c_int), ("incr", ctypes.c_double * 64),
                ("final_incr", ctypes.c_double), ("seconds", ctypes.c_double),
                ("fine_steps", ctypes.c_int64), ("coarse_steps", ctypes.c_int64)]


class Job(ctypes.Structure):
    """``mrs_job``."""
    _fields_ = [("kind", ctypes.c_int), ("n_points", ctypes.c_int64), ("mu", ctypes.c_double),
                ("eps", ctypes.c_double), ("X", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("n", ctypes.c_void_p), ("u", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("n_rods", ctypes.c_int), ("rod_off", ctypes.POINTER(ctypes.c_int64)),
                ("Xr", ctypes.c_void_p), ("Dr", ctypes.c_void_p), ("params", RodParams),
                ("t0", ctypes.c_double), ("dt", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("scheme", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load the library (built by ``paper_2604_12083_gb300.build``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.mrs_last_error.restype = ctypes.c_char_p
        L.mrs_version.restype = ctypes.c_char_p
        L.mrs_ctx_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
        L.mrs_ctx_destroy.argtypes = [_vp]
        L.mrs_ctx_num_sms.argtypes = [_vp]
        L.mrs_ctx_set_fused_steps.argtypes = [_vp, ctypes.c_int]
        L.mrs_ctx_set_rod_force_kernel.argtypes = [_vp, ctypes.c_int]
        L.mrs_ctx_set_sym_pass_bytes.argtypes = [_vp, ctypes.c_size_t]
        L.mrs_fma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                    ctypes.POINTER(ctypes.c_float)]
        L.mrs_device_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint)]
        L.mrs_velocity.argtypes = [_vp, ctypes.c_int, _i64p, _vp, _vp, _vp, _vp, _vp, _vp,
                                   ctypes.c_double, ctypes.c_double, _dp, ctypes.c_int, _vp]
        L.mrs_plan_create.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.c_double, ctypes.c_double,
                                      _dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]
        L.mrs_reserve.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.c_double, ctypes.c_double, _dp,
                                  ctypes.c_int]
        L.mrs_plan_execute.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.mrs_plan_destroy.argtypes = [_vp]
        L.mrs_plan_config_info.argtypes = [_vp, ctypes.c_int, _ip, _ip, _ip]
        L.mrs_plan_info.argtypes = [_vp, _ip, _i64p, _ip]
        L.mrs_plan_scratch.argtypes = [_vp, _ip, ctypes.POINTER(ctypes.c_size_t)]
        L.rod_forces.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.POINTER(RodParams), _vp, _vp,
                                 ctypes.c_double, _vp, _vp, _vp]
        L.rod_step.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.POINTER(RodParams), _vp, _vp,
                               ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, _vp]
        L.rot_sqrt_batch.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
        L.rod_checkpoint_save.argtypes = [ctypes.c_char_p, ctypes.c_int, _i64p, _vp, _vp,
                                          ctypes.c_double, _vp]
        L.rod_checkpoint_load.argtypes = [ctypes.c_char_p, ctypes.c_int, _i64p, _vp, _vp, _dp, _vp]
        L.rod_advance.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.c_double,
                                  ctypes.c_int, _vp]
        L.parareal_run_pipelined.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.POINTER(RodParams),
                                             _vp, _vp, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             ctypes.POINTER(PararealStats), _vp]
        L.mrs_autotune.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.c_double, ctypes.c_double, _dp,
                                   ctypes.c_int, ctypes.c_int, _ip, ctypes.POINTER(ctypes.c_float)]
        L.mrs_autotune_save.argtypes = [_vp, ctypes.c_char_p]
        L.mrs_autotune_load.argtypes = [_vp, ctypes.c_char_p]
        L.serve_create.argtypes = [ctypes.POINTER(_vp), _vp, ctypes.c_size_t, ctypes.c_int]
        L.serve_submit.argtypes = [_vp, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]
        L.serve_poll.argtypes = [_vp, ctypes.c_uint64, _ip, _dp]
        L.serve_drain.argtypes = [_vp, ctypes.c_double]
        L.serve_set_policy.argtypes = [_vp, ctypes.c_double, ctypes.c_int]
        L.serve_inject_alloc_failure.argtypes = [_vp, ctypes.c_uint64]
        L.serve_cancel.argtypes = [_vp, ctypes.c_uint64]
        L.serve_stats.argtypes = [_vp, _i64p, _i64p, _dp, _ip, ctypes.POINTER(ctypes.c_size_t), _i64p]
        L.serve_destroy.argtypes = [_vp]
        L.mrs_velocity_noalloc.argtypes = [ctypes.c_int64, _vp, _vp, _vp, _vp, _vp,
                                           ctypes.c_double, ctypes.c_double, _vp]
        L.parareal_run.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.POINTER(RodParams), _vp,
                                   _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.POINTER(PararealStats), _vp]
        _lib = L
        return L


def _check(status):
    if status != MRS_OK:
        raise MrsError(status, lib().mrs_last_error().decode())


def _ptr(t):
    """Device pointer of a torch tensor (must be contiguous), or None."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _offsets(offsets):
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    return off, off.ctypes.data_as(_i64p)


class Context:
    """``mrs_ctx`` on one device."""

    def __init__(self, device: int = 0):
        self.handle = _vp()
        _check(lib().mrs_ctx_create(ctypes.byref(self.handle), int(device)))
        self.device = device

    @property
    def num_sms(self) -> int:
        return int(lib().mrs_ctx_num_sms(self.handle))

    def set_sym_pass_bytes(self, nbytes: int) -> None:
        """``mrs_ctx_set_sym_pass_bytes``: column-partial buffer of one pass of a symmetric plan
        (plans created afterwards; larger plans run in several passes)."""
        _check(lib().mrs_ctx_set_sym_pass_bytes(self.handle, int(nbytes)))

    def set_fused_steps(self, mode: int) -> None:
        """``mrs_ctx_set_fused_steps``: 1 (default) one fused launch per rod-stepping call for
        instances of at most 128 nodes in batches of more than 4096 nodes, 2 whenever the
        instance fits shared memory, 0 never."""
        _check(lib().mrs_ctx_set_fused_steps(self.handle, int(mode)))

    def set_rod_force_kernel(self, mode: int) -> None:
        """``mrs_ctx_set_rod_force_kernel``: 0 (default) warp-cooperative force kernel for
        batches of at most 4096 nodes, 1 always one thread per segment, 2 always
        warp-cooperative."""
        _check(lib().mrs_ctx_set_rod_force_kernel(self.handle, int(mode)))

    def device_status(self) -> int:
        """``mrs_device_status``: anomaly flags since the last call (synchronizes, clears)."""
        f = ctypes.c_uint()
        _check(lib().mrs_device_status(self.handle, ctypes.byref(f)))
        return f.value

    def close(self):
        if self.handle:
            _check(lib().mrs_ctx_destroy(self.handle))
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mrs_velocity(ctx: Context, offsets, X, f, n, u, w, mu, eps, eps_per_sys=None,
                 precision=MRS_F32_COMP, Xt=None, stream=None):
    """``mrs_velocity``: u, w (device tensors, overwritten) from X, f, n (device tensors)."""
    off, poff = _offsets(offsets)
    eps_arr = None
    peps = None
    if eps_per_sys is not None:
        eps_arr = np.ascontiguousarray(np.asarray(eps_per_sys, dtype=np.float64))
        peps = eps_arr.ctypes.data_as(_dp)
    _check(lib().mrs_velocity(ctx.handle, len(off) - 1, poff, _ptr(X), _ptr(f), _ptr(n), _ptr(Xt),
                              _ptr(u), _ptr(w), float(mu), float(eps), peps, int(precision),
                              _stream(stream)))


def mrs_reserve(ctx: Context, offsets, mu, eps, eps_per_sys=None, precision=MRS_F32_COMP):
    """``mrs_reserve``: build and cache the plan ``mrs_velocity`` uses for this shape, so that
    later calls with it allocate nothing (and can be captured in a CUDA graph)."""
    off, poff = _offsets(offsets)
    peps = None
    if eps_per_sys is not None:
        eps_arr = np.ascontiguousarray(np.asarray(eps_per_sys, dtype=np.float64))
        peps = eps_arr.ctypes.data_as(_dp)
    _check(lib().mrs_reserve(ctx.handle, len(off) - 1, poff, float(mu), float(eps), peps,
                             int(precision)))


def fma_probe(device, kind, iters=1 << 16, warps_per_scheduler=0):
    """``mrs_fma_probe``: (TFLOP/s, ms) of the FP32 FMA pipe for kind 0 (FFMA), 1 (FFMA2),
    2 (interleaved), or of the FP64 pipe (kind 3: all lanes; kind 4: lane 0 of each warp, its
    flops only); warps_per_scheduler 0 fills the device."""
    tf, ms = ctypes.c_double(), ctypes.c_float()
    _check(lib().mrs_fma_probe(int(device), int(kind), int(iters), int(warps_per_scheduler),
                               ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def mrs_velocity_noalloc(n_points, X, f, n, u, w, mu, eps, stream=None):
    """``mrs_velocity_noalloc``: one system, float32 compensated, no device allocation (for
    callers that must not allocate); u, w (device float32 tensors) are overwritten."""
    _check(lib().mrs_velocity_noalloc(int(n_points), _ptr(X), _ptr(f), _ptr(n), _ptr(u), _ptr(w),
                                      float(mu), float(eps), _stream(stream)))


class Plan:
    """``mrs_plan``: a pair-sum plan built once and executed many times."""

    def __init__(self, ctx: Context, offsets, mu, eps, eps_per_sys=None,
                 precision=MRS_F32_COMP, config=-1):
        off, poff = _offsets(offsets)
        peps = None
        if eps_per_sys is not None:
            self._eps = np.ascontiguousarray(np.asarray(eps_per_sys, dtype=np.float64))
            peps = self._eps.ctypes.data_as(_dp)
        self.handle = _vp()
        self.ctx = ctx
        _check(lib().mrs_plan_create(ctx.handle, len(off) - 1, poff, float(mu), float(eps), peps,
                                     int(precision), int(config), ctypes.byref(self.handle)))

    def execute(self, X, f, n, u, w, Xt=None, stream=None):
        _check(lib().mrs_plan_execute(self.handle, _ptr(X), _ptr(f), _ptr(n), _ptr(Xt), _ptr(u),
                                      _ptr(w), _stream(stream)))

    def scratch(self):
        """``mrs_plan_scratch``: {"passes": executions' passes, "bytes": partial-sum scratch}."""
        npass, nbytes = ctypes.c_int(), ctypes.c_size_t()
        _check(lib().mrs_plan_scratch(self.handle, ctypes.byref(npass), ctypes.byref(nbytes)))
        return {"passes": npass.value, "bytes": nbytes.value}

    def info(self):
        g, c = ctypes.c_int(), ctypes.c_int()
        wu = ctypes.c_int64()
        _check(lib().mrs_plan_info(self.handle, ctypes.byref(g), ctypes.byref(wu), ctypes.byref(c)))
        return {"grid": g.value, "work_units": wu.value, "config": c.value}

    def close(self):
        if self.handle:
            _check(lib().mrs_plan_destroy(self.handle))
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(ctx: Context, offsets, mu, eps, eps_per_sys=None, precision=MRS_F32_COMP, reps=3):
    """``mrs_autotune``: (best config, its time in ms) for this batch shape."""
    off, poff = _offsets(offsets)
    peps = None
    if eps_per_sys is not None:
        ev = np.ascontiguousarray(np.asarray(eps_per_sys, dtype=np.float64))
        peps = ev.ctypes.data_as(_dp)
    c, ms = ctypes.c_int(), ctypes.c_float()
    _check(lib().mrs_autotune(ctx.handle, len(off) - 1, poff, float(mu), float(eps), peps,
                              int(precision), int(reps), ctypes.byref(c), ctypes.byref(ms)))
    return c.value, ms.value


def autotune_save(ctx: Context, path: str):
    _check(lib().mrs_autotune_save(ctx.handle, path.encode()))


def autotune_load(ctx: Context, path: str):
    _check(lib().mrs_autotune_load(ctx.handle, path.encode()))


def plan_config_count() -> int:
    return int(lib().mrs_plan_config_count())


def plan_config_symmetric(config: int) -> bool:
    """``mrs_plan_config_symmetric``: whether a configuration evaluates each unordered pair once."""
    r = int(lib().mrs_plan_config_symmetric(int(config)))
    if r < 0:
        raise MrsError(MRS_EINVAL, "config %d out of range" % config)
    return bool(r)


def plan_config_info(ctx: Context, config: int):
    t, k, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().mrs_plan_config_info(ctx.handle, int(config), ctypes.byref(t), ctypes.byref(k),
                                      ctypes.byref(o)))
    return {"threads": t.value, "targets_per_thread": k.value, "ctas_per_sm": o.value}


def rod_forces(ctx: Context, rod_off, params: RodParams, X, D, t, g, m, stream=None):
    """``rod_forces``: g, m (device float64 tensors, overwritten) from X, D at time t."""
    off, poff = _offsets(rod_off)
    _check(lib().rod_forces(ctx.handle, len(off) - 1, poff, ctypes.byref(params), _ptr(X), _ptr(D),
                            float(t), _ptr(g), _ptr(m), _stream(stream)))


def rod_step(ctx: Context, rod_off, params: RodParams, X, D, t0, dt, nsteps, scheme,
             precision=MRS_F32_COMP, stream=None):
    """``rod_step``: nsteps steps in place on device float64 tensors X, D."""
    off, poff = _offsets(rod_off)
    _check(lib().rod_step(ctx.handle, len(off) - 1, poff, ctypes.byref(params), _ptr(X), _ptr(D),
                          float(t0), float(dt), int(nsteps), int(scheme), int(precision),
                          _stream(stream)))


def rod_advance(ctx: Context, X, D, u, w, dt, stream=None):
    """``rod_advance``: X += u dt, frames rotated by |w| dt about w (in place, device float64
    state; u, w float32 or float64 tensors)."""
    import torch
    _check(lib().rod_advance(ctx.handle, int(X.shape[0]), _ptr(X), _ptr(D), _ptr(u), _ptr(w),
                             float(dt), 1 if u.dtype == torch.float64 else 0, _stream(stream)))


def rod_checkpoint_save(path, rod_off, X, D, t, stream=None):
    """``rod_checkpoint_save``: write t, offsets, X, D (device float64 tensors) to a file."""
    off, poff = _offsets(rod_off)
    _check(lib().rod_checkpoint_save(path.encode(), len(off) - 1, poff, _ptr(X), _ptr(D), float(t),
                                     _stream(stream)))


def rod_checkpoint_load(path, rod_off, X, D, stream=None):
    """``rod_checkpoint_load``: fill X, D from a checkpoint file; returns its time t."""
    off, poff = _offsets(rod_off)
    t = ctypes.c_double()
    _check(lib().rod_checkpoint_load(path.encode(), len(off) - 1, poff, _ptr(X), _ptr(D),
                                     ctypes.byref(t), _stream(stream)))
    return t.value


def rot_sqrt_batch(ctx: Context, R, S, stream=None):
    """``rot_sqrt_batch``: S[n,3,3] (device float64, overwritten) = principal sqrt of R[n,3,3]."""
    _check(lib().rot_sqrt_batch(ctx.handle, int(R.shape[0]), _ptr(R), _ptr(S), _stream(stream)))


def parareal_run(ctx: Context, rod_off, params: RodParams, X, D, T0, T1, n_slices, dt_fine,
                 coarse_ratio, max_iter, tol, stream=None, raise_on_noconv=True, group_size=0):
    """``parareal_run`` (group_size 0) or ``parareal_run_pipelined`` (group_size >= 1): Parareal
    in place on device float64 X, D; returns the statistics."""
    off, poff = _offsets(rod_off)
    st = PararealStats()
    if group_size:
        status = lib().parareal_run_pipelined(
            ctx.handle, len(off) - 1, poff, ctypes.byref(params), _ptr(X), _ptr(D), float(T0),
            float(T1), int(n_slices), float(dt_fine), int(coarse_ratio), int(max_iter),
            float(tol), int(group_size), ctypes.byref(st), _stream(stream))
    else:
        status = lib().parareal_run(ctx.handle, len(off) - 1, poff, ctypes.byref(params), _ptr(X),
                                    _ptr(D), float(T0), float(T1), int(n_slices), float(dt_fine),
                                    int(coarse_ratio), int(max_iter), float(tol), ctypes.byref(st),
                                    _stream(stream))
    if status == MRS_ENOCONV and not raise_on_noconv:
        return st
    _check(status)
    return st


class Server:
    """``mrs_server``: continuous batching of velocity and rod jobs on one GPU."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, max_slots: int):
        self.handle = _vp()
        self.ctx = ctx
        self._keep = {}
        _check(lib().serve_create(ctypes.byref(self.handle), ctx.handle, int(hbm_budget_bytes),
                                  int(max_slots)))

    def submit_velocity(self, X, f, n, u, w, mu, eps):
        j = Job()
        j.kind, j.n_points, j.mu, j.eps = MRS_JOB_VELOCITY, int(X.shape[0]), float(mu), float(eps)
        j.X, j.f, j.n, j.u, j.w = (t.data_ptr() for t in (X, f, n, u, w))
        return self._submit(j, (X, f, n, u, w))

    def submit_rod(self, rod_off, X, D, params: RodParams, t0, dt, nsteps, scheme, mu, eps):
        off, poff = _offsets(rod_off)
        j = Job()
        j.kind, j.n_points, j.mu, j.eps = MRS_JOB_ROD, int(X.shape[0]), float(mu), float(eps)
        j.n_rods, j.rod_off = len(off) - 1, poff
        j.Xr, j.Dr = X.data_ptr(), D.data_ptr()
        j.params = params
        j.t0, j.dt, j.nsteps, j.scheme = float(t0), float(dt), int(nsteps), int(scheme)
        return self._submit(j, (X, D, off))

    def _submit(self, j, keep):
        t = ctypes.c_uint64()
        _check(lib().serve_submit(self.handle, ctypes.byref(j), ctypes.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def poll(self, ticket):
        """(done, latency_s); raises if the job failed."""
        d, lat = ctypes.c_int(), ctypes.c_double()
        st = lib().serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(d), ctypes.byref(lat))
        if st == MRS_PENDING:
            return False, None
        _check(st)
        self._keep.pop(ticket, None)
        return True, lat.value

    def set_policy(self, big_job_pairs=1.3e10, max_big_jobs=1):
        """``serve_set_policy``: big-job threshold (pair interactions) and big jobs per iteration."""
        _check(lib().serve_set_policy(self.handle, float(big_job_pairs), int(max_big_jobs)))

    def inject_alloc_failure(self, ticket):
        """``serve_inject_alloc_failure``: make the admission of a waiting job fail (tests)."""
        _check(lib().serve_inject_alloc_failure(self.handle, ctypes.c_uint64(ticket)))

    def cancel(self, ticket):
        """``serve_cancel``: cancel a job that has not been admitted yet."""
        _check(lib().serve_cancel(self.handle, ctypes.c_uint64(ticket)))

    def drain(self, timeout_s=600.0):
        _check(lib().serve_drain(self.handle, float(timeout_s)))

    def stats(self):
        it, done, peak = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        pairs, pool, sym = ctypes.c_double(), ctypes.c_size_t(), ctypes.c_int64()
        _check(lib().serve_stats(self.handle, ctypes.byref(it), ctypes.byref(done),
                                 ctypes.byref(pairs), ctypes.byref(peak), ctypes.byref(pool),
                                 ctypes.byref(sym)))
        return {"iterations": it.value, "completed": done.value, "pairs": pairs.value,
                "peak_active": peak.value, "peak_pool_bytes": pool.value,
                "symmetric_iterations": sym.value}

    def close(self):
        if self.handle:
            _check(lib().serve_destroy(self.handle))
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
