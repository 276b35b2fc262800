"""Python binding of the C ABI in include/pimc.h (argument marshalling only).

Every step of the sampler runs in the CUDA library ``_build/libpimc.so``; this
module only converts numpy/torch arguments to pointers and error codes to
exceptions.  There is no CPU fallback: without the built library every entry
point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

from . import build as _build

FP64, FP32_MIXED = 0, 1
MODEL_HH, MODEL_LINGAUSS, MODEL_TOY1D, MODEL_HH_PAPER = 0, 1, 2, 3
MODEL_DIMS = {MODEL_HH: (4, 7), MODEL_LINGAUSS: (2, 1), MODEL_TOY1D: (1, 1), MODEL_HH_PAPER: (4, 7)}
SCHEME_RK4, SCHEME_TRAPEZOID = 0, 1
PROPOSAL_GAUSS, PROPOSAL_UNIFORM = 0, 1

OK, ERR_ARG, ERR_STATE, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NUMERIC, ERR_IO = 0, -1, -2, -3, -4, -5, -6, -7
_ERRNAMES = {ERR_ARG: "PIMC_ERR_ARG", ERR_STATE: "PIMC_ERR_STATE", ERR_CUDA: "PIMC_ERR_CUDA",
             ERR_OOM: "PIMC_ERR_OOM", ERR_TIMEOUT: "PIMC_ERR_TIMEOUT", ERR_NUMERIC: "PIMC_ERR_NUMERIC",
             ERR_IO: "PIMC_ERR_IO"}

# Every symbol include/pimc.h declares (checked by the test suite).
EXPORTS = [
    "pimc_create", "pimc_destroy", "pimc_last_error", "pimc_set_stream", "pimc_set_precision",
    "pimc_set_scheme", "pimc_set_proposal",
    "pimc_set_data", "pimc_load_data", "pimc_set_params", "pimc_set_path", "pimc_set_steps", "pimc_set_schedule",
    "pimc_set_chain", "pimc_sweep", "pimc_hmc", "pimc_sync", "pimc_action", "pimc_grad", "pimc_action_dev",
    "pimc_grad_dev", "pimc_site_delta", "pimc_param_delta", "pimc_moments", "pimc_set_histograms",
    "pimc_histograms", "pimc_histogram_shape", "pimc_set_param_trace", "pimc_param_trace", "pimc_get_state", "pimc_params_async", "pimc_get_steps", "pimc_get_sweep", "pimc_accept_stats",
    "pimc_launch_info", "pimc_sweep_form", "pimc_set_sweep_form", "pimc_residual_moments", "pimc_forecast", "pimc_checkpoint_save", "pimc_checkpoint_load", "pimc_set_wait_limit",
    "pimc_debug_skip_arrive", "pimc_debug_check_counts", "pimc_debug_fix_sum", "pimc_debug_map_rate", "pimc_debug_lane_maps", "pimc_set_grid", "pimc_action_static",
    "pimc_batch_create", "pimc_batch_destroy", "pimc_batch_last_error", "pimc_batch_sweep", "pimc_batch_sync",
    "pimc_batch_set_tuning", "pimc_batch_info", "pimc_batch_autotune",
]


class PimcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_d = ctypes.c_double


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the CUDA library (fails loudly when it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _build.LIB
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA sampler library not built ({p}); run __graft_entry__.build()")
            L = ctypes.CDLL(p)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    sig = {
        "pimc_create": [_vp, _int, _i64, _int, _int, _d, _vp, _vp],
        "pimc_destroy": [_vp],
        "pimc_set_stream": [_vp, _vp],
        "pimc_set_precision": [_vp, _int],
        "pimc_set_scheme": [_vp, _int],
        "pimc_set_proposal": [_vp, _int],
        "pimc_set_data": [_vp, _vp, _vp],
        "pimc_load_data": [_vp, _vp, _vp],
        "pimc_set_params": [_vp, _vp, _vp, _vp, _vp, _int],
        "pimc_set_path": [_vp, _vp],
        "pimc_set_steps": [_vp, _vp, _int, _vp],
        "pimc_set_schedule": [_vp, _i64, _i64, _d, _i64, _d, _d],
        "pimc_set_chain": [_vp, ctypes.c_uint32],
        "pimc_sweep": [_vp, _i64, ctypes.c_uint64],
        "pimc_sync": [_vp],
        "pimc_hmc": [_vp, _i64, _int, _d, _vp, ctypes.c_uint64, _vp],
        "pimc_action": [_vp, _vp, _vp, _vp],
        "pimc_grad": [_vp, _d, _vp, _vp],
        "pimc_action_dev": [_vp, _vp, _vp, _vp, _vp],
        "pimc_grad_dev": [_vp, _vp, _vp, _d, _vp, _vp, _vp],
        "pimc_site_delta": [_vp, _vp, _d, _vp],
        "pimc_param_delta": [_vp, _int, _d, _d, _vp],
        "pimc_moments": [_vp, _vp, _vp, _vp],
        "pimc_set_histograms": [_vp, _int, _vp, _vp, _vp, _int],
        "pimc_histograms": [_vp, _vp],
        "pimc_histogram_shape": [_vp, _vp, _vp],
        "pimc_set_param_trace": [_vp, _i64],
        "pimc_param_trace": [_vp, _vp, _i64, _vp],
        "pimc_get_state": [_vp, _vp, _vp],
        "pimc_get_steps": [_vp, _vp, _vp],
        "pimc_get_sweep": [_vp, _vp, _vp],
        "pimc_accept_stats": [_vp, _vp, _vp, _vp, _vp],
        "pimc_launch_info": [_vp, _vp, _vp],
        "pimc_sweep_form": [_vp, _vp],
        "pimc_set_sweep_form": [_vp, _int],
        "pimc_residual_moments": [_vp, _vp, _vp, _vp],
        "pimc_forecast": [_vp, _i64, _vp, _int, _int, ctypes.c_uint64, _vp],
        "pimc_checkpoint_save": [_vp, ctypes.c_char_p],
        "pimc_checkpoint_load": [_vp, ctypes.c_char_p],
        "pimc_set_wait_limit": [_vp, _i64],
        "pimc_debug_skip_arrive": [_vp, _int],
        "pimc_debug_fix_sum": [_vp, _i64, _int, _vp],
        "pimc_debug_check_counts": [_vp, _vp, _vp, _vp, _vp, _vp, _int],
        "pimc_debug_lane_maps": [_vp, _vp, _vp, _d, _i64, _vp, _vp],
        "pimc_debug_map_rate": [_int, _int, _i64, _vp],
        "pimc_params_async": [_vp, _vp],
        "pimc_set_grid": [_vp, _int],
        "pimc_action_static": [_int, _i64, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
        "pimc_batch_create": [_vp, _vp, _int],
        "pimc_batch_destroy": [_vp],
        "pimc_batch_sweep": [_vp, _i64, ctypes.c_uint64],
        "pimc_batch_sync": [_vp],
        "pimc_batch_set_tuning": [_vp, _int, _int, _int],
        "pimc_batch_info": [_vp, _vp, _vp, _vp],
        "pimc_batch_autotune": [_vp, _i64, ctypes.c_uint64, _vp, _vp, _vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _int
    L.pimc_last_error.argtypes = [_vp]
    L.pimc_last_error.restype = ctypes.c_char_p
    L.pimc_batch_last_error.argtypes = [_vp]
    L.pimc_batch_last_error.restype = ctypes.c_char_p


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def action_static(model, M, dt, Rm, Rf, X_ptr, p_ptr, y_ptr, I_ptr, out_ptr, stream_ptr):
    """Allocation-free FP64 action of caller-owned device arrays (no handle).
    Rf must hold exactly D doubles for the model: the library reads D of them."""
    L = load()
    rf = _f64(Rf).ravel()
    if int(model) not in MODEL_DIMS or rf.size != MODEL_DIMS[int(model)][0]:
        raise PimcError(ERR_ARG, f"Rf must hold D = {MODEL_DIMS.get(int(model), ('?',))[0]} values for model "
                                 f"{model}, got {rf.size}")
    r = L.pimc_action_static(int(model), int(M), float(dt), float(Rm), _p(rf), _vp(X_ptr), _vp(p_ptr),
                             _vp(y_ptr), _vp(I_ptr), _vp(out_ptr), _vp(stream_ptr))
    if r != OK:
        raise PimcError(r, L.pimc_last_error(None).decode())


def debug_fix_sum(terms, as_float=False, acc128=False):
    """The exact sum parameter moves use, applied to a host array (test hook);
    acc128: FP32 terms through the general form's 128-bit per-thread sum."""
    L = load()
    t = _f64(terms)
    out = np.zeros(1)
    mode = 2 if acc128 else (1 if as_float else 0)
    r = L.pimc_debug_fix_sum(_p(t), int(t.size), mode, _p(out))
    if r != OK:
        raise PimcError(r, L.pimc_last_error(None).decode())
    return float(out[0])


def debug_map_rate(packed, ctas_per_sm, iters=2000, fp64=False):
    """HH maps per second of the map alone, iterated from registers (test
    hook): FP32 single or packed lanes, or the FP64 map."""
    L = load()
    out = np.zeros(1)
    form = 2 if fp64 else (1 if packed else 0)
    r = L.pimc_debug_map_rate(form, int(ctas_per_sm), int(iters), _p(out))
    if r != OK:
        raise PimcError(r, L.pimc_last_error(None).decode())
    return float(out[0])


def debug_lane_maps(X, I, p, dt):
    """FP32 HH maps of the sites (columns of X) in the single-site form, and the
    number of pair components whose packed two-lane map differs (test hook)."""
    L = load()
    Xc = _f64(X).reshape(4, -1)
    n = Xc.shape[1]
    Ic, pc = _f64(I), _f64(p)
    assert Ic.size == n and pc.size == 7
    f = np.zeros((4, n))
    m = np.zeros(1, dtype=np.int64)
    r = L.pimc_debug_lane_maps(_p(Xc), _p(Ic), _p(pc), float(dt), int(n), _p(f), _p(m))
    if r != OK:
        raise PimcError(r, L.pimc_last_error(None).decode())
    return f, int(m[0])


class Sampler:
    """Handle of the GPU sampler for one chain over one data set."""

    def __init__(self, model, M, dt, Rm, Rf, precision=FP64):
        self._L = load()
        self.model = int(model)
        self.D, self.Np = MODEL_DIMS[self.model]
        self.M = int(M)
        h = ctypes.c_void_p()
        rm = np.array([float(Rm)])
        rf = _f64(Rf)
        r = self._L.pimc_create(ctypes.byref(h), self.model, self.M, self.D, 1, float(dt), _p(rm), _p(rf))
        if r != OK:
            raise PimcError(r, self._L.pimc_last_error(None).decode())
        self._h = h
        if precision != FP64:
            self.set_precision(precision)

    @classmethod
    def from_problem(cls, prob, precision=FP64):
        s = cls(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf, precision)
        if getattr(prob, "scheme", 0):
            s.set_scheme(prob.scheme)
        if getattr(prob, "proposal", 0):
            s.set_proposal(prob.proposal)
        s.set_data(prob.y, prob.I)
        s.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
        s.set_steps(prob.sig_x, prob.sig_p)
        return s

    def _ck(self, r):
        if r != OK:
            raise PimcError(r, self._L.pimc_last_error(self._h).decode())

    def close(self):
        # a batch holding this handle goes first (its launches use the handle's
        # stream and buffers)
        for b in list(getattr(self, "_batches", ())):
            b.close()
        if getattr(self, "_h", None):
            self._L.pimc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- setup
    def set_stream(self, stream_ptr):
        self._ck(self._L.pimc_set_stream(self._h, ctypes.c_void_p(int(stream_ptr))))

    def set_precision(self, precision):
        self._ck(self._L.pimc_set_precision(self._h, int(precision)))

    def set_scheme(self, scheme):
        self._ck(self._L.pimc_set_scheme(self._h, int(scheme)))

    def set_proposal(self, kind):
        self._ck(self._L.pimc_set_proposal(self._h, int(kind)))

    def set_data(self, y, I):
        self._ck(self._L.pimc_set_data(self._h, _p(_f64(y)), _p(_f64(I))))

    def load_data(self, y_ptr, I_ptr):
        """New data (host pointers, e.g. pinned tensors) for the running chain."""
        self._ck(self._L.pimc_load_data(self._h, _vp(y_ptr), _vp(I_ptr)))

    def set_params(self, p, lo=None, hi=None, free=None):
        fr = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
        self._ck(self._L.pimc_set_params(self._h, _p(_f64(p)), _p(None if lo is None else _f64(lo)),
                                         _p(None if hi is None else _f64(hi)), _p(fr), self.Np))

    def set_path(self, X=None):
        self._ck(self._L.pimc_set_path(self._h, _p(None if X is None else _f64(X).reshape(-1))))

    def set_steps(self, sig_x, sig_p):
        sx = _f64(sig_x).reshape(-1)
        per_site = 1 if sx.size == self.D * (self.M + 1) else 0
        self._ck(self._L.pimc_set_steps(self._h, _p(sx), per_site, _p(_f64(sig_p))))

    def set_schedule(self, n_init=0, n_skip=1, beta0=1.0, n_cool=0, f_acc=0.4, alpha=0.0):
        self._ck(self._L.pimc_set_schedule(self._h, int(n_init), int(n_skip), float(beta0), int(n_cool),
                                           float(f_acc), float(alpha)))

    def set_chain(self, chain):
        self._ck(self._L.pimc_set_chain(self._h, int(chain)))

    def set_grid(self, grid):
        self._ck(self._L.pimc_set_grid(self._h, int(grid)))

    def set_wait_limit(self, ns):
        self._ck(self._L.pimc_set_wait_limit(self._h, int(ns)))

    def debug_skip_arrive(self, cta):
        self._ck(self._L.pimc_debug_skip_arrive(self._h, int(cta)))

    # ---- run
    def sweep(self, n, seed, sync=True):
        self._ck(self._L.pimc_sweep(self._h, int(n), int(seed)))
        if sync:
            self.sync()

    def hmc(self, n_traj, n_leap, eps, inv_mass=None, seed=0, wait=True):
        """Whole-path HMC trajectories; returns the number accepted.  With
        wait=False the trajectories are only enqueued on the handle's stream
        (no accept count, no synchronisation) and None is returned."""
        im = None if inv_mass is None else _f64(inv_mass)
        if im is not None:
            assert im.size == self.D * (self.M + 1) + self.Np
        n = np.zeros(1, dtype=np.int64)
        self._ck(self._L.pimc_hmc(self._h, int(n_traj), int(n_leap), float(eps), _p(im), int(seed),
                                  _p(n) if wait else None))
        return int(n[0]) if wait else None

    def sync(self):
        self._ck(self._L.pimc_sync(self._h))

    # ---- queries
    def action(self):
        a = np.zeros(3)
        self._ck(self._L.pimc_action(self._h, _p(a[0:1]), _p(a[1:2]), _p(a[2:3])))
        return float(a[0]), float(a[1]), float(a[2])

    def grad(self, beta=1.0):
        gX = np.zeros(self.D * (self.M + 1))
        gp = np.zeros(self.Np)
        self._ck(self._L.pimc_grad(self._h, float(beta), _p(gX), _p(gp)))
        return gX.reshape(self.D, self.M + 1), gp

    def action_dev(self, X_ptr, p_ptr, out_ptr, stream_ptr):
        self._ck(self._L.pimc_action_dev(self._h, _vp(X_ptr), _vp(p_ptr), _vp(out_ptr), _vp(stream_ptr)))

    def grad_dev(self, X_ptr, p_ptr, beta, gX_ptr, gp_ptr, stream_ptr):
        self._ck(self._L.pimc_grad_dev(self._h, _vp(X_ptr), _vp(p_ptr), float(beta), _vp(gX_ptr),
                                       _vp(gp_ptr), _vp(stream_ptr)))

    def site_delta(self, Xp, beta=1.0):
        out = np.zeros(self.M + 1)
        self._ck(self._L.pimc_site_delta(self._h, _p(_f64(Xp).reshape(-1)), float(beta), _p(out)))
        return out

    def param_delta(self, l, pl_new, beta=1.0):
        out = np.zeros(1)
        self._ck(self._L.pimc_param_delta(self._h, int(l), float(pl_new), float(beta), _p(out)))
        return float(out[0])

    def moments(self):
        nc = self.D * (self.M + 1) + self.Np
        mean = np.zeros(nc)
        var = np.zeros(nc)
        J = np.zeros(1, dtype=np.int64)
        self._ck(self._L.pimc_moments(self._h, _p(mean), _p(var), _p(J)))
        return mean, var, int(J[0])

    def residual_moments(self):
        nr = (self.D + 1) * self.M
        mean, var = np.zeros(nr), np.zeros(nr)
        J = np.zeros(1, dtype=np.int64)
        self._ck(self._L.pimc_residual_moments(self._h, _p(mean), _p(var), _p(J)))
        return mean, var, int(J[0])

    def forecast(self, n_steps, I_future, n_ens, noise, seed):
        out = np.zeros(int(n_ens) * self.D * (int(n_steps) + 1))
        self._ck(self._L.pimc_forecast(self._h, int(n_steps), _p(_f64(I_future)), int(n_ens), int(noise),
                                       int(seed), _p(out)))
        return out.reshape(int(n_ens), self.D, int(n_steps) + 1)

    def set_histograms(self, comp, lo, hi, n_bins):
        comp = np.ascontiguousarray(comp, dtype=np.int64)
        self._ck(self._L.pimc_set_histograms(self._h, comp.size, _p(comp), _p(_f64(lo)), _p(_f64(hi)),
                                             int(n_bins)))

    def histograms(self):
        ns, nb = ctypes.c_int(), ctypes.c_int()
        self._ck(self._L.pimc_histogram_shape(self._h, ctypes.byref(ns), ctypes.byref(nb)))
        out = np.zeros(ns.value * (nb.value + 2), dtype=np.uint64)
        self._ck(self._L.pimc_histograms(self._h, _p(out)))
        return out.reshape(ns.value, nb.value + 2)

    def set_param_trace(self, cap):
        self._ck(self._L.pimc_set_param_trace(self._h, int(cap)))

    def param_trace(self):
        n = np.zeros(1, dtype=np.int64)
        self._ck(self._L.pimc_param_trace(self._h, None, 0, _p(n)))
        out = np.zeros(int(n[0]) * self.Np)
        self._ck(self._L.pimc_param_trace(self._h, _p(out), int(n[0]), _p(n)))
        return out.reshape(int(n[0]), self.Np)

    def state(self):
        X = np.zeros(self.D * (self.M + 1))
        p = np.zeros(self.Np)
        self._ck(self._L.pimc_get_state(self._h, _p(X), _p(p)))
        return X.reshape(self.D, self.M + 1), p

    def params(self):
        p = np.zeros(self.Np)
        self._ck(self._L.pimc_get_state(self._h, None, _p(p)))
        return p

    def params_async(self, p_ptr):
        """Enqueue a copy of p into caller-owned host memory (Np doubles at
        p_ptr, page-locked for asynchrony); valid after the stream syncs."""
        self._ck(self._L.pimc_params_async(self._h, _vp(p_ptr)))

    def steps(self):
        sx = np.zeros(self.D * (self.M + 1))
        sp = np.zeros(self.Np)
        self._ck(self._L.pimc_get_steps(self._h, _p(sx), _p(sp)))
        return sx.reshape(self.D, self.M + 1), sp

    def sweep_counter(self):
        s = np.zeros(1, dtype=np.int64)
        b = np.zeros(1)
        self._ck(self._L.pimc_get_sweep(self._h, _p(s), _p(b)))
        return int(s[0]), float(b[0])

    def accept_stats(self):
        sa = np.zeros(2, dtype=np.uint64)
        sp = np.zeros(2, dtype=np.uint64)
        pa = np.zeros(self.Np, dtype=np.uint64)
        pp = np.zeros(self.Np, dtype=np.uint64)
        self._ck(self._L.pimc_accept_stats(self._h, _p(sa), _p(sp), _p(pa), _p(pp)))
        return sa, sp, pa, pp

    def launch_info(self):
        g = ctypes.c_int()
        b = ctypes.c_int()
        self._ck(self._L.pimc_launch_info(self._h, ctypes.byref(g), ctypes.byref(b)))
        return g.value, b.value

    def check_counts(self, reset=True):
        """Checked builds: per-site visit counts (even phase, odd phase,
        parameter-move cache writes), the executed parameter moves and the
        sticky status (test hook)."""
        n1 = self.M + 1
        ev, od, pa = (np.zeros(n1, dtype=np.uint32) for _ in range(3))
        mv = np.zeros(1, dtype=np.uint64)
        st = np.zeros(1, dtype=np.int32)
        self._ck(self._L.pimc_debug_check_counts(self._h, _p(ev), _p(od), _p(pa), _p(mv), _p(st), 1 if reset else 0))
        return ev, od, pa, int(mv[0]), int(st[0])

    def set_sweep_form(self, form):
        """'auto' (the resident form where it fits) or 'general'."""
        self._ck(self._L.pimc_set_sweep_form(self._h, {"auto": 0, "general": 1}.get(form, -1)))

    def sweep_form(self):
        """'resident' (one site a thread for the whole launch) or 'general'."""
        r = ctypes.c_int()
        self._ck(self._L.pimc_sweep_form(self._h, ctypes.byref(r)))
        return "resident" if r.value else "general"

    def checkpoint_save(self, path):
        self._ck(self._L.pimc_checkpoint_save(self._h, os.fsencode(path)))

    def checkpoint_load(self, path):
        self._ck(self._L.pimc_checkpoint_load(self._h, os.fsencode(path)))


class Batch:
    """Many chains (each a Sampler) in one launch; chain state stays in the Samplers."""

    def __init__(self, samplers):
        self._L = load()
        self.samplers = list(samplers)
        arr = (ctypes.c_void_p * len(self.samplers))(*[s._h.value for s in self.samplers])
        b = ctypes.c_void_p()
        r = self._L.pimc_batch_create(ctypes.byref(b), arr, len(self.samplers))
        if r != OK:
            raise PimcError(r, self._L.pimc_batch_last_error(None).decode())
        self._b = b
        for s in self.samplers:
            if not hasattr(s, "_batches"):
                s._batches = weakref.WeakSet()
            s._batches.add(self)

    def _ck(self, r):
        if r != OK:
            raise PimcError(r, self._L.pimc_batch_last_error(self._b).decode())

    def sweep(self, n, seed, sync=True):
        self._ck(self._L.pimc_batch_sweep(self._b, int(n), int(seed)))
        if sync:
            self.sync()

    def sync(self):
        self._ck(self._L.pimc_batch_sync(self._b))

    def set_tuning(self, threads_per_cta, ctas_per_sm, ctas_per_chain=1):
        self._ck(self._L.pimc_batch_set_tuning(self._b, int(threads_per_cta), int(ctas_per_sm), int(ctas_per_chain)))

    def info(self):
        """(CTAs of a launch, threads per CTA, chains split over several CTAs)."""
        n, t, sp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._ck(self._L.pimc_batch_info(self._b, ctypes.byref(n), ctypes.byref(t), ctypes.byref(sp)))
        return n.value, t.value, sp.value

    def autotune(self, trial_sweeps, seed):
        """Returns (threads per CTA, CTAs per SM, CTAs per long chain)."""
        t, k, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._ck(self._L.pimc_batch_autotune(self._b, int(trial_sweeps), int(seed), ctypes.byref(t), ctypes.byref(k),
                                             ctypes.byref(g)))
        return t.value, k.value, g.value

    def close(self):
        if getattr(self, "_b", None):
            self._L.pimc_batch_destroy(self._b)
            self._b = None
            for s in self.samplers:
                getattr(s, "_batches", set()).discard(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
