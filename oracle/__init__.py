"""Plain serial FP64 CPU oracle (ctypes wrapper around ``pimc_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  The CUDA library and
its Python binding never import it, and it imports nothing from them.

The C source follows the paper step by step: Eq. (action) with the Gaussian
assumptions of Sec. 2.1, the Metropolis rule of Eq. (Paccept), the checkerboard
state update and the sequential parameter moves of Fig. 1 / Sec. 4.1, the
annealing schedule of Eq. (fbeta) and the step-size rule of Sec. 4.2, and the
running path statistics of Sec. 4.1.  Which function is pinned by what is listed
in the header comment of ``pimc_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pimc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

MODEL_HH, MODEL_LINGAUSS, MODEL_TOY1D, MODEL_HH_PAPER = 0, 1, 2, 3
MODEL_DIMS = {MODEL_HH: (4, 7), MODEL_LINGAUSS: (2, 1), MODEL_TOY1D: (1, 1), MODEL_HH_PAPER: (4, 7)}
SCHEME_RK4, SCHEME_TRAPEZOID = 0, 1
PROPOSAL_GAUSS, PROPOSAL_UNIFORM = 0, 1


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with the host C compiler (no FMA contraction).
    openmp=True builds liboracle_omp.so from the same source with OpenMP on:
    the sites of a parity phase and the parameter-move sums split over host
    threads.  That build only times the method on all host cores; its sums add
    in another order, so the tests use the serial build."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "pimc_oracle.h")
    path = _OMP_PATH if openmp else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return path
    tmp = path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", _SRC, "-o", tmp, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.check_call(cmd)
    os.replace(tmp, path)
    return path


def lib(openmp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if openmp:
            if _lib_omp is None:
                L = ctypes.CDLL(build(openmp=True))
                _declare(L)
                _lib_omp = L
            return _lib_omp
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def threads(openmp: bool = False) -> int:
    return int(lib(openmp).orc_threads())


_d = ctypes.c_double
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_int = ctypes.c_int
_vp = ctypes.c_void_p


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_vp, _vp, _vp]
    L.orc_u01.argtypes = [_u32, _u32]
    L.orc_u01.restype = _d
    L.orc_site_draws.argtypes = [_u64, _u32, _u64, _i64, _int, _vp, _vp]
    L.orc_param_draws.argtypes = [_u64, _u32, _u64, _int, _vp, _vp]
    L.orc_model_rhs.argtypes = [_int, _vp, _vp, _d, _vp]
    L.orc_model_map.argtypes = [_int, _d, _vp, _vp, _d, _vp]
    L.orc_model_map_vjp.argtypes = [_int, _d, _vp, _vp, _d, _vp, _vp, _vp]
    L.orc_hh_rates.argtypes = [_d, _vp, _vp]
    L.orc_paper_gates.argtypes = [_d, _vp, _vp]
    L.orc_set_scheme.argtypes = [_vp, _int]
    L.orc_set_proposal.argtypes = [_vp, _int]
    L.orc_create.argtypes = [_int, _i64, _d, _d, _vp]
    L.orc_create.restype = _vp
    L.orc_destroy.argtypes = [_vp]
    L.orc_set_data.argtypes = [_vp, _vp, _vp]
    L.orc_set_params.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.orc_set_path.argtypes = [_vp, _vp]
    L.orc_set_steps.argtypes = [_vp, _vp, _int, _vp]
    L.orc_set_schedule.argtypes = [_vp, _i64, _i64, _d, _i64, _d, _d]
    L.orc_set_chain.argtypes = [_vp, _u32]
    L.orc_set_sweep_counter.argtypes = [_vp, _i64, _d]
    L.orc_sweep.argtypes = [_vp, _i64, _u64]
    L.orc_action.argtypes = [_vp, _vp, _vp, _vp]
    L.orc_site_delta_all.argtypes = [_vp, _vp, _d, _vp, _vp]
    L.orc_param_delta.argtypes = [_vp, _int, _d, _d, _vp]
    L.orc_param_delta.restype = _d
    L.orc_grad.argtypes = [_vp, _d, _vp, _vp]
    L.orc_get_state.argtypes = [_vp, _vp, _vp]
    L.orc_get_cache.argtypes = [_vp, _vp]
    L.orc_get_steps.argtypes = [_vp, _vp, _vp]
    L.orc_get_sweep.argtypes = [_vp, _vp]
    L.orc_get_sweep.restype = _i64
    L.orc_last_margins.argtypes = [_vp, _vp, _vp]
    L.orc_accept_stats.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.orc_moments.argtypes = [_vp, _vp, _vp]
    L.orc_moments.restype = _i64
    L.orc_set_histograms.argtypes = [_vp, _int, _vp, _vp, _vp, _int]
    L.orc_histograms.argtypes = [_vp, _vp]
    L.orc_hmc.argtypes = [_vp, _i64, _int, _d, _vp, _u64, _vp]
    L.orc_residual_moments.argtypes = [_vp, _vp, _vp]
    L.orc_residual_moments.restype = _i64
    L.orc_forecast.argtypes = [_vp, _i64, _vp, _int, _int, _u64, _vp]
    L.orc_fill_site_uniforms.argtypes = [_u64, _u32, _i64, _i64, _u64, _i64, _vp]
    L.orc_set_state_box.argtypes = [_vp, _vp, _vp]
    L.orc_site_update.argtypes = [_vp, _i64, _vp, _d]
    L.orc_param_update.argtypes = [_vp, _int, _d, _d]
    L.orc_threads.argtypes = []
    L.orc_threads.restype = _int


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- RNG -------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u01(hi, lo):
    return lib().orc_u01(int(hi), int(lo))


def site_draws(seed, chain, sweep, n, D):
    z = np.zeros(D)
    u = np.zeros(1)
    lib().orc_site_draws(seed, chain, sweep, n, D, _p(z), _p(u))
    return z, float(u[0])


def param_draws(seed, chain, sweep, l):
    z = np.zeros(1)
    u = np.zeros(1)
    lib().orc_param_draws(seed, chain, sweep, l, _p(z), _p(u))
    return float(z[0]), float(u[0])


def fill_site_uniforms(seed, chain, n0, nn, sweep0, ns):
    out = np.zeros((nn, ns))
    lib().orc_fill_site_uniforms(seed, chain, n0, nn, sweep0, ns, _p(out))
    return out


# ---- model -------------------------------------------------------------------
def model_rhs(model, x, p, I):
    D, _ = MODEL_DIMS[model]
    out = np.zeros(D)
    lib().orc_model_rhs(model, _p(_f64(x)), _p(_f64(p)), float(I), _p(out))
    return out


def model_map(model, dt, x, p, I):
    D, _ = MODEL_DIMS[model]
    out = np.zeros(D)
    lib().orc_model_map(model, float(dt), _p(_f64(x)), _p(_f64(p)), float(I), _p(out))
    return out


def model_map_vjp(model, dt, x, p, I, w):
    D, Np = MODEL_DIMS[model]
    gx = np.zeros(D)
    gp = np.zeros(Np)
    lib().orc_model_map_vjp(model, float(dt), _p(_f64(x)), _p(_f64(p)), float(I),
                            _p(_f64(w)), _p(gx), _p(gp))
    return gx, gp


def hh_rates(V):
    a = np.zeros(3)
    b = np.zeros(3)
    lib().orc_hh_rates(float(V), _p(a), _p(b))
    return a, b


def paper_gates(V):
    ainf = np.zeros(3)
    tau = np.zeros(3)
    lib().orc_paper_gates(float(V), _p(ainf), _p(tau))
    return ainf, tau


class Chain:
    """One Markov chain of the oracle sampler (serial FP64)."""

    def __init__(self, model, M, dt, Rm, Rf, openmp=False):
        self._L = lib(openmp)
        self.model = model
        self.D, self.Np = MODEL_DIMS[model]
        self.M = int(M)
        self._Rf = _f64(Rf)
        h = self._L.orc_create(model, self.M, float(dt), float(Rm), _p(self._Rf))
        if not h:
            raise ValueError("oracle: invalid arguments")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    # setup
    def set_data(self, y, I):
        y = _f64(y)
        I = _f64(I)
        assert y.shape == (self.M + 1,) and I.shape == (self.M,)
        self._L.orc_set_data(self._h, _p(y), _p(I))

    def set_params(self, p, lo=None, hi=None, free=None):
        p = _f64(p)
        lo = None if lo is None else _f64(lo)
        hi = None if hi is None else _f64(hi)
        fr = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
        self._L.orc_set_params(self._h, _p(p), _p(lo), _p(hi), _p(fr))

    def set_path(self, X=None):
        Xc = None if X is None else _f64(X).reshape(self.D * (self.M + 1))
        self._L.orc_set_path(self._h, _p(Xc))

    def set_steps(self, sig_x, sig_p):
        sx = _f64(sig_x)
        per_site = 1 if sx.size == self.D * (self.M + 1) else 0
        self._L.orc_set_steps(self._h, _p(sx.reshape(-1)), per_site, _p(_f64(sig_p)))

    def set_schedule(self, n_init=0, n_skip=1, beta0=1.0, n_cool=0, f_acc=0.4, alpha=0.0):
        r = self._L.orc_set_schedule(self._h, n_init, n_skip, float(beta0), n_cool,
                                   float(f_acc), float(alpha))
        if r != 0:
            raise ValueError("oracle: bad schedule")

    def set_state_box(self, lo, hi):
        self._L.orc_set_state_box(self._h, _p(_f64(lo)), _p(_f64(hi)))

    def site_update(self, n, z, u):
        return int(self._L.orc_site_update(self._h, int(n), _p(_f64(z)), float(u)))

    def param_update(self, l, z, u):
        return int(self._L.orc_param_update(self._h, int(l), float(z), float(u)))

    def set_scheme(self, scheme):
        if self._L.orc_set_scheme(self._h, int(scheme)) != 0:
            raise ValueError("bad scheme")

    def set_proposal(self, kind):
        if self._L.orc_set_proposal(self._h, int(kind)) != 0:
            raise ValueError("bad proposal kind")

    def set_chain(self, chain):
        self._L.orc_set_chain(self._h, chain)

    def set_sweep_counter(self, sweep, beta):
        self._L.orc_set_sweep_counter(self._h, sweep, float(beta))

    # run
    def sweep(self, n, seed):
        r = self._L.orc_sweep(self._h, int(n), int(seed))
        if r != 0:
            raise RuntimeError(f"oracle sweep failed ({r})")

    def hmc(self, n_traj, n_leap, eps, inv_mass, seed):
        im = _f64(inv_mass)
        assert im.size == self.D * (self.M + 1) + self.Np
        nacc = np.zeros(1, dtype=np.int64)
        r = self._L.orc_hmc(self._h, int(n_traj), int(n_leap), float(eps), _p(im), int(seed), _p(nacc))
        if r != 0:
            raise RuntimeError(f"oracle hmc failed ({r})")
        return int(nacc[0])

    # queries
    def action(self):
        out = np.zeros(3)
        a = out[0:1]; ao = out[1:2]; af = out[2:3]
        self._L.orc_action(self._h, _p(a), _p(ao), _p(af))
        return float(a[0]), float(ao[0]), float(af[0])

    def site_delta_all(self, Xp, beta=1.0):
        Xp = _f64(Xp).reshape(self.D * (self.M + 1))
        dA = np.zeros(self.M + 1)
        sc = np.zeros(self.M + 1)
        self._L.orc_site_delta_all(self._h, _p(Xp), float(beta), _p(dA), _p(sc))
        return dA, sc

    def param_delta(self, l, pl_new, beta=1.0):
        sc = np.zeros(1)
        dA = self._L.orc_param_delta(self._h, int(l), float(pl_new), float(beta), _p(sc))
        return float(dA), float(sc[0])

    def grad(self, beta=1.0):
        gX = np.zeros(self.D * (self.M + 1))
        gp = np.zeros(self.Np)
        self._L.orc_grad(self._h, float(beta), _p(gX), _p(gp))
        return gX.reshape(self.D, self.M + 1), gp

    def state(self):
        X = np.zeros(self.D * (self.M + 1))
        p = np.zeros(self.Np)
        self._L.orc_get_state(self._h, _p(X), _p(p))
        return X.reshape(self.D, self.M + 1), p

    def cache(self):
        f = np.zeros(self.D * (self.M + 1))
        self._L.orc_get_cache(self._h, _p(f))
        return f.reshape(self.D, self.M + 1)

    def steps(self):
        sx = np.zeros(self.D * (self.M + 1))
        sp = np.zeros(self.Np)
        self._L.orc_get_steps(self._h, _p(sx), _p(sp))
        return sx.reshape(self.D, self.M + 1), sp

    def sweep_counter(self):
        b = np.zeros(1)
        s = self._L.orc_get_sweep(self._h, _p(b))
        return int(s), float(b[0])

    def last_margins(self):
        sm = np.zeros(self.M + 1)
        pm = np.zeros(self.Np)
        self._L.orc_last_margins(self._h, _p(sm), _p(pm))
        return sm, pm

    def accept_stats(self):
        sa = np.zeros(2, dtype=np.uint64)
        sp = np.zeros(2, dtype=np.uint64)
        pa = np.zeros(self.Np, dtype=np.uint64)
        pp = np.zeros(self.Np, dtype=np.uint64)
        self._L.orc_accept_stats(self._h, _p(sa), _p(sp), _p(pa), _p(pp))
        return sa, sp, pa, pp

    def moments(self):
        nc = self.D * (self.M + 1) + self.Np
        mean = np.zeros(nc)
        var = np.zeros(nc)
        J = self._L.orc_moments(self._h, _p(mean), _p(var))
        return mean, var, int(J)

    def residual_moments(self):
        nr = (self.D + 1) * self.M
        mean = np.zeros(nr)
        var = np.zeros(nr)
        J = self._L.orc_residual_moments(self._h, _p(mean), _p(var))
        return mean, var, int(J)

    def forecast(self, n_steps, I, n_ens, noise, seed):
        out = np.zeros(n_ens * self.D * (n_steps + 1))
        self._L.orc_forecast(self._h, int(n_steps), _p(_f64(I)), int(n_ens), int(noise), int(seed), _p(out))
        return out.reshape(n_ens, self.D, n_steps + 1)

    def set_histograms(self, comp, lo, hi, n_bins):
        comp = np.ascontiguousarray(comp, dtype=np.int64)
        self._nsel = comp.size
        self._nbins = int(n_bins)
        self._L.orc_set_histograms(self._h, comp.size, _p(comp), _p(_f64(lo)), _p(_f64(hi)), int(n_bins))

    def histograms(self):
        out = np.zeros(self._nsel * (self._nbins + 2), dtype=np.uint64)
        self._L.orc_histograms(self._h, _p(out))
        return out.reshape(self._nsel, self._nbins + 2)
