"""Seeded synthetic inputs for the Hodgkin-Huxley data-assimilation workload.

This module holds the input recipe only: the Ornstein-Uhlenbeck drive current,
a finely integrated HH "physical system" that produces the true path, the noisy
voltage observations, the prior box, the initial parameter guess and initial
proposal scales.  It holds none of the sampler's arithmetic: the CUDA library
and the test oracle each compute the action, the model map and the initial
path with their own code, and both receive exactly the arrays made here.

Recipe (the paper's Sec. 5.1 setting, re-parameterised for the textbook HH
model in the modern convention):

* drive I: OU with mean 10, sd 5 uA/cm^2, correlation time 2 ms, exact
  discretisation I_{n+1} = mu + (I_n - mu) e^{-dt/tau} + sd sqrt(1 - e^{-2dt/tau}) xi_n,
  I_0 ~ N(mu, sd^2); held constant over each sample interval.
* truth: HH with (gNa, gK, gL, ENa, EK, EL, C) = (120, 36, 0.3, 50, -77, -54.4, 1),
  relaxed 50 ms at rest without current, then integrated at `substeps` RK4
  substeps per interval dt = 0.02 ms.
* observations y_n = V_n + 0.5 xi'_n (so Rm = 1/0.25), n = 0..M.
* Rf = (1e2, 1e4, 1e4, 1e4).
* prior box: +-50 % of |truth| around the truth for every parameter.
* initial guess p = truth (1 + 0.2 u_l), u_l ~ U(-1, 1), for the free parameters.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "synth_hh.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsynth_hh.so")
_lock = threading.Lock()
_lib = None

HH_TRUTH = np.array([120.0, 36.0, 0.3, 50.0, -77.0, -54.4, 1.0])
HH_NAMES = ("gNa", "gK", "gL", "ENa", "EK", "EL", "C")
HH_RF = np.array([1e2, 1e4, 1e4, 1e4])
HH_SIGMA_Y = 0.5
HH_DT = 0.02


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.synth_hh_truth.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                         ctypes.c_void_p]
            L.synth_hh_truth.restype = ctypes.c_int
            _lib = L
    return _lib


def ou_current(M: int, dt: float, seed: int, mean: float = 10.0, sd: float = 5.0,
               tau: float = 2.0) -> np.ndarray:
    """Exactly discretised OU current I_0..I_{M-1} (seeded)."""
    rng = np.random.default_rng([seed, 0x0C])
    a = np.exp(-dt / tau)
    b = sd * np.sqrt(1.0 - a * a)
    xi = rng.standard_normal(M)
    out = np.empty(M)
    # linear recursion I_n - mean = a (I_{n-1} - mean) + b xi_n, I_0 - mean = sd xi_0
    from scipy.signal import lfilter
    drive = b * xi
    drive[0] = sd * xi[0]
    out[:] = lfilter([1.0], [1.0, -a], drive) + mean
    return out


def hh_truth(M: int, dt: float, I: np.ndarray, q=HH_TRUTH, substeps: int = 10,
             relax_ms: float = 50.0) -> np.ndarray:
    X = np.zeros(4 * (M + 1))
    q = np.ascontiguousarray(q, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.float64)
    r = _load().synth_hh_truth(int(M), float(dt), int(substeps), q.ctypes.data, I.ctypes.data,
                               float(relax_ms), X.ctypes.data)
    if r != 0:
        raise ValueError("synth_hh_truth: bad arguments")
    return X.reshape(4, M + 1)


@dataclasses.dataclass
class Problem:
    """One data-assimilation problem instance (host arrays, FP64)."""
    model: int
    M: int
    dt: float
    Rm: float
    Rf: np.ndarray
    y: np.ndarray            # (M+1,)
    I: np.ndarray            # (M,)
    p_true: np.ndarray
    p_init: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    free: np.ndarray         # uint8
    sig_x: np.ndarray        # (D,) initial proposal scale per component
    sig_p: np.ndarray        # (Np,)
    X_true: np.ndarray | None = None
    data_seed: int = 0
    scheme: int = 0          # 0: explicit RK4 map, 1: trapezoid rule
    proposal: int = 0        # 0: Gaussian, 1: uniform U(-1, 1) increments

    @property
    def D(self) -> int:
        return int(self.Rf.size)

    @property
    def Np(self) -> int:
        return int(self.p_true.size)


def hh_problem(M: int, data_seed: int = 0, free=("gNa", "gK", "gL"), p_true=None,
               substeps: int = 10, dt: float = HH_DT) -> Problem:
    """HH problem: OU drive, fine-grid truth, y = V + 0.5 noise (Sec. 5.1 recipe)."""
    q = HH_TRUTH.copy() if p_true is None else np.asarray(p_true, dtype=np.float64).copy()
    I = ou_current(M, dt, data_seed)
    X = hh_truth(M, dt, I, q, substeps=substeps)
    rng = np.random.default_rng([data_seed, 0x0B5])
    y = X[0] + HH_SIGMA_Y * rng.standard_normal(M + 1)
    if free == "all":
        free = HH_NAMES
    fmask = np.array([1 if nm in free else 0 for nm in HH_NAMES], dtype=np.uint8)
    u = np.random.default_rng([data_seed, 0x1A17]).uniform(-1.0, 1.0, 7)
    p0 = np.where(fmask == 1, q * (1.0 + 0.2 * u), q)
    lo = q - 0.5 * np.abs(q)
    hi = q + 0.5 * np.abs(q)
    return Problem(model=0, M=M, dt=dt, Rm=1.0 / HH_SIGMA_Y ** 2, Rf=HH_RF.copy(), y=y, I=I,
                   p_true=q, p_init=p0, lo=lo, hi=hi, free=fmask,
                   sig_x=np.array([0.05, 0.005, 0.005, 0.005]),
                   sig_p=0.002 * np.abs(p0), X_true=X, data_seed=data_seed)


def random_path_near(prob: Problem, X0: np.ndarray, scale, seed: int) -> np.ndarray:
    """A seeded perturbation of a path (test input: states away from the chain's)."""
    rng = np.random.default_rng([seed, 0x9A7])
    return X0 + np.asarray(scale)[:, None] * rng.standard_normal(X0.shape)


def lingauss_problem(M: int, data_seed: int = 0, dt: float = 0.1, Rm: float = 4.0,
                     Rf=(25.0, 25.0), b_free: bool = True) -> Problem:
    """Linear-Gaussian test problem (D = 2, one offset parameter b); any y gives
    a Gaussian posterior, so y is a noisy sinusoid and I a seeded sequence."""
    rng = np.random.default_rng([data_seed, 0x11])
    t = np.arange(M + 1) * dt
    y = np.sin(1.3 * t) + 0.3 * rng.standard_normal(M + 1)
    I = 0.5 * rng.standard_normal(M)
    return Problem(model=1, M=M, dt=dt, Rm=Rm, Rf=np.asarray(Rf, dtype=np.float64), y=y, I=I,
                   p_true=np.array([0.2]), p_init=np.array([0.0]), lo=np.array([-50.0]),
                   hi=np.array([50.0]), free=np.array([1 if b_free else 0], dtype=np.uint8),
                   sig_x=np.array([0.25, 0.25]), sig_p=np.array([0.2]), data_seed=data_seed)


def toy_problem(M: int, data_seed: int = 0, dt: float = 0.1, Rm: float = 4.0, Rf: float = 9.0,
                p0: float = 1.0, p_free: bool = False, lo: float = 0.0, hi: float = 2.0) -> Problem:
    """Scalar nonlinear test problem dx/dt = p sin(x) - x/2 + I (D = 1)."""
    rng = np.random.default_rng([data_seed, 0x70])
    y = 0.8 + 0.3 * rng.standard_normal(M + 1)
    I = 0.1 * rng.standard_normal(M)
    return Problem(model=2, M=M, dt=dt, Rm=Rm, Rf=np.array([Rf]), y=y, I=I,
                   p_true=np.array([p0]), p_init=np.array([p0]), lo=np.array([lo]),
                   hi=np.array([hi]), free=np.array([1 if p_free else 0], dtype=np.uint8),
                   sig_x=np.array([0.4]), sig_p=np.array([0.3]), data_seed=data_seed)


# ---------------------------------------------------------------------------
# The paper's own HH variant (Sec. 5.1): tanh gate kinetics with the Table 1
# constants, the p1..p7 voltage equation in the shifted convention (rest near
# 0 mV), 25 kHz sampling, R_d = diag(100, 1e6, 1e6, 1e6), R_o = 100.
# ---------------------------------------------------------------------------
PAPER_TRUTH = np.array([1.0, 120.0, 115.0, 20.0, -12.0, 0.3, 10.6])
PAPER_NAMES = ("p1", "p2", "p3", "p4", "p5", "p6", "p7")
_PAPER_GATES = np.array([[25.0, 15.0, 0.1, 0.4],     # m: V_a, dV_a, tau0, tau1
                         [5.0, -15.0, 1.0, 7.0],     # h
                         [10.0, 30.0, 1.0, 5.0]])    # n


def _paper_field(s, q, I):
    V, m, h, n = s
    t = np.tanh((V - _PAPER_GATES[:, 0]) / _PAPER_GATES[:, 1])
    ainf = 0.5 + 0.5 * t
    tau = _PAPER_GATES[:, 2] + _PAPER_GATES[:, 3] * (1.0 - t * t)
    dV = q[0] * I + q[1] * m ** 3 * h * (q[2] - V) + q[3] * n ** 4 * (q[4] - V) + q[5] * (q[6] - V)
    return np.concatenate([[dV], (ainf - s[1:]) / tau])


def paper_truth(M, dt, I, q=PAPER_TRUTH, substeps=10, relax_ms=50.0):
    """Fine-grid integration of the paper's HH variant (drive held per interval)."""
    h = dt / substeps
    t = np.tanh((0.0 - _PAPER_GATES[:, 0]) / _PAPER_GATES[:, 1])
    s = np.concatenate([[0.0], 0.5 + 0.5 * t])

    def adv(s, I):
        k1 = _paper_field(s, q, I)
        k2 = _paper_field(s + 0.5 * h * k1, q, I)
        k3 = _paper_field(s + 0.5 * h * k2, q, I)
        k4 = _paper_field(s + h * k3, q, I)
        return s + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)

    for _ in range(int(relax_ms / h)):
        s = adv(s, 0.0)
    X = np.zeros((4, M + 1))
    X[:, 0] = s
    for n in range(M):
        for _ in range(substeps):
            s = adv(s, I[n])
        X[:, n + 1] = s
    return X


def paper_problem(M, data_seed=0, free="all", dt=0.04, scheme=1, proposal=1, substeps=10):
    """Problem in the paper's setting: HH variant, trapezoid rule, uniform proposals."""
    q = PAPER_TRUTH.copy()
    I = ou_current(M, dt, data_seed)
    X = paper_truth(M, dt, I, q, substeps=substeps)
    rng = np.random.default_rng([data_seed, 0xA9])
    y = X[0] + 0.1 * rng.standard_normal(M + 1)
    if free == "all":
        free = PAPER_NAMES
    fmask = np.array([1 if nm in free else 0 for nm in PAPER_NAMES], dtype=np.uint8)
    u = np.random.default_rng([data_seed, 0x1A18]).uniform(-1.0, 1.0, 7)
    p0 = np.where(fmask == 1, q * (1.0 + 0.2 * u), q)
    lo = q - 0.5 * np.abs(q)
    hi = q + 0.5 * np.abs(q)
    return Problem(model=3, M=M, dt=dt, Rm=100.0, Rf=np.array([1e2, 1e6, 1e6, 1e6]), y=y, I=I,
                   p_true=q, p_init=p0, lo=lo, hi=hi, free=fmask,
                   sig_x=np.array([2e-3, 1e-3, 1e-3, 1e-3]), sig_p=0.002 * np.abs(p0), X_true=X,
                   data_seed=data_seed, scheme=scheme, proposal=proposal)
