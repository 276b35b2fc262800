"""Statistical and system tests of the CUDA sampler through the C ABI.

* T-LG on the GPU: the linear-Gaussian posterior is closed form; means and
  variances of 16 independent GPU chains match it within 4 standard errors.
* running moments and histograms equal numpy over the recorded GPU samples.
* T-MIX: FP32-mixed against FP64 -- Delta A relative error, accept-flip rate
  and posterior-mean shift (reported; loose bounds asserted).
* T-ERR, T-FAULT (bounded barrier wait, no hang), T-CKPT (bitwise resume).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import pimc, synth
from tests import _linear_gaussian as lgc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme,proposal", [(0, 0), (1, 1)])
def test_T_LG_gpu_chains_match_closed_form(scheme, proposal):
    prob = synth.lingauss_problem(M=10, data_seed=3, dt=0.5, Rm=4.0, Rf=(2.0, 2.0))
    prob.scheme, prob.proposal = scheme, proposal
    L, r, w = lgc.system(prob.M, prob.dt, prob.Rm, prob.Rf, prob.y, prob.I, p_free=True, scheme=scheme)
    mu, cov = lgc.posterior(L, r, w)
    csd = 1.0 / np.sqrt(np.diag(np.linalg.inv(cov)))
    nx = 2 * (prob.M + 1)
    means, vars_ = [], []
    for k in range(16):
        g = pimc.Sampler.from_problem(prob)
        kk = 1.0 if proposal == 0 else 1.7
        g.set_steps(kk * csd[:nx].reshape(2, prob.M + 1), np.array([2.0 * kk * csd[-1]]))
        g.set_chain(k)
        g.set_schedule(n_init=3000, n_skip=1)
        g.sweep(3000 + 25000, seed=2024)
        m, v, J = g.moments()
        assert J == 25000
        means.append(m)
        vars_.append(v)
    means = np.array(means)
    vars_ = np.array(vars_)
    se_m = means.std(0, ddof=1) / np.sqrt(16)
    se_v = vars_.std(0, ddof=1) / np.sqrt(16)
    assert np.all(np.abs(means.mean(0) - mu) < 4 * se_m)
    assert np.all(np.abs(vars_.mean(0) - np.diag(cov)) < 4 * se_v)


def test_moments_and_histograms_match_numpy_trace():
    prob = synth.hh_problem(300, data_seed=2)
    g = pimc.Sampler.from_problem(prob)
    n_init, n_skip = 5, 2
    g.set_schedule(n_init=n_init, n_skip=n_skip)
    M = prob.M
    comps = np.array([0 * (M + 1) + 5, 2 * (M + 1) + 150, 3 * (M + 1) + M, 4 * (M + 1) + 1])
    lo = np.array([-70.0, 0.2, 0.1, 20.0])
    hi = np.array([-60.0, 0.8, 0.6, 50.0])
    g.set_histograms(comps, lo, hi, 32)
    S = []
    for s in range(45):
        g.sweep(1, 31)
        if s >= n_init and (s - n_init) % n_skip == 0:
            X, p = g.state()
            S.append(np.concatenate([X.ravel(), p]))
    S = np.array(S)
    mean, var, J = g.moments()
    assert J == S.shape[0] == 20
    np.testing.assert_allclose(mean, S.mean(0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(var, S.var(0, ddof=1), rtol=1e-7, atol=1e-15)
    H = g.histograms()
    for k, c in enumerate(comps):
        v = S[:, c]
        inside, _ = np.histogram(v[(v >= lo[k]) & (v < hi[k])], bins=32, range=(lo[k], hi[k]))
        assert H[k, 0] == np.sum(v < lo[k]) and H[k, -1] == np.sum(v >= hi[k])
        assert np.array_equal(H[k, 1:-1], inside)


def test_T_MIX_fp32_mixed_against_fp64():
    prob = synth.hh_problem(4096, data_seed=1, free="all")
    X = synth.random_path_near(prob, prob.X_true, 0.3 * prob.sig_x, seed=1)
    Xp = synth.random_path_near(prob, X, 1.0 * prob.sig_x, seed=2)
    o = oracle.Chain(0, prob.M, prob.dt, prob.Rm, prob.Rf)
    o.set_data(prob.y, prob.I)
    o.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    o.set_path(X)
    d64, scale = o.site_delta_all(Xp)
    g32 = pimc.Sampler.from_problem(prob, precision=pimc.FP32_MIXED)
    g32.set_path(X)
    d32 = g32.site_delta(Xp)
    rel = np.abs(d32 - d64) / scale
    # FP32 arithmetic: error a few ulps of float relative to the condition scale
    assert np.median(rel) < 1e-5 and np.percentile(rel, 99) < 1e-3
    # accept-flip rate over one sweep from the same state and counters
    g64 = pimc.Sampler.from_problem(prob)
    for g in (g64, g32):
        g.set_path(X)
        g.sweep(1, 5)
    X64, _ = g64.state()
    X32, _ = g32.state()
    moved64 = np.any(X64 != X, axis=0)
    moved32 = np.any(np.abs(X32 - X) > 1e-5 * (1 + np.abs(X)), axis=0)
    flip_rate = np.mean(moved64 != moved32)
    assert flip_rate < 0.01, flip_rate


def test_T_ERR_boundary_rejects_bad_arguments():
    L = pimc.load()
    import ctypes
    h = ctypes.c_void_p()
    rm = np.array([4.0])
    rf = np.array([1e2, 1e4, 1e4, 1e4])
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert L.pimc_create(ctypes.byref(h), 0, 0, 4, 1, 0.02, P(rm), P(rf)) == pimc.ERR_ARG
    assert L.pimc_create(ctypes.byref(h), 0, 100, 3, 1, 0.02, P(rm), P(rf)) == pimc.ERR_ARG
    assert L.pimc_create(ctypes.byref(h), 0, 100, 4, 2, 0.02, P(rm), P(rf)) == pimc.ERR_ARG
    assert L.pimc_create(ctypes.byref(h), 0, 100, 4, 1, -1.0, P(rm), P(rf)) == pimc.ERR_ARG
    assert L.pimc_create(ctypes.byref(h), 0, 100, 4, 1, 0.02, P(np.array([0.0])), P(rf)) == pimc.ERR_ARG
    assert L.pimc_create(ctypes.byref(h), 9, 100, 4, 1, 0.02, P(rm), P(rf)) == pimc.ERR_ARG
    assert L.pimc_create(ctypes.byref(h), 0, 100, 4, 1, 0.02, P(rm), P(np.array([1.0, np.nan, 1, 1]))) == pimc.ERR_ARG
    prob = synth.hh_problem(50, data_seed=0)
    g = pimc.Sampler(0, 50, 0.02, prob.Rm, prob.Rf)
    with pytest.raises(pimc.PimcError) as e:
        g.sweep(1, 0)
    assert e.value.code == pimc.ERR_STATE
    y = prob.y.copy()
    y[3] = np.nan
    with pytest.raises(pimc.PimcError) as e:
        g.set_data(y, prob.I)
    assert e.value.code == pimc.ERR_ARG
    g.set_data(prob.y, prob.I)
    # streaming data: non-finite values anywhere (also in the last, unrolled-off
    # entries of the check) are rejected before anything is enqueued
    for which, idx, val in (("y", prob.M, np.inf), ("I", prob.M - 1, -np.inf), ("I", 2, np.nan)):
        yy, II = prob.y.copy(), prob.I.copy()
        (yy if which == "y" else II)[idx] = val
        with pytest.raises(pimc.PimcError) as e:
            g.load_data(yy.ctypes.data, II.ctypes.data)
        assert e.value.code == pimc.ERR_ARG
    bad = prob.p_init.copy()
    bad[0] = prob.hi[0] + 1.0
    with pytest.raises(pimc.PimcError) as e:
        g.set_params(bad, prob.lo, prob.hi, prob.free)
    assert e.value.code == pimc.ERR_ARG
    with pytest.raises(pimc.PimcError) as e:
        g.checkpoint_load("/nonexistent/file.ckpt")
    assert e.value.code == pimc.ERR_IO
    with pytest.raises(pimc.PimcError) as e:
        g.set_histograms([10 ** 9], [0.0], [1.0], 8)
    assert e.value.code == pimc.ERR_ARG
    # the handle and the CUDA context stay usable after every rejected call
    g.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    g.set_steps(prob.sig_x, prob.sig_p)
    g.sweep(3, 1)
    A, Ao, Af = g.action()
    assert np.isfinite(A)


@pytest.mark.parametrize("precision", ["fp64", "fp32mixed"])
def test_T_FAULT_bounded_barrier_wait_reports_timeout(precision):
    """One CTA skips its barrier arrivals (a flag nothing else sets): the other
    CTAs' bounded waits expire, the launch returns, the status reads
    PIMC_ERR_TIMEOUT, and the handle works again afterwards.  FP64 runs the
    general form (grid barriers), FP32-mixed the resident form (counted
    parameter-move sums and neighbour flags)."""
    prob = synth.hh_problem(2000, data_seed=0)
    g = pimc.Sampler.from_problem(prob, precision=pimc.FP64 if precision == "fp64" else pimc.FP32_MIXED)
    assert g.sweep_form() == ("general" if precision == "fp64" else "resident")
    grid, _ = g.launch_info()
    assert grid >= 2
    g.set_wait_limit(200_000_000)  # 0.2 s
    g.debug_skip_arrive(1)
    import time
    t0 = time.time()
    with pytest.raises(pimc.PimcError) as e:
        g.sweep(1, 3)
    assert e.value.code == pimc.ERR_TIMEOUT
    assert time.time() - t0 < 30
    g.debug_skip_arrive(-1)
    g.set_path(prob.X_true)
    g.sweep(5, 3)
    assert np.isfinite(g.action()[0])


def test_T_CKPT_resume_is_bitwise(tmp_path):
    prob = synth.hh_problem(777, data_seed=4, free="all")
    a = pimc.Sampler.from_problem(prob)
    a.set_schedule(n_init=10, n_skip=3, beta0=0.1, n_cool=15, f_acc=0.4, alpha=0.2)
    a.set_histograms([5, 900, 4 * 778], [-80.0, 0.0, 80.0], [-50.0, 1.0, 160.0], 10)
    a.sweep(20, 11)
    path = str(tmp_path / "run.ckpt")
    a.checkpoint_save(path)
    a.sweep(20, 11)
    Xa, pa = a.state()
    ma, va, Ja = a.moments()
    b = pimc.Sampler(0, prob.M, prob.dt, prob.Rm, prob.Rf)
    b.checkpoint_load(path)
    b.sweep(20, 11)
    Xb, pb = b.state()
    mb, vb, Jb = b.moments()
    assert np.array_equal(Xa, Xb) and np.array_equal(pa, pb)
    assert Ja == Jb and np.array_equal(ma, mb) and np.array_equal(va, vb, equal_nan=True)
    assert np.array_equal(a.histograms(), b.histograms())
    assert a.sweep_counter() == b.sweep_counter()
    # truncated and corrupted files are refused
    raw = open(path, "rb").read()
    open(path + ".short", "wb").write(raw[: len(raw) // 2])
    bad = bytearray(raw)
    bad[100] ^= 0xFF
    open(path + ".bad", "wb").write(bytes(bad))
    for p in (path + ".short", path + ".bad"):
        with pytest.raises(pimc.PimcError) as e:
            b.checkpoint_load(p)
        assert e.value.code == pimc.ERR_IO


def test_residual_moments_and_forecast_parity():
    prob = synth.hh_problem(120, data_seed=6, free="all")
    g = pimc.Sampler.from_problem(prob)
    g.set_schedule(n_init=3, n_skip=2)
    eps, dl = [], []
    for s in range(21):
        g.sweep(1, 19)
        if s >= 3 and (s - 3) % 2 == 0:
            X, p = g.state()
            f = np.array([oracle.model_map(0, prob.dt, X[:, n], p, prob.I[n]) for n in range(prob.M)]).T
            eps.append((X[:, 1:] - f).ravel())
            dl.append(X[0, 1:] - prob.y[1:])
    R = np.hstack([np.array(eps), np.array(dl)])
    mean, var, J = g.residual_moments()
    assert J == R.shape[0] == 9
    scale = np.abs(R).max(axis=0) + 1e-300
    assert np.all(np.abs(mean - R.mean(0)) <= 1e-10 * scale)
    np.testing.assert_allclose(var, R.var(0, ddof=1), rtol=1e-6, atol=1e-12 * scale.max() ** 2)
    # ensemble forecast from the same state: oracle and GPU, with and without noise
    X, p = g.state()
    o = oracle.Chain(0, prob.M, prob.dt, prob.Rm, prob.Rf)
    o.set_data(prob.y, prob.I)
    o.set_params(p, prob.lo, prob.hi, prob.free)
    o.set_path(X)
    Ifut = synth.ou_current(50, prob.dt, 99)
    for noise in (0, 1):
        fg = g.forecast(50, Ifut, 64, noise, 5)
        fo = o.forecast(50, Ifut, 64, noise, 5)
        np.testing.assert_allclose(fg, fo, rtol=1e-10, atol=1e-10)


def test_params_async_matches_the_synchronous_read():
    torch = pytest.importorskip("torch")
    prob = synth.hh_problem(500, data_seed=3, free="all")
    g = pimc.Sampler.from_problem(prob)
    buf = torch.zeros((3, 7), dtype=torch.float64).pin_memory()
    for k in range(3):
        g.sweep(2, 11, sync=False)
        g.params_async(buf[k].data_ptr())
    g.sync()
    assert np.array_equal(buf[2].numpy(), g.params())
    assert not np.array_equal(buf[0].numpy(), buf[2].numpy()) or np.all(np.isfinite(buf.numpy()))


@pytest.mark.parametrize("precision", [pimc.FP64, pimc.FP32_MIXED])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("M", [300, 512])
def test_load_data_equals_set_data(precision, scheme, M):
    """Streaming new data into a handle whose parameters are set (one launch:
    conversion and cache refresh) leaves it where a handle given that data
    from the start is: the sweeps that follow are bit for bit the same.  M =
    512 puts the trapezoid rule's last cached value (site M) at a multiple of
    the launch width."""
    p1 = synth.hh_problem(M, data_seed=1)
    p2 = synth.hh_problem(M, data_seed=2)

    def handle(y, I):
        g = pimc.Sampler(0, M, p1.dt, p1.Rm, p1.Rf)
        g.set_precision(precision)
        g.set_scheme(scheme)
        g.set_data(y, I)
        g.set_path(p1.X_true)
        g.set_params(p1.p_init, p1.lo, p1.hi, p1.free)
        g.set_steps(p1.sig_x, p1.sig_p)
        g.set_schedule(n_init=0, n_skip=1)
        return g

    direct = handle(p2.y, p2.I)
    streamed = handle(p1.y, p1.I)
    y2, I2 = np.ascontiguousarray(p2.y), np.ascontiguousarray(p2.I)
    streamed.load_data(y2.ctypes.data, I2.ctypes.data)
    for g in (direct, streamed):
        g.sweep(6, 11)
    (Xa, pa), (Xb, pb) = direct.state(), streamed.state()
    assert np.array_equal(Xa, Xb) and np.array_equal(pa, pb)
    ma, mb = direct.moments(), streamed.moments()
    assert np.array_equal(ma[0], mb[0]) and np.array_equal(ma[1], mb[1])
    assert direct.action() == streamed.action()
    direct.close()
    streamed.close()
