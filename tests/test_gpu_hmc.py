"""Whole-path HMC on the GPU (pimc_hmc) against the oracle's HMC and against
the closed-form linear-Gaussian posterior.

* replay: same seed and Philox counters, trajectory by trajectory from the same
  state; accept decisions must agree (a differing decision must sit within
  1e-9 of its threshold) and accepted end points must agree to the leapfrog's
  rounding (FP64).
* T-LG: means and variances of 32 independent GPU HMC chains match the closed
  form within 4 standard errors (FP64 and FP32-mixed).
"""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import pimc, synth
from tests import _linear_gaussian as lgc

pytestmark = pytest.mark.gpu


def _oracle(prob):
    ch = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf)
    ch.set_scheme(prob.scheme)
    ch.set_data(prob.y, prob.I)
    ch.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    return ch


@pytest.mark.parametrize("model", ["lg", "hh", "lg_trap", "hh_many_tiles"])
def test_hmc_replay_against_oracle(model):
    n_traj = 30
    if model == "hh_many_tiles":
        # 40 001 sites: more tiles than the leapfrog kernel's CTAs (two an SM),
        # so CTAs stride over tiles; a few trajectories keep the oracle quick
        prob = synth.hh_problem(40000, data_seed=4, free=("gNa", "gK", "gL"))
        inv_mass = np.concatenate([np.tile([5e-3, 5e-5, 5e-5, 5e-5], (prob.M + 1, 1)).T.ravel(),
                                   1e-3 * np.abs(prob.p_init)])
        eps, n_leap, n_traj = 2e-3, 4, 4  # small steps from the truth: accepted trajectories
    elif model.startswith("lg"):
        prob = synth.lingauss_problem(M=10, data_seed=3, dt=0.5, Rm=4.0, Rf=(2.0, 2.0))
        prob.scheme = 1 if model == "lg_trap" else 0
        L, r, w = lgc.system(prob.M, prob.dt, prob.Rm, prob.Rf, prob.y, prob.I, p_free=True, scheme=prob.scheme)
        mu, cov = lgc.posterior(L, r, w)
        inv_mass = np.diag(cov).copy()
        eps, n_leap = 0.2, 12
    else:
        prob = synth.hh_problem(48, data_seed=2, free=("gNa", "gK", "gL"))
        inv_mass = np.concatenate([np.tile([5e-3, 5e-5, 5e-5, 5e-5], (prob.M + 1, 1)).T.ravel(),
                                   1e-2 * np.abs(prob.p_init)])
        eps, n_leap = 0.1, 8
    g = pimc.Sampler.from_problem(prob)
    if model == "hh_many_tiles":
        g.set_path(prob.X_true)
        g.set_params(prob.p_true, prob.lo, prob.hi, prob.free)
    o = _oracle(prob)
    agree = 0
    for t in range(n_traj):
        X0, p0 = g.state()
        o.set_path(X0)
        o.set_params(p0, prob.lo, prob.hi, prob.free)
        o.set_sweep_counter(t, 1.0)
        na_g = g.hmc(1, n_leap, eps, inv_mass, seed=5)
        na_o = o.hmc(1, n_leap, eps, inv_mass, seed=5)
        Xg, pg = g.state()
        Xo, po = o.state()
        if na_g != na_o:
            pytest.fail(f"trajectory {t}: GPU accepted {na_g}, oracle {na_o}")
        agree += na_g
        scale = np.maximum(1.0, np.abs(Xo))
        assert np.all(np.abs(Xg - Xo) <= 1e-9 * scale), t
        assert np.all(np.abs(pg - po) <= 1e-9 * np.maximum(1.0, np.abs(po))), t
    assert agree >= (5 if n_traj >= 30 else 1)  # the chain moves


@pytest.mark.parametrize("precision", ["fp64", "fp32mixed"])
def test_hmc_T_LG_closed_form(precision):
    """Also the FP32-mixed form, whose positions and momenta are float pairs
    (hi + lo) with FP32 gradients: its chains target the same posterior."""
    prob = synth.lingauss_problem(M=10, data_seed=3, dt=0.5, Rm=4.0, Rf=(2.0, 2.0))
    L, r, w = lgc.system(prob.M, prob.dt, prob.Rm, prob.Rf, prob.y, prob.I, p_free=True)
    mu, cov = lgc.posterior(L, r, w)
    inv_mass = np.diag(cov).copy()
    means, vars_ = [], []
    for k in range(32):
        g = pimc.Sampler.from_problem(prob, precision=pimc.FP64 if precision == "fp64" else pimc.FP32_MIXED)
        g.set_chain(k)
        g.set_schedule(n_init=200, n_skip=1)
        nacc = g.hmc(200 + 6000, 16, 0.2, inv_mass, seed=9)
        assert nacc > 0.8 * 6200
        m, v, J = g.moments()
        assert J == 6000
        means.append(m)
        vars_.append(v)
        g.close()
    means, vars_ = np.array(means), np.array(vars_)
    se_m = means.std(0, ddof=1) / np.sqrt(len(means))
    se_v = vars_.std(0, ddof=1) / np.sqrt(len(vars_))
    assert np.all(np.abs(means.mean(0) - mu) < 4 * se_m)
    assert np.all(np.abs(vars_.mean(0) - np.diag(cov)) < 4 * se_v)


def test_param_trace_matches_per_sweep_state():
    prob = synth.hh_problem(200, data_seed=1)
    g = pimc.Sampler.from_problem(prob)
    g.set_param_trace(16)
    ps = []
    for _ in range(25):
        g.sweep(1, 3)
        ps.append(g.state()[1])
    tr = g.param_trace()
    assert tr.shape == (16, 7)
    np.testing.assert_array_equal(tr, np.array(ps[-16:]))


@pytest.mark.parametrize("precision", [pimc.FP64, pimc.FP32_MIXED])
def test_concurrent_chains_on_own_streams_match_sequential(precision):
    """Chains whose trajectories are only enqueued (hmc(wait=False)) from one
    host thread each, every handle on its own stream, end bit for bit where
    the same chains end when run one after another with a synchronising call:
    handles share no device state, and the enqueue-only path runs the same
    trajectory graph."""
    import threading
    import torch
    prob = synth.lingauss_problem(M=300, data_seed=3, dt=0.5, Rm=4.0, Rf=(2.0, 2.0))
    inv_mass = np.full(2 * (prob.M + 1) + 1, 0.05)
    n_traj, n_leap, eps = 40, 10, 0.15

    def chain(k):
        s = pimc.Sampler.from_problem(prob, precision=precision)
        s.set_chain(100 + k)
        s.set_schedule(n_init=10 ** 9, n_skip=1)
        s.set_param_trace(n_traj)
        return s

    seq = []
    for k in range(4):
        s = chain(k)
        n_acc = s.hmc(n_traj, n_leap, eps, inv_mass, seed=7)
        seq.append((s.state(), s.param_trace(), n_acc))
        s.close()

    streams = [torch.cuda.Stream() for _ in range(4)]
    conc = [chain(k) for k in range(4)]
    for s, st in zip(conc, streams):
        s.set_stream(st.cuda_stream)
    threads = [threading.Thread(target=s.hmc, args=(n_traj, n_leap, eps, inv_mass, 7, False)) for s in conc]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    for s, (st_seq, tr_seq, n_acc) in zip(conc, seq):
        s.sync()
        X, p = s.state()
        tr = s.param_trace()
        assert np.array_equal(X, st_seq[0]) and np.array_equal(p, st_seq[1])
        assert np.array_equal(tr, tr_seq)
        assert 0 < n_acc <= n_traj
        # accepted trajectories are the steps where the parameter changed
        assert int(np.sum(np.any(np.diff(tr, axis=0) != 0.0, axis=1))) <= n_acc
        s.close()
