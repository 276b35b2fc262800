"""Parity of the CUDA sampler (through the C ABI) with the FP64 CPU oracle.

* T-dA: per-site Delta A_n for random paths and proposals, every site, at
  M in {1, 2, 17, 1000, 4097}: |dA_gpu - dA_cpu| <= 1e-12 * sum 1/2 R (d'^2 + d^2).
* parameter-move Delta A, full action and gradient (FP64).
* T-REPLAY: same seed and Philox counters, 1000 sweeps in lockstep; every
  sweep starts both sides from the GPU state; an accept that differs must be
  within 1e-9 of its threshold (|log u + dA| of the oracle) and is counted.
* grid independence (ragged tiles, one CTA vs many).
"""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import pimc, synth

pytestmark = pytest.mark.gpu


def oracle_chain(prob):
    ch = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf)
    ch.set_scheme(prob.scheme)
    ch.set_proposal(prob.proposal)
    ch.set_data(prob.y, prob.I)
    ch.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    ch.set_steps(prob.sig_x, prob.sig_p)
    return ch


def base_path(prob):
    if prob.X_true is not None:
        return prob.X_true.copy()
    X = np.zeros((prob.D, prob.M + 1))
    X[0] = prob.y
    return X


def hh(M, seed=0, free=("gNa", "gK", "gL")):
    return synth.hh_problem(M, data_seed=seed, free=free)


def trap(prob, proposal=0):
    prob.scheme = 1
    prob.proposal = proposal
    return prob


@pytest.mark.parametrize("M", [1, 2, 17, 1000, 4097])
@pytest.mark.parametrize("model", ["hh", "lg", "toy", "paper_trap", "hh_trap", "lg_trap"])
def test_site_delta_parity(M, model):
    if model == "hh":
        prob = hh(M, seed=M)
    elif model == "lg":
        prob = synth.lingauss_problem(M, data_seed=M)
    elif model == "paper_trap":
        if M > 1000:
            pytest.skip("paper-variant generator is slow at this size")
        prob = synth.paper_problem(M, data_seed=M)
    elif model == "hh_trap":
        prob = trap(hh(M, seed=M))
    elif model == "lg_trap":
        prob = trap(synth.lingauss_problem(M, data_seed=M))
    else:
        prob = synth.toy_problem(M, data_seed=M, p_free=True)
    X = synth.random_path_near(prob, base_path(prob), 0.5 * prob.sig_x, seed=M)
    Xp = synth.random_path_near(prob, X, 3.0 * prob.sig_x, seed=M + 1)
    g = pimc.Sampler.from_problem(prob)
    g.set_path(X)
    o = oracle_chain(prob)
    o.set_path(X)
    for beta in (1.0, 0.25):
        dg = g.site_delta(Xp, beta)
        do, scale = o.site_delta_all(Xp, beta)
        err = np.abs(dg - do)
        assert np.all(err <= 1e-12 * scale + 1e-300), (np.argmax(err / (scale + 1e-300)), err.max())


@pytest.mark.parametrize("M,variant", [(1, "hh"), (17, "hh"), (1000, "hh"), (4097, "hh"), (17, "hh_trap"),
                                       (1000, "hh_trap"), (2, "paper_trap"), (300, "paper_trap"),
                                       (300, "paper_rk4")])
def test_param_delta_action_and_grad_parity(M, variant):
    if variant == "hh":
        prob = hh(M, seed=3, free="all")
    elif variant == "hh_trap":
        prob = trap(hh(M, seed=3, free="all"))
    else:
        prob = synth.paper_problem(M, data_seed=3, scheme=1 if variant == "paper_trap" else 0)
    X = synth.random_path_near(prob, base_path(prob), 0.3 * prob.sig_x, seed=7)
    g = pimc.Sampler.from_problem(prob)
    g.set_path(X)
    o = oracle_chain(prob)
    o.set_path(X)
    rng = np.random.default_rng(M)
    for l in range(7):
        pl = prob.p_init[l] * (1 + 0.003 * rng.standard_normal())
        dg = g.param_delta(l, pl, 0.7)
        do, scale = o.param_delta(l, pl, 0.7)
        assert abs(dg - do) <= 1e-12 * scale + 1e-300, (l, dg, do, scale)
    Ag = np.array(g.action())
    Ao = np.array(o.action())
    np.testing.assert_allclose(Ag, Ao, rtol=1e-12, atol=0)
    gXg, gpg = g.grad(0.6)
    gXo, gpo = o.grad(0.6)
    # gradient entries are sums of O(1) terms of either sign: compare on the
    # scale of the largest contribution of each component
    scale = np.abs(gXo).max(axis=1, keepdims=True) + 1e-300
    assert np.all(np.abs(gXg - gXo) <= 1e-11 * scale)
    np.testing.assert_allclose(gpg, gpo, rtol=1e-10, atol=1e-10 * np.abs(gpo).max())


def _replay(prob, n_sweeps, seed, grid=0):
    g = pimc.Sampler.from_problem(prob)
    if grid:
        g.set_grid(grid)
    o = oracle_chain(prob)
    flips = 0
    decisions = 0
    for s in range(n_sweeps):
        Xg0, pg0 = g.state()
        o.set_path(Xg0)
        o.set_params(pg0, prob.lo, prob.hi, prob.free)
        o.set_sweep_counter(s, 1.0)
        g.sweep(1, seed)
        o.sweep(1, seed)
        Xg, pg = g.state()
        Xo, po = o.state()
        sm, pm = o.last_margins()
        moved_g = np.any(Xg != Xg0, axis=0)
        moved_o = np.any(Xo != Xg0, axis=0)
        differ = moved_g != moved_o
        decisions += prob.M + 1 + int(np.sum(prob.free))
        if np.any(differ):
            assert np.all(sm[differ] < 1e-9), (s, np.where(differ)[0], sm[differ])
            flips += int(np.sum(differ))
        same = ~differ
        tol = 1e-12 * np.maximum(1.0, np.abs(Xo))
        assert np.all(np.abs(Xg - Xo)[:, same] <= tol[:, same]), s
        for l in range(prob.Np):
            if (pg[l] != pg0[l]) != (po[l] != pg0[l]):
                assert pm[l] < 1e-9, (s, l, pm[l])
                flips += 1
            else:
                assert abs(pg[l] - po[l]) <= 1e-12 * max(1.0, abs(po[l]))
    return flips, decisions


def test_replay_1000_sweeps_hh_config0():
    prob = hh(1000, seed=0)
    flips, decisions = _replay(prob, 1000, seed=1)
    assert flips <= 2, flips


@pytest.mark.parametrize("grid", [1, 3, 7])
def test_replay_ragged_tiles(grid):
    """Tiles of uneven length and one-CTA launches agree with the oracle."""
    prob = hh(237, seed=5, free="all")
    flips, _ = _replay(prob, 40, seed=9, grid=grid)
    assert flips == 0


@pytest.mark.parametrize("model", ["lg", "toy", "lg_trap", "toy_trap_uniform"])
def test_replay_test_models(model):
    if model.startswith("lg"):
        prob = synth.lingauss_problem(50, 1)
    else:
        prob = synth.toy_problem(50, 2, p_free=True)
    if "trap" in model:
        trap(prob, proposal=1 if "uniform" in model else 0)
    flips, _ = _replay(prob, 200, seed=4)
    assert flips == 0


def test_replay_paper_setting():
    """The paper's variant: tanh kinetics, trapezoid rule, uniform proposals, 7 free parameters."""
    prob = synth.paper_problem(400, data_seed=8, free="all")
    flips, _ = _replay(prob, 150, seed=6)
    assert flips <= 1


def test_sweep_counter_and_annealing_match_oracle():
    prob = hh(64, seed=2)
    g = pimc.Sampler.from_problem(prob)
    o = oracle_chain(prob)
    for ch in (g, o):
        ch.set_schedule(n_init=30, n_skip=5, beta0=0.05, n_cool=20, f_acc=0.4, alpha=0.3)
    g.sweep(40, 77)
    o.sweep(40, 77)
    sg, bg = g.sweep_counter()
    so, bo = o.sweep_counter()
    assert sg == so == 40 and bg == bo == 1.0
    Xg, pg = g.state()
    Xo, po = o.state()
    # annealed, adapted 40-sweep chains from the same counters stay together
    assert np.max(np.abs(Xg - Xo)) < 1e-9 * 100
    sxg, spg = g.steps()
    sxo, spo = o.steps()
    np.testing.assert_allclose(sxg, sxo, rtol=1e-12)
    np.testing.assert_allclose(spg, spo, rtol=1e-12)
