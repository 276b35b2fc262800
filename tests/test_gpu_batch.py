"""T-BATCH: many chains of uneven M in one batched launch.

Each chain of a batch runs exactly the sweeps it runs alone on one CTA
(pimc_set_grid(h, 1)): states, parameters and moments are bit-identical.
Counters are keyed by the chain id, never by the CTA, so the assignment of
chains to CTAs (the tiling, the autotuner's choice) does not change a chain.
Chains of a batch are also replayed against the FP64 oracle sweep by sweep
(the rule of the single-chain replays: a differing decision must sit within
1e-9 of its threshold, Eq. (Paccept), and is counted).
"""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import pimc, synth

pytestmark = pytest.mark.gpu

MS = [37, 200, 511, 1000, 2500, 64, 1, 300]


def _make(prec, grid1=False, paper=False):
    out = []
    for k, M in enumerate(MS):
        if paper:
            prob = synth.paper_problem(min(M, 600), data_seed=100 + k)
        else:
            prob = synth.hh_problem(M, data_seed=100 + k, free="all" if k % 2 == 0 else ("gNa", "gK", "gL"))
        s = pimc.Sampler.from_problem(prob, precision=prec)
        s.set_chain(k)
        s.set_schedule(n_init=12, n_skip=3, beta0=0.2, n_cool=8, f_acc=0.4, alpha=0.3)
        if grid1:
            s.set_grid(1)
        out.append(s)
    return out


@pytest.mark.parametrize("prec,paper", [(pimc.FP64, False), (pimc.FP32_MIXED, False), (pimc.FP64, True)])
def test_batched_chains_equal_single_chain_runs_bitwise(prec, paper):
    alone = _make(prec, grid1=True, paper=paper)
    for s in alone:
        s.sweep(25, 77)
    grouped = _make(prec, paper=paper)
    b = pimc.Batch(grouped)
    b.set_tuning(256, 0)
    b.sweep(10, 77)
    b.sweep(15, 77)   # a second graph (different length) continues the counters
    for s1, s2 in zip(alone, grouped):
        X1, p1 = s1.state()
        X2, p2 = s2.state()
        assert np.array_equal(X1, X2) and np.array_equal(p1, p2)
        m1, v1, J1 = s1.moments()
        m2, v2, J2 = s2.moments()
        assert J1 == J2 and np.array_equal(m1, m2) and np.array_equal(v1, v2, equal_nan=True)
        assert s1.sweep_counter() == s2.sweep_counter()
        a1, a2 = s1.accept_stats(), s2.accept_stats()
        for x, y in zip(a1, a2):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", [pimc.FP64, pimc.FP32_MIXED])
def test_tiling_does_not_change_a_chain(prec):
    """128- and 256-thread CTAs, few or many chains per CTA, long chains split
    over up to 4 CTAs of the launch: the same chains, bit for bit (the
    parameter-move sums are exact, so the order in which threads and CTAs add
    their terms does not matter)."""
    ref = _make(prec)
    b = pimc.Batch(ref)
    b.set_tuning(256, 1)
    b.sweep(20, 5)
    assert b.info()[2] == 0
    for nt, k, g in ((128, 0, 1), (128, 0, 4), (256, 0, 2)):
        other = _make(prec)
        b2 = pimc.Batch(other)
        b2.set_tuning(nt, k, g)
        if g > 1:
            assert b2.info()[2] >= 1  # the 2501-site chain (and at 128 threads the 1001-site one) is split
        b2.sweep(7, 5)
        b2.sweep(13, 5)  # a second launch continues the chains' barrier words and sums
        for s1, s2 in zip(ref, other):
            X1, p1 = s1.state()
            X2, p2 = s2.state()
            assert np.array_equal(X2, X1) and np.array_equal(p2, p1), (nt, k, g)
            m1, v1, J1 = s1.moments()
            m2, v2, J2 = s2.moments()
            assert J1 == J2 == 3 and np.array_equal(m1, m2) and np.array_equal(v1, v2, equal_nan=True)
            assert s1.sweep_counter() == s2.sweep_counter()


def test_autotune_picks_a_valid_shape():
    chains = _make(pimc.FP32_MIXED)
    b = pimc.Batch(chains)
    nt, k, g = b.autotune(3, 1)
    assert nt in (128, 256) and k >= 1 and g in (1, 2, 4)
    n_ctas, t, n_split = b.info()
    assert t == nt and 1 <= n_ctas and (n_split == 0) == (g == 1 or n_split == 0)
    b.sweep(5, 2)
    for s in chains:
        assert np.all(np.isfinite(s.state()[0]))


@pytest.mark.parametrize("ctas_per_chain", [1, 4])
def test_batched_chains_replay_against_oracle(ctas_per_chain):
    """The shortest and the longest chain of an FP64 batch (M = 37 and 5000,
    3 and 7 free parameters, chain ids 0 and 5) follow the oracle chain with
    the same data, steps and chain id, one batched sweep at a time; with
    ctas_per_chain = 4 the long chains run as tiles over 2 to 4 CTAs."""
    Ms = [37, 800, 2500, 64, 1200, 5000]
    probs, samplers = [], []
    for k, M in enumerate(Ms):
        prob = synth.hh_problem(M, data_seed=300 + k, free="all" if k % 2 else ("gNa", "gK", "gL"))
        s = pimc.Sampler.from_problem(prob)
        s.set_chain(k)
        probs.append(prob)
        samplers.append(s)
    b = pimc.Batch(samplers)
    b.set_tuning(256, 0, ctas_per_chain)
    assert (b.info()[2] > 0) == (ctas_per_chain > 1)
    watch = [0, 5]
    oracles = {}
    for k in watch:
        prob = probs[k]
        o = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf)
        o.set_data(prob.y, prob.I)
        o.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
        o.set_steps(prob.sig_x, prob.sig_p)
        o.set_chain(k)
        oracles[k] = o
    flips = {k: 0 for k in watch}
    moves = {k: 0 for k in watch}
    seed = 31
    for s_idx in range(40):
        before = {k: samplers[k].state() for k in watch}
        for k in watch:
            X0, p0 = before[k]
            o = oracles[k]
            o.set_path(X0)
            o.set_params(p0, probs[k].lo, probs[k].hi, probs[k].free)
            o.set_sweep_counter(s_idx, 1.0)
        b.sweep(1, seed)
        for k in watch:
            prob, o = probs[k], oracles[k]
            X0, p0 = before[k]
            o.sweep(1, seed)
            Xg, pg = samplers[k].state()
            Xo, po = o.state()
            sm, pm = o.last_margins()
            moved_g = np.any(Xg != X0, axis=0)
            moved_o = np.any(Xo != X0, axis=0)
            differ = moved_g != moved_o
            moves[k] += int(np.sum(moved_g))
            if np.any(differ):
                assert np.all(sm[differ] < 1e-9), (k, s_idx, np.where(differ)[0])
                flips[k] += int(np.sum(differ))
            same = ~differ
            tol = 1e-12 * np.maximum(1.0, np.abs(Xo))
            assert np.all(np.abs(Xg - Xo)[:, same] <= tol[:, same]), (k, s_idx)
            for l in range(prob.Np):
                if (pg[l] != p0[l]) != (po[l] != p0[l]):
                    assert pm[l] < 1e-9, (k, s_idx, l)
                    flips[k] += 1
                else:
                    assert abs(pg[l] - po[l]) <= 1e-12 * max(1.0, abs(po[l]))
    for k in watch:
        assert flips[k] <= 2, (k, flips[k])
        assert moves[k] > 0
        assert samplers[k].sweep_counter()[0] == 40
