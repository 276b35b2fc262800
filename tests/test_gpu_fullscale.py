"""Parity at the benchmark's scale and grid, and the FP32-mixed Metropolis
sampler against the closed-form posterior.

* FP64 replay against the oracle on the benchmark workload (HH, M = 32768,
  all 7 parameters free): the sweep runs on one CTA per SM (152 tiles of 216
  sites on GB300), so the grid barrier, the exact-sum slots with 152
  arrivals and the cross-tile neighbours are the ones the benchmark times.
  Same rule as the small replays: a decision that differs must sit within
  1e-9 of its threshold (Eq. (Paccept)) and is counted.
* The FP32-mixed resident form (neighbour flags, speculative parameter maps,
  CTA sums formed during the barrier) against the general form, bit for bit,
  on the same full grid: M = 32768 and M = 34047 (224 sites a tile, the
  resident form's largest), 20 sweeps over two launches with statistics,
  adaptation and annealing.
* T-LG for FP32-mixed Metropolis (checkerboard of Sec. 4.1, Eq. (Paccept)):
  the resident form on one CTA and on three, and the general form; means and
  variances of 64 independent chains within 4 standard errors of the
  closed-form Gaussian posterior.
"""
import numpy as np
import pytest

from paper_1103_4887_gb300 import pimc, synth
from tests import _linear_gaussian as lgc
from tests.test_gpu_parity import _replay
from tests.test_gpu_resident import _run, _same

pytestmark = pytest.mark.gpu


def test_replay_fp64_bench_workload_full_grid():
    prob = synth.hh_problem(32768, data_seed=0, free="all")
    g = pimc.Sampler.from_problem(prob)
    grid, _ = g.launch_info()
    assert grid >= 147  # one tile per SM: at most 224 sites a CTA
    g.close()
    flips, decisions = _replay(prob, 30, seed=1)
    assert flips <= 2, (flips, decisions)


@pytest.mark.parametrize("M", [32768, 34047])
def test_resident_equals_general_bitwise_full_grid(M):
    prob = synth.hh_problem(M, data_seed=3, free="all")
    a = _run(prob, "auto", 20)
    b = _run(prob, "general", 20)
    assert a.sweep_form() == "resident"
    assert b.sweep_form() == "general"
    grid, _ = a.launch_info()
    assert grid >= 147 and a.launch_info() == b.launch_info()
    if M == 34047:
        assert (M + 1 + grid - 1) // grid == 224
    _same(a, b)


@pytest.mark.parametrize("case", ["resident_grid1", "resident_grid3", "general"])
def test_T_LG_fp32_mixed_metropolis(case):
    M, grid, form = {"resident_grid1": (10, 0, "auto"), "resident_grid3": (23, 3, "auto"),
                     "general": (10, 0, "general")}[case]
    prob = synth.lingauss_problem(M=M, data_seed=3, dt=0.5, Rm=4.0, Rf=(2.0, 2.0))
    L, r, w = lgc.system(prob.M, prob.dt, prob.Rm, prob.Rf, prob.y, prob.I, p_free=True)
    mu, cov = lgc.posterior(L, r, w)
    csd = 1.0 / np.sqrt(np.diag(np.linalg.inv(cov)))
    nx = 2 * (prob.M + 1)
    n_chains = 64
    means, vars_ = [], []
    for k in range(n_chains):
        g = pimc.Sampler.from_problem(prob, precision=pimc.FP32_MIXED)
        if grid:
            g.set_grid(grid)
        g.set_sweep_form(form)
        assert g.sweep_form() == ("general" if form == "general" else "resident")
        if grid:
            assert g.launch_info()[0] == grid
        g.set_steps(csd[:nx].reshape(2, prob.M + 1), np.array([2.0 * csd[-1]]))
        g.set_chain(k)
        g.set_schedule(n_init=3000, n_skip=1)
        g.sweep(3000 + 25000, seed=2024)
        m, v, J = g.moments()
        assert J == 25000
        means.append(m)
        vars_.append(v)
        g.close()
    means = np.array(means)
    vars_ = np.array(vars_)
    se_m = means.std(0, ddof=1) / np.sqrt(n_chains)
    se_v = vars_.std(0, ddof=1) / np.sqrt(n_chains)
    assert np.all(np.abs(means.mean(0) - mu) < 4 * se_m)
    assert np.all(np.abs(vars_.mean(0) - np.diag(cov)) < 4 * se_v)
