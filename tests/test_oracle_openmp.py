"""The OpenMP build of the oracle (used only to time the method on all host
cores) runs the same chain as the serial build: the site phases are
order-independent and only the parameter-move sums add in another order, so
states and parameters agree to rounding."""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import synth


def _chain(prob, openmp):
    ch = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf, openmp=openmp)
    ch.set_data(prob.y, prob.I)
    ch.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    ch.set_steps(prob.sig_x, prob.sig_p)
    ch.set_schedule(n_init=4, n_skip=2, f_acc=0.4, alpha=0.3)
    return ch


def test_openmp_build_runs_the_same_chain():
    try:
        n_threads = oracle.threads(openmp=True)
    except Exception as e:  # no OpenMP in the host compiler
        pytest.skip(f"OpenMP build unavailable: {e}")
    assert n_threads >= 1 and oracle.threads() == 1
    prob = synth.hh_problem(301, data_seed=4, free="all")
    a, b = _chain(prob, False), _chain(prob, True)
    a.sweep(8, 5)
    b.sweep(8, 5)
    Xa, pa = a.state()
    Xb, pb = b.state()
    np.testing.assert_allclose(Xb, Xa, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pb, pa, rtol=1e-12)
    for x, y in zip(a.accept_stats(), b.accept_stats()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
