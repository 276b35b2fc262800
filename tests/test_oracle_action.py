"""Pins of the oracle's action, local change of action and gradient.

* Linear-Gaussian model: the full action equals the closed-form quadratic
  1/2 (L z - r)^T W (L z - r) built from the RK4 polynomials (no oracle code),
  and the gradient equals L^T W (L z - r).
* Every model: the local change of action of Fig. 1 equals the difference of
  two full actions (Eq. (Paccept) only needs Delta A = A(X') - A(X)); the
  parameter move likewise; the gradient equals central finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import synth
from tests import _linear_gaussian as lgc


def make_chain(prob, X=None):
    ch = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf)
    ch.set_scheme(prob.scheme)
    ch.set_data(prob.y, prob.I)
    ch.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    if X is not None:
        ch.set_path(X)
    return ch


@pytest.mark.parametrize("scheme", [0, 1])
def test_lingauss_action_closed_form(scheme):
    prob = synth.lingauss_problem(12, data_seed=3)
    prob.scheme = scheme
    L, r, w = lgc.system(prob.M, prob.dt, prob.Rm, prob.Rf, prob.y, prob.I, p_free=True, scheme=scheme)
    rng = np.random.default_rng(0)
    for _ in range(10):
        z = rng.standard_normal(L.shape[1])
        ch = make_chain(prob)
        ch.set_params(z[-1:], prob.lo, prob.hi, prob.free)
        ch.set_path(z[:-1].reshape(2, prob.M + 1))
        A, Ao, Af = ch.action()
        np.testing.assert_allclose(A, lgc.action(L, r, w, z), rtol=1e-12)
        assert abs(A - (Ao + Af)) <= 1e-12 * abs(A)
        gX, gp = ch.grad()
        g = L.T @ (w * (L @ z - r))
        np.testing.assert_allclose(np.concatenate([gX.ravel(), gp]), g, rtol=1e-10, atol=1e-10)


def _with_scheme(prob, scheme):
    prob.scheme = scheme
    return prob


def _problems():
    hh = synth.hh_problem(40, data_seed=1, free="all")
    return [("hh", hh), ("lg", synth.lingauss_problem(25, 2)), ("toy", synth.toy_problem(25, 4, p_free=True)),
            ("paper_trap", synth.paper_problem(40, data_seed=2)),
            ("paper_rk4", synth.paper_problem(40, data_seed=3, scheme=0)),
            ("hh_trap", _with_scheme(synth.hh_problem(40, data_seed=4, free="all"), 1)),
            ("lg_trap", _with_scheme(synth.lingauss_problem(25, 5), 1)),
            ("toy_trap", _with_scheme(synth.toy_problem(25, 6, p_free=True), 1))]


@pytest.mark.parametrize("name,prob", _problems())
def test_site_delta_equals_full_action_difference(name, prob):
    X0 = prob.X_true if prob.X_true is not None else np.vstack([prob.y] + [np.zeros(prob.M + 1)] * (prob.D - 1))
    X = synth.random_path_near(prob, X0, 0.5 * prob.sig_x, seed=1)
    Xp = synth.random_path_near(prob, X, 2.0 * prob.sig_x, seed=2)
    ch = make_chain(prob, X)
    for beta in (1.0, 0.3):
        dA, scale = ch.site_delta_all(Xp, beta)
        for n in range(prob.M + 1):
            ref = make_chain(prob, X)
            Xn = X.copy()
            Xn[:, n] = Xp[:, n]
            A0 = _beta_action(ref, beta)
            ref.set_path(Xn)
            A1 = _beta_action(ref, beta)
            # the difference of two full sums carries their rounding error
            tol = 1e-12 * scale[n] + 4e-16 * (abs(A0) + abs(A1))
            assert abs(dA[n] - (A1 - A0)) <= tol, (n, dA[n], A1 - A0)


def _beta_action(ch, beta):
    A, Ao, Af = ch.action()
    return Ao + beta * Af


@pytest.mark.parametrize("name,prob", _problems())
def test_param_delta_equals_full_action_difference(name, prob):
    X0 = prob.X_true if prob.X_true is not None else np.vstack([prob.y] + [np.zeros(prob.M + 1)] * (prob.D - 1))
    ch = make_chain(prob, X0)
    rng = np.random.default_rng(9)
    for l in range(prob.Np):
        for beta in (1.0, 0.5):
            pl = prob.p_init[l] * (1 + 0.01 * rng.standard_normal()) + 1e-3 * rng.standard_normal()
            dA, scale = ch.param_delta(l, pl, beta)
            ref = make_chain(prob, X0)
            A0 = _beta_action(ref, beta)
            p2 = prob.p_init.copy()
            p2[l] = pl
            ref.set_params(p2, prob.lo, prob.hi, prob.free)
            A1 = _beta_action(ref, beta)
            assert abs(dA - (A1 - A0)) <= 1e-12 * scale + 4e-16 * (abs(A0) + abs(A1))


@pytest.mark.parametrize("name,prob", _problems())
def test_action_gradient_matches_central_differences(name, prob):
    M = prob.M
    X0 = prob.X_true if prob.X_true is not None else np.vstack([prob.y] + [np.zeros(M + 1)] * (prob.D - 1))
    X = synth.random_path_near(prob, X0, 0.3 * prob.sig_x, seed=5)
    ch = make_chain(prob, X)
    gX, gp = ch.grad(1.0)
    rng = np.random.default_rng(1)
    idx = rng.choice(prob.D * (M + 1), size=min(40, prob.D * (M + 1)), replace=False)
    for k in idx:
        a, n = divmod(int(k), M + 1)
        h = 1e-6 * max(1.0, abs(X[a, n]))
        Xa = X.copy(); Xa[a, n] += h
        Xb = X.copy(); Xb[a, n] -= h
        ch.set_path(Xa); Aa = ch.action()[0]
        ch.set_path(Xb); Ab = ch.action()[0]
        fd = (Aa - Ab) / (2 * h)
        assert abs(gX[a, n] - fd) <= 1e-7 * max(1.0, abs(fd)) + 1e-13 * abs(Aa) / h
    ch.set_path(X)
    for l in range(prob.Np):
        h = 1e-6 * max(1.0, abs(prob.p_init[l]))
        pa = prob.p_init.copy(); pa[l] += h
        pb = prob.p_init.copy(); pb[l] -= h
        ch.set_params(pa, prob.lo, prob.hi, prob.free); Aa = ch.action()[0]
        ch.set_params(pb, prob.lo, prob.hi, prob.free); Ab = ch.action()[0]
        fd = (Aa - Ab) / (2 * h)
        assert abs(gp[l] - fd) <= 1e-7 * max(1.0, abs(fd)) + 1e-13 * abs(Aa) / h
