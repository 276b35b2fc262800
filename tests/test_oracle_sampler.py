"""Pins of the oracle sampler against what the mathematics fixes.

* T-LG: linear-Gaussian model (x and the offset parameter jointly Gaussian):
  posterior means and variances from the closed-form precision matrix; the
  checkerboard Metropolis chain must match within 4 batch-means standard errors.
* T-QUAD: scalar nonlinear model with M = 2: posterior moments by brute-force
  Gauss-Legendre quadrature of exp(-A) over the whole path (and parameter).
* T-DB: exact detailed balance of every half-sweep and parameter move on a
  finite lattice (discrete symmetric proposals, state and parameter boxes),
  and invariance of exp(-A) under the composed sweep.
* Running moments and histograms against numpy over the recorded samples;
  annealing (Eq. (fbeta)) and step-size adaptation (Sec. 4.2) behaviour.
"""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import synth
from tests import _linear_gaussian as lgc


def new_chain(prob, sig_x=None, sig_p=None):
    ch = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf)
    ch.set_scheme(prob.scheme)
    ch.set_proposal(prob.proposal)
    ch.set_data(prob.y, prob.I)
    ch.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    ch.set_steps(prob.sig_x if sig_x is None else sig_x, prob.sig_p if sig_p is None else sig_p)
    return ch


def run_trace(ch, n, seed):
    D, M, Np = ch.D, ch.M, ch.Np
    tr = np.empty((n, D * (M + 1) + Np))
    for k in range(n):
        ch.sweep(1, seed)
        X, p = ch.state()
        tr[k, :D * (M + 1)] = X.ravel()
        tr[k, D * (M + 1):] = p
    return tr


def batch_se(v, B=100):
    bm = v[: (v.shape[0] // B) * B].reshape(B, -1, *v.shape[1:]).mean(axis=1)
    return bm.std(axis=0, ddof=1) / np.sqrt(B)


LG_ARGS = dict(M=10, data_seed=3, dt=0.5, Rm=4.0, Rf=(2.0, 2.0))


def lg_setup():
    prob = synth.lingauss_problem(**LG_ARGS)
    L, r, w = lgc.system(prob.M, prob.dt, prob.Rm, prob.Rf, prob.y, prob.I, p_free=True)
    mu, cov = lgc.posterior(L, r, w)
    csd = 1.0 / np.sqrt(np.diag(np.linalg.inv(cov)))
    nx = 2 * (prob.M + 1)
    return prob, mu, cov, csd, nx


def test_T_LG_closed_form_posterior():
    prob, mu, cov, csd, nx = lg_setup()
    ch = new_chain(prob, sig_x=csd[:nx].reshape(2, prob.M + 1), sig_p=np.array([2.0 * csd[-1]]))
    ch.set_schedule(n_init=0, n_skip=1)
    ch.sweep(3000, 11)
    tr = run_trace(ch, 200000, 11)
    se = batch_se(tr)
    assert np.all(np.abs(tr.mean(0) - mu) < 4 * se)
    sq = (tr - mu) ** 2
    assert np.all(np.abs(sq.mean(0) - np.diag(cov)) < 4 * batch_se(sq))
    # the oracle's own running moments equal numpy's over the same samples
    ch2 = new_chain(prob, sig_x=csd[:nx].reshape(2, prob.M + 1), sig_p=np.array([2.0 * csd[-1]]))
    ch2.set_schedule(n_init=3000, n_skip=1)
    ch2.sweep(3000, 11)
    tr2 = run_trace(ch2, 5000, 11)
    mean, var, J = ch2.moments()
    assert J == 5000
    np.testing.assert_allclose(mean, tr2.mean(0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(var, tr2.var(0, ddof=1), rtol=1e-9)


def test_T_LG_fixed_parameter_block_tridiagonal():
    """Parameter held fixed: the path posterior alone (block-tridiagonal precision)."""
    prob = synth.lingauss_problem(**LG_ARGS, b_free=False)
    prob.p_init = np.array([0.7])
    L, r, w = lgc.system(prob.M, prob.dt, prob.Rm, prob.Rf, prob.y, prob.I, p_free=False, p_value=0.7)
    mu, cov = lgc.posterior(L, r, w)
    Q = L.T @ (w[:, None] * L)
    # block-tridiagonal in time: no coupling between sites more than one step apart
    for a in range(2):
        for b in range(2):
            for n in range(prob.M + 1):
                for m in range(prob.M + 1):
                    if abs(n - m) > 1:
                        assert Q[a * (prob.M + 1) + n, b * (prob.M + 1) + m] == 0.0
    csd = 1.0 / np.sqrt(np.diag(Q))
    ch = new_chain(prob, sig_x=1.2 * csd.reshape(2, prob.M + 1), sig_p=np.array([0.0]))
    ch.sweep(1000, 5)
    tr = run_trace(ch, 100000, 5)
    se = batch_se(tr)
    assert np.all(np.abs(tr.mean(0)[:-1] - mu) < 4 * se[:-1])
    assert np.all(tr[:, -1] == 0.7)
    sq = (tr[:, :-1] - mu) ** 2
    assert np.all(np.abs(sq.mean(0) - np.diag(cov)) < 4 * batch_se(sq))


def _gauss_legendre(lo, hi, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (hi - lo) * x + 0.5 * (hi + lo), 0.5 * (hi - lo) * w


def test_T_QUAD_brute_force_path_integral():
    """M = 2, D = 1: <x_n> and Var x_n from a 3-D tensor Gauss-Legendre grid
    (160 nodes per axis) of exp(-A); f evaluated by the oracle's map on each axis."""
    prob = synth.toy_problem(2, data_seed=1, dt=0.3, Rm=4.0, Rf=6.0, p0=1.0)
    yv, Iv, p = prob.y, prob.I, prob.p_init
    g0, w0 = _gauss_legendre(-4.5, 6.0, 160)
    g1, w1 = _gauss_legendre(-3.0, 4.5, 160)
    g2, w2 = _gauss_legendre(-3.0, 4.5, 160)
    f0 = np.array([oracle.model_map(2, prob.dt, [v], p, Iv[0])[0] for v in g0])
    f1 = np.array([oracle.model_map(2, prob.dt, [v], p, Iv[1])[0] for v in g1])
    A = (0.5 * prob.Rm * ((g1[None, :, None] - yv[1]) ** 2 + (g2[None, None, :] - yv[2]) ** 2)
         + 0.5 * prob.Rf[0] * ((g1[None, :, None] - f0[:, None, None]) ** 2
                               + (g2[None, None, :] - f1[None, :, None]) ** 2))
    W = w0[:, None, None] * w1[None, :, None] * w2[None, None, :] * np.exp(-(A - A.min()))
    Z = W.sum()
    grids = (g0[:, None, None], g1[None, :, None], g2[None, None, :])
    m = np.array([(W * g).sum() / Z for g in grids])
    v = np.array([(W * (g - mm) ** 2).sum() / Z for g, mm in zip(grids, m)])
    # the box holds all the mass
    for ax in range(3):
        edge = np.take(W, [0, -1], axis=ax).sum() / Z
        assert edge < 1e-12
    ch = new_chain(prob, sig_x=np.array([0.6]), sig_p=np.array([0.0]))
    ch.sweep(2000, 3)
    tr = run_trace(ch, 200000, 3)[:, :3]
    se = batch_se(tr)
    assert np.all(np.abs(tr.mean(0) - m) < 4 * se)
    sq = (tr - m) ** 2
    assert np.all(np.abs(sq.mean(0) - v) < 4 * batch_se(sq))


def test_T_QUAD_with_free_parameter():
    """M = 2, D = 1 and the nonlinear parameter p free in a box: a 4-D grid."""
    prob = synth.toy_problem(2, data_seed=2, dt=0.3, Rm=4.0, Rf=6.0, p0=1.0, p_free=True,
                             lo=0.0, hi=2.0)
    yv, Iv = prob.y, prob.I
    n = 48
    gx, wx = _gauss_legendre(-4.5, 6.0, n)
    gy, wy = _gauss_legendre(-3.0, 4.5, n)
    gp, wp = _gauss_legendre(0.0, 2.0, n)
    f0 = np.array([[oracle.model_map(2, prob.dt, [v], [q], Iv[0])[0] for q in gp] for v in gx])
    f1 = np.array([[oracle.model_map(2, prob.dt, [v], [q], Iv[1])[0] for q in gp] for v in gy])
    # axes: (x0, x1, x2, p)
    x1 = gy[None, :, None, None]
    x2 = gy[None, None, :, None]
    A = (0.5 * prob.Rm * ((x1 - yv[1]) ** 2 + (x2 - yv[2]) ** 2)
         + 0.5 * prob.Rf[0] * ((x1 - f0[:, None, None, :]) ** 2 + (x2 - f1[None, :, None, :]) ** 2))
    W = (wx[:, None, None, None] * wy[None, :, None, None] * wy[None, None, :, None]
         * wp[None, None, None, :] * np.exp(-(A - A.min())))
    Z = W.sum()
    grids = (gx[:, None, None, None], x1, x2, gp[None, None, None, :])
    m = np.array([(W * g).sum() / Z for g in grids])
    v = np.array([(W * (g - mm) ** 2).sum() / Z for g, mm in zip(grids, m)])
    ch = new_chain(prob, sig_x=np.array([0.6]), sig_p=np.array([0.5]))
    ch.sweep(2000, 4)
    tr = run_trace(ch, 200000, 4)
    se = batch_se(tr)
    assert np.all(np.abs(tr.mean(0) - m) < 4 * se)
    sq = (tr - m) ** 2
    assert np.all(np.abs(sq.mean(0) - v) < 4 * batch_se(sq))


# ---------------------------------------------------------------------------
# T-DB: exact detailed balance on a lattice
# ---------------------------------------------------------------------------
H = 0.25            # lattice spacing (exact in binary)
XS = np.arange(-0.5, 1.51, H)   # 9 values
PS = np.arange(0.5, 1.51, H)    # 5 values


def _db_chain(x0, x1, pv, prob):
    ch = oracle.Chain(2, 1, prob.dt, prob.Rm, prob.Rf)
    ch.set_data(prob.y, prob.I)
    ch.set_params([pv], [PS[0]], [PS[-1]], [1])
    ch.set_path(np.array([[x0, x1]]))
    ch.set_steps([H], [H])
    ch.set_state_box([XS[0]], [XS[-1]])
    return ch


def _accept_probability(state, prob, move):
    """P(accept) of one proposal, measured on the oracle's update as a black
    box: the decision is monotone in u, so bisect the threshold u*."""
    def trial(u):
        ch = _db_chain(*state, prob)
        return move(ch, u)
    if trial(1.0 - 2.0 ** -53):
        return 1.0
    lo, hi = 0.0, 1.0 - 2.0 ** -53
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if trial(mid):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _index(state):
    x0, x1, pv = state
    i0 = int(round((x0 - XS[0]) / H)); i1 = int(round((x1 - XS[0]) / H)); ip = int(round((pv - PS[0]) / H))
    return (i0 * XS.size + i1) * PS.size + ip


def test_T_DB_exact_detailed_balance():
    prob = synth.toy_problem(1, data_seed=5, dt=0.3, Rm=2.0, Rf=3.0, p0=1.0, p_free=True)
    states = [(a, b, c) for a in XS for b in XS for c in PS]
    ns = len(states)
    logpi = np.empty(ns)
    for s in states:
        logpi[_index(s)] = -_db_chain(*s, prob).action()[0]
    pi = np.exp(logpi - logpi.max())
    pi /= pi.sum()
    kernels = []
    for kind in ("site0", "site1", "param"):
        P = np.zeros((ns, ns))
        for s in states:
            i = _index(s)
            for z in (-1.0, 1.0):
                if kind == "param":
                    tgt = (s[0], s[1], s[2] + H * z)
                    move = lambda ch, u, z=z: ch.param_update(0, z, u)
                else:
                    k = 0 if kind == "site0" else 1
                    t = list(s); t[k] = s[k] + H * z; tgt = tuple(t)
                    move = lambda ch, u, z=z, k=k: ch.site_update(k, [z], u)
                inside = (XS[0] <= tgt[0] <= XS[-1] and XS[0] <= tgt[1] <= XS[-1]
                          and PS[0] <= tgt[2] <= PS[-1])
                pa = _accept_probability(s, prob, move) if inside else 0.0
                if not inside:
                    # the oracle must reject an out-of-box proposal outright
                    assert not move(_db_chain(*s, prob), 1e-300)
                if inside:
                    P[i, _index(tgt)] += 0.5 * pa
                P[i, i] += 0.5 * (1.0 - pa)
        np.testing.assert_allclose(P.sum(1), 1.0, atol=1e-12)
        F = pi[:, None] * P
        np.testing.assert_allclose(F, F.T, atol=1e-12 * pi.max())
        kernels.append(P)
    sweep = kernels[0] @ kernels[1] @ kernels[2]
    np.testing.assert_allclose(pi @ sweep, pi, atol=1e-12)


# ---------------------------------------------------------------------------
# statistics, histograms, schedule
# ---------------------------------------------------------------------------
def test_moments_and_histograms_match_numpy():
    prob = synth.hh_problem(30, data_seed=2)
    ch = new_chain(prob)
    n_init, n_skip = 7, 3
    ch.set_schedule(n_init=n_init, n_skip=n_skip)
    M = prob.M
    comps = np.array([0 * (M + 1) + 5, 2 * (M + 1) + 11, 4 * (M + 1) + 0])  # V_5, h_11, p_gNa
    lo = np.array([-70.0, 0.3, 100.0]); hi = np.array([-60.0, 0.7, 140.0])
    ch.set_histograms(comps, lo, hi, 16)
    samples = []
    for s in range(60):
        ch.sweep(1, 21)
        if s >= n_init and (s - n_init) % n_skip == 0:
            X, p = ch.state()
            samples.append(np.concatenate([X.ravel(), p]))
    S = np.array(samples)
    mean, var, J = ch.moments()
    assert J == len(samples) == 18
    np.testing.assert_allclose(mean, S.mean(0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(var, S.var(0, ddof=1), rtol=1e-8, atol=1e-18)
    H_ = ch.histograms()
    for k, c in enumerate(comps):
        v = S[:, c]
        inside, _ = np.histogram(v[(v >= lo[k]) & (v < hi[k])], bins=16, range=(lo[k], hi[k]))
        assert H_[k, 0] == np.sum(v < lo[k])
        assert H_[k, -1] == np.sum(v >= hi[k])
        assert np.array_equal(H_[k, 1:-1], inside)


def test_annealing_schedule_eq_fbeta():
    prob = synth.hh_problem(10, data_seed=2)
    ch = new_chain(prob)
    beta0, n_cool = 0.01, 50
    ch.set_schedule(n_init=100, n_skip=10, beta0=beta0, n_cool=n_cool)
    fb = (1.0 / beta0) ** (1.0 / n_cool)
    for s in range(60):
        sw, beta = ch.sweep_counter()
        assert sw == s
        if s < n_cool:
            assert abs(beta - beta0 * fb ** s) <= 1e-13 * beta
        else:
            assert beta == 1.0
        ch.sweep(1, 2)
    # one step before N_cool the product is within rounding of (1/beta0)^(-1/N_cool)
    assert abs(beta0 * fb ** (n_cool - 1) - fb ** -1) < 1e-13


def test_step_size_adaptation_reaches_target_acceptance():
    """The Sec. 4.2 rule is a proportional controller on the acceptance rate:
    after a burn-in with adaptation the frozen steps accept near f_acc."""
    prob = synth.hh_problem(120, data_seed=4)
    ch = new_chain(prob)
    ch.set_schedule(n_init=3000, n_skip=25, f_acc=0.4, alpha=0.5)
    ch.sweep(3000, 8)
    sig_before, sp_before = ch.steps()
    sa0, sp0, pa0, pp0 = ch.accept_stats()
    ch.sweep(1000, 8)
    sig_after, sp_after = ch.steps()
    assert np.array_equal(sig_before, sig_after) and np.array_equal(sp_before, sp_after)
    sa1, sp1, pa1, pp1 = ch.accept_stats()
    rate = (sa1 - sa0).sum() / (sp1 - sp0).sum()
    assert abs(rate - 0.4) < 0.05
    prate = (pa1 - pa0)[:3] / (pp1 - pp0)[:3]
    assert np.all(np.abs(prate - 0.4) < 0.15)


def test_hmc_closed_form_posterior():
    """Whole-path HMC on the linear-Gaussian model reproduces the closed form.
    Mass = posterior marginal variances; the leapfrog is stable for
    eps < 2 / sqrt(max eig(M^-1 Q)) (= 0.34 here), so eps = 0.2."""
    prob, mu, cov, csd, nx = lg_setup()
    ch = new_chain(prob)
    ch.set_schedule(n_init=200, n_skip=1)
    inv_mass = np.diag(cov).copy()
    nacc = ch.hmc(200, 16, 0.2, inv_mass, 17)
    tr = np.empty((20000, nx + 1))
    for k in range(tr.shape[0]):
        nacc += ch.hmc(1, 16, 0.2, inv_mass, 17)
        X, p = ch.state()
        tr[k, :nx] = X.ravel()
        tr[k, nx:] = p
    assert 0.8 < nacc / 20200 < 0.99
    mean, var, J = ch.moments()
    assert J == 20000
    np.testing.assert_allclose(mean, tr.mean(0), rtol=1e-12, atol=1e-12)
    se = batch_se(tr)
    assert np.all(np.abs(tr.mean(0) - mu) < 4 * se)
    sq = (tr - mu) ** 2
    assert np.all(np.abs(sq.mean(0) - np.diag(cov)) < 4 * batch_se(sq))


def test_residual_moments_match_numpy():
    """Residual accumulators (eps_{n+1} = x_{n+1} - f(x_n), delta_n = x_{n,0} - y_n)
    against numpy over the recorded samples, with f from the (pinned) map."""
    prob = synth.hh_problem(25, data_seed=3)
    ch = new_chain(prob)
    ch.set_schedule(n_init=4, n_skip=2)
    eps, dl = [], []
    for s in range(30):
        ch.sweep(1, 13)
        if s >= 4 and (s - 4) % 2 == 0:
            X, p = ch.state()
            f = np.array([oracle.model_map(0, prob.dt, X[:, n], p, prob.I[n]) for n in range(prob.M)]).T
            eps.append((X[:, 1:] - f).ravel())
            dl.append(X[0, 1:] - prob.y[1:])
    R = np.hstack([np.array(eps), np.array(dl)])
    mean, var, J = ch.residual_moments()
    assert J == R.shape[0] == 13
    np.testing.assert_allclose(mean, R.mean(0), rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(var, R.var(0, ddof=1), rtol=1e-7, atol=1e-18)


def test_forecast_deterministic_and_noise_law():
    prob = synth.hh_problem(40, data_seed=1)
    ch = new_chain(prob)
    Ifut = 10.0 + np.zeros(25)
    det = ch.forecast(25, Ifut, 3, 0, 1)
    X, p = ch.state()
    x = X[:, -1].copy()
    for k in range(25):
        assert np.array_equal(det[0, :, k], x)
        x = oracle.model_map(0, prob.dt, x, p, Ifut[k])
    assert np.array_equal(det[0], det[2])
    # one noisy step: x_1 = f(x_0) + xi, xi_a ~ N(0, 1/Rf_a)
    ens = ch.forecast(1, Ifut[:1], 20000, 1, 7)
    d = ens[:, :, 1] - det[0, :, 1]
    se = 1.0 / np.sqrt(prob.Rf) / np.sqrt(d.shape[0])
    assert np.all(np.abs(d.mean(0)) < 4 * se)
    assert np.all(np.abs(d.var(0) * prob.Rf - 1.0) < 4 * np.sqrt(2.0 / d.shape[0]))



@pytest.mark.parametrize("scheme,proposal", [(1, 0), (1, 1), (0, 1)])
def test_T_LG_trapezoid_and_uniform_proposals(scheme, proposal):
    """The trapezoid rule of Eq. (modelError) keeps the linear model's posterior
    Gaussian (closed form), and the uniform increments of Fig. 1 sample it too."""
    prob = synth.lingauss_problem(**LG_ARGS)
    prob.scheme, prob.proposal = scheme, proposal
    L, r, w = lgc.system(prob.M, prob.dt, prob.Rm, prob.Rf, prob.y, prob.I, p_free=True, scheme=scheme)
    mu, cov = lgc.posterior(L, r, w)
    csd = 1.0 / np.sqrt(np.diag(np.linalg.inv(cov)))
    nx = 2 * (prob.M + 1)
    k = 1.0 if proposal == 0 else 1.7  # U(-1,1) has sd 1/sqrt(3)
    ch = new_chain(prob, sig_x=k * csd[:nx].reshape(2, prob.M + 1), sig_p=np.array([2.0 * k * csd[-1]]))
    ch.sweep(3000, 21)
    tr = run_trace(ch, 150000, 21)
    se = batch_se(tr)
    assert np.all(np.abs(tr.mean(0) - mu) < 4 * se)
    sq = (tr - mu) ** 2
    assert np.all(np.abs(sq.mean(0) - np.diag(cov)) < 4 * batch_se(sq))
