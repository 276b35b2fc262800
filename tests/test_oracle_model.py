"""Pins of the oracle's model layer: the RK4 map, the HH vector field and the
reverse-mode products, against closed forms, textbook properties of the
Hodgkin-Huxley model and finite differences (none of which reuse oracle code
for the expected value)."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle

HH = oracle.MODEL_HH
LG = oracle.MODEL_LINGAUSS
TOY = oracle.MODEL_TOY1D
P_HH = np.array([120.0, 36.0, 0.3, 50.0, -77.0, -54.4, 1.0])
K_LG = np.array([[-0.5, -2.0], [2.0, -0.5]])


def rk4_polys(Z):
    """RK4 applied to x' = K x + b over one step h (Z = h K) is exactly
    x -> T(Z) x + h S(Z) b with T the 4th-order Taylor polynomial of e^Z and
    S(Z) = I + Z/2 + Z^2/6 + Z^3/24 (the RK4 stability polynomial)."""
    I2 = np.eye(Z.shape[0])
    Z2 = Z @ Z
    Z3 = Z2 @ Z
    Z4 = Z3 @ Z
    return I2 + Z + Z2 / 2 + Z3 / 6 + Z4 / 24, I2 + Z / 2 + Z2 / 6 + Z3 / 24


@pytest.mark.parametrize("dt", [0.01, 0.1, 0.37])
def test_rk4_linear_model_closed_form(dt):
    rng = np.random.default_rng(5)
    T, S = rk4_polys(dt * K_LG)
    for _ in range(20):
        x = rng.standard_normal(2) * 3
        p = rng.standard_normal(1)
        I = rng.standard_normal()
        expect = T @ x + dt * S @ np.array([p[0], I])
        got = oracle.model_map(LG, dt, x, p, I)
        np.testing.assert_allclose(got, expect, rtol=1e-14, atol=1e-14)


def test_rk4_local_error_is_fifth_order():
    """One RK4 step against the exact flow (scipy DOP853 at rtol 1e-13) of the
    oracle's own vector field: the local error scales as h^5, so halving h
    divides it by ~32 (a wrong stage weight drops the order)."""
    x0 = np.array([0.7])
    p = np.array([1.3])
    I = 0.2

    def flow(h):
        sol = solve_ivp(lambda t, x: oracle.model_rhs(TOY, x, p, I), (0, h), x0,
                        method="DOP853", rtol=1e-13, atol=1e-15)
        return sol.y[:, -1]

    errs = []
    for h in (0.2, 0.1, 0.05):
        errs.append(abs(oracle.model_map(TOY, h, x0, p, I)[0] - flow(h)[0]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 24 < r1 < 40 and 24 < r2 < 40


def test_hh_resting_state_textbook():
    """With no current the HH membrane (modern convention) rests at -65 mV with
    m = 0.0529, h = 0.5961, n = 0.3177 (Hodgkin & Huxley 1952; e.g. Dayan & Abbott)."""
    x = np.array([-60.0, 0.05, 0.6, 0.3])
    for _ in range(int(200 / 0.02)):
        x = oracle.model_map(HH, 0.02, x, P_HH, 0.0)
    assert abs(x[0] + 65.0) < 0.01
    np.testing.assert_allclose(x[1:], [0.0529, 0.5961, 0.3177], atol=2e-4)
    assert np.max(np.abs(oracle.model_rhs(HH, x, P_HH, 0.0))) < 1e-9


def _spike_times(I, T=600.0, dt=0.02):
    x = np.array([-65.0, 0.0529, 0.5961, 0.3177])
    V = np.empty(int(T / dt))
    for k in range(V.size):
        x = oracle.model_map(HH, dt, x, P_HH, I)
        V[k] = x[0]
    t = np.arange(V.size) * dt
    up = np.where((V[1:] > 0) & (V[:-1] <= 0))[0]
    return t[up], V


def test_hh_repetitive_firing_textbook():
    """At 10 uA/cm^2 the HH model fires periodically at about 68 Hz with
    overshooting spikes; at 5 uA/cm^2 (below the ~6.2 uA/cm^2 onset of
    repetitive firing) it settles without a sustained train."""
    ts, V = _spike_times(10.0)
    late = ts[ts > 150]
    rate = 1000.0 / np.mean(np.diff(late))
    assert 62.0 < rate < 74.0
    assert V[int(150 / 0.02):].max() > 20.0
    ts5, _ = _spike_times(5.0)
    assert np.sum(ts5 > 200) == 0


def test_hh_rates_continuous_at_removable_singularities():
    for V0, g in ((-40.0, 0), (-55.0, 2)):
        vals = [oracle.hh_rates(V0 + d)[0][g] for d in (-1e-4, -1e-7, 0.0, 1e-7, 1e-4)]
        # limits: alpha_m(-40) = 1, alpha_n(-55) = 0.1
        lim = 1.0 if g == 0 else 0.1
        assert abs(vals[2] - lim) < 1e-15
        assert max(abs(v - lim) for v in vals) < 1e-5 * lim + 1e-6


def test_paper_variant_behaviour():
    """The paper's HH variant (Sec. 5.1, Table 1) in the shifted convention:
    a_inf(V_a) = 1/2 and tau(V_a) = tau0 + tau1 for each gate; the membrane
    rests near 0 mV, and a 10 uA/cm^2 drive gives repeated overshooting spikes
    ("qualitatively similar" to Hodgkin-Huxley)."""
    for g, (Va, t0, t1) in enumerate([(25.0, 0.1, 0.4), (5.0, 1.0, 7.0), (10.0, 1.0, 5.0)]):
        ainf, tau = oracle.paper_gates(Va)
        assert ainf[g] == 0.5 and abs(tau[g] - (t0 + t1)) < 1e-15
    p = np.array([1.0, 120.0, 115.0, 20.0, -12.0, 0.3, 10.6])
    x = np.array([0.0, *oracle.paper_gates(0.0)[0]])
    for _ in range(int(200 / 0.04)):
        x = oracle.model_map(3, 0.04, x, p, 0.0)
    assert abs(x[0]) < 2.0
    assert np.max(np.abs(oracle.model_rhs(3, x, p, 0.0))) < 1e-9
    V = []
    for _ in range(int(300 / 0.04)):
        x = oracle.model_map(3, 0.04, x, p, 10.0)
        V.append(x[0])
    V = np.array(V)
    assert 90.0 < V.max() < 125.0
    assert np.sum((V[1:] > 50) & (V[:-1] <= 50)) >= 8


@pytest.mark.parametrize("model", [HH, LG, TOY, 3])
def test_map_vjp_matches_central_differences(model):
    D, Np = oracle.MODEL_DIMS[model]
    rng = np.random.default_rng(11 + model)
    dt = 0.02 if model == HH else (0.04 if model == 3 else 0.1)
    for trial in range(6):
        if model == HH:
            x = np.array([rng.uniform(-80, 40), rng.uniform(0.05, 0.95),
                          rng.uniform(0.05, 0.95), rng.uniform(0.05, 0.95)])
            if trial == 0:
                x[0] = -40.0 + 1e-5  # near the removable singularity of alpha_m
            p = P_HH * (1 + 0.1 * rng.uniform(-1, 1, 7))
            I = rng.uniform(0, 20)
        elif model == 3:
            x = np.array([rng.uniform(-10, 100), rng.uniform(0.05, 0.95),
                          rng.uniform(0.05, 0.95), rng.uniform(0.05, 0.95)])
            p = np.array([1.0, 120.0, 115.0, 20.0, -12.0, 0.3, 10.6]) * (1 + 0.1 * rng.uniform(-1, 1, 7))
            I = rng.uniform(0, 20)
        else:
            x = rng.standard_normal(D)
            p = rng.standard_normal(Np)
            I = rng.standard_normal()
        w = rng.standard_normal(D)
        gx, gp = oracle.model_map_vjp(model, dt, x, p, I, w)
        for i in range(D):
            h = 1e-6 * max(1.0, abs(x[i]))
            e = np.zeros(D); e[i] = h
            fd = (w @ oracle.model_map(model, dt, x + e, p, I)
                  - w @ oracle.model_map(model, dt, x - e, p, I)) / (2 * h)
            assert abs(gx[i] - fd) <= 1e-7 * max(1.0, abs(fd))
        for l in range(Np):
            h = 1e-6 * max(1.0, abs(p[l]))
            e = np.zeros(Np); e[l] = h
            fd = (w @ oracle.model_map(model, dt, x, p + e, I)
                  - w @ oracle.model_map(model, dt, x, p - e, I)) / (2 * h)
            assert abs(gp[l] - fd) <= 1e-7 * max(1.0, abs(fd))
