"""The adjoint of the action on the GPU (workload of the differentiation
config: HH, M = 16384, all 7 parameters), through the C ABI and through the
torch.autograd.Function:

* against the oracle's independent reverse mode (FP64, every component);
* against central finite differences (h = 1e-6 max(1, |x|)) of the GPU's own
  local changes of action (pimc_site_delta / pimc_param_delta, which equal
  differences of the full action without its cancellation): 1e-8 relative;
* FP32-mixed against FP64 (reported, loose bound).
"""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import pimc, synth

pytestmark = pytest.mark.gpu

M = 16384


@pytest.fixture(scope="module")
def setup():
    prob = synth.hh_problem(M, data_seed=7, free="all")
    X = synth.random_path_near(prob, prob.X_true, 0.5 * prob.sig_x, seed=3)
    g = pimc.Sampler.from_problem(prob)
    g.set_path(X)
    return prob, X, g


def test_gpu_grad_matches_oracle_reverse_mode(setup):
    prob, X, g = setup
    o = oracle.Chain(0, prob.M, prob.dt, prob.Rm, prob.Rf)
    o.set_data(prob.y, prob.I)
    o.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    o.set_path(X)
    gXg, gpg = g.grad(1.0)
    gXo, gpo = o.grad(1.0)
    scale = np.abs(gXo).max(axis=1, keepdims=True)
    assert np.max(np.abs(gXg - gXo) / scale) < 1e-11
    np.testing.assert_allclose(gpg, gpo, rtol=1e-10)


@pytest.mark.parametrize("scheme", [0, 1])
def test_gpu_grad_strided_tiles_matches_oracle(scheme):
    """600 001 sites: more tiles than CTAs, so every CTA of the gather-form
    gradient kernel strides over several tiles (both discretisations)."""
    prob = synth.hh_problem(600000, data_seed=1)
    prob.scheme = scheme
    X = synth.random_path_near(prob, prob.X_true, 0.5 * prob.sig_x, seed=3)
    g = pimc.Sampler.from_problem(prob)
    g.set_path(X)
    o = oracle.Chain(0, prob.M, prob.dt, prob.Rm, prob.Rf)
    o.set_scheme(scheme)
    o.set_data(prob.y, prob.I)
    o.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    o.set_path(X)
    gXg, gpg = g.grad(0.7)
    gXo, gpo = o.grad(0.7)
    scale = np.abs(gXo).max(axis=1, keepdims=True)
    assert np.max(np.abs(gXg - gXo) / scale) < 1e-11
    np.testing.assert_allclose(gpg, gpo, rtol=1e-9)


def test_gpu_grad_matches_central_differences(setup):
    prob, X, g = setup
    gX, gp = g.grad(1.0)
    rng = np.random.default_rng(0)
    for k in rng.choice(4 * (M + 1), size=48, replace=False):
        a, n = divmod(int(k), M + 1)
        h = 1e-6 * max(1.0, abs(X[a, n]))
        Xa = X.copy(); Xa[a, n] += h
        Xb = X.copy(); Xb[a, n] -= h
        fd = (g.site_delta(Xa)[n] - g.site_delta(Xb)[n]) / (2 * h)
        assert abs(gX[a, n] - fd) <= 1e-8 * max(abs(fd), 1e-3 * np.abs(gX[a]).max()), (a, n, gX[a, n], fd)
    for l in range(7):
        h = 1e-6 * max(1.0, abs(prob.p_init[l]))
        fd = (g.param_delta(l, prob.p_init[l] + h) - g.param_delta(l, prob.p_init[l] - h)) / (2 * h)
        assert abs(gp[l] - fd) <= 1e-8 * abs(fd), (l, gp[l], fd)


def test_fp32_mixed_gradient_against_fp64(setup):
    prob, X, g = setup
    g32 = pimc.Sampler.from_problem(prob, precision=pimc.FP32_MIXED)
    g32.set_path(X)
    gX64, gp64 = g.grad(1.0)
    gX32, gp32 = g32.grad(1.0)
    scale = np.abs(gX64).max(axis=1, keepdims=True)
    err = np.abs(gX32 - gX64) / scale
    assert np.median(err) < 1e-5
    assert np.all(np.abs(gp32 - gp64) <= 1e-3 * np.abs(gp64) + 1e-3)


def test_autograd_function(setup):
    torch = pytest.importorskip("torch")
    from paper_1103_4887_gb300.autograd import path_action
    prob, X, g = setup
    dev = torch.device("cuda", 0)
    Xt = torch.tensor(X, dtype=torch.float64, device=dev, requires_grad=True)
    pt = torch.tensor(prob.p_init, dtype=torch.float64, device=dev, requires_grad=True)
    A = path_action(Xt, pt, g)
    (3.0 * A).backward()
    A_ref = g.action()[0]
    assert abs(A.item() - A_ref) <= 1e-12 * abs(A_ref)
    gX, gp = g.grad(1.0)
    np.testing.assert_allclose(Xt.grad.cpu().numpy(), 3.0 * gX, rtol=0, atol=1e-12 * np.abs(gX).max())
    np.testing.assert_allclose(pt.grad.cpu().numpy(), 3.0 * gp, rtol=1e-12)
