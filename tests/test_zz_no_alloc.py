"""The allocation-free action entry point (pimc_action_static) against the
handle-based one (pimc_action_dev) and the FP64 oracle, through the C ABI.

pimc_action_static serves callers that cannot allocate device memory at call
time (fixed budgets or caller-owned pools, plugin hosts that forbid
cudaMalloc/cudaFree, real-time loops).  Its scratch is one fixed device array
shared by every call, so two calls in a row must both be right: the second
sees whatever the first left in the array.  The cases cover every model the
entry point supports, the smallest path (M = 1) and the full scratch
(M = 262,143: 2048 CTAs, the last slot of the array).  This file is collected
last so that a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import pimc, synth

pytestmark = pytest.mark.gpu

STATIC_MAX_M = 262143


def _problem(model, M):
    if model == pimc.MODEL_HH:
        return synth.hh_problem(M, data_seed=11, free="all")
    if model == pimc.MODEL_LINGAUSS:
        return synth.lingauss_problem(M, data_seed=12)
    return synth.toy_problem(M, data_seed=13, p_free=True)


def _base(prob):
    if prob.X_true is not None:
        return prob.X_true
    X = np.zeros((prob.D, prob.M + 1))
    X[0] = prob.y
    return X


@pytest.mark.parametrize("model,M", [(pimc.MODEL_HH, STATIC_MAX_M), (pimc.MODEL_HH, 1),
                                     (pimc.MODEL_LINGAUSS, 300), (pimc.MODEL_TOY1D, 90)])
def test_action_static_matches_handle_action_and_oracle_on_two_calls(model, M):
    torch = pytest.importorskip("torch")
    prob = _problem(model, M)
    g = pimc.Sampler.from_problem(prob)
    o = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf)
    o.set_data(prob.y, prob.I)
    o.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    y = torch.tensor(prob.y, dtype=torch.float64, device=dev)
    I = torch.tensor(prob.I, dtype=torch.float64, device=dev)
    p = torch.tensor(prob.p_init, dtype=torch.float64, device=dev)
    out_ref = torch.zeros(3, dtype=torch.float64, device=dev)
    out_new = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    for k in range(2):
        Xh = synth.random_path_near(prob, _base(prob), (0.2 + 0.3 * k) * prob.sig_x, seed=40 + k)
        X = torch.tensor(Xh, dtype=torch.float64, device=dev).contiguous()
        g.action_dev(X.data_ptr(), p.data_ptr(), out_ref.data_ptr(), stream.cuda_stream)
        pimc.action_static(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf, X.data_ptr(), p.data_ptr(),
                           y.data_ptr(), I.data_ptr(), out_new.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        ref = out_ref.cpu().numpy()
        new = out_new.cpu().numpy()
        np.testing.assert_allclose(new, ref, rtol=1e-12, atol=0.0)
        assert abs(new[0] - (new[1] + new[2])) <= 1e-12 * abs(new[0])
        o.set_path(Xh)
        np.testing.assert_allclose(new, np.array(o.action()), rtol=1e-12, atol=0.0)
        out_new.fill_(float("nan"))


def test_action_static_rejects_sizes_beyond_its_scratch():
    with pytest.raises(pimc.PimcError) as e:
        pimc.action_static(0, STATIC_MAX_M + 1, 0.02, 4.0, [1e2, 1e4, 1e4, 1e4], 1, 1, 1, 1, 1, 0)
    assert e.value.code == pimc.ERR_ARG
    assert str(STATIC_MAX_M) in str(e.value)


def test_action_static_rejects_unsupported_model_and_short_Rf():
    with pytest.raises(pimc.PimcError) as e:
        pimc.action_static(pimc.MODEL_HH_PAPER, 100, 0.04, 100.0, [1e2, 1e6, 1e6, 1e6], 1, 1, 1, 1, 1, 0)
    assert e.value.code == pimc.ERR_ARG
    assert "not supported" in str(e.value)
    with pytest.raises(pimc.PimcError) as e:
        pimc.action_static(pimc.MODEL_HH, 100, 0.02, 4.0, [1e2], 1, 1, 1, 1, 1, 0)
    assert e.value.code == pimc.ERR_ARG
