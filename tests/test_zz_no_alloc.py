"""The allocation-free action entry point (pimc_action_static) against the
handle-based one (pimc_action_dev), through the C ABI.

pimc_action_static serves callers that cannot allocate device memory at call
time (fixed budgets or caller-owned pools, plugin hosts that forbid
cudaMalloc/cudaFree, real-time loops).  Its scratch is one fixed device array
shared by every call, so two calls in a row must both be right: the second
sees whatever the first left in the array.  This file is collected last so
that a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

from paper_1103_4887_gb300 import pimc, synth

pytestmark = pytest.mark.gpu


def test_action_static_matches_handle_action_on_two_calls():
    torch = pytest.importorskip("torch")
    prob = synth.hh_problem(5000, data_seed=11, free="all")
    g = pimc.Sampler.from_problem(prob)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    y = torch.tensor(prob.y, dtype=torch.float64, device=dev)
    I = torch.tensor(prob.I, dtype=torch.float64, device=dev)
    p = torch.tensor(prob.p_init, dtype=torch.float64, device=dev)
    out_ref = torch.zeros(3, dtype=torch.float64, device=dev)
    out_new = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    for k in range(2):
        Xh = synth.random_path_near(prob, prob.X_true, (0.2 + 0.3 * k) * prob.sig_x, seed=40 + k)
        X = torch.tensor(Xh, dtype=torch.float64, device=dev).contiguous()
        g.action_dev(X.data_ptr(), p.data_ptr(), out_ref.data_ptr(), stream.cuda_stream)
        pimc.action_static(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf, X.data_ptr(), p.data_ptr(),
                           y.data_ptr(), I.data_ptr(), out_new.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        ref = out_ref.cpu().numpy()
        new = out_new.cpu().numpy()
        np.testing.assert_allclose(new, ref, rtol=1e-12, atol=0.0)
        assert abs(new[0] - (new[1] + new[2])) <= 1e-12 * abs(new[0])


def test_action_static_rejects_sizes_beyond_its_scratch():
    with pytest.raises(pimc.PimcError) as e:
        pimc.action_static(0, 262144, 0.02, 4.0, [1e2, 1e4, 1e4, 1e4], 1, 1, 1, 1, 1, 0)
    assert e.value.code == pimc.ERR_ARG
    assert "262143" in str(e.value)
