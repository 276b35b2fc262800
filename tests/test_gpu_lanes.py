"""The FP32 HH map in its two lane forms, through the C ABI.

The FP32-mixed sweep evaluates the model map one site alone (site phases,
the resident form's first parameter move) or two at a time as the lanes of
one packed f32x2 evaluation (the general and batched forms' parameter moves,
the resident form's speculative outcomes).  Every operation of the lane form
is explicitly rounded and no packed product feeds an addition, so both forms
must give the same bits; the single-site map must also agree with the FP64
oracle's map to FP32 accuracy."""
import numpy as np
import pytest

import oracle
from paper_1103_4887_gb300 import pimc, synth

pytestmark = pytest.mark.gpu

DT = 0.02


def _states(n, seed):
    rng = np.random.default_rng(seed)
    X = np.empty((4, n))
    X[0] = rng.uniform(-90.0, 60.0, n)
    X[1:] = rng.uniform(0.0, 1.0, (3, n))
    # the removable singularities of alpha_m, alpha_n and both sides of the
    # series cut of psi (|u| = 1e-2, u = (V + 40)/10 or (V + 55)/10)
    special = np.array([-40.0, -55.0, -40.1, -39.9, -55.1, -54.9, -40.0999, -39.9001, -65.0, 0.0, 50.0])
    m = min(n, special.size)
    X[0, :m] = special[:m]
    I = rng.uniform(0.0, 20.0, n)
    return X, I


@pytest.mark.parametrize("n", [1, 2, 7, 100001])
def test_packed_lanes_match_single_site_map_bitwise(n):
    X, I = _states(n, seed=n)
    f, mismatch = pimc.debug_lane_maps(X, I, synth.HH_TRUTH, DT)
    assert mismatch == 0
    assert np.all(np.isfinite(f))


def test_single_site_map_against_fp64_oracle():
    n = 20001
    X, I = _states(n, seed=5)
    p = synth.HH_TRUTH
    f, mismatch = pimc.debug_lane_maps(X, I, p, DT)
    assert mismatch == 0
    X32 = X.astype(np.float32).astype(np.float64)  # the device rounds the inputs to FP32
    I32 = I.astype(np.float32).astype(np.float64)
    p32 = np.asarray(p, dtype=np.float32).astype(np.float64)
    for k in list(range(0, 11)) + list(range(11, n, 97)):
        ref = oracle.model_map(oracle.MODEL_HH, DT, X32[:, k], p32, I32[k])
        # FP32 arithmetic over one RK4 step of the HH field (about 230 rounded
        # operations and SFU exponentials of ~2^-22 relative error)
        assert np.all(np.abs(f[:, k] - ref) <= 1e-4 * np.maximum(1.0, np.abs(ref))), (k, f[:, k], ref)


def test_rejects_bad_arguments():
    X, I = _states(4, seed=1)
    with pytest.raises(pimc.PimcError) as e:
        pimc.debug_lane_maps(X, I, synth.HH_TRUTH, 0.0)
    assert e.value.code == pimc.ERR_ARG


def test_map_rate_probe_is_positive_and_packed_not_slower():
    single = pimc.debug_map_rate(False, 2, 500)
    packed = pimc.debug_map_rate(True, 2, 500)
    assert single > 0 and packed > 0.9 * single
    fp64 = pimc.debug_map_rate(False, 1, 50, fp64=True)
    assert 0 < fp64 < single
    with pytest.raises(pimc.PimcError):
        pimc.debug_map_rate(True, 3, 500)
