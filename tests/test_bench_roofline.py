"""The roofline denominators bench.py reports, against the arithmetic stated
for them: the per-map cost of the FP32 HH RK4 map counted from its formula
(4 field evaluations of 50 FP32 operations, 16 of them fmas, and 5 SFU
operations; 28 stage combinations, 24 of them fmas), and the derived peak from
the unit counts (FP32 lanes 128 and SFU 16 per clock and SM)."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_map_cost_matches_its_count(bench):
    per_field_ops, per_field_fmas, per_field_sfu = 50, 16, 5
    combos, combo_fmas = 28, 24
    assert bench.FP32_OPS_PER_MAP == 4 * per_field_ops + combos
    assert bench.MUFU_OPS_PER_MAP == 4 * per_field_sfu
    # flops with an fma counted as two
    assert bench.FLOP_PER_MAP == bench.FP32_OPS_PER_MAP + 4 * per_field_fmas + combo_fmas


def test_derived_peak_is_fp32_bound(bench):
    n_sm, mhz = 152, 2070.0
    fp32_clk = bench.FP32_OPS_PER_MAP / 128.0
    sfu_clk = bench.MUFU_OPS_PER_MAP / 16.0
    assert fp32_clk > sfu_clk  # the map is bound by the FP32 lanes, not the SFU
    peak = bench._peak_fp32_tflops(n_sm, mhz)
    assert peak == pytest.approx(bench.FLOP_PER_MAP * n_sm * mhz * 1e6 / fp32_clk / 1e12, rel=1e-12)
    assert peak == pytest.approx(55.8, abs=0.05)


def test_maps_per_sweep(bench):
    # one map per site and sweep for the state moves, one per site and free
    # parameter for the parameter moves (sites 0..M-1 carry a map)
    assert bench.maps_per_sweep(32768, 7) == 8 * 32768


def test_survey_count_fraction(bench):
    # the scope table's count: 24 ex2 + 14 rcp a map on 16 SFU lanes per clock
    # and SM is the binding unit (its ~250 flop take fewer FP32 clocks)
    maps, t, n_sm, mhz = 10 * 8 * 32768, 242e-6, 152, 2070.0
    fr = bench.roofline_fracs(maps, t, n_sm, mhz)
    t_sfu = maps * 38 / (16 * n_sm * mhz * 1e6)
    assert fr["frac_survey_count"] == pytest.approx(t_sfu / t, rel=1e-12)
    t_fp32 = maps * 228 / (128 * n_sm * mhz * 1e6)
    assert fr["frac_recount"] == pytest.approx(t_fp32 / t, rel=1e-12)


def test_traffic_only_for_the_captured_kernel_sources(bench, monkeypatch):
    rec = {("resident", 32768): {"bytes": 8.0e6, "sweeps": 10, "src": bench.kernel_source_hash(), "profile": "x"}}
    monkeypatch.setattr(bench, "TRAFFIC", rec)
    assert bench.traffic_of("resident", 32768, 10) == pytest.approx(8.0e6)
    assert bench.traffic_of("resident", 32768, 20) == pytest.approx(16.0e6)
    assert bench.traffic_of("general", 32768, 10) is None
    rec[("resident", 32768)]["src"] = "0" * 16
    assert bench.traffic_of("resident", 32768, 10) is None


def test_ess_block_flags_agreement_and_length(bench):
    rng = np.random.default_rng(0)
    K, n, phi = 32, 2000, 0.5
    x = np.empty((K, n, 2))
    x[:, 0] = rng.standard_normal((K, 2)) / np.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[:, t] = phi * x[:, t - 1] + rng.standard_normal((K, 2))
    blk = bench._ess_block(x, 2.0, ["a", "b"], n_boot=20)
    assert blk["established"] and blk["max_rhat"] < 1.05
    assert blk["min_ess"] == min(v["ess"] for v in blk["params"].values())
    assert blk["min_ess_per_s"] == pytest.approx(blk["min_ess"] / 2.0)
    # AR(1) with phi = 1/2: tau = 3
    assert abs(blk["min_ess"] - K * n / 3) < 0.15 * K * n / 3
    y = x.copy()
    y[: K // 2, :, 1] += 5.0  # half the chains elsewhere in one parameter
    blk2 = bench._ess_block(y, 2.0, ["a", "b"], n_boot=20)
    assert not blk2["established"] and blk2["params"]["b"]["rhat"] > 1.5
