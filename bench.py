"""Benchmark: HH Metropolis site-updates/s of the GB300 sampler.

Workload: Hodgkin-Huxley D = 4, all 7 parameters free, M = 32768 time steps
(dt = 0.02 ms), seeded OU drive, noisy voltage observations.  One step is one
launch of N_skip = 10 full checkerboard sweeps -- each sweep: even sites, odd
sites, 7 sequential parameter moves (each a full-path RK4 pass plus an FP64
reduction and accept test) -- ending with one moment/histogram/residual
record, so that a step runs every row of the hot path once.  value =
(M + 1) * N_skip site updates per step / device time per step, summed over
ranks (independent replica chains, weak scaling).  The L2 is flushed (a
256 MiB write) before every timed step; each step is timed with CUDA events on
the sampler's stream.

--impl reference times the serial FP64 CPU oracle (the method's plain
statement) on the host for the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

# concurrent HMC chains, one stream each: up to 32 hardware work queues (the
# default is 8); set before the process creates its CUDA context
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HH Metropolis site-updates/s (M=32768, 7 free params, checkerboard sweep)"
UNIT = "site-updates/s"
M_DEFAULT = 32768
NSKIP = 10
# The paper's own speedup (Sec. 5, Fig. speedup): other hardware, its FP32
# tanh-model workload, against a different CPU code; context, not a target.
PAPER_SPEEDUP_CONTEXT = ("T_CPU/T_GPU up to about 300 (GTX 470, 448 cores) and 200 (GTX 460) against one "
                         "Intel Core i3 core, FP32, M = 100..40000, 1e5 sweeps")
SEED = 1
REF_BUDGET_S = 120.0
# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum, cold cache)
# of one launch of a sweep kernel, with the hash of the kernel sources it was
# captured on: a figure is reported only while the sources still hash the same
# (a changed kernel has no traffic figure until it is captured again).
KERNEL_SOURCES = ("paper_1103_4887_gb300/csrc/sweep.cu", "paper_1103_4887_gb300/csrc/device.cuh",
                  "paper_1103_4887_gb300/csrc/scheme.cuh", "paper_1103_4887_gb300/csrc/stats.cuh",
                  "paper_1103_4887_gb300/csrc/internal.h")
TRAFFIC = {
    # one 10-sweep bench step of sweep_resident_kernel<HH<float>>, M = 32768
    ("resident", 32768): {"bytes": 7.8523e6, "sweeps": 10, "src": "3933e0b65b73c5e5",
                          "profile": "profiles/sweep_resident_kernel_hh_M32768_full.md"},
    # one 10-sweep launch of sweep_kernel<HH<float>,float>, M = 2^20
    ("general", 1048576): {"bytes": 586.50e6, "sweeps": 10, "src": "3933e0b65b73c5e5",
                           "profile": "profiles/sweep_kernel_hh_M1048576_full.md"},
}

# Algorithmic cost of one RK4 map of the HH vector field in the FP32-mixed
# form, counted from the formula (4 field evaluations of 50 FP32 operations
# -- 16 of them fmas -- and 5 SFU operations: exponentials of -(V+65)/80,
# -(V+65)/18 and the two psi arguments, one shared reciprocal; 28 stage
# combinations, 24 of them fmas): FP32 instructions and SFU (MUFU) operations.
FP32_OPS_PER_MAP = 228
MUFU_OPS_PER_MAP = 20
# FP32 floating-point operations per map (an FMA counted as 2).
FLOP_PER_MAP = 316
# The scope table's own count of one RK4 map of the HH field (6 exponentials and
# 3-4 divides per field evaluation): 24 ex2 and 14 rcp on the SFU, about 250
# FP32 flop; at 16 SFU operations per clock and SM it is SFU-bound.
SURVEY_SFU_OPS_PER_MAP = 38
SURVEY_FLOP_PER_MAP = 250


def maps_per_sweep(M, n_free):
    # one map per site move (sites 0..M-1 have a successor) and M per free parameter
    return M * (1 + n_free)


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_of(form, M, n_sweeps):
    """DRAM bytes of one launch of n_sweeps sweeps from the recorded capture,
    scaled by the sweeps (a launch's traffic grows with its sweeps), or None
    when there is no capture for this kernel and size, or the kernel sources
    changed since it was taken."""
    rec = TRAFFIC.get((form, M))
    if rec is None or rec["src"] != kernel_source_hash():
        return None
    return rec["bytes"] * n_sweeps / rec["sweeps"]


def roofline_fracs(maps, seconds, n_sm, sm_mhz):
    """Fractions of the FP32/SFU compute roofline reached by `maps` RK4 maps in
    `seconds`: against the map's recount (228 FP32 + 20 SFU operations,
    FP32-bound) and against the scope table's count (24 ex2 + 14 rcp on the
    SFU, SFU-bound)."""
    f = sm_mhz * 1e6
    t_recount = maps * max(FP32_OPS_PER_MAP / 128.0, MUFU_OPS_PER_MAP / 16.0) / (n_sm * f)
    t_survey = maps * max(SURVEY_FLOP_PER_MAP / 2.0 / 128.0, SURVEY_SFU_OPS_PER_MAP / 16.0) / (n_sm * f)
    return {"frac_recount": t_recount / seconds, "frac_survey_count": t_survey / seconds,
            "t_min_recount_s": t_recount, "t_min_survey_count_s": t_survey}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while active."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is not None:
            time.sleep(0.06)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.rows = [[c.strip() for c in ln.split(",")] for ln in out.splitlines() if ln.strip()]
        return False


def summarize_clocks(rows):
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
    mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 4 + i and r[4 + i].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(prob, budget_s=12.0):
    """The serial FP64 oracle as it stands, on one host core, for a bounded
    number of full sweeps of the same workload."""
    import oracle
    ch = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf)
    ch.set_data(prob.y, prob.I)
    ch.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    ch.set_steps(prob.sig_x, prob.sig_p)
    ch.set_schedule(n_init=0, n_skip=NSKIP)
    n = 0
    t0 = time.perf_counter()
    while True:
        ch.sweep(1, SEED)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 200:
            break
    return {"value": (prob.M + 1) * n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full sweeps of the M={prob.M} workload (all 7 params free), serial FP64, "
                      f"{el:.1f} s"}


def workload_config(M):
    """The workload a step runs, the same in both arms: HH with all 7
    parameters free, N_skip sweeps a step, one statistics record a step."""
    return {"workload": f"hh_M{M}_7free", "M": M, "n_free": 7, "sweeps_per_step": NSKIP, "n_skip": NSKIP}


def run_reference(args):
    """The serial FP64 oracle on one host core, same workload, step, metric and
    unit: a step is N_skip full sweeps with one statistics record, after
    W warm-up steps that adapt the steps (as the GPU arm's warm-up does); the
    timed steps stop after REF_BUDGET_S seconds so the run ends within a few
    minutes whatever K is."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1103_4887_gb300 import synth
    import oracle
    prob = synth.hh_problem(args.M, data_seed=0, free="all")
    ch = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf)
    ch.set_data(prob.y, prob.I)
    ch.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
    ch.set_steps(prob.sig_x, prob.sig_p)
    ch.set_schedule(n_init=args.warmup * NSKIP, n_skip=NSKIP, f_acc=0.4, alpha=0.5)
    for _ in range(args.warmup):
        ch.sweep(NSKIP, SEED)
    times = []
    t_start = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ch.sweep(NSKIP, SEED)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > REF_BUDGET_S:
            break
    tot = sum(times)
    n = len(times)
    value = (prob.M + 1) * NSKIP * n / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * tot / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.M),
            "run": {"precision": "fp64", "where": "host, one core (serial oracle)", "steps_requested": args.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{n} steps of {NSKIP} full sweeps of the M={args.M} workload (of "
                                       f"{args.steps} requested, bounded at {REF_BUDGET_S:.0f} s), serial FP64 "
                                       f"oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile_case(args):
    """Three launches of one bench step (N_skip sweeps) of the sweep kernel in
    each precision on the bench workload (no timing); the case the ncu
    captures use."""
    from paper_1103_4887_gb300 import pimc, synth
    prob = synth.hh_problem(args.M, data_seed=0, free="all")
    for prec in (pimc.FP32_MIXED, pimc.FP64):
        s = pimc.Sampler.from_problem(prob, precision=prec)
        s.set_schedule(n_init=0, n_skip=NSKIP)
        for _ in range(3):
            s.sweep(NSKIP, SEED)
        print(json.dumps({"precision": prec, "form": s.sweep_form(), "grid_block": list(s.launch_info())}))
        s.close()
    print("profile case done")


def run_profile_hmc(args):
    """Three whole-path HMC trajectories (L = 20) in each precision on the
    ESS workload (HH, M = 16384, all 7 parameters free; no timing); the case
    the ncu captures of the leapfrog kernel use."""
    from paper_1103_4887_gb300 import pimc, synth
    prob = synth.hh_problem(16384, data_seed=0, free="all")
    for prec in (pimc.FP32_MIXED, pimc.FP64):
        s = pimc.Sampler.from_problem(prob, precision=prec)
        s.set_params(prob.p_true, prob.lo, prob.hi, prob.free)
        s.set_path(prob.X_true)
        s.set_schedule(n_init=10 ** 9, n_skip=1)
        n = s.hmc(3, 20, 0.005, None, seed=SEED)
        print(json.dumps({"precision": prec, "accepted": n}))
        s.close()
    print("profile case done")


def _peak_fp32_tflops(n_sm, sm_mhz):
    t_map = max(FP32_OPS_PER_MAP / (n_sm * 128 * sm_mhz * 1e6), MUFU_OPS_PER_MAP / (n_sm * 16 * sm_mhz * 1e6))
    return FLOP_PER_MAP / t_map / 1e12


def map_ceiling():
    """Maps per second of the FP32 HH map alone, iterated from registers by
    every SM (pimc_debug_map_rate): one site a thread or two on the packed
    f32x2 lanes, at 1 and 2 CTAs of 256 threads an SM -- the ceiling of a
    sweep's map arithmetic on this device, beside the derived peak."""
    import torch
    from paper_1103_4887_gb300 import pimc
    peaks, _ = load_peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_maps = n_sm * 128.0 * sm_mhz * 1e6 / FP32_OPS_PER_MAP  # derived peak in maps/s (FP32-bound)
    out = {"derived_peak_maps_per_s": peak_maps}
    for packed in (False, True):
        for k in (1, 2):
            r = pimc.debug_map_rate(packed, k, 4000)
            out[f"{'packed' if packed else 'single'}_{k}cta_per_sm"] = {"maps_per_s": r, "frac_of_derived_peak":
                                                                         r / peak_maps}
    # the FP64 map (software exponentials on the FP64 pipe), the plain sweep's ceiling
    out["fp64_1cta_per_sm"] = {"maps_per_s": pimc.debug_map_rate(False, 1, 200, fp64=True)}
    return out


def sweep_M_rows(exps=range(10, 21, 2), cpu_budget_s=4.0, ceiling=None):
    """Observation-length sweep (HH, all 7 parameters free): per M, device time
    per sweep in one persistent launch (state L2-resident between sweeps, as in
    a sampling run), FP32-mixed and FP64, and the oracle timed on the host for a
    bounded number of sweeps -- the serial build on one core and the OpenMP
    build on all cores (its thread count stated)."""
    import torch
    import oracle
    from paper_1103_4887_gb300 import pimc, synth
    peaks, peak_src = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    rows = []
    for e in exps:
        M = 1 << e
        prob = synth.hh_problem(M, data_seed=0, free="all")
        row = {"M": M}
        for name, prec, n in (("fp32mixed", pimc.FP32_MIXED, 400 if M <= 1 << 16 else 100),
                              ("fp64", pimc.FP64, 40 if M <= 1 << 16 else 10)):
            s = pimc.Sampler.from_problem(prob, precision=prec)
            s.set_schedule(n_init=0, n_skip=NSKIP)
            s.sweep(5, SEED)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            st = torch.cuda.current_stream()
            s.set_stream(st.cuda_stream)
            e0.record(st)
            s.sweep(n, SEED, sync=False)
            e1.record(st)
            torch.cuda.synchronize()
            s.sync()
            ms = e0.elapsed_time(e1) / n
            maps = maps_per_sweep(M, 7)
            form = s.sweep_form()
            entry = {"ms_per_sweep": ms, "site_updates_per_s": (M + 1) / (ms * 1e-3),
                     "rk4_maps_per_s": maps / (ms * 1e-3), "sweeps_timed": n, "form": form,
                     "grid_block": list(s.launch_info())}
            if prec == pimc.FP32_MIXED:
                tf = maps * FLOP_PER_MAP / (ms * 1e-3) / 1e12
                entry.update({"achieved_tflops": tf, **roofline_fracs(maps, ms * 1e-3, n_sm, sm_mhz)})
                if ceiling:
                    entry["frac_of_map_ceiling"] = (maps / (ms * 1e-3)) / ceiling["packed_2cta_per_sm"]["maps_per_s"]
                tr = traffic_of(form, M, 10)
                if tr is not None:
                    entry["traffic_bytes_per_10_sweeps"] = tr
                    entry["dram_gbs"] = tr / (10 * ms * 1e-3) / 1e9
            else:
                # FP64 transcendental functions are software sequences on the FP64
                # pipe: the achieved rate is stated as maps/s against the FP64 map's
                # own measured ceiling; the FP32 count does not apply
                entry["note"] = "FP64 pipe-bound (software exp); compare maps/s"
                if ceiling and "fp64_1cta_per_sm" in ceiling:
                    entry["frac_of_fp64_map_ceiling"] = (maps / (ms * 1e-3)) / ceiling["fp64_1cta_per_sm"]["maps_per_s"]
            row[name] = entry
            s.close()
        n_cpu = 100 if M <= 1 << 12 else (10 if M <= 1 << 16 else 2)
        for key, omp in (("oracle_1core", False), ("oracle_allcores", True)):
            try:
                ch = oracle.Chain(prob.model, prob.M, prob.dt, prob.Rm, prob.Rf, openmp=omp)
            except Exception as ex:  # no OpenMP build on this host
                row[key] = {"error": repr(ex)}
                continue
            ch.set_data(prob.y, prob.I)
            ch.set_params(prob.p_init, prob.lo, prob.hi, prob.free)
            ch.set_steps(prob.sig_x, prob.sig_p)
            t0 = time.perf_counter()
            k = 0
            while k < n_cpu:
                ch.sweep(1, SEED)
                k += 1
                if time.perf_counter() - t0 > cpu_budget_s:
                    break
            cpu_s = (time.perf_counter() - t0) / k
            row[key] = {"s_per_sweep": cpu_s, "site_updates_per_s": (M + 1) / cpu_s, "sweeps_timed": k,
                        "threads": oracle.threads(omp), "nproc": os.cpu_count()}
        cpu_s = row["oracle_1core"]["s_per_sweep"]
        row["speedup_fp32_vs_oracle_1core"] = cpu_s / (row["fp32mixed"]["ms_per_sweep"] * 1e-3)
        row["speedup_fp64_vs_oracle_1core"] = cpu_s / (row["fp64"]["ms_per_sweep"] * 1e-3)
        if "s_per_sweep" in row["oracle_allcores"]:
            row["speedup_fp32_vs_oracle_allcores"] = (row["oracle_allcores"]["s_per_sweep"]
                                                      / (row["fp32mixed"]["ms_per_sweep"] * 1e-3))
        rows.append(row)
    return {"rows": rows, "paper_speedup_context": PAPER_SPEEDUP_CONTEXT,
            "peak_clock": f"{sm_mhz:.0f} MHz ({peak_src})", "n_sm": n_sm,
            "frac_recount": "maps x max(228/128, 20/16) clocks / (SMs x clock) / time",
            "frac_survey_count": "maps x max(125/128, 38/16) clocks / (SMs x clock) / time"}


def run_sweep_M(args):
    ceil = map_ceiling()
    print(json.dumps({"map_ceiling": ceil}), flush=True)
    for row in sweep_M_rows(cpu_budget_s=30.0, ceiling=ceil)["rows"]:
        print(json.dumps(row), flush=True)


def run_batch(args):
    """Many chains in one launch: 64 seeded HH data sets with M uniform in
    [2048, 65536] and true (gNa, gK, gL) within +-20 % of nominal, 8 chains each
    (512 chains), FP32-mixed, tile shape chosen by the autotuner; device time of
    a block of sweeps (every chain advances by `steps` sweeps)."""
    import torch
    from paper_1103_4887_gb300 import pimc, synth
    rng = np.random.default_rng(2024)
    st = torch.cuda.current_stream()  # the batch launches on its first handle's stream
    n_sets, per_set = 64, 8
    Ms = rng.integers(2048, 65537, size=n_sets)
    samplers = []
    for d in range(n_sets):
        q = synth.HH_TRUTH.copy()
        q[:3] *= 1.0 + 0.2 * rng.uniform(-1.0, 1.0, 3)
        prob = synth.hh_problem(int(Ms[d]), data_seed=100 + d, free=("gNa", "gK", "gL"), p_true=q)
        for k in range(per_set):
            s = pimc.Sampler.from_problem(prob, precision=pimc.FP32_MIXED)
            s.set_stream(st.cuda_stream)
            s.set_chain(k)
            s.set_schedule(n_init=10 ** 6, n_skip=20, f_acc=0.4, alpha=0.5)
            samplers.append(s)
    b = pimc.Batch(samplers)
    nt, k, g = b.autotune(4, SEED)
    steps = max(args.steps // 30, 20)
    b.sweep(steps, SEED)  # warm-up: also captures the graph of a `steps`-sweep block
    torch.cuda.synchronize()
    el = _timer(st)(lambda: b.sweep(steps, SEED, sync=False))
    sites = int(sum(int(m) + 1 for m in Ms)) * per_set
    maps = int(sum(maps_per_sweep(int(m), 3) for m in Ms)) * per_set
    n_ctas, _, n_split = b.info()
    peaks, _ = load_peaks()
    fr = roofline_fracs(maps * steps, el, torch.cuda.get_device_properties(0).multi_processor_count,
                        float(peaks.get("sm_max_mhz", 2070.0)))
    res = {"mode": "batch", "chains": n_sets * per_set, "data_sets": n_sets, "sites_per_sweep": sites,
           "sweeps": steps, "seconds": el, "site_updates_per_s": sites * steps / el,
           "ms_per_sweep_all_chains": 1e3 * el / steps, "tuning": {"threads_per_cta": nt,
           "ctas_per_sm": k, "ctas_per_long_chain": g, "chains_split": n_split, "ctas": n_ctas}, "precision": "fp32mixed",
           "rk4_maps_per_s": maps * steps / el, "frac_recount": fr["frac_recount"],
           "frac_survey_count": fr["frac_survey_count"]}
    b.close()
    for s in samplers:
        s.close()
    return res


def run_paper(args):
    """The paper's Sec. 5.1 workload shape (M = 8000, D = 4, 7 free parameters,
    trapezoid model error, tanh gate kinetics, uniform proposals) on synthetic
    OU-driven data: device time per sweep and the time 10^6 sweeps would take,
    beside the paper's 683 s for 10^6 sweeps on a GTX 460 in FP32 (context: other
    hardware and other data)."""
    import torch
    from paper_1103_4887_gb300 import pimc, synth
    prob = synth.paper_problem(8000, data_seed=0, free="all")
    out = {"mode": "paper_setting", "M": 8000, "dt_ms": 0.04, "scheme": "trapezoid", "proposal": "uniform"}
    st = torch.cuda.current_stream()
    for name, prec, n in (("fp32mixed", pimc.FP32_MIXED, 2000), ("fp64", pimc.FP64, 200)):
        s = pimc.Sampler.from_problem(prob, precision=prec)
        s.set_stream(st.cuda_stream)
        s.set_schedule(n_init=10 ** 9, n_skip=400)
        s.sweep(20, SEED)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.sweep(n, SEED, sync=False)
        e1.record(st)
        torch.cuda.synchronize()
        s.sync()
        ms = e0.elapsed_time(e1) / n
        out[name] = {"ms_per_sweep": ms, "site_updates_per_s": 8001 / (ms * 1e-3),
                     "seconds_per_1e6_sweeps": ms * 1e3, "vs_paper_gtx460_683s": 683.0 / (ms * 1e3)}
        s.close()
    return out


def run_mixed(args):
    """FP32-mixed against plain FP64 on the bench workload (HH, M = 32768, all 7
    parameters free): (1) per-site Delta A error on the same path and
    proposals; (2) accept-flip rate -- the fraction of site decisions of one
    sweep from the same state, seed and counters that differ; (3) shift of the
    posterior parameter means in Monte Carlo standard errors (batch means of
    the parameter traces), both chains from the true path after a burn-in."""
    import torch
    from paper_1103_4887_gb300 import diagnostics, pimc, synth
    M = args.M
    prob = synth.hh_problem(M, data_seed=0, free="all")
    out = {"M": M, "n_free": 7}
    st = torch.cuda.current_stream()
    # (1) Delta A on the same states and proposals
    X = synth.random_path_near(prob, prob.X_true, 0.5 * prob.sig_x, seed=11)
    Xp = synth.random_path_near(prob, X, 2.0 * prob.sig_x, seed=12)
    d = {}
    for name, prec in (("fp64", pimc.FP64), ("fp32", pimc.FP32_MIXED)):
        s = pimc.Sampler.from_problem(prob, precision=prec)
        s.set_path(X)
        d[name] = s.site_delta(Xp)
        s.close()
    err = np.abs(d["fp32"] - d["fp64"])
    big = np.abs(d["fp64"]) > 1.0
    out["delta_A"] = {"abs_err_median": float(np.median(err)), "abs_err_p99": float(np.quantile(err, 0.99)),
                      "abs_err_max": float(err.max()),
                      "rel_err_median_where_abs_dA_gt_1": float(np.median(err[big] / np.abs(d["fp64"][big]))),
                      "rel_err_p99_where_abs_dA_gt_1": float(np.quantile(err[big] / np.abs(d["fp64"][big]), 0.99)),
                      "sites": int(M + 1)}
    # (2) accept flips: one sweep from the same state (path near the truth, adapted steps)
    base = pimc.Sampler.from_problem(prob, precision=pimc.FP64)
    base.set_schedule(n_init=200, n_skip=20, f_acc=0.4, alpha=0.5)
    base.sweep(200, SEED)
    X0, p0 = base.state()
    sx, sp = base.steps()
    base.close()
    moved = {}
    for name, prec in (("fp64", pimc.FP64), ("fp32", pimc.FP32_MIXED)):
        s = pimc.Sampler.from_problem(prob, precision=prec)
        s.set_params(p0, prob.lo, prob.hi, prob.free)
        s.set_path(X0)
        s.set_steps(sx, sp)
        s.set_schedule(n_init=10 ** 9, n_skip=10 ** 6)
        flips_site, flips_par = [], []
        res = []
        for k in range(5):
            s.set_path(X0)
            s.set_params(p0, prob.lo, prob.hi, prob.free)
            Xb, pb = s.state()  # as stored (FP32-mixed rounds the path)
            s.sweep(1, SEED + k)
            X1, p1 = s.state()
            res.append((np.any(X1 != Xb, axis=0), p1 != pb))
        moved[name] = res
        s.close()
    fs = sum(int(np.sum(a[0] != b[0])) for a, b in zip(moved["fp64"], moved["fp32"]))
    fp_ = sum(int(np.sum(a[1] != b[1])) for a, b in zip(moved["fp64"], moved["fp32"]))
    out["accept_flips"] = {"site_flips": fs, "site_decisions": 5 * (M + 1), "site_flip_rate": fs / (5 * (M + 1)),
                           "param_flips": fp_, "param_decisions": 5 * 7}
    # (3) posterior parameter means
    tr = {}
    for name, prec, n in (("fp64", pimc.FP64, 8000), ("fp32", pimc.FP32_MIXED, 8000)):
        s = pimc.Sampler.from_problem(prob, precision=prec)
        s.set_params(prob.p_true, prob.lo, prob.hi, prob.free)
        s.set_path(prob.X_true)
        s.set_stream(st.cuda_stream)
        s.set_schedule(n_init=2000, n_skip=20, f_acc=0.4, alpha=0.5)
        s.sweep(2000, SEED, sync=False)
        s.set_param_trace(n)
        s.sweep(n, SEED, sync=False)
        s.sync()
        tr[name] = s.param_trace()
        s.close()
    m64, m32 = tr["fp64"].mean(0), tr["fp32"].mean(0)
    se64, se32 = diagnostics.batch_means_se(tr["fp64"], 20), diagnostics.batch_means_se(tr["fp32"], 20)
    z = np.abs(m32 - m64) / np.sqrt(se64 ** 2 + se32 ** 2 + 1e-300)
    out["posterior_mean_shift"] = {"sweeps_each": 8000, "burn_in": 2000, "mean_fp64": m64.tolist(),
                                   "mean_fp32": m32.tolist(), "shift_in_se": z.tolist(),
                                   "max_shift_in_se": float(z.max())}
    return out


def _timer(st):
    import torch

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3
    return timed


def _ess_block(tr, secs, names, n_boot=100):
    """Per parameter: multi-chain ESS with a bootstrap-over-chains SE, the
    chain-means cross-check, split R-hat, mean and its MC standard error; the
    minimum over parameters as ESS/s (tr: [K, n, P] parameter traces of K
    chains, secs: device seconds of the sampling phase)."""
    from paper_1103_4887_gb300 import diagnostics as dg
    out = {"chains": int(tr.shape[0]), "steps_per_chain": int(tr.shape[1]), "seconds": secs, "params": {}}
    ess_l = []
    for j, nm in enumerate(names):
        x = tr[:, :, j]
        ess, se = dg.ess_with_se(x, n_boot=n_boot)
        sd = float(x.std())
        out["params"][nm] = {"ess": ess, "ess_se": se, "ess_chain_means": dg.ess_chain_means(x),
                             "rhat": dg.split_rhat(x), "mean": float(x.mean()), "sd": sd,
                             "mc_se": sd / np.sqrt(max(ess, 1.0))}
        ess_l.append((ess, se, nm))
    ess, se, nm = min(ess_l)
    out.update({"min_ess": ess, "min_ess_se": se, "min_ess_param": nm, "min_ess_per_s": ess / secs,
                "min_ess_per_s_se": se / secs, "max_rhat": max(v["rhat"] for v in out["params"].values())})
    out["established"] = bool(out["max_rhat"] < 1.05 and ess >= 100.0)
    return out


def ess_study(prob, K=64, K_hmc=16, pilot=(2000, 2000), n_metro=(20000, 4000), n_hmc=(1000, 200), n_leap=20,
              names=None, seed=SEED, anneal=None, f_acc=0.4, alpha=0.5):
    """Parameter ESS per second of the four samplers on one posterior, from
    independent chains that start in it.  A pilot of K batched FP32-mixed
    Metropolis chains (from the data's initial path, adapting during its first
    half; optionally annealed there as in Sec. 4.2, anneal = (beta0, N_cool))
    supplies each chain's starting state and steps, and the pooled
    variances that serve as HMC's inverse mass.  Then, from those states and
    with fresh seeds: K chains of batched checkerboard Metropolis in FP32-mixed
    and in FP64 (n_metro sweeps each), and K_hmc chains of whole-path HMC in
    FP32-mixed and FP64 (n_hmc trajectories of n_leap steps each, the step
    tuned per chain to ~70 % acceptance first; the chains run concurrently,
    one stream each).  ESS/s divides by the device
    time of the sampling phase; R-hat and the spread of chain means tell
    whether the chains agree (ESS is meaningful only where they do)."""
    import torch
    from paper_1103_4887_gb300 import diagnostics as dg
    from paper_1103_4887_gb300 import pimc
    st = torch.cuda.current_stream()
    timed = _timer(st)
    free = np.flatnonzero(prob.free)
    names = names or [f"p{j}" for j in free]
    out = {"M": prob.M, "n_free": int(free.size), "K_metropolis": K, "K_hmc": K_hmc}

    def make(prec, chain):
        s = pimc.Sampler.from_problem(prob, precision=prec)
        s.set_stream(st.cuda_stream)
        s.set_chain(chain)
        return s

    # pilot
    P = [make(pimc.FP32_MIXED, k) for k in range(K)]
    for s in P:
        if anneal is None:
            s.set_schedule(n_init=pilot[0], n_skip=10, f_acc=f_acc, alpha=alpha)
        else:
            s.set_schedule(n_init=pilot[0], n_skip=10, beta0=anneal[0], n_cool=anneal[1], f_acc=f_acc, alpha=alpha)
        s.set_param_trace(pilot[1])
    b = pimc.Batch(P)
    out["pilot_seconds"] = timed(lambda: b.sweep(pilot[0] + pilot[1], seed + 100, sync=False))
    b.close()
    ptr = np.array([s.param_trace() for s in P])[:, :, free]
    out["pilot"] = {"sweeps": pilot[0] + pilot[1], "adapting": pilot[0], "anneal": anneal,
                    "rhat_after_adaptation": {nm: dg.split_rhat(ptr[:, :, j]) for j, nm in enumerate(names)},
                    "mean": dict(zip(names, ptr.mean(axis=(0, 1)).tolist()))}
    starts = [s.state() for s in P]
    steps = [s.steps() for s in P]
    mv = np.array([s.moments()[:2] for s in P])  # [K, 2, D(M+1)+NP]
    inv_mass = mv[:, 1].mean(axis=0) + mv[:, 0].var(axis=0)  # pooled variance
    inv_mass = np.where(np.isfinite(inv_mass) & (inv_mass > 0), inv_mass, 1e-12)
    for s in P:
        s.close()

    for key, prec, n in (("metropolis_fp32mixed", pimc.FP32_MIXED, n_metro[0]),
                         ("metropolis_fp64", pimc.FP64, n_metro[1])):
        S = [make(prec, k) for k in range(K)]
        for s, (X, p), (sx, sp) in zip(S, starts, steps):
            s.set_path(X)
            s.set_params(p, prob.lo, prob.hi, prob.free)
            s.set_steps(sx, sp)
            s.set_schedule(n_init=10 ** 9, n_skip=10 ** 6)  # no statistics records, no adaptation
            s.set_param_trace(n)
        b = pimc.Batch(S)
        chunk = max(n // 4, 1)
        b.sweep(chunk, seed + 1)  # warm-up: captures the chunk's graph
        secs = sum(timed(lambda: b.sweep(chunk, seed + 1, sync=False)) for _ in range(4))
        b.close()
        tr = np.array([s.param_trace() for s in S])[:, :, free]
        out[key] = {"sweeps": 4 * chunk, **_ess_block(tr, secs, names)}
        for s in S:
            s.close()

    # HMC: each chain's trajectory is one CUDA graph on its handle's stream;
    # the K_hmc chains run concurrently, one stream each (the timed region
    # spans all of them), after their steps are tuned one chain at a time
    for key, prec, n in (("hmc_fp32mixed", pimc.FP32_MIXED, n_hmc[0]), ("hmc_fp64", pimc.FP64, n_hmc[1])):
        chains, eps_l = [], []
        streams = [torch.cuda.Stream() for _ in range(K_hmc)]
        for k in range(K_hmc):
            s = make(prec, 10000 + k)
            s.set_stream(streams[k].cuda_stream)  # before the graph capture (a new stream re-captures)
            X, p = starts[k]
            s.set_path(X)
            s.set_params(p, prob.lo, prob.hi, prob.free)
            s.set_schedule(n_init=10 ** 9, n_skip=1)
            eps = 0.05
            for _ in range(10):
                a = s.hmc(10, n_leap, eps, inv_mass, seed=seed + 2) / 10.0
                eps *= float(np.exp(1.5 * (a - 0.7)))
            s.set_param_trace(n)
            s.hmc(0, n_leap, eps, inv_mass, seed=seed + 3)  # captures the trajectory graph
            chains.append(s)
            eps_l.append(eps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for ss in streams:
            ss.wait_event(e0)
        # one host thread a chain enqueues its graph launches (the launch
        # loop runs in the library with the interpreter lock released)
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(len(chains), os.cpu_count() or 1)) as pool:
            list(pool.map(lambda ce: ce[0].hmc(n, n_leap, ce[1], inv_mass, seed=seed + 3, wait=False),
                          zip(chains, eps_l)))
        for ss in streams:
            ev = torch.cuda.Event()
            ev.record(ss)
            st.wait_event(ev)
        e1.record(st)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) * 1e-3
        trs, acc = [], []
        for s in chains:
            s.sync()
            tr = s.param_trace()
            trs.append(tr[:, free])
            # a rejected trajectory leaves p unchanged, bit for bit
            acc.append(float(np.mean(np.any(np.diff(tr, axis=0) != 0.0, axis=1))))
            s.close()
        out[key] = {"trajectories": n, "n_leap": n_leap, "eps_median": float(np.median(eps_l)),
                    "accept": float(np.mean(acc)), "concurrent_streams": len(chains),
                    **_ess_block(np.array(trs), secs, names)}

    # equal posterior accuracy: each sampler's means against plain FP64
    # Metropolis, in pooled Monte Carlo standard errors
    ref = out["metropolis_fp64"]["params"]
    for key in ("metropolis_fp32mixed", "hmc_fp32mixed", "hmc_fp64"):
        out[key]["mean_shift_vs_fp64_metropolis_in_se"] = {
            nm: abs(v["mean"] - ref[nm]["mean"]) / np.hypot(v["mc_se"], ref[nm]["mc_se"])
            for nm, v in out[key]["params"].items()}
    base = out["metropolis_fp64"]["min_ess_per_s"]
    for key in ("metropolis_fp32mixed", "hmc_fp32mixed", "hmc_fp64", "metropolis_fp64"):
        out[key]["min_ess_per_s_vs_fp64_metropolis"] = out[key]["min_ess_per_s"] / base if base > 0 else None
    return out


def ess_default():
    """The bounded ESS study of the default line (about half a minute): the
    linear-Gaussian posterior at M = 200, and the HH problem at M = 2048 with
    all 7 parameters free."""
    from paper_1103_4887_gb300 import synth
    lg = synth.lingauss_problem(200, data_seed=3, dt=0.5, Rm=4.0, Rf=(2.0, 2.0))
    hh = synth.hh_problem(2048, data_seed=0, free="all")
    return {"lingauss_M200": ess_study(lg, K=64, K_hmc=32, pilot=(20000, 20000), n_metro=(40000, 32000),
                                       n_hmc=(2000, 1000), n_leap=16, names=["b"]),
            "hh_M2048_7free": ess_study(hh, K=64, K_hmc=16, pilot=(5000, 5000), n_metro=(20000, 2000),
                                        n_hmc=(1000, 150), names=list(synth.HH_NAMES))}


def run_ess(args):
    """ESS study on the two posteriors: the linear-Gaussian test model (a
    posterior every sampler mixes, at two path lengths) and the HH problem
    with all 7 parameters free (M = 16384: the chains' R-hat shows whether they
    agree within the run)."""
    from paper_1103_4887_gb300 import synth
    res = {}
    for M in (200, 2000):
        prob = synth.lingauss_problem(M, data_seed=3, dt=0.5, Rm=4.0, Rf=(2.0, 2.0))
        res[f"lingauss_M{M}"] = ess_study(prob, K=64, K_hmc=32, pilot=(20000, 20000), n_metro=(40000, 32000),
                                          n_hmc=(2000, 1000), n_leap=16, names=["b"])
        print(json.dumps({f"lingauss_M{M}": res[f"lingauss_M{M}"]}), flush=True)
    prob = synth.hh_problem(16384, data_seed=0, free="all")
    res["hh_M16384_7free"] = ess_study(prob, K=64, K_hmc=16, pilot=(20000, 20000), n_metro=(40000, 2000),
                                       n_hmc=(1000, 150), names=list(synth.HH_NAMES))
    print(json.dumps({"hh_M16384_7free": res["hh_M16384_7free"]}), flush=True)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32mixed", choices=["fp32mixed", "fp64"])
    ap.add_argument("--M", type=int, default=M_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the batched and ESS measurements")
    ap.add_argument("--fp64-steps", type=int, default=40)
    ap.add_argument("--profile", action="store_true",
                    help="no timing: 3 launches of one bench step per precision (a small case for ncu)")
    ap.add_argument("--profile-hmc", action="store_true",
                    help="no timing: 3 HMC trajectories per precision on the ESS workload (a small case for ncu)")
    ap.add_argument("--map-ceiling", action="store_true",
                    help="maps/s of the FP32 HH map alone from registers (single and packed lanes, 1 and 2 CTAs/SM)")
    ap.add_argument("--sweep-M", action="store_true",
                    help="observation-length sweep M = 2^10..2^20: site-updates/s and roofline per M, FP32-mixed "
                         "and FP64, with the serial oracle timed on the host for the same M")
    ap.add_argument("--batch", action="store_true",
                    help="batched launch: 64 data sets (M ~ U[2048, 65536]) x 8 chains, FP32-mixed, autotuned")
    ap.add_argument("--paper", action="store_true",
                    help="the paper's own setting: HH variant with tanh kinetics, trapezoid rule, uniform "
                         "proposals, M = 8000 at 25 kHz, all 7 parameters free")
    ap.add_argument("--mixed", action="store_true",
                    help="FP32-mixed vs FP64 on the bench workload: Delta A error, accept-flip rate, "
                         "posterior-mean shift in MC standard errors")
    ap.add_argument("--ess", action="store_true",
                    help="parameter ESS/s of FP32-mixed and FP64 Metropolis and whole-path HMC from independent "
                         "chains: linear-Gaussian posterior at M = 200 and 2000, HH with 7 free parameters at "
                         "M = 16384")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile:
        run_profile_case(args)
        return
    if args.map_ceiling:
        print(json.dumps(map_ceiling()), flush=True)
        return
    if args.profile_hmc:
        run_profile_hmc(args)
        return
    if args.sweep_M:
        run_sweep_M(args)
        return
    if args.ess:
        run_ess(args)
        return
    if args.mixed:
        print(json.dumps(run_mixed(args)), flush=True)
        return
    if args.batch:
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.paper:
        print(json.dumps(run_paper(args)), flush=True)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1103_4887_gb300 import pimc, synth
    prec = pimc.FP32_MIXED if args.precision == "fp32mixed" else pimc.FP64
    prob = synth.hh_problem(args.M, data_seed=rank, free="all")
    n_free = int(prob.free.sum())
    stream = torch.cuda.current_stream()

    def make(precision):
        s = pimc.Sampler.from_problem(prob, precision=precision)
        s.set_stream(stream.cuda_stream)
        s.set_chain(rank)
        s.set_schedule(n_init=args.warmup * NSKIP, n_skip=NSKIP, f_acc=0.4, alpha=0.5)
        return s

    samp = make(prec)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed_steps(s, K, warm):
        for _ in range(warm):
            s.sweep(NSKIP, SEED, sync=False)
        torch.cuda.synchronize()
        s.sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            s.sweep(NSKIP, SEED, sync=False)
            e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        s.sync()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    # clocks during the timed region
    with ClockSampler(local) as clk:
        ms = timed_steps(samp, args.steps, args.warmup)
    total_ms = sum(ms)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    sites = prob.M + 1
    value = world * sites * NSKIP * args.steps / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps

    # steady state: one persistent launch of many sweeps, no flush in between
    n_ss = 2000 if prec == pimc.FP32_MIXED else 100
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    samp.sweep(n_ss, SEED, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    samp.sync()
    ss_ms = e0.elapsed_time(e1)
    steady = {"sweeps_per_launch": n_ss, "ms_per_sweep": ss_ms / n_ss,
              "site_updates_per_s": world * sites * n_ss / (ss_ms * 1e-3)}

    # e2e through the public API with host buffers: per step the data arrays
    # go host->device from pinned memory (pimc_load_data), the step's sweeps
    # run, and the parameter vector comes back into pinned host memory
    # (pimc_params_async: a copy on the stream, no host stall per step); the
    # clock stops when the last step's parameters have arrived
    y_pin = torch.from_numpy(prob.y.copy()).pin_memory()
    I_pin = torch.from_numpy(prob.I.copy()).pin_memory()
    p_pin = torch.zeros((args.steps, samp.Np), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        samp.load_data(y_pin.data_ptr(), I_pin.data_ptr())
        samp.sweep(NSKIP, SEED, sync=False)
        samp.params_async(p_pin[k].data_ptr())
    samp.sync()
    e2e_s = time.perf_counter() - t0
    assert np.all(np.isfinite(p_pin.numpy())) and np.array_equal(p_pin[-1].numpy(), samp.params())
    e2e = {"value": world * sites * NSKIP * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 8 * (2 * prob.M + 1), "d2h_bytes_per_step": 8 * 7}

    # FP64 form on the same workload (for the FP32-mixed vs FP64 comparison)
    fp64 = None
    if prec == pimc.FP32_MIXED and args.fp64_steps > 0:
        s64 = make(pimc.FP64)
        ms64 = timed_steps(s64, args.fp64_steps, 3)
        fp64 = {"value": world * sites * NSKIP * args.fp64_steps / (sum(ms64) * 1e-3),
                "ms_per_step": sum(ms64) / len(ms64)}
        s64.close()

    grid_block = list(samp.launch_info())
    form = samp.sweep_form()
    peaks, peak_src = load_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    maps = maps_per_sweep(args.M, n_free)
    if prec == pimc.FP32_MIXED:
        # compute roofline of the map's instruction mix: FP32 lanes 128/clk/SM,
        # SFU 16/clk/SM at the maximum SM clock
        t_map = max(FP32_OPS_PER_MAP / (n_sm * 128 * sm_mhz * 1e6), MUFU_OPS_PER_MAP / (n_sm * 16 * sm_mhz * 1e6))
        peak_tflops = FLOP_PER_MAP / t_map / 1e12
    else:
        peak_tflops = 1.25  # nominal FP64 rate of the part
    achieved = maps * NSKIP * FLOP_PER_MAP / (ms_per_step * 1e-3) / 1e12
    kname = "sweep_resident_kernel<HH>" if form == "resident" else "sweep_kernel<HH>"
    # DRAM bytes (read + write) of one bench-step launch of this kernel, from
    # an ncu capture of it on this workload (None once the kernel changed)
    traffic = traffic_of(form, args.M, NSKIP) if prec == pimc.FP32_MIXED else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": traffic,
            "kernel": kname, "peak_source": f"derived from unit counts at {sm_mhz:.0f} MHz ({peak_src} clocks)",
            "kernel_src_hash": kernel_source_hash()}
    if prec == pimc.FP32_MIXED:
        roof.update({k: v for k, v in roofline_fracs(maps * NSKIP, ms_per_step * 1e-3, n_sm, sm_mhz).items()
                     if k.startswith("frac_")})
    if traffic is not None:  # the memory side of the same launch, against the copy peak
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        roof["dram_gbs"] = traffic / (ms_per_step * 1e-3) / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / hbm
        roof["dram_peak_gbs"] = hbm

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob)
    extras = {}
    if rank == 0 and world == 1 and not args.quick:
        samp.close()
        try:
            extras["map_ceiling"] = map_ceiling()
        except Exception as e:  # reported, not hidden
            extras["map_ceiling"] = {"error": repr(e)}
        try:
            extras["sweep_M"] = sweep_M_rows(ceiling=extras["map_ceiling"])
        except Exception as e:
            extras["sweep_M"] = {"error": repr(e)}
        try:
            extras["batch"] = run_batch(args)
        except Exception as e:  # reported, not hidden
            extras["batch"] = {"error": repr(e)}
        try:
            extras["mixed"] = run_mixed(args)
        except Exception as e:
            extras["mixed"] = {"error": repr(e)}
        try:
            extras["ess"] = ess_default()
        except Exception as e:
            extras["ess"] = {"error": repr(e)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if prec == pimc.FP32_MIXED else "f64", "data": "synthetic",
                "config": workload_config(args.M),
                "run": {"precision": args.precision, "l2": "flushed (256 MiB write) before every timed step",
                        "grid_block": grid_block, "form": form},
                # per step: the sweep kernel, and for the resident form the
                # parameter-draws kernel before it
                "gpu_launches": args.steps * (2 if form == "resident" else 1),
                "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "clocks": summarize_clocks(clk.rows),
                "steady_state": steady, "fp64": fp64,
                "rk4_maps_per_s": world * maps * NSKIP / (ms_per_step * 1e-3),
                "param_moves_per_s": world * n_free * NSKIP / (ms_per_step * 1e-3)}
        line.update(extras)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
