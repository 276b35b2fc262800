"""Race and bounds check of the checkerboard (Sec. 4.1: sites of one parity
move together; Sec. 4.3: one thread a site) on the checked build.

libpimc_check.so is the same library with the sweep kernels compiled with
PIMC_CHECK: every site visit of a site phase and every cache write of a
parameter move is counted per site, and a site index outside [0, M] sets a
status bit and skips the access (nothing traps).  On the benchmark workload
(HH, M = 32768, all 7 parameters free, 152 CTAs) in both sweep forms, and
on a batched launch, each site must be visited exactly once per phase of its
parity and never in the other, and written exactly once per executed
parameter move.  Each case runs in a child process that loads the checked
library.
"""
import json
import os
import subprocess
import sys

import pytest

from paper_1103_4887_gb300 import build as pbuild

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
from paper_1103_4887_gb300 import pimc, synth
pimc.load(sys.argv[1])
case = sys.argv[2]
out = {}

def check(s, n_sweeps):
    ev, od, pa, moves, status = s.check_counts()
    M = s.M
    n = np.arange(M + 1)
    return {"even_ok": bool(np.all(ev[n % 2 == 0] == n_sweeps) and np.all(ev[n % 2 == 1] == 0)),
            "odd_ok": bool(np.all(od[n % 2 == 1] == n_sweeps) and np.all(od[n % 2 == 0] == 0)),
            "param_ok": bool(np.all(pa[:M] == moves) and pa[M] == 0), "moves": moves,
            "bounds_bit": bool(status & 2), "even_max": int(ev.max()), "odd_max": int(od.max()),
            "param_max": int(pa.max()), "param_min": int(pa[:M].min())}

if case in ("resident", "general", "fp64"):
    prob = synth.hh_problem(32768, data_seed=0, free="all")
    prec = pimc.FP64 if case == "fp64" else pimc.FP32_MIXED
    s = pimc.Sampler.from_problem(prob, precision=prec)
    s.set_sweep_form("general" if case == "general" else "auto")
    s.set_schedule(n_init=0, n_skip=10)
    s.check_counts()  # reset
    s.sweep(10, 3)
    s.sweep(10, 3)
    out = check(s, 20)
    out["form"] = s.sweep_form()
    out["grid"] = s.launch_info()[0]
else:
    chains = []
    for k, M in enumerate((37, 800, 2500, 64)):
        prob = synth.hh_problem(M, data_seed=50 + k, free="all")
        s = pimc.Sampler.from_problem(prob, precision=pimc.FP32_MIXED)
        s.set_chain(k)
        s.check_counts()
        chains.append(s)
    b = pimc.Batch(chains)
    b.sweep(15, 4)
    res = [check(s, 15) for s in chains]
    out = {k: all(r[k] for r in res) for k in ("even_ok", "odd_ok", "param_ok")}
    out["bounds_bit"] = any(r["bounds_bit"] for r in res)
    out["moves"] = min(r["moves"] for r in res)
    b.close()  # the batch goes before its handles
    for s in chains:
        s.close()
print("RESULT " + json.dumps(out), flush=True)
"""


@pytest.mark.parametrize("case", ["resident", "general", "fp64", "batch"])
def test_every_site_written_once_per_phase(case):
    pbuild.build()
    lib = pbuild.LIB_CHECK
    assert os.path.exists(lib)
    r = subprocess.run([sys.executable, "-c", CHILD, lib, case], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    if case in ("resident", "general", "fp64"):
        assert res["form"] == ("resident" if case == "resident" else "general")
        assert res["grid"] >= 147
    assert res["even_ok"] and res["odd_ok"] and res["param_ok"], res
    assert not res["bounds_bit"], res
    assert res["moves"] > 0, res


def test_unchecked_build_refuses_the_counts():
    from paper_1103_4887_gb300 import pimc, synth
    s = pimc.Sampler.from_problem(synth.hh_problem(50, data_seed=0))
    with pytest.raises(pimc.PimcError) as e:
        s.check_counts()
    assert e.value.code == pimc.ERR_STATE
