"""The two forms of the FP32-mixed sweep agree bit for bit.

The resident form (one site a thread for the whole launch, flags between
neighbouring CTAs, speculative parameter maps) and the general form (threads
striding over the tile, grid barriers) evaluate the same per-site terms and
sum the parameter-move partials exactly, so on the same tiles every state,
parameter, statistic and counter is identical.  The FP32 HH map runs one site
alone or two as the lanes of a packed map (general form: sites n, n + 1;
resident form: a site's two speculative outcomes); the cached values that
the residual statistics read expose any bit of difference between the two."""
import numpy as np
import pytest

from paper_1103_4887_gb300 import pimc, synth

pytestmark = pytest.mark.gpu


def _run(prob, form, n_sweeps, grid=0, seed=21):
    s = pimc.Sampler.from_problem(prob, precision=pimc.FP32_MIXED)
    if grid:
        s.set_grid(grid)
    s.set_sweep_form(form)
    s.set_schedule(n_init=12, n_skip=3, beta0=0.2, n_cool=10, f_acc=0.4, alpha=0.3)
    s.sweep(n_sweeps // 2, seed)
    s.sweep(n_sweeps - n_sweeps // 2, seed)  # a second launch continues the flags' epochs
    return s


def _same(a, b):
    Xa, pa = a.state()
    Xb, pb = b.state()
    assert np.array_equal(Xa, Xb) and np.array_equal(pa, pb)
    ma, va, Ja = a.moments()
    mb, vb, Jb = b.moments()
    assert Ja == Jb and np.array_equal(ma, mb) and np.array_equal(va, vb, equal_nan=True)
    for x, y in zip(a.accept_stats(), b.accept_stats()):
        assert np.array_equal(x, y)
    for x, y in zip(a.residual_moments(), b.residual_moments()):
        assert np.array_equal(np.asarray(x), np.asarray(y), equal_nan=True)
    for x, y in zip(a.steps(), b.steps()):
        assert np.array_equal(x, y)
    assert a.sweep_counter() == b.sweep_counter()


@pytest.mark.parametrize("case", ["hh_M1000", "hh_M1000_one_free", "hh_M237_grid3", "hh_M150_grid1", "hh_M1_grid1",
                                  "paper_M400", "hh_trap_M600", "lg_M300", "toy_M90"])
def test_resident_and_general_forms_agree_bitwise(case):
    grid = 0
    if case == "hh_M1000":
        prob = synth.hh_problem(1000, data_seed=3, free="all")
    elif case == "hh_M1000_one_free":
        # one parameter: the resident form evaluates every move's map one site
        # at a time, the general form two sites a thread on the packed map
        prob = synth.hh_problem(1000, data_seed=3, free=("gNa",))
    elif case == "hh_M237_grid3":
        prob, grid = synth.hh_problem(237, data_seed=5, free="all"), 3
    elif case == "hh_M150_grid1":
        prob, grid = synth.hh_problem(150, data_seed=6, free=("gNa", "EK")), 1
    elif case == "hh_M1_grid1":
        prob, grid = synth.hh_problem(1, data_seed=7, free="all"), 1
    elif case == "paper_M400":
        prob = synth.paper_problem(400, data_seed=8, free="all")
    elif case == "hh_trap_M600":
        prob = synth.hh_problem(600, data_seed=9, free="all")
        prob.scheme = 1
        prob.proposal = 1
    elif case == "lg_M300":
        prob = synth.lingauss_problem(300, 1)
    else:
        prob = synth.toy_problem(90, 2, p_free=True)
    a = _run(prob, "auto", 40, grid)
    b = _run(prob, "general", 40, grid)
    assert a.sweep_form() == "resident"
    assert b.sweep_form() == "general"
    assert a.launch_info() == b.launch_info()
    _same(a, b)


def test_form_selection():
    s = pimc.Sampler.from_problem(synth.hh_problem(32768, data_seed=0, free="all"), precision=pimc.FP32_MIXED)
    assert s.sweep_form() == "resident"
    grid, _ = s.launch_info()
    assert grid >= 147  # at most 224 sites a CTA
    s.set_precision(pimc.FP64)
    assert s.sweep_form() == "general"
    s2 = pimc.Sampler.from_problem(synth.hh_problem(1 << 17, data_seed=0, free="all"), precision=pimc.FP32_MIXED)
    assert s2.sweep_form() == "general"
    with pytest.raises(pimc.PimcError):
        s2.set_sweep_form("fastest")
