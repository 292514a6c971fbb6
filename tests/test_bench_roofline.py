"""The bench's roofline arithmetic on CPU: the derived vector peaks from the
unit counts, the formula flops of a step's stencil launches, and which peak
each precision form is quoted against."""
import math
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_derived_peaks_from_unit_counts():
    assert math.isclose(bench.fp64_peak_tflops(2070.0), 152 * 2 * 2 * 2.07e9 / 1e12)
    assert math.isclose(bench.fp32_peak_tflops(2070.0), 152 * 128 * 2 * 2.07e9 / 1e12)
    assert math.isclose(bench.fp32_peak_tflops() / bench.fp64_peak_tflops(), 64.0)


def test_step_flops_average_the_three_stages():
    cells = 1000
    per_stage = [bench.alg_flops_per_cell("vanleer", False, False, True),
                 bench.alg_flops_per_cell("vanleer", False, True, False),
                 bench.alg_flops_per_cell("vanleer", False, True, False)]
    assert per_stage[0] - per_stage[1] == 20 - 10   # norm partials vs U^n blending
    assert math.isclose(bench.step_flops_per_launch("vanleer", False, cells), cells * sum(per_stage) / 3)
    # 3D van Leer: 3 Roe fluxes of 155, 3 directions of face states of 45,
    # primitives 12, flux sums 25, update 17, +20 / +10
    assert math.isclose(bench.step_flops_per_launch("vanleer", False, 1), (674 + 664 + 664) / 3)


def test_pipe_roofline_peaks_per_form():
    flops, ms = 1.0e10, 10.0
    achieved = flops / (ms / 1e3) / 1e12
    r64 = bench.pipe_roofline("fp64", flops, ms)
    assert r64["bound"] == "alu" and r64["unit"] == "TFLOP/s"
    assert math.isclose(r64["achieved"], achieved)
    assert math.isclose(r64["frac"], achieved / bench.fp64_peak_tflops())
    for form in ("fp32_flux", "fp32_store"):
        r = bench.pipe_roofline(form, flops, ms)
        assert math.isclose(r["frac"], achieved / bench.fp32_peak_tflops())
    rdf = bench.pipe_roofline("df64", flops, ms)
    assert math.isclose(rdf["frac"], r64["frac"]) and "double-float" in rdf["peak_source"]
