"""The bench's JSON line on a GPU: every key of the contract, with the
types and relations it promises (a small case of the default workload)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_the_contract_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--n", "64", "--steps", "3", "--warmup", "3",
                        "--no-cpu-baseline", "--no-perf-model", "--no-variants"],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["gpu_launches"] > 0
    assert "workload" in line["config"]
    roof = line["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in roof, key
    assert roof["bound"] in ("alu", "hbm", "tensor") and 0 < roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    e2e = line["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    clk = line["clocks"]
    assert clk["sm_mhz"] > 0 and clk["sm_max_mhz"] > 0 and isinstance(clk["reasons"], list)
    # one mean launch time per Runge-Kutta stage, averaging to the per-launch mean
    by_stage = roof["kernel_ms_by_stage"]
    assert len(by_stage) == 3 and all(t > 0 for t in by_stage)
    assert sum(by_stage) / 3 == pytest.approx(roof["kernel_ms_per_launch"], rel=1e-6)


def test_profile_launches_lists_each_stencil_launch():
    import torch
    from paper_2305_18057_gb300 import sensei, workloads as wl
    w = wl.periodic_3d(n=32)
    g = sensei.Grid(w.dims, w.nodes, limiter=sensei.LIM_VANLEER, precision=sensei.FP32_STORE)
    for f in range(6):
        g.set_bc(0, f, sensei.BC_PERIODIC)
    U = [g.new_state(0)]
    g.upload(U[0], 0, w.U0[0])
    g.profile(True)
    g.profile_read(reset=True)
    for _ in range(2):
        g.rk_step(U, sensei.RK3_SSP, cfl=0.5)
    torch.cuda.synchronize()
    per = g.profile_launches()
    ms, n, _ = g.profile_read(reset=True)
    g.profile(False)
    assert n == 6 and len(per) == 6 and all(t > 0 for t in per)
    assert sum(per) == pytest.approx(ms, rel=1e-6)
    assert g.profile_launches() == []
