"""The reference arm of bench.py (the FP64 oracle on the host cores) prints
one JSON line with the keys the benchmark contract names, on the same
workload configuration as the GPU arm; under several ranks only rank 0
prints.  CPU only: a bounded sample of the default scene."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                          "--cpu-budget", "0.5", "--cpu-threads", "2", *args],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_line_has_the_contract_keys():
    lines = _run()
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the GPU arm's workload object, built by the same function
    import bench
    args = type("A", (), {"scene": bench.DEFAULT_SCENE, "seed": None, "h_max": None})()
    sc = bench.scene_for_rank(args, 0)
    want = bench.workload_config(args, sc, bench.filter_cfg(sc))
    assert d["config"] == want
    assert want["scene"] == "sweep_N200" and want["h_max"] == 20000 and want["timed_frames"] == [10, 49]


def test_reference_arm_prints_only_on_rank_0():
    assert _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}) == []


def test_clock_summary_reads_reasons_for_its_own_gpu():
    """The clock record beside every number: median SM clock under load,
    the maximum, and any throttle reason seen while the timed steps ran."""
    import bench
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2010, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "1, 900, 2070, 300.0, 0x40, Active, Not Active, Active, Not Active",
             "garbage line"]
    c = bench.summarize_clocks(lines, 0)
    assert c == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c1 = bench.summarize_clocks(lines, 1)
    assert c1["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and c1["sm_mhz"] == 900.0
    assert bench.summarize_clocks([], 0)["reasons"] == ["unavailable"]
