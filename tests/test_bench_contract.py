"""The benchmark's JSON line, on CPU.

The reference arm (the oracle on the host cores) runs here without a GPU: it
must print exactly one JSON line with the contract's keys, describe the same
workload, in the same ``config`` dict, as the GPU arm of the default command,
and time the oracle only (no host-device copies).
"""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", *extra],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line_has_the_contract_keys():
    line = _reference_line()
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["metric"] == line["unit"] == "aligned pairs/s"
    assert line["higher_is_better"] is True
    assert (line["steps"], line["warmup"], line["n_gpus"]) == (2, 1, 1)
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_config_equals_the_gpu_arms():
    """The GPU arm builds its config with bench.workload_config from the whole
    default workload (no sample, no read ranges); the reference arm must print
    the identical dict, although it times a bounded sample of that workload."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads

    old = sys.argv
    sys.argv = ["bench.py"]
    try:
        args = bench.parse()
    finally:
        sys.argv = old
    assert args.workload == bench.WORKLOAD and tuple(args.xdrops) == tuple(bench.XDROPS)
    w = workloads.generate(args.workload)
    gpu_cfg = bench.workload_config(w, len(workloads.pair_groups(w.pairs)) - 1, len(w.pairs), args.xdrops)
    assert _reference_line()["config"] == gpu_cfg
    assert gpu_cfg["workload"] == "c2_ecoli" and gpu_cfg["xdrop"] == [7, 25]


@pytest.mark.parametrize("world", [2])
def test_reference_arm_prints_on_rank_zero_only(world):
    """Under torchrun only rank 0 runs the oracle and prints; the other ranks
    exit 0 without work."""
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 0

    import contextlib
    import io
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A(), world, 1)
    assert buf.getvalue() == ""
