"""The benchmark's reference arm (the oracle on the host cores) prints one JSON
line with the keys the measurement contract asks for, the same workload
config as the GPU arm, and a finite positive rate (CPU only)."""
import argparse
import contextlib
import io
import json

import bench


def test_reference_arm_line():
    args = argparse.Namespace(gpus=1, steps=1, warmup=1, impl="reference")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"] == bench.arm_config(1)
    assert line["value"] > 0.0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
