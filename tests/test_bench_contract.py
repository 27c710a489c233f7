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


def test_clock_summary_keeps_the_samples_of_the_timed_region():
    """nvidia-smi lines (timestamp first) outside [mark_start, mark_end] are
    dropped; the throttle reasons are those seen inside; without samples in
    the region every sample counts."""
    import datetime

    def line(t, sm, thermal="Not Active", cap="Not Active"):
        ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {sm}, 2070, 900.0, 0x0, Not Active, {thermal}, Not Active, {cap}"

    t0 = 1_800_000_000.0
    c = bench.ClockSampler(0)
    c.out = "\n".join([line(t0 - 0.2, 1100, thermal="Active"), line(t0 + 0.05, 2070),
                       line(t0 + 0.10, 2040, cap="Active"), line(t0 + 0.15, 2070),
                       line(t0 + 0.5, 900)])
    c.t_start, c.t_end = t0, t0 + 0.2
    s = c.summary()
    assert s["samples"] == 5 and s["samples_in_timed_region"] == 3
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    c.t_start, c.t_end = t0 + 1.0, t0 + 1.01          # no sample inside: all count
    s = c.summary()
    assert s["samples_in_timed_region"] == 0 and s["sm_mhz"] == 2040
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_issue_roof_arithmetic():
    """The alu object of the bench line: ncu's warp instructions per launch of
    the fused FP64 element kernel over its CUDA-event time, against 152 SMs x
    4 schedulers x 2.07 GHz (a GB300 run: 0.35244 ms -> 0.680 of the roof)."""
    tiles = {"f64_stages": 1}
    assert bench.ax_kernel_name(tiles) == "ax_df_kernel<8, 1, 1>"
    assert bench.ax_traffic(tiles) == 1_064_131_328
    roof = bench.alu_roof(tiles, 0.3524431988596916)
    assert roof["peak"] == 152 * 4 * 2.07e9
    assert abs(roof["frac"] - 301_503_392 / 0.3524431988596916e-3 / roof["peak"]) < 1e-12
    assert abs(roof["frac"] - 0.6797) < 1e-3
    # a kernel variant no ncu capture covers reports no traffic and no roof
    assert bench.ax_traffic({"f64_stages": 2}) is None
    assert bench.alu_roof({"f64_stages": 2}, 0.3) is None
