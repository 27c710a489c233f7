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
    c.t_start, c.t_end = t0 + 0.3, t0 + 0.31          # no sample inside: the adjacent ones
    s = c.summary()
    assert s["samples_in_timed_region"] == 0 and s["window"] == "adjacent"
    assert s["samples_used"] == 2 and s["sm_mhz"] == (2070 + 900) / 2
    assert s["reasons"] == []
    c.t_start, c.t_end = t0 + 1.0, t0 + 1.01          # only samples before it
    s = c.summary()
    assert s["window"] == "adjacent" and s["samples_used"] == 1 and s["sm_mhz"] == 900
    c.t_start = c.t_end = None                        # no region marked: every sample
    s = c.summary()
    assert s["window"] == "all" and s["samples_used"] == 5
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_issue_roof_arithmetic():
    """The alu object of the bench line: ncu's warp instructions per launch of
    the fused FP64 element kernel over its CUDA-event time, against 152 SMs x
    4 schedulers x 2.07 GHz (a GB300 run: 0.35244 ms -> 0.680 of the roof)."""
    tiles = {"f64_stages": 1}
    assert bench.ax_kernel_name(tiles) == "ax_df_kernel<8, 1, 1>"
    caps = {"ax_df_kernel<8, 1, 1>": {"source": "abc", "dram_bytes": 1_064_131_328,
                                      "warp_instructions": 301_503_392}}
    assert bench.ax_traffic(tiles, captures=caps, digest="abc") == 1_064_131_328
    roof = bench.alu_roof(tiles, 0.3524431988596916, captures=caps, digest="abc")
    assert roof["peak"] == 152 * 4 * 2.07e9
    assert abs(roof["frac"] - 301_503_392 / 0.3524431988596916e-3 / roof["peak"]) < 1e-12
    assert abs(roof["frac"] - 0.6797) < 1e-3
    # a kernel variant no ncu capture covers reports no traffic and no roof
    assert bench.ax_traffic({"f64_stages": 2}, captures=caps, digest="abc") is None
    assert bench.alu_roof({"f64_stages": 2}, 0.3, captures=caps, digest="abc") is None
    # nor does a capture of an older source of the kernel
    assert bench.ax_traffic(tiles, captures=caps, digest="abd") is None
    assert bench.alu_roof(tiles, 0.3, captures=caps, digest="abd") is None


def test_recorded_captures_match_the_current_kernel_source():
    """Every ncu figure the bench reports is tied to a digest of the kernel's
    sources; the digest is reproducible, and a stale entry reads as null."""
    d = bench.ax_source_digest()
    assert len(d) == 16 and d == bench.ax_source_digest()
    for name, cap in bench.AX_CAPTURES.items():
        assert set(cap) == {"source", "dram_bytes", "warp_instructions"}, name


def test_capture_figures_match_the_committed_profile():
    """The ncu figures the bench reports for the FP64 element kernel are the
    ones its committed profile summary states: the same source digest, warp
    instructions and DRAM bytes per launch."""
    import os
    import re
    cap = bench.AX_CAPTURES["ax_df_kernel<8, 1, 1>"]
    path = os.path.join(bench.ROOT, "profiles", "ax_df_kernel_fused_f64_e32768_n7.md")
    with open(path) as fh:
        text = fh.read()
    assert "Source digest of the captured kernel (bench.ax_source_digest): %s." % cap["source"] in text
    warp = re.search(r"\| smsp__inst_executed\.sum \| ([0-9.]+) M warp instructions", text)
    assert warp and abs(float(warp.group(1)) * 1e6 - cap["warp_instructions"]) < 0.05e6
    dram = re.search(r"\| dram__bytes_read\.sum \+ dram__bytes_write\.sum \| ([0-9.]+) \+ ([0-9.]+) = ", text)
    assert dram
    total_mb = float(dram.group(1)) + float(dram.group(2))
    assert abs(total_mb * 1e6 - cap["dram_bytes"]) < 0.1e6


def _counted_element_flops(N):
    """Adds and multiplies of one sum-factorised element operator, counted by
    running it on values that count the operations applied to them."""
    count = [0]

    class C:
        def __add__(self, o):
            count[0] += 1
            return C()

        def __mul__(self, o):
            count[0] += 1
            return C()

        __radd__ = __add__
        __rmul__ = __mul__

    P = N + 1
    D = [[C() for _ in range(P)] for _ in range(P)]
    u = {(i, j, k): C() for i in range(P) for j in range(P) for k in range(P)}

    def dsum(terms):
        acc = None
        for t in terms:
            acc = t if acc is None else acc + t
        return acc

    wr, ws, wt = {}, {}, {}
    for (i, j, k) in u:
        ur = dsum(D[i][l] * u[l, j, k] for l in range(P))
        us = dsum(D[j][l] * u[i, l, k] for l in range(P))
        ut = dsum(D[k][l] * u[i, j, l] for l in range(P))
        g = [C() for _ in range(6)]
        wr[i, j, k] = g[0] * ur + g[3] * us + g[4] * ut
        ws[i, j, k] = g[3] * ur + g[1] * us + g[5] * ut
        wt[i, j, k] = g[4] * ur + g[5] * us + g[2] * ut
    for (i, j, k) in u:
        _ = (dsum(D[l][i] * wr[l, j, k] for l in range(P))
             + dsum(D[l][j] * ws[i, l, k] for l in range(P))
             + dsum(D[l][k] * wt[i, j, l] for l in range(P)))
    return count[0] / P ** 3


def test_cost_model_bookkeeping():
    """Eq. 12 per local point as the model section uses it: W of the element
    operator equals the operations of a sum-factorised element counted one by
    one; Q is u, w and six G per point; the gather-scatter's share of points is
    the fraction of an interior element's points that other elements also hold
    (multiplicity > 1 on the oracle's mesh); Eq. 13 takes the larger time."""
    from oracle import mesh
    for N in (1, 2, 3):
        W_ax, Q_ax, W_gs, Q_gs = bench.model_costs(N, fp64=True)
        assert W_ax == _counted_element_flops(N)
    for N in (2, 5, 7):
        gid = mesh.global_ids(3, 3, 3, N)
        mult = mesh.multiplicity(gid)
        shared = float((mult[13] > 1).mean())            # the centre element of 27
        for fp64, wsz in ((True, 8), (False, 4)):
            W_ax, Q_ax, W_gs, Q_gs = bench.model_costs(N, fp64)
            assert Q_ax == 8 * wsz
            assert abs(Q_gs - 2 * wsz * shared) < 1e-12
            assert abs(W_gs - 0.5 * shared) < 1e-12
    ms, bound = bench.model_time_ms(100, 8, 1_000_000, 1e12, 1e12)
    assert bound == "flops" and abs(ms - 0.1) < 1e-12
    ms, bound = bench.model_time_ms(100, 64, 1_000_000, 1e14, 1e12)
    assert bound == "bytes" and abs(ms - 0.064) < 1e-12
