"""Benchmark: SEM operator throughput and solve time on one GB300 (or N replicas).

A step is one application of the assembled operator w = mask o QQ^T A_L u
(Ax kernel + gather-scatter kernel) in FP64 on the 32x32x32-element
deformed box [0, 2 pi]^3 at N = 7 (16,777,216 local GLL points), u ~ U(-1,1)
seeded.  value = local points per second over all ranks (GDOF/s).  Extra
keys report the FP32 operator, the Poisson solve to 1e-8 on the 48^3-element
box (FP64 PCG against FP32-inner / FP64-refinement), the roofline of the Ax
kernel, the end-to-end rate through the host-buffer C-ABI call and the
oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-solve] [--no-batch] [--no-cpu] [--sections a,b,...]
                  [--pressure-nel NEL] [--tiles SPEC] [--model-sweep]
"""
import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402

WORKLOAD = si.THROUGHPUT          # 32^3 elements, N = 7, deformed [0, 2 pi]^3
SOLVE = si.SOLVE                  # 48^3 elements, N = 7, RHS of 8 Fourier modes, tol 1e-8
METRIC = "Ax+dssum GDOF/s (FP64, N=7, E=32^3 deformed); CG solve to 1e-8 mixed vs FP64"
UNIT = "GDOF/s"


def arm_config(world, n=32 ** 3 * 8 ** 3):
    """The workload of the operator line, shared by both arms."""
    return {"workload": "Ax+dssum (mask), 32x32x32 deformed hex elements on [0,2pi]^3, "
                        "N=7, u~U(-1,1) seed 42",
            "local_points": n, "l2": "inputs larger than L2 (u 134 MB, G 805 MB)",
            "parallelism": f"replicas x{world}"}


def max_over_ranks(values, device):
    """Each timing in `values` (ms) replaced by its maximum over the ranks of
    the default process group (unchanged without one): the slowest replica
    sets the whole-job rate.  `device` holds the reduction tensor (a CUDA
    device under NCCL, the CPU under gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(points_per_rank, steps, world, ms):
    """G points per second over all replicas: every rank processes
    points_per_rank per step, and the job ends with its slowest rank (ms)."""
    return world * points_per_rank * steps / (ms / 1e3) / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Source files the FP64 element kernel is built from.  An ncu capture below
# holds only for the kernel built from files with the recorded digest: after
# any change to them the bench reports null until the kernel is captured again.
AX_SOURCES = tuple(os.path.join("paper_2107_01243_gb300", "csrc", f) for f in (
    "ax_df.cu", "df.cuh", "df_tables.cuh", "ax_tile.cuh", "tma.cuh", "reduce.cuh",
    "cg_state.cuh"))


def ax_source_digest(root=ROOT):
    import hashlib
    d = hashlib.sha256()
    for f in AX_SOURCES:
        with open(os.path.join(root, f), "rb") as fh:
            d.update(fh.read())
    return d.hexdigest()[:16]


# Per launch of the FP64 Ax kernel on the 32^3, N=7 throughput mesh, from one
# ncu capture (summary and command under profiles/): DRAM bytes
# (dram__bytes_read.sum + dram__bytes_write.sum) and warp instructions
# (smsp__inst_executed.sum).  The double-float kernel is bound by instruction
# issue on the FP32 pipe, so its second roof is the issue rate, 152 SMs x 4
# schedulers x the maximum SM clock.
AX_CAPTURES = {
    "ax_df_kernel<8, 1, 1>": {
        "source": "337018094dbfaa39",
        "dram_bytes": 939_699_456 + 78_679_552,
        "warp_instructions": 249_740_848,       # profiles/ax_df_kernel_fused_f64_e32768_n7.md
    },
}
ISSUE_PEAK = 152 * 4 * 2.07e9         # warp instructions per second


def ax_kernel_name(tiles):
    """The FP64 element kernel of the operator step at N=7 (double-float
    arithmetic on the FP32 pipes, 1 or 2 shared-memory stages, fused output)."""
    return f"ax_df_kernel<8, {tiles['f64_stages']}, 1>"


def ax_capture(tiles, captures=None, digest=None):
    """The capture of this kernel variant, if one was taken of the current source."""
    c = (AX_CAPTURES if captures is None else captures).get(ax_kernel_name(tiles))
    if c is None:
        return None
    if c["source"] != (ax_source_digest() if digest is None else digest):
        return None
    return c


def ax_traffic(tiles, **kw):
    c = ax_capture(tiles, **kw)
    return None if c is None else c["dram_bytes"]


def alu_roof(tiles, ax_ms, **kw):
    """Issue roof of the FP64 Ax kernel: warp instructions per launch (ncu)
    over its CUDA-event duration, against the SMs' issue rate at max clock."""
    c = ax_capture(tiles, **kw)
    if c is None:
        return None
    instr = c["warp_instructions"]
    achieved = instr / (ax_ms / 1e3)
    return {"bound": "alu", "kernel": ax_kernel_name(tiles), "unit": "warp instr/s",
            "achieved": achieved, "peak": ISSUE_PEAK, "frac": achieved / ISSUE_PEAK,
            "warp_instructions_per_launch": instr}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 20 ms) around the timed region; the summary
    keeps the samples whose timestamps fall between mark_start() and
    mark_end() (host times taken after the synchronisations that bracket the
    region).  A region shorter than the sampling interval may hold none: the
    summary then uses the last sample before it and the first after it, and
    says so ("window": "adjacent" instead of "timed_region")."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t_start = self.t_end = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def mark_start(self):
        self.t_start = time.time()

    def mark_end(self):
        self.t_end = time.time()

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not getattr(self, "out", ""):
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []                              # (host time or None, sm, max, reasons)
        for line in self.out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm, smax = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, sm, smax, {n for n, v in zip(names, parts[6:10])
                                        if v.lower().startswith("active")}))
        if not rows:
            return None
        inside, window = [], "all"
        if self.t_start is not None and self.t_end is not None:
            timed = [r for r in rows if r[0] is not None]
            inside = [r for r in timed if self.t_start <= r[0] <= self.t_end]
            window = "timed_region"
            if not inside:
                before = [r for r in timed if r[0] < self.t_start]
                after = [r for r in timed if r[0] > self.t_end]
                inside = before[-1:] + after[:1]
                window = "adjacent"
        use = inside or rows
        if not inside:
            window = "all"
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": use[-1][2],
                "reasons": sorted(set().union(*(r[3] for r in use))), "samples": len(rows),
                "samples_in_timed_region": len(inside) if window == "timed_region" else 0,
                "window": window, "samples_used": len(use)}


# ---------------------------------------------------------------- oracle timing
def oracle_sample(nz):
    """Oracle data for a 32 x 32 x nz slab of the throughput mesh (same element
    size and deformation as the full mesh's first nz element layers)."""
    from tests.helpers import OracleProblem
    nel = (WORKLOAD["nel"][0], WORKLOAD["nel"][1], nz)
    L = list(WORKLOAD["length"])
    L[2] = L[2] * nz / WORKLOAD["nel"][2]
    o = OracleProblem(nel, WORKLOAD["N"], length=tuple(L), deform=WORKLOAD["deform"])
    u = si.uniform(o.shape, WORKLOAD["seed"])
    return o, u


def time_oracle(nz, min_seconds):
    o, u = oracle_sample(nz)
    runs, t0 = 0, time.perf_counter()
    while True:
        o.matvec(u)
        runs += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    n = u.size * runs
    return n / el / 1e9, dict(points=u.size, runs=runs, seconds=el, nel=o.nel)


def _oracle_worker(nz, min_seconds, barrier, queue):
    """One host core: the oracle operator on its own slab, timed once every
    worker has built its data (so that the timed loops overlap)."""
    o, u = oracle_sample(nz)
    o.matvec(u)
    barrier.wait()
    runs, t0 = 0, time.perf_counter()
    while True:
        o.matvec(u)
        runs += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    queue.put((u.size * runs / el / 1e9, u.size, runs, el))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def time_oracle_all_cores(nz, min_seconds):
    """The oracle on every host core at once: one spawned process per core
    (numpy single-threaded in each), each on a 32 x 32 x nz slab; the rate is
    the sum over the workers."""
    import multiprocessing as mp
    n = host_cores()
    keep = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                           "MKL_NUM_THREADS")}
    for v in keep:
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")      # never fork a process that holds a CUDA context
    barrier, queue = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(nz, min_seconds, barrier, queue))
             for _ in range(n)]
    try:
        for pr in procs:
            pr.start()
        res = [queue.get(timeout=900) for _ in procs]
    finally:
        for pr in procs:
            pr.join(timeout=60)
        for v, old in keep.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
    return sum(r[0] for r in res), dict(workers=n, points=res[0][1],
                                        runs=sum(r[2] for r in res),
                                        seconds=max(r[3] for r in res))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    o, u = oracle_sample(2)
    for _ in range(args.warmup):
        o.matvec(u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.matvec(u)
    el = time.perf_counter() - t0
    value = u.size * args.steps / el / 1e9
    sample = (f"oracle Ax+dssum on a 32x32x2 slab ({u.size} local points) of the "
              f"32^3-element N=7 mesh per step, numpy, 1 thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--model-sweep", action="store_true",
                    help="print the Eq. 12-13 cost model against measured kernel times for "
                         "N = 2..9 instead of the benchmark line")
    ap.add_argument("--sections",
                    default="model,solve,batch,manufactured,projection,pressure,adjoint",
                    help="comma list of the solver sections to run after the operator line "
                         "(--no-solve and --no-batch remove theirs)")
    ap.add_argument("--pressure-nel", type=int, default=48,
                    help="elements per direction of the pressure-solver section (48: the "
                         "solve mesh; smaller for profiling)")
    ap.add_argument("--tiles", default=None,
                    help="pin the Ax tiles instead of autotuning: "
                         "<bulk-copy|global-load>:<fp32 stages>:<fp32 elements per CTA>:<fp64 stages>")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    import paper_2107_01243_gb300 as sem

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    if args.model_sweep:
        if rank == 0:
            print(json.dumps(run_model_sweep(sem, torch, dev)))
        return 0

    cfg = WORKLOAD
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    if args.tiles:
        k32, st32, el32, st64 = args.tiles.split(":")
        sem.sem_set_tuning(h, ax32_kernel=k32, ax32_stages=int(st32),
                           ax32_elems_per_cta=int(el32), f64_stages=int(st64))
        tiles = dict(ax32_kernel=k32, ax32_stages=int(st32), ax32_elems_per_cta=int(el32),
                     f64_stages=int(st64), pinned=True)
    else:
        tiles = sem.sem_autotune(h)
    n = h.n_local
    u_host = torch.from_numpy(si.uniform(n, cfg["seed"])).pin_memory()
    u = u_host.to(dev)
    w = torch.empty_like(u)
    u32 = u.float()
    w32 = torch.empty_like(u32)

    def step64():
        sem.sem_apply(h, u, w)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def ev3():
        return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                 torch.cuda.Event(enable_timing=True)) for _ in range(K)]

    for _ in range(args.warmup):
        step64()
    barrier()
    K = args.steps
    # a step is the assembled operator, split into its element phase (Ax with
    # the x-face sums) and its finishing gather-scatter passes by events
    ev = ev3()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        clk.mark_start()
        t0.record(stream)
        for s in range(K):
            ev[s][0].record(stream)
            sem.sem_apply(h, u, w, phase=sem.SEM_APPLY_LOCAL)
            ev[s][1].record(stream)
            sem.sem_apply(h, u, w, phase=sem.SEM_APPLY_FINISH)
            ev[s][2].record(stream)
        t1.record(stream)
        barrier()
        clk.mark_end()
    ms = t0.elapsed_time(t1)
    ax_ms = statistics.mean(a.elapsed_time(b) for a, b, _ in ev)
    ds_ms = statistics.mean(b.elapsed_time(c) for _, b, c in ev)
    (ms,) = max_over_ranks([ms], dev)
    value = whole_job_rate(n, K, world, ms)

    def split_times(local, finish, warm=3, reps=None):
        for _ in range(warm):
            local()
            finish()
        torch.cuda.synchronize()
        e = ev3()[:reps or K]
        for s in range(len(e)):
            e[s][0].record(stream)
            local()
            e[s][1].record(stream)
            finish()
            e[s][2].record(stream)
        torch.cuda.synchronize()
        return (statistics.mean(a.elapsed_time(b) for a, b, _ in e),
                statistics.mean(b.elapsed_time(c) for _, b, c in e))

    # FP32 operator, and both precisions as element kernel + separate gather-scatter
    ax32, ds32 = split_times(lambda: sem.sem_apply(h, u32, w32, phase=sem.SEM_APPLY_LOCAL),
                             lambda: sem.sem_apply(h, u32, w32, phase=sem.SEM_APPLY_FINISH))
    sep64 = split_times(lambda: sem.sem_ax(h, u, w), lambda: sem.sem_dssum(h, w))
    sep32 = split_times(lambda: sem.sem_ax(h, u32, w32), lambda: sem.sem_dssum(h, w32))
    # the IEEE FP64 element kernel (DFMA on the FP64 pipe) on the same mesh
    sem.sem_set_f64_kernel(h, sem.SEM_F64_KERNEL_NATIVE)
    nat64 = split_times(lambda: sem.sem_ax(h, u, w), lambda: None, reps=min(K, 50))[0]
    sem.sem_set_f64_kernel(h, sem.SEM_F64_KERNEL_AUTO)
    # FP32 operator on global vectors (the inner-solve operator): clearing w_g,
    # then the element kernel that gathers u_g and assembles w_g by reductions
    ng = h.n_global
    ug32 = torch.empty(ng, dtype=torch.float32, device=dev)
    sem.sem_to_global(h, u32, ug32)
    wg32 = torch.empty_like(ug32)
    glob32 = sum(split_times(lambda: sem.sem_apply_global(h, ug32, wg32), lambda: None))
    glob_bytes = 24 * n + 8 * ng            # G 6 x 4 per local point, u_g and w_g 4 + 4 per global

    # end to end through the host-buffer call
    w_host = torch.empty_like(u_host).pin_memory()
    for _ in range(3):
        sem.sem_apply_host(h, u_host, w_host)
    Ke = max(5, min(K, 50))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    a.record(stream)
    for _ in range(Ke):
        sem.sem_apply_host(h, u_host, w_host)
    b.record(stream)
    barrier()
    (e2e_ms,) = max_over_ranks([a.elapsed_time(b)], dev)
    e2e = whole_job_rate(n, Ke, world, e2e_ms)

    hbm, peak_kind = peaks()
    ax_bytes = 64 * n                       # u 8 + w 8 + 6 G x 8 per point
    achieved = ax_bytes / (ax_ms / 1e3) / 1e9
    nb_shared = 0.578125 * n                # boundary fraction at N = 7: 1 - (6/8)^3
    ds_bytes = (8 + 8 + 4) * nb_shared
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "arithmetic": ("FP64 inputs, outputs and gather-scatter; the element kernel "
                       "evaluates in double-float (pairs of FP32, 48-bit significand) with "
                       "exact power-of-two rescaling of elements, geometric factors and "
                       "coefficients outside FP32's exponent range, and matches the FP64 "
                       "oracle to 1e-12 for finite inputs of any magnitude; "
                       "kernels.ax_f64_native_* is the IEEE FP64 kernel on the same mesh"),
        "config": arm_config(world, n),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": ax_traffic(tiles),
                     "kernel": ax_kernel_name(tiles),
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": ax_bytes},
        "alu": alu_roof(tiles, ax_ms),
        "kernels": {"ax_f64_ms": ax_ms, "gs_finish_f64_ms": ds_ms,
                    "ax_f64_native_ms": nat64,
                    "ax_f64_native_gdofs": n / (nat64 / 1e3) / 1e9,
                    "ax_f64_native_frac": ax_bytes / (nat64 / 1e3) / 1e9 / hbm,
                    "ax_f64_native_note": ("sem_ax with SEM_F64_KERNEL_NATIVE: IEEE FP64 "
                                           "arithmetic (DFMA), bound by the FP64 pipe"),
                    "ax_f32_ms": ax32, "ax_f32_gbs": 32 * n / (ax32 / 1e3) / 1e9,
                    "ax_f32_frac": 32 * n / (ax32 / 1e3) / 1e9 / hbm,
                    "gs_finish_f32_ms": ds32,
                    "ax_f64_gdofs": n / (ax_ms / 1e3) / 1e9,
                    "operator_f32_gdofs": n / ((ax32 + ds32) / 1e3) / 1e9,
                    "global_f32": {"note": "sem_apply_global: w_g cleared, then gather of "
                                           "u_g and assembly of w_g by L2 reductions; "
                                           "GDOF/s counted in local points",
                                   "ms": glob32, "gdofs": n / (glob32 / 1e3) / 1e9,
                                   "global_points": ng,
                                   "algorithmic_gbs": glob_bytes / (glob32 / 1e3) / 1e9,
                                   "frac": glob_bytes / (glob32 / 1e3) / 1e9 / hbm},
                    "separate": {"note": "sem_ax then sem_dssum (increasing-index gather-scatter)",
                                 "ax_f64_ms": sep64[0], "dssum_f64_ms": sep64[1],
                                 "dssum_f64_gbs": ds_bytes / (sep64[1] / 1e3) / 1e9,
                                 "ax_f32_ms": sep32[0], "dssum_f32_ms": sep32[1],
                                 "operator_f64_gdofs": n / (sum(sep64) / 1e3) / 1e9,
                                 "operator_f32_gdofs": n / (sum(sep32) / 1e3) / 1e9}},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": 4 * K,              # element kernel + 3 gather-scatter passes
        "autotune": tiles,
        "clocks": clk.summary(),
    }
    del w, w32, u32, ug32, wg32
    sem.sem_destroy(h)

    sections = set(args.sections.split(","))
    if args.no_solve:
        sections -= {"solve", "manufactured", "projection", "pressure", "adjoint"}
    if args.no_batch:
        sections.discard("batch")
    if "model" in sections:
        line["model"] = run_model_sweep(sem, torch, dev, orders=(5, 7, 9),
                                        target_points=8_388_608, reps=10)
    if "solve" in sections:
        line["solve"] = run_solves(sem, torch, dev)
    if "batch" in sections:
        line["batch"] = run_batch(sem, torch, dev)
        # small problems, where one launch per stage for all problems pays most
        line["batch"]["small_problems"] = run_batch(sem, torch, dev, n_problems=16, e_hi=4096)
    if "manufactured" in sections:
        line["manufactured"] = run_manufactured(sem, torch, dev)
    if "projection" in sections:
        line["projection"] = run_projection(sem, torch, dev)
    if "pressure" in sections:
        line["pressure"] = run_pressure(sem, torch, dev, nel=args.pressure_nel)
    if "adjoint" in sections:
        line["adjoint"] = run_adjoint(sem, torch, dev)

    if rank == 0 and world == 1 and not args.no_cpu:
        gd1, meta1 = time_oracle(8, 10.0)
        gdn, metan = time_oracle_all_cores(2, 10.0)
        line["cpu_baseline"] = {
            "value": gdn, "unit": UNIT, "cores": metan["workers"], "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": (f"oracle Ax+dssum (numpy, FP64) on every host core at once: "
                       f"{metan['workers']} processes, each on its own 32x32x2 slab of the "
                       f"throughput mesh ({metan['points']} points), {metan['runs']} runs in "
                       f"all over {metan['seconds']:.1f} s; rate = sum over the processes"),
            "one_core": {
                "value": gd1, "unit": UNIT, "cores": 1,
                "sample": (f"the same on one core: a 32x32x8 slab ({meta1['points']} points) "
                           f"x {meta1['runs']} runs, {meta1['seconds']:.1f} s")}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(sem, torch, dev, n_problems=64, e_hi=32768):
    """64 independent deformed-box Helmholtz problems (E in [512, 32768], N in
    {5,7,9}, h2 = lambda in [0.1, 10]): one batched solve against the same
    problems solved one after another, FP32 inner / FP64 refinement to 1e-8."""
    probs = si.batch_problems(n_problems, e_hi=e_hi)
    hs, bs = [], []
    for q in probs:
        h = sem.sem_setup(q["nel"], q["N"], length=(si.TWO_PI,) * 3, deform=0.1,
                          precision=sem.SEM_PREC_F64 | sem.SEM_PREC_F32)
        xs = [torch.empty(h.n_local, dtype=torch.float64, device=dev) for _ in range(3)]
        for t, f in zip(xs, (sem.SEM_FIELD_X, sem.SEM_FIELD_Y, sem.SEM_FIELD_Z)):
            sem.sem_get_field(h, f, t)
        X, Y, Z = (t.cpu().numpy() for t in xs)
        f = torch.from_numpy(si.eval_fourier(q["rhs_modes"], X, Y, Z)).to(dev)
        b = torch.empty_like(f)
        sem.sem_rhs(h, f, b)
        hs.append(h)
        bs.append(b)
        del xs, f
    lams = [q["lam"] for q in probs]
    npts = [h.n_local for h in hs]
    batch = sem.sem_batch_create(hs)
    xb = [torch.empty_like(b) for b in bs]

    def batched(concurrent):
        sem.sem_batch_set_concurrency(batch, concurrent)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        inf = sem.sem_batch_solve(batch, bs, xb, [1.0] * len(hs), lams, tol=1e-8)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, inf

    batched(False)                     # warm-up (graph instantiation, first-call set-up)
    tb, infos = batched(False)         # order classes one after another (the default)
    tcon, _ = batched(True)            # the same as concurrent graph branches
    xs_ = [torch.empty_like(b) for b in bs]
    torch.cuda.synchronize()
    seq, tper = [], []
    t0 = time.perf_counter()
    for h, b, x, lam in zip(hs, bs, xs_, lams):
        t1 = time.perf_counter()
        seq.append(sem.sem_cg_solve(h, b, x, h1=1.0, h2=lam, tol=1e-8,
                                    precision=sem.SEM_SOLVE_MIXED))
        tper.append(time.perf_counter() - t1)         # the call synchronises
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    work = sum(n * i["iters"] for n, i in zip(npts, infos))
    per_order = {}
    for N in sorted({q["N"] for q in probs}):
        ix = [k for k, q in enumerate(probs) if q["N"] == N]
        w_n = sum(npts[k] * seq[k]["iters"] for k in ix)
        per_order[str(N)] = {"problems": len(ix), "local_points": int(sum(npts[k] for k in ix)),
                             "sequential_seconds": sum(tper[k] for k in ix),
                             "gdof_iters_per_s": w_n / sum(tper[k] for k in ix) / 1e9}
    out = {"workload": f"{len(hs)} Helmholtz problems, E in [512, {e_hi}], N in {{5,7,9}}, "
                       "h2 in [0.1, 10], deformed boxes, tol 1e-8, FP32 inner / FP64 refine",
           "local_points": int(sum(npts)),
           "batched_seconds": tb, "batched_concurrent_classes_seconds": tcon,
           "sequential_seconds": ts, "speedup": ts / tb,
           "gdof_iters_per_s": work / tb / 1e9,
           "sequential_per_order": per_order,
           "note": "each timing after one untimed batched solve; sequential = the same "
                   "problems through sem_cg_solve one after another",
           "all_converged": all(i["status"] == "SEM_OK" for i in infos),
           "max_rel_res": max(i["rel_res"] for i in infos),
           "iters_total": int(sum(i["iters"] for i in infos)),
           "sequential_iters_total": int(sum(i["iters"] for i in seq))}
    sem.sem_batch_destroy(batch)
    del hs, bs, xb, xs_
    return out


def run_solves(sem, torch, dev):
    cfg = SOLVE
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    sem.sem_autotune(h)
    n = h.n_local
    xs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(3)]
    sem.sem_get_field(h, sem.SEM_FIELD_X, xs[0])
    sem.sem_get_field(h, sem.SEM_FIELD_Y, xs[1])
    sem.sem_get_field(h, sem.SEM_FIELD_Z, xs[2])
    X, Y, Z = (t.cpu().numpy() for t in xs)
    f = torch.from_numpy(si.eval_fourier(si.fourier_modes(cfg["seed"]), X, Y, Z)).to(dev)
    del xs, X, Y, Z
    b = torch.empty_like(f)
    sem.sem_rhs(h, f, b)
    out = {"workload": "Poisson, 48^3 deformed hex elements, N=7, 8 Fourier-mode RHS",
           "local_points": n, "tol": cfg["tol"]}
    # mixed: FP32 inner PCG on global (unique-dof) vectors; mixed_local_inner:
    # the same solve with the inner PCG on L-vectors (assembled operator with
    # gather-scatter passes)
    # fp64_pipelined: the FP64 solve with the pipelined recurrences (one
    # reduction per iteration; more vector traffic, fewer kernels)
    for name, prec, inner, var in (
            ("fp64", sem.SEM_SOLVE_F64, sem.SEM_INNER_AUTO, sem.SEM_CG_STANDARD),
            ("fp64_pipelined", sem.SEM_SOLVE_F64, sem.SEM_INNER_AUTO, sem.SEM_CG_PIPELINED),
            ("mixed", sem.SEM_SOLVE_MIXED, sem.SEM_INNER_GLOBAL, sem.SEM_CG_STANDARD),
            ("mixed_local_inner", sem.SEM_SOLVE_MIXED, sem.SEM_INNER_LOCAL, sem.SEM_CG_STANDARD)):
        sem.sem_set_inner_vectors(h, inner)
        sem.sem_set_cg_variant(h, var)
        x = torch.empty_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = sem.sem_cg_solve(h, b, x, tol=cfg["tol"], precision=prec)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        out[name] = {"seconds": el, "iters": info["iters"], "outer": info["outer_iters"],
                     "rel_res": info["rel_res"], "status": info["status"]}
    out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    out["speedup_global_vs_local_inner"] = (out["mixed_local_inner"]["seconds"] /
                                            out["mixed"]["seconds"])
    sem.sem_destroy(h)
    return out


def _coords(sem, torch, h, dev):
    xs = [torch.empty(h.n_local, dtype=torch.float64, device=dev) for _ in range(3)]
    for t, f in zip(xs, (sem.SEM_FIELD_X, sem.SEM_FIELD_Y, sem.SEM_FIELD_Z)):
        sem.sem_get_field(h, f, t)
    return [t.cpu().numpy() for t in xs]


def run_pressure(sem, torch, dev, restart=10, nel=48):
    """Neko's pressure-solver path (§4, Table 2) on the 48^3 solve mesh: flexible
    GMRES(10) preconditioned by the two-level Schwarz method (10 coarse CG
    iterations), FP64 to 1e-8 (Jacobi-PCG on the same problem is the "solve"
    section; point-Jacobi GMRES(30) took 9779 iterations, 119 s, and is not
    rerun here).  With this preconditioner the iteration count hardly depends
    on the restart length (38 at 10, 37 at 30), while the Gram-Schmidt work
    grows with it (0.31 s at 10, 0.43 s at 30)."""
    cfg = SOLVE
    h = sem.sem_setup((nel,) * 3, cfg["N"], length=cfg["length"], deform=cfg["deform"])
    X, Y, Z = _coords(sem, torch, h, dev)
    f = torch.from_numpy(si.eval_fourier(si.fourier_modes(cfg["seed"]), X, Y, Z)).to(dev)
    del X, Y, Z
    b = torch.empty_like(f)
    sem.sem_rhs(h, f, b)
    del f
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pre = sem.sem_schwarz_create(h, 1.0, 0.0, coarse_iters=10)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    out = {"workload": f"Poisson, {nel}^3 deformed hex elements, N=7, 8 Fourier-mode RHS, "
                       "FP64 to 1e-8", "restart": restart, "schwarz_setup_seconds": t_setup}
    # gmres_schwarz_mixed: FP32 inner FGMRES on global vectors, FP64 refinement
    for name, prec in (("gmres_schwarz", sem.SEM_SOLVE_F64),
                       ("gmres_schwarz_mixed", sem.SEM_SOLVE_MIXED)):
        x = torch.empty_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = sem.sem_gmres_solve(h, b, x, tol=cfg["tol"], restart=restart, precond=pre,
                                   maxit=20000, precision=prec, raise_on_fail=False)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "iters": info["iters"],
                     "restarts": info["outer_iters"], "rel_res": info["rel_res"],
                     "status": info["status"]}
    # one preconditioner application and one FP64 operator, CUDA events
    r = b.clone()
    z = torch.empty_like(b)
    w = torch.empty_like(b)
    for _ in range(2):
        sem.sem_schwarz_apply(pre, r, z)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    for _ in range(5):
        sem.sem_schwarz_apply(pre, r, z)
    e[1].record()
    e[2].record()
    for _ in range(5):
        sem.sem_apply(h, r, w)
    e[3].record()
    torch.cuda.synchronize()
    out["schwarz_apply_ms"] = e[0].elapsed_time(e[1]) / 5
    out["operator_f64_ms"] = e[2].elapsed_time(e[3]) / 5
    sem.sem_schwarz_destroy(pre)
    sem.sem_destroy(h)
    return out


def run_projection(sem, torch, dev, nsolve=8, m=20):
    """Successive right-hand sides (8 Fourier modes whose phases drift, as
    successive time steps produce) on the 32^3 throughput mesh, N = 7,
    mixed-precision PCG to 1e-8: from zero each time, and from the projection
    onto the space of previous solutions (m = 20, as Neko keeps for its
    pressure solves)."""
    cfg = WORKLOAD
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    sem.sem_autotune(h)
    X, Y, Z = _coords(sem, torch, h, dev)
    bs = []
    for k in range(nsolve):
        f = torch.from_numpy(si.eval_fourier(si.drifting_modes(cfg["seed"] + 1, k), X, Y, Z)).to(dev)
        b = torch.empty_like(f)
        sem.sem_rhs(h, f, b)
        bs.append(b)
    del X, Y, Z
    x = torch.empty_like(bs[0])
    sem.sem_cg_solve(h, bs[0], x, tol=1e-8, precision=sem.SEM_SOLVE_MIXED)   # warm-up
    out = {"workload": f"{nsolve} successive right-hand sides (drifting Fourier modes), 32^3 "
                       "deformed elements, N=7, mixed precision to 1e-8", "space": m}
    for name in ("plain", "projected"):
        p = sem.sem_proj_create(h, m) if name == "projected" else None
        its = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b in bs:
            if p is None:
                info = sem.sem_cg_solve(h, b, x, tol=1e-8, precision=sem.SEM_SOLVE_MIXED)
            else:
                info = sem.sem_proj_solve(p, b, x, tol=1e-8, precision=sem.SEM_SOLVE_MIXED)
            its.append(info["iters"])
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "iters": its}
        if p is not None:
            sem.sem_proj_destroy(p)
    sem.sem_destroy(h)
    return out


def run_manufactured(sem, torch, dev):
    """Unit cube, 4^3 undeformed elements, u = sin(pi x) sin(pi y) sin(pi z):
    FP64 PCG to 1e-10 at N = 7 (iterations, time, time per iteration, max
    nodal error against the exact solution) and the spectral-convergence sweep
    N = 2..10 (max nodal error per order)."""
    cfg = si.MANUFACTURED

    def solve(N, reps=1):
        h = sem.sem_setup(cfg["nel"], N, length=cfg["length"], deform=cfg["deform"])
        X, Y, Z = _coords(sem, torch, h, dev)
        f = torch.from_numpy(si.manufactured_f(X, Y, Z)).to(dev)
        b = torch.empty_like(f)
        sem.sem_rhs(h, f, b)
        x = torch.empty_like(b)
        info = sem.sem_cg_solve(h, b, x, tol=cfg["tol"])          # warm-up (graph, dinv)
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = sem.sem_cg_solve(h, b, x, tol=cfg["tol"])
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        err = float(np.abs(x.cpu().numpy() - si.manufactured_u(X, Y, Z)).max())
        sem.sem_destroy(h)
        return info, statistics.median(times), err

    info, sec, err = solve(cfg["N"], reps=5)
    sweep = {}
    for N in range(2, 11):
        i2, _, e2 = solve(N)
        sweep[str(N)] = {"max_nodal_error": e2, "iters": i2["iters"]}
    return {"workload": "Poisson on the unit cube, 4^3 undeformed elements, N=7, "
                        "u = sin(pi x) sin(pi y) sin(pi z), FP64 PCG to 1e-10",
            "iters": info["iters"], "seconds": sec, "ms_per_iter": 1e3 * sec / max(1, info["iters"]),
            "rel_res": info["rel_res"], "status": info["status"], "max_nodal_error": err,
            "spectral_sweep_E4cubed": sweep}


def run_adjoint(sem, torch, dev):
    """16^3 deformed elements, N = 7, h1 = 1 + 0.5 tanh(smooth field), h2 = 1:
    forward solve + adjoint solve + dL/dh1 kernel through autograd (time), and
    the gradient along a smooth direction against central differences."""
    cfg = si.ADJOINT
    h = sem.sem_setup(cfg["nel"], cfg["N"], length=cfg["length"], deform=cfg["deform"])
    X, Y, Z = _coords(sem, torch, h, dev)
    h1 = torch.from_numpy(si.smooth_coefficient(X, Y, Z, cfg["h1_seed"])).to(dev)
    ut = torch.from_numpy(0.01 * si.eval_fourier(si.fourier_modes(cfg["target_seed"]),
                                                 X, Y, Z)).to(dev)
    f = torch.from_numpy(si.eval_fourier(si.fourier_modes(cfg["rhs_seed"]), X, Y, Z)).to(dev)
    d = torch.from_numpy(si.eval_fourier(si.fourier_modes(80), X, Y, Z)).to(dev)
    b = torch.empty_like(f)
    sem.sem_rhs(h, f, b)
    mult = torch.empty_like(b)
    sem.sem_get_field(h, sem.SEM_FIELD_MULT, mult)
    tol = 1e-13

    def fwd_bwd():
        h1_t = h1.clone().requires_grad_(True)
        x = sem.helmholtz_solve(h1_t, b, h, h2=1.0, tol=tol)
        loss = (((x - ut) ** 2) / mult).sum()
        loss.backward()
        return h1_t.grad

    fwd_bwd()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = fwd_bwd()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0

    def L(h1v):
        x = torch.empty_like(b)
        sem.sem_cg_solve(h, b, x, h1_field=h1v, h2=1.0, tol=tol)
        return float((((x - ut) ** 2) / mult).sum())

    eps = 1e-5 * float(h1.abs().max())
    fd = (L(h1 + eps * d) - L(h1 - eps * d)) / (2 * eps)
    gd = float((g * d).sum())
    n = h.n_local
    sem.sem_destroy(h)
    return {"workload": "variable-coefficient Helmholtz, 16^3 deformed elements, N=7, "
                        "loss ||u - u_target||^2, dL/dh1 by adjoint PCG, FP64, tol 1e-13",
            "local_points": n,
            "forward_backward_seconds": sec, "fd": fd, "grad_dot_dir": gd,
            "fd_rel_diff": abs(fd - gd) / abs(fd)}


# ---------------------------------------------------------------- cost model
FP64_PEAK = 1.20e12        # FLOP/s, FMA probe on this GB300 (independent FMA chains)
FP32_PEAK = 71.4e12


def model_costs(N, fp64):
    """Eq. 12 per local point: W (adds + mults) and Q (bytes loaded and stored,
    cold cache) of the element operator and of the gather-scatter."""
    P = N + 1
    wsz = 8 if fp64 else 4
    W_ax = 3 * (2 * P - 1) + 15 + 3 * (2 * P - 1) + 2      # D, G (9 mult 6 add), D^T, sum
    Q_ax = (1 + 1 + 6) * wsz                              # u, w, G
    shared = 1.0 - ((P - 2) / P) ** 3 if P > 2 else 1.0   # interior elements
    W_gs = 0.5 * shared                                   # one add per extra copy
    Q_gs = 2 * wsz * shared                               # read + write of shared copies
    return W_ax, Q_ax, W_gs, Q_gs


def model_time_ms(W, Q, n, pi, beta):
    """Eq. 13 for one kernel: n points of W flops and Q bytes each, on a
    machine of pi flop/s and beta bytes/s; (ms, the bound that decides it)."""
    tw, tq = W * n / pi, Q * n / beta
    return max(tw, tq) * 1e3, ("flops" if tw > tq else "bytes")


def run_model_sweep(sem, torch, dev, target_points=16_777_216, reps=20, orders=range(2, 10)):
    """Eq. 13 (T = max(W / pi, Q / beta)) against the measured kernel times for
    the given orders on deformed boxes of about target_points local points
    (the bench line's section: N = 5, 7, 9 on 8.4 M points; --model-sweep:
    N = 2..9 on 16.8 M)."""
    beta = peaks()[0] * 1e9
    rows = []
    for N in orders:
        P = N + 1
        nel = si.near_cubic_box(target_points / P ** 3, max_side=128)
        h = sem.sem_setup(nel, N, length=(si.TWO_PI,) * 3, deform=0.1)
        sem.sem_autotune(h)
        n = h.n_local
        row = {"N": N, "nel": list(nel), "local_points": n}
        for fp64 in (True, False):
            dt = torch.float64 if fp64 else torch.float32
            u = torch.rand(n, dtype=dt, device=dev) - 0.5
            w = torch.empty_like(u)
            W_ax, Q_ax, W_gs, Q_gs = model_costs(N, fp64)
            pi = FP64_PEAK if fp64 else FP32_PEAK
            kinds = [("ax", lambda: sem.sem_ax(h, u, w), W_ax, Q_ax),
                     ("dssum", lambda: sem.sem_dssum(h, w), W_gs, Q_gs),
                     ("apply", lambda: sem.sem_apply(h, u, w), W_ax + W_gs, Q_ax + Q_gs)]
            if fp64:
                def native():
                    sem.sem_set_f64_kernel(h, sem.SEM_F64_KERNEL_NATIVE)
                    sem.sem_ax(h, u, w)
                    sem.sem_set_f64_kernel(h, sem.SEM_F64_KERNEL_AUTO)
                kinds.append(("ax_native", native, W_ax, Q_ax))
            tag = "f64" if fp64 else "f32"
            for name, fn, W, Q in kinds:
                for _ in range(3):
                    fn()
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(reps):
                    fn()
                b.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / reps
                t_model, bound = model_time_ms(W, Q, n, pi, beta)
                row[f"{name}_{tag}"] = {"ms": ms, "model_ms": t_model, "bound": bound,
                                        "measured_over_model": ms / t_model}
            del u, w
        sem.sem_destroy(h)
        rows.append(row)
    return {"model": "Eq. 13: T = max(W / pi, Q / beta), cold cache, per kernel",
            "pi_fp64": FP64_PEAK, "pi_fp32": FP32_PEAK, "beta": beta, "rows": rows}


if __name__ == "__main__":
    sys.exit(main())
