"""Throughput benchmark of the curved-space LBM hot path on GB300.

Workload (default): the 256^3 deformed channel -- 256 span on axis 0, 256
along the flow on axis 1, 256 wall-normal on axis 2 -- walls across axis 2,
periodic span, parabolic inflow / outflow along the flow axis, tau = 0.6
(Re ~ 100), an 8-mode seeded wall deformation of 8 % amplitude under the
time law sin^2(pi t / 2000), FP32 storage.  One bench step is one cycle of
that schedule: metric update + transformation of f (every 10 LBM steps), 10
LBM steps, then the FP64 mass and wall-force reductions.  Metric snapshots
are generated up front (the caller's job) and cycled.  MLUPS = lattice nodes
x LBM steps / time.  The line also carries the 128 x 128 x 256 dynamic
channel (16 modes, 10 %) under the same schedule (`dynamic_channel`).

Inputs (5.6 GB of state per LBM step at 256^3) exceed the 129 MB L2, so no
flush is needed between timed iterations.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 every rank advances its own channel (independent problems, weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1803_07822_gb300 import inputs as I  # noqa: E402

METRIC = "curved-space LBM MLUPS and HBM GB/s vs peak; adjoint/forward step-time ratio"
UNIT = "MLUPS"
STEPS_PER_CYCLE = 10
# algorithmic bytes per node update: 19 f read + 19 written, 10 history
# coefficients read + written (FP32), 25 geometry values read (FP32)
BYTES_PER_NODE = {"fp32": 19 * 4 * 2 + 10 * 4 * 2 + 25 * 4, "fp16": 19 * 2 * 2 + 80 + 100,
                  "bf16": 19 * 2 * 2 + 80 + 100, "fp64": 19 * 8 * 2 + 80 + 100}
# DRAM bytes per node update (dram__bytes_read.sum + dram__bytes_write.sum of
# the kernels of one LBM step, per launch, divided by the nodes) from an ncu
# capture of the kernels as they stand, keyed by (pass, storage, workload);
# a workload too large for a capture takes the figure of a smaller lattice of
# the same tile shape (the note says which).  A pass with no entry reports
# traffic null.
MEASURED_DRAM_BYTES_PER_NODE = {("fused", "fp32", "target256"): 325.2, ("fused", "fp32", "slab256"): 325.2}
TRAFFIC_NOTE = {
    ("fused", "fp32", "target256"): "k_step_fused alone, from an ncu capture of one launch on the 256x256x64 slab of "
                                    "the same generator (the same one-row tiles, 1/4 of the nodes), scaled by the "
                                    "nodes: 885.8 MB read + 478.2 MB written for 4,194,304 nodes",
    ("fused", "fp32", "slab256"): "k_step_fused alone, one launch captured by ncu on this lattice",
}
NO_CAPTURE = "no ncu capture of the step kernels as they stand"


def step_pass(n, storage, step_kernel, axis2_periodic=False):
    """The step pass the library takes for this lattice (the rule
    include/cslbm.h states for cslbm_step_kernel): "fused", "rows" or "flat"."""
    sb = {"fp32": 4, "fp16": 2, "bf16": 2}.get(storage)
    rows = (step_kernel in ("auto", "rows") and sb is not None and n[0] <= 256 and n[0] % 4 == 0
            and (n[0] * sb) % 16 == 0 and n[0] * n[1] * n[2] >= 256)
    if rows and step_kernel == "auto" and not axis2_periodic:
        return "fused"
    return "rows" if rows else "flat"


PASS_KERNELS = {"fused": "k_step_fused + k_step_faces", "rows": "k_momentum_flat + k_step_rows + k_step_faces",
                "flat": "k_momentum_flat + k_step_flat"}


def workload_spec(name):
    if name == "dynamic":
        return dict(key="dynamic", n=(128, 256, 128), seed=2000, n_modes=16, amp=0.10, tau=0.6, re=100.0,
                    storage="fp32", label="deformed channel 128x128x256, dynamic metric (16 modes, 10 %), "
                                          "inflow/outflow, tau 0.6, Re 100, FP32, transform every 10 steps")
    if name == "crop64":
        return dict(key="crop64", n=(64, 128, 64), seed=2000, n_modes=16, amp=0.10, tau=0.6, re=100.0, storage="fp32",
                    label="deformed channel 64x64x128 (profiling case), dynamic metric, inflow/outflow, FP32")
    if name == "slab256":
        return dict(key="slab256", n=(256, 256, 64), seed=3000, n_modes=8, amp=0.08, tau=0.6, re=100.0, storage="fp32",
                    label="deformed channel 256x256x64 slab (profiling case: the 256^3 tile shape at a quarter "
                          "of its nodes), dynamic metric (8 modes, 8 %), inflow/outflow, tau 0.6, FP32")
    if name == "target256":
        return dict(key="target256", n=(256, 256, 256), seed=3000, n_modes=8, amp=0.08, tau=0.6, re=100.0, storage="fp32",
                    label="deformed channel 256^3, dynamic metric (8 modes, 8 %), inflow/outflow, tau 0.6, FP32")
    raise ValueError(name)


def snapshots(w, times):
    out = []
    for t in times:
        ch, faces = I.dynamic_channel_at(w, t)
        out.append((ch, faces))
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (every 50 ms,
    timestamped), started before the warm-up; stop() keeps the samples taken
    between mark_start() and mark_end(), or the one nearest that window when
    it is shorter than the sampling interval."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.t0 = self.t1 = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def wait_first(self, limit_s=5.0):
        t = time.time()
        while self.p is not None and time.time() - t < limit_s:
            if os.path.getsize(self.f.name) > 0:
                return
            time.sleep(0.02)

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        samples = []
        for r in rows:
            try:
                ts = r[0].strip()
                t = time.mktime(time.strptime(ts.split(".")[0], "%Y/%m/%d %H:%M:%S")) + float("0." + ts.split(".")[1])
                samples.append((t, float(r[1]), float(r[2]),
                                {name for k, name in enumerate(names) if len(r) > 4 + k and r[4 + k].strip() == "Active"}))
            except (ValueError, IndexError):
                continue
        if not samples:
            return None
        inside = [x for x in samples if self.t0 is not None and self.t0 <= x[0] <= (self.t1 or x[0])]
        window = "timed region"
        if not inside:
            mid = 0.5 * ((self.t0 or 0.0) + (self.t1 or self.t0 or 0.0))
            inside = [min(samples, key=lambda x: abs(x[0] - mid))]
            window = "nearest sample to a timed region shorter than the 50 ms interval"
        reasons = set().union(*[x[3] for x in inside])
        return {"sm_mhz": statistics.median(x[1] for x in inside), "sm_max_mhz": max(x[2] for x in samples),
                "reasons": sorted(reasons), "samples": len(inside), "window": window,
                "sm_mhz_min": min(x[1] for x in inside)}


def dist_setup(args):
    """(rank, world, local) from the launcher's environment; a process group
    when world > 1 -- NCCL on the GPUs, gloo where there is no GPU (the
    host-logic tests).  Every rank then runs its own, independent problem."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def reduce_max(x, world):
    """The maximum of x over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_mlups(world, nodes_per_rank, lbm_steps, ms):
    """Whole-job throughput: every rank updates its own nodes_per_rank nodes
    lbm_steps times; ms is the slowest rank's time (weak scaling)."""
    return world * nodes_per_rank * lbm_steps / (ms * 1e-3) / 1e6


def oracle_cycle_sample(spec, steps, warm, div=2):
    """The FP64 oracle on a bounded sample of the same workload: the same
    generator on a crop of 1/div the extent per axis (1/8 of the volume by
    default), timed over whole cycles (metric transform + 10 steps).  Returns
    (MLUPS, seconds, nodes, cores)."""
    import oracle
    n = tuple(v // div for v in spec["n"])
    w = I.dynamic_channel(n=n, seed=spec["seed"], n_modes=spec["n_modes"], amp=spec["amp"], tau=spec["tau"],
                          re=spec["re"])
    snaps = snapshots(w, [500.0 + STEPS_PER_CYCLE * k for k in range(steps + warm + 1)])
    o = oracle.Lattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    ch0, f0 = snaps[0]
    o.set_metric(ch0.g6, ch0.dg18)
    for (a, s), u in f0.items():
        o.set_face_velocity(a, s, u)
    o.init()
    prev = ch0
    t_total = 0.0
    for k in range(1, steps + warm + 1):
        ch, faces = snaps[k]
        t0 = time.perf_counter()
        o.transform(ch.g6, ch.dg18, prev.J9, ch.J9)
        for (a, s), u in faces.items():
            o.set_face_velocity(a, s, u)
        o.step(STEPS_PER_CYCLE)
        o.mass()
        o.wall_force(0, 1, ch.J9)
        dt = time.perf_counter() - t0
        prev = ch
        if k > warm:
            t_total += dt
    N = int(np.prod(n))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return N * STEPS_PER_CYCLE * steps / t_total / 1e6, t_total, n, cores


ORACLE_C1_STEPS = 200


def oracle_c1_sample():
    """The FP64 oracle on the 16 x 16 x 32 plain channel (walls, body force,
    one-mode deformation), ORACLE_C1_STEPS timed steps after 20, with the
    threads OpenMP was given in this process.  Returns (MLUPS, seconds)."""
    import oracle
    w = I.plain_fp64_channel()
    o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    o.set_metric(w["chart"].g6, w["chart"].dg18)
    o.init()
    o.step(20)
    t0 = time.perf_counter()
    o.step(ORACLE_C1_STEPS)
    dt = time.perf_counter() - t0
    return int(np.prod(w["n"])) * ORACLE_C1_STEPS / dt / 1e6, dt


def oracle_single_thread():
    """oracle_c1_sample in a child process started with OMP_NUM_THREADS=1."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-c1"], capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, OMP_NUM_THREADS="1"), cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("single-thread oracle run failed:\n" + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": UNIT, "cores": 1,
            "sample": f"16x16x32 plain FP64 channel, {ORACLE_C1_STEPS} steps after 20 ({d['secs']:.1f} s)"}


def cpu_model(path="/proc/cpuinfo"):
    """The host CPU as /proc/cpuinfo names it: the model name where there is
    one (x86), else the implementer and part codes (Arm)."""
    try:
        with open(path) as fh:
            txt = fh.read()
    except OSError:
        return platform.machine()
    m = re.search(r"^model name\s*:\s*(.+)$", txt, re.M)
    if m:
        return m.group(1).strip()
    imp = re.search(r"^CPU implementer\s*:\s*(\S+)", txt, re.M)
    part = re.search(r"^CPU part\s*:\s*(\S+)", txt, re.M)
    return f"{platform.machine()}, implementer {imp.group(1) if imp else '?'}, part {part.group(1) if part else '?'}"


def oracle_batch_sample(ws, count=3, steps=10):
    """The FP64 oracle on the `count` smallest channels of a batch, one after
    another (as the per-channel form runs them), `steps` steps each after 2.
    Returns the cpu_baseline object."""
    import oracle
    order = sorted(range(len(ws)), key=lambda i: int(np.prod(ws[i]["n"])))[:count]
    nodes, secs = 0, 0.0
    for i in order:
        w = ws[i]
        o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
        o.set_metric(w["chart"].g6, w["chart"].dg18)
        o.init()
        o.step(2)
        t0 = time.perf_counter()
        o.step(steps)
        secs += time.perf_counter() - t0
        nodes += int(np.prod(w["n"]))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": nodes * steps / secs / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the {count} smallest channels of the batch ({nodes} nodes), {steps} steps each after 2, "
                      f"FP64 ({secs:.1f} s)"}


def bench_batch(args):
    """The batched form: 64 independent periodic channels with sides drawn from
    U{32..96} per axis, 4-mode deformations of 2-10 % amplitude, tau in
    [0.55, 1.0], FP32, all advanced by one persistent launch per LBM step (a
    device-side queue of work items over every channel, a grid barrier
    between the momentum and step phases) replayed from a CUDA graph, tile
    shape from the library's autotuner.  A bench step is 10
    LBM steps of every channel.  Also timed: the same channels stepped one
    channel at a time (each its own launches), the per-channel baseline."""
    import torch

    from paper_1803_07822_gb300.lattice import CurvedBatch
    rank, world, local = dist_setup(args)
    ws = I.batch_channels(nb=64, seed0=4000 + 1000 * rank)
    b = CurvedBatch([dict(n=w["n"], bc_lo=w["bc_lo"], bc_hi=w["bc_hi"], tau=w["tau"], fext=w["fext"]) for w in ws])
    for i, w in enumerate(ws):
        b[i].set_chart(w["chart"])
        b[i].init_equilibrium()
    shape, tune_table = b.tune(reps=5)
    stream = b.stream
    N = b.nodes

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    clocks = Clocks(local)
    for _ in range(args.warmup):
        b.step(STEPS_PER_CYCLE)
    clocks.wait_first()
    l0 = b.launches()
    clocks.mark_start()
    ms = timed(lambda: b.step(STEPS_PER_CYCLE), args.steps)
    clocks.mark_end()
    clk = clocks.stop()
    launches = b.launches() - l0
    ms = reduce_max(ms, world)

    def per_channel():
        for c in b:
            c.step(STEPS_PER_CYCLE)

    kpc = max(1, args.steps // 3)
    per_channel()
    ms_pc = reduce_max(timed(per_channel, kpc), world) / kpc
    bad = [i for i, c in enumerate(b) if not c.check()]
    # end to end: the same steps with the 64 channel masses read back to the host every bench step
    t0 = time.perf_counter()
    for _ in range(kpc):
        b.step(STEPS_PER_CYCLE)
        masses = [c.total_mass() for c in b]
    e2e_s = (time.perf_counter() - t0) / kpc
    peak, peak_kind = peaks()
    steps_total = STEPS_PER_CYCLE * args.steps
    value = world * N * steps_total / (ms * 1e-3) / 1e6
    ach = BYTES_PER_NODE["fp32"] * N * steps_total / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "64 independent deformed periodic channels, sides U{32..96}, 4 modes 2-10 %, "
                               "tau U[0.55, 1.0], FP32, batched (one persistent launch per LBM step over a "
                               "work-item queue, CUDA graph)", "nodes": N, "lbm_steps_per_step": STEPS_PER_CYCLE,
                   "l2": "inputs > L2 (5.8 GB of state per LBM step), no flush",
                   "tile_shape": {"block_nodes": shape[0], "item_nodes": shape[1], "blocks_per_sm": shape[2]},
                   "tune_ms_per_lbm_step": {f"{k[0]}/{k[1]}/{k[2]}": v for k, v in sorted(tune_table.items())},
                   "state_finite_after_run": not bad and b.check(), "unstable_channels": bad},
        "per_channel_launches": {"value": world * N * STEPS_PER_CYCLE / (ms_pc * 1e-3) / 1e6, "unit": UNIT,
                                 "ms_per_step": ms_pc},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": None, "peak_kind": peak_kind,
                     "kernel": "one batched LBM step: k_batch_persistent", "bytes_per_node": 332},
        "e2e": {"value": world * N * STEPS_PER_CYCLE / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 8 * len(masses)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = oracle_batch_sample(ws)
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"] = {"error": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


ADJOINT_STEPS, ADJOINT_EVERY = 200, 20


def bench_side(args):
    """One JSON line for the adjoint (adjoint/forward step-time ratio on the
    adjoint-form channel) or for the lattice gradient of the six metric
    fields on the 128 x 128 x 256 bench channel (FP64 GFLOP/s)."""
    import torch

    from paper_1803_07822_gb300.lattice import CurvedLattice
    torch.cuda.set_device(0)
    base = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic"}
    if args.workload == "adjoint64":
        r = adjoint_report(args.step_kernel, args.adjoint_steps)
        line = dict(base, metric="adjoint/forward step-time ratio", value=r["ratio"], unit="ratio",
                    higher_is_better=False, dtype="f32", ms_per_step=r["backward_ms_per_step"],
                    config={"workload": r["workload"]}, adjoint=r)
    else:
        w = I.dynamic_channel(n=(128, 256, 128), t=500.0)
        lat = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], storage="fp32")
        r = lattice_gradient_report(lat, torch.as_tensor(w["chart"].g6, device="cuda"), 4, reps=max(args.steps, 1))
        line = dict(base, metric="lattice gradient of the metric (App. D, order 4), FP64 GFLOP/s",
                    value=r["roofline"]["achieved"], unit="GFLOP/s", higher_is_better=True, dtype="f64",
                    ms_per_step=r["ms"], config={"workload": "six metric fields of the 128x128x256 dynamic channel"},
                    lattice_gradient=r)
        if not args.no_cpu_baseline:
            try:
                line["cpu_baseline"] = oracle_gradient_sample(workload_spec("dynamic"))
            except Exception as e:  # noqa: BLE001
                line["cpu_baseline"] = {"error": str(e)[-300:]}
    print(json.dumps(line), flush=True)


# algorithmic bytes per D2Q9 node update (FP32): 9 slots read + written, 6
# forcing coefficients read + written, 10 geometry values read
BYTES_PER_NODE_2D = 9 * 4 * 2 + 6 * 4 * 2 + 10 * 4


def d2q9_channel(n):
    """The D2Q9 benchmark channel at size n: periodic along x, walls across
    y, the top wall displaced by 6 % of the height x cos(2 pi x / n0), body
    force for a centre-line speed of 0.05 at tau 0.8.  (chart, tau, force)."""
    H = n[1] - 1
    x = I.grid2d(n)[0]
    k = 2 * np.pi / n[0]
    a = 0.06 * H
    ch = I.channel_chart2d(n, a * np.cos(k * x), -a * k * np.sin(k * x), -a * k * k * np.cos(k * x))
    tau = 0.8
    return ch, tau, 8.0 * (tau - 0.5) / 3.0 * 0.05 / H ** 2


def oracle2d_sample(n=(1024, 256), steps=40):
    """The FP64 D2Q9 oracle on the same channel at a quarter of the size per
    axis: `steps` timed steps after 2.  Returns (MLUPS, seconds, n, cores)."""
    import oracle
    ch, tau, F = d2q9_channel(n)
    o = oracle.Lattice2D(n, (0, 1), (0, 1), tau=tau, fext=(F, 0.0))
    o.set_metric(ch.g3, ch.dg6)
    o.init()
    o.step(2)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n[0] * n[1] * steps / dt / 1e6, dt, n, cores


def bench_d2q9(args):
    """The D2Q9 path on a 4096 x 1024 periodic channel (walls across, the top
    wall displaced by 6 % of the height x cos(2 pi x / 4096), body-force
    drive, FP32): MLUPS and the fraction of the measured HBM bandwidth against
    160 B per node update; 10 LBM steps per bench step."""
    import torch

    from paper_1803_07822_gb300.lattice import CurvedLattice2D
    torch.cuda.set_device(0)
    n = (4096, 1024)
    ch, tau, F = d2q9_channel(n)
    lat = CurvedLattice2D(n, (0, 1), (0, 1), tau=tau, fext=(F, 0.0), storage="fp32")
    lat.set_chart(ch)
    lat.init_equilibrium()
    N = lat.N
    for _ in range(args.warmup):
        lat.step(STEPS_PER_CYCLE)
    clocks = Clocks(0)
    clocks.wait_first()
    torch.cuda.synchronize()
    clocks.mark_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        lat.step(STEPS_PER_CYCLE)
    e1.record()
    torch.cuda.synchronize()
    clocks.mark_end()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    step_ms = ms / (args.steps * STEPS_PER_CYCLE)
    peak, peak_kind = peaks()
    achieved = BYTES_PER_NODE_2D * N / (step_ms * 1e-3) / 1e9
    line = {"metric": "curved-space LBM MLUPS (D2Q9)", "value": N * STEPS_PER_CYCLE * args.steps / (ms * 1e-3) / 1e6,
            "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "D2Q9 periodic deformed channel 4096x1024, 6 % cosine top wall, body force, FP32",
                       "nodes": N, "lbm_steps_per_step": STEPS_PER_CYCLE,
                       "l2": "inputs > L2 (0.7 GB of state per LBM step), no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_kind": peak_kind, "kernel": "one LBM step: k2_momentum + k2_step",
                         "bytes_per_node": BYTES_PER_NODE_2D, "step_ms": step_ms},
            "gpu_launches": 2 * STEPS_PER_CYCLE * args.steps, "clocks": clk}
    if not args.no_cpu_baseline:
        v, secs, nc, cores = oracle2d_sample()
        line["cpu_baseline"] = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                "sample": f"the same channel at {nc[0]}x{nc[1]}, 40 steps after 2, FP64 "
                                          f"({secs:.1f} s)"}
    print(json.dumps(line), flush=True)


def adjoint_report(step_kernel, steps=None):
    """Adjoint/forward step-time ratio on the adjoint-form channel
    (inputs.adjoint_channel: 64 x 128 x 64, 32 deformation coefficients,
    tau 0.8, FP32 storage): the gradient of the streamwise force on the
    deformed wall after 200 steps from rest with respect to the metric inputs
    (g, dg, J), through the library's adjoint with checkpoints every 20 steps.
    backward_ms_per_step is that gradient's device time (CUDA events) over the
    200 steps: every step recomputed from its checkpoint, its state reloaded
    and reversed, plus the seed, the rest initialisation and the metric
    kernel reversed.  forward_ms_per_step is the plain FP32 step of the same
    lattice.  The chain rule from (g, dg, J) to the coefficients is the
    caller's torch code and is timed apart.  Accuracy: three coefficient
    derivatives against central differences (h = 1e-4) of the FP64 forward."""
    import torch

    from paper_1803_07822_gb300.adjoint import chart_from_coeffs, wall_force_objective
    from paper_1803_07822_gb300.lattice import CurvedLattice
    w = I.adjoint_channel()
    axis = w["layout"][0]
    e3 = [0.0, 0.0, 0.0]
    e3[w["layout"][2]] = 1.0
    T = ADJOINT_STEPS if steps is None else int(steps)
    lat = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp32",
                        step_kernel=step_kernel)
    c = torch.tensor(w["c"], dtype=torch.float64, device="cuda", requires_grad=True)
    chart = chart_from_coeffs(c, w["n"], w["modes"], w["scale"])
    leaves = [t.detach().requires_grad_(True) for t in chart]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    for rep in range(2):  # the first pass allocates the adjoint workspace and the checkpoints
        torch.cuda.synchronize()
        ev[0].record()
        J = wall_force_objective(lat, *leaves, T, ADJOINT_EVERY, axis=axis, side=1, e3=e3)
        ev[1].record()
        grads = torch.autograd.grad(J, leaves)
        ev[2].record()
        torch.cuda.synchronize()
    lat.init_equilibrium()
    ev[3].record()
    lat.step(T)
    ev[4].record()
    torch.autograd.backward(chart, grads, retain_graph=True)  # first call: lazy initialisation in torch
    c.grad = None
    torch.cuda.synchronize()
    ev[5].record()
    torch.autograd.backward(chart, grads)
    ev[6].record()
    torch.cuda.synchronize()
    fwd = ev[3].elapsed_time(ev[4]) / T
    bwd = ev[1].elapsed_time(ev[2]) / T
    sb = lat.state_bytes()
    mem = lat._adjoint.workspace.numel() + (-(-T // ADJOINT_EVERY) + 1 + min(T, ADJOINT_EVERY)) * sb
    g = c.grad.cpu().numpy()

    f64 = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp64",
                        step_kernel="flat")

    def objective(cv):
        g6, dg18, J9 = chart_from_coeffs(torch.tensor(cv, dtype=torch.float64, device="cuda"), w["n"], w["modes"],
                                         w["scale"])
        f64.set_metric(g6, dg18)
        f64.set_jacobian(J9)
        f64.init_equilibrium()
        f64.step(T)
        return float(np.dot(e3, f64.wall_force(axis, 1)))

    picks, h, fd = [0, 9, 27], 1e-4, []
    for m in picks:
        cp, cm = w["c"].copy(), w["c"].copy()
        cp[m] += h
        cm[m] -= h
        fd.append((objective(cp) - objective(cm)) / (2 * h))
    err = float(np.linalg.norm(g[picks] - np.array(fd)) / np.linalg.norm(fd))
    for x in (lat, f64):
        x.close()
    return {"workload": "adjoint-form channel 64x128x64 (span, flow, wall), 32 coefficients, tau 0.8, FP32 storage; "
                        f"objective: streamwise force on the deformed wall after {T} steps from rest",
            "ratio": bwd / fwd, "forward_ms_per_step": fwd, "backward_ms_per_step": bwd,
            "forward_kernel": step_kernel, "checkpoint_every": ADJOINT_EVERY,
            "chart_backward_ms": ev[5].elapsed_time(ev[6]),
            "memory_bytes": mem, "state_bytes": sb,
            "grad_rel_err_vs_fp64_fd": err, "fd": "central, h = 1e-4, coefficients 0, 9, 27, FP64 GPU forward"}


# FP64 operations (an FMA counts 2) per lattice site and field of the
# lattice-derivative kernels as written: k_pad 16 additions + 2 FMAs + 1
# multiply per padded site (order 4), k_grad 9 pair differences + 15 FMAs
LAP_FLOP, GRAD_FLOP = {2: 0, 4: 21}, {2: 39, 4: 39}
# FP64 peak from the unit counts: 152 SMs x 2 FP64 FMA per clock x 2 x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


def lattice_gradient_report(lat, g6, order=4, reps=5):
    """Device time of the library's lattice gradient (App. D) of the six
    metric components on the bench lattice, against the FP64 peak."""
    import torch
    for _ in range(2):
        lat.lattice_gradient(g6, order)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        lat.lattice_gradient(g6, order)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    N = lat.N
    pad = [(0 if (lo == 0 and hi == 0) else 1) for lo, hi in zip(list(lat.params.bc_lo), list(lat.params.bc_hi))]
    Ne = int(np.prod([k + 2 * p for k, p in zip(lat.n, pad)]))
    flop = 6 * (LAP_FLOP[order] * Ne + GRAD_FLOP[order] * N)
    nbytes = 6 * 8 * (N + 2 * Ne) + 18 * 8 * N
    gf = flop / (ms * 1e-3) / 1e9
    return {"order": order, "fields": 6, "nodes": N, "ms": ms, "flop_per_node": flop / N,
            "bytes_per_node": nbytes / N, "hbm_gbs": nbytes / (ms * 1e-3) / 1e9,
            "roofline": {"bound": "alu", "achieved": gf, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (FP64)",
                         "frac": gf / FP64_PEAK_GFLOPS, "peak_kind": "derived from unit counts and clock"}}


def transform_interp_report(lat, dev, layout, reps=5):
    """Device time of one chart change of the bench channel (metric kernel +
    transformation) with the interpolating form against the node-wise one.
    The transition map of the channel chart h^w = x_w (1 + d/H) between two
    snapshots: x_w = x~_w J~^w_w / J^w_w (J^w_w = 1 + d/H), the rest fixed."""
    import torch
    w = layout[0]
    grid = torch.as_tensor(np.stack(I.grid(lat.n)), device="cuda")
    # both forms with FP64 inputs (the interpolating call takes no other),
    # converted once outside the timed region
    dev = [{k: (v.double() if k in ("g6", "dg18", "J9") else v) for k, v in d.items()} for d in dev]
    pairs = [(dev[i], dev[i + 1]) for i in range(len(dev) - 1)]
    psis = []
    for a, b in pairs:
        psi = grid.clone()
        psi[w] = psi[w] * b["J9"][w * 3 + w] / a["J9"][w * 3 + w]
        psis.append(psi)
    out = {}
    for mode in ("node", "interp"):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(reps + 2):
            if rep == 2:
                e0.record()
            for (a, b), psi in zip(pairs, psis):
                if mode == "interp":
                    lat.update_metric_interp(b["g6"], b["dg18"], b["J9"], psi)
                else:
                    lat.update_metric(b["g6"], b["dg18"], b["J9"])
                lat.set_jacobian(a["J9"])  # back to the pair's old chart for the next change
        e1.record()
        torch.cuda.synchronize()
        out[mode] = e0.elapsed_time(e1) / (reps * len(pairs))
    return {"node_wise_ms": out["node"], "interp_ms": out["interp"], "nodes": lat.N,
            "note": "one chart change incl. the metric kernel; the interpolating form adds the moment-field pass "
                    "and reads 8 corners per node (20 fields + the Jacobian)"}


def oracle_gradient_sample(spec, order=4):
    """The FP64 oracle's lattice gradient (App. D) of the six metric
    components of the channel `spec` at half the extent per axis, in the
    lattice-gradient line's unit (GFLOP/s, by the same algorithmic FLOP count
    as the library's figure) and in Mnode/s."""
    import oracle
    n = tuple(v // 2 for v in spec["n"])
    w = I.dynamic_channel(n=n, seed=spec["seed"], n_modes=spec["n_modes"], amp=spec["amp"], tau=spec["tau"],
                          re=spec["re"])
    (c0, _), = snapshots(w, [500.0])
    N = int(np.prod(n))
    pad = [(0 if (lo == 0 and hi == 0) else 1) for lo, hi in zip(w["bc_lo"], w["bc_hi"])]
    Ne = int(np.prod([k + 2 * p for k, p in zip(n, pad)]))
    flop = 6 * (LAP_FLOP[order] * Ne + GRAD_FLOP[order] * N)
    t0 = time.perf_counter()
    oracle.lattice_gradient(n, c0.g6, order, w["bc_lo"], w["bc_hi"])
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": flop / dt / 1e9, "unit": "GFLOP/s (FP64)", "mnode_per_s": N / dt / 1e6, "cores": cores,
            "kind": "oracle", "sample": f"order-{order} gradient of the 6 metric components, {n[0]}x{n[1]}x{n[2]} "
                                        f"crop of the same generator, FP64 oracle ({dt:.2f} s)"}


def oracle_side_samples(spec):
    """The FP64 oracle on a half-size crop of the bench channel (the same
    generator at n / 2 per axis): the fourth-order lattice gradient of the six
    metric components (App. D, oracle_gradient_sample), and one chart change
    node-wise and with interpolation (Sec. IV.B) between the snapshots t = 500
    and 510.  Returns the cpu_baseline objects of the lattice_gradient and
    transform_interp reports."""
    import oracle
    n = tuple(v // 2 for v in spec["n"])
    w = I.dynamic_channel(n=n, seed=spec["seed"], n_modes=spec["n_modes"], amp=spec["amp"], tau=spec["tau"],
                          re=spec["re"])
    (c0, f0), (c1, f1) = snapshots(w, [500.0, 510.0])
    N = int(np.prod(n))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    crop = f"{n[0]}x{n[1]}x{n[2]} crop of the same generator, FP64 oracle"
    wa = w["layout"][0]
    psi = np.stack(I.grid(n))
    psi[wa] = psi[wa] * c1.J9[wa * 3 + wa] / c0.J9[wa * 3 + wa]
    times = {}
    for mode in ("node", "interp"):
        o = oracle.Lattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
        o.set_metric(c0.g6, c0.dg18)
        for (a, s), u in f0.items():
            o.set_face_velocity(a, s, u)
        o.init()
        t0 = time.perf_counter()
        if mode == "node":
            o.transform(c1.g6, c1.dg18, c0.J9, c1.J9)
        else:
            o.transform_interp(c1.g6, c1.dg18, c0.J9, c1.J9, psi)
        times[mode] = time.perf_counter() - t0
    grad = oracle_gradient_sample(spec)
    trans = {"node_wise_ms": times["node"] * 1e3, "interp_ms": times["interp"] * 1e3, "nodes": N, "cores": cores,
             "kind": "oracle", "sample": f"one chart change (metric + transform) on the {crop}"}
    return grad, trans


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec = workload_spec(args.workload)
    # the crop: half the extent per axis, or a quarter where that would take
    # more than about 3e8 node updates (under a minute on the host cores)
    div = 2
    while int(np.prod([v // div for v in spec["n"]])) * STEPS_PER_CYCLE * (args.steps + args.warmup) > 3e8 and div < 8:
        div *= 2
    mlups, secs, n, cores = oracle_cycle_sample(spec, args.steps, args.warmup, div)
    sample = (f"{n[0]}x{n[1]}x{n[2]} crop of the same generator, {args.steps} timed cycles "
              f"({STEPS_PER_CYCLE} steps + transform + reductions each), FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": spec["label"], "sample": sample},
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def channel_cycles(spec, args, rank, world, local, steps):
    """The channel of `spec` through `steps` timed bench cycles after
    args.warmup, inputs resident in HBM: metric snapshots pre-generated and
    cycled, each cycle a chart change with transformation, 10 LBM steps and
    the mass and wall-force reductions.  Device time with CUDA events on the
    library's stream, the slowest rank's; one LBM step timed by the library
    (profiling on) for the roofline.  For FP32-arithmetic storage the chart
    change takes its derivatives and Jacobian in FP32
    (cslbm_update_metric_mixed: the library rounds them to FP32 before use,
    so the state is the one FP64 inputs give, bit for bit)."""
    import torch

    from paper_1803_07822_gb300.lattice import CurvedLattice
    w = I.dynamic_channel(n=spec["n"], seed=spec["seed"] + rank, n_modes=spec["n_modes"], amp=spec["amp"],
                          tau=spec["tau"], re=spec["re"])
    N = int(np.prod(spec["n"]))
    times = [500.0 + STEPS_PER_CYCLE * k for k in range(args.snapshots + 1)]
    snaps = snapshots(w, times)
    lat = CurvedLattice(spec["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage=spec["storage"],
                        step_kernel=args.step_kernel)
    # device-resident inputs for the kernel-throughput run
    mixed = spec["storage"] != "fp64"
    dev = []
    for ch, faces in snaps:
        d = {k: torch.as_tensor(getattr(ch, k), device="cuda") for k in ("g6", "dg18", "J9")}
        if mixed:
            d["dg18"], d["J9"] = d["dg18"].float(), d["J9"].float()
        d["faces"] = {key: torch.as_tensor(u, device="cuda") for key, u in faces.items()}
        dev.append(d)
    ch0, faces0 = snaps[0]
    lat.set_chart(ch0)
    for (a, s), u in faces0.items():
        lat.set_boundary_velocity(a, s, u)
    lat.init_equilibrium()

    def cycle_dev(k):
        d = dev[1 + k % args.snapshots]
        if mixed:
            lat.update_metric_mixed(d["g6"], d["dg18"], d["J9"])
        else:
            lat.update_metric(d["g6"], d["dg18"], d["J9"])
        for (a, s), u in d["faces"].items():
            lat.set_boundary_velocity(a, s, u)
        lat.step(STEPS_PER_CYCLE)
        lat.total_mass()
        lat.wall_force(0, 1)

    clocks = Clocks(local)
    for k in range(args.warmup):
        cycle_dev(k)
    clocks.wait_first()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks.mark_start()
    lat.profile(True)
    stream = lat.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        cycle_dev(args.warmup + k)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    step_ms_total, nprof, launches = lat.profile_read()
    lat.profile(False)
    ms = reduce_max(ms, world)
    return dict(lat=lat, w=w, N=N, snaps=snaps, dev=dev, ms=ms, step_ms=step_ms_total / max(nprof, 1),
                launches=launches, clk=clk, ok=lat.check())


def roofline_of(spec, args, N, step_ms):
    peak, peak_kind = peaks()
    bpn = BYTES_PER_NODE[spec["storage"]]
    achieved = bpn * N / (step_ms * 1e-3) / 1e9
    sp = step_pass(spec["n"], spec["storage"], args.step_kernel)
    mb = MEASURED_DRAM_BYTES_PER_NODE.get((sp, spec["storage"], spec["key"]))
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None if mb is None else mb * N, "peak_kind": peak_kind,
            "kernel": "one LBM step: " + PASS_KERNELS[sp], "bytes_per_node": bpn,
            "traffic_note": TRAFFIC_NOTE.get((sp, spec["storage"], spec["key"]), NO_CAPTURE), "step_ms": step_ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cslbm", choices=["cslbm", "reference"])
    ap.add_argument("--workload", default="target256",
                    choices=["target256", "dynamic", "slab256", "crop64", "batch64", "adjoint64", "lgrad", "d2q9"])
    ap.add_argument("--adjoint-steps", type=int, default=ADJOINT_STEPS,
                    help="LBM steps of the adjoint objective (adjoint64 workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward step-time ratio")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 128x128x256 dynamic channel reported beside the 256^3 line")
    ap.add_argument("--snapshots", type=int, default=3)
    ap.add_argument("--step-kernel", default="auto", choices=["auto", "rows", "flat"])
    ap.add_argument("--storage", default=None, choices=["fp32", "fp16", "bf16", "fp64"],
                    help="storage of the populations (default: the workload's, FP32)")
    ap.add_argument("--oracle-c1", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_c1:  # the child process of oracle_single_thread
        v, secs = oracle_c1_sample()
        print(json.dumps({"value": v, "secs": secs}), flush=True)
        return None
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return bench_batch(args)
    if args.workload in ("adjoint64", "lgrad"):
        return bench_side(args)
    if args.workload == "d2q9":
        return bench_d2q9(args)

    import torch

    rank, world, local = dist_setup(args)
    spec = workload_spec(args.workload)
    if args.storage:
        spec["storage"] = args.storage
        spec["label"] = spec["label"].replace(
            "FP32", args.storage.upper() + (" weight-shifted storage, FP32 arithmetic" if args.storage in ("fp16", "bf16")
                                            else " storage"))
    r = channel_cycles(spec, args, rank, world, local, args.steps)
    lat, N = r["lat"], r["N"]
    ms_per_step = r["ms"] / args.steps
    value = whole_job_mlups(world, N, STEPS_PER_CYCLE * args.steps, r["ms"])
    state_gb = BYTES_PER_NODE[spec["storage"]] * N / 1e9
    e2e = None if args.no_e2e else end_to_end(args, lat, r["snaps"], N, world, mixed=spec["storage"] != "fp64")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if spec["storage"] == "fp32" else spec["storage"], "data": "synthetic",
        "config": {"workload": spec["label"], "nodes": N, "lbm_steps_per_step": STEPS_PER_CYCLE,
                   "l2": f"inputs > L2 ({state_gb:.1f} GB of state per LBM step), no flush",
                   "chart_inputs": ("g FP64, dg and J FP32 (cslbm_update_metric_mixed: the state of FP64 inputs, "
                                    "bit for bit)" if spec["storage"] != "fp64" else "g, dg, J FP64"),
                   "state_finite_after_run": r["ok"]},
        "roofline": roofline_of(spec, args, N, r["step_ms"]),
        "e2e": e2e,
        "gpu_launches": r["launches"],
        "clocks": r["clk"],
    }
    if rank == 0 and world == 1:
        line["lattice_gradient"] = lattice_gradient_report(lat, r["dev"][0]["g6"])
        line["transform_interp"] = transform_interp_report(lat, r["dev"], r["w"]["layout"])
    del lat, r
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.workload == "target256" and not args.no_secondary:
        # the dynamic channel of the plain FP32 form, beside the target line
        s2 = workload_spec("dynamic")
        if args.storage:
            s2["storage"] = args.storage
        r2 = channel_cycles(s2, args, rank, world, local, max(3, args.steps // 2))
        k2 = max(3, args.steps // 2)
        line["dynamic_channel"] = {"workload": s2["label"], "value": whole_job_mlups(1, r2["N"], STEPS_PER_CYCLE * k2,
                                                                                    r2["ms"]),
                                   "unit": UNIT, "ms_per_step": r2["ms"] / k2, "steps": k2,
                                   "roofline": roofline_of(s2, args, r2["N"], r2["step_ms"]),
                                   "state_finite_after_run": r2["ok"]}
        del r2
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_report(args.step_kernel)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups, secs, n, cores = oracle_cycle_sample(spec, 2, 0)
        line["cpu_baseline"] = {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n[0]}x{n[1]}x{n[2]} crop of the same generator, 2 cycles "
                                          f"(transform + {STEPS_PER_CYCLE} steps + reductions), FP64",
                                "cpu": cpu_model()}
        # secondary oracle timings: a failure is reported in the line, not raised
        try:
            line["cpu_baseline"]["single_thread"] = oracle_single_thread()
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"]["single_thread"] = {"error": str(e)[-300:]}
        try:
            grad_cpu, trans_cpu = oracle_side_samples(spec)
            line["lattice_gradient"]["cpu_baseline"] = grad_cpu
            line["transform_interp"]["cpu_baseline"] = trans_cpu
        except Exception as e:  # noqa: BLE001
            line["lattice_gradient"]["cpu_baseline"] = {"error": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def end_to_end(args, lat, snaps, N, world, mixed=True):
    """The same cycles through the public API with every cycle's inputs
    copied from pinned host buffers: the metric, its derivatives, the
    Jacobian and the face velocities go host -> device on a copy stream into
    one of two device buffers while the previous cycle computes (the next
    cycle's chart change waits for its copy), and the mass and wall force are
    read back every cycle.  All copies and reads are inside the timed
    region.  With `mixed` (FP32-arithmetic storage) the derivatives and the
    Jacobian travel in FP32 and the chart change is
    cslbm_update_metric_mixed, which leaves the same state as the FP64-input
    call (the library rounds both to FP32 before use): 156 instead of 264
    bytes per node over a host link of about 210 GB/s."""
    import torch
    keys = ("g6", "dg18", "J9")
    dtype = {"g6": torch.float64, "dg18": torch.float32 if mixed else torch.float64,
             "J9": torch.float32 if mixed else torch.float64}
    pinned = []
    for ch, faces in snaps:
        p = {}
        for k in keys:
            p[k] = torch.empty(getattr(ch, k).shape, dtype=dtype[k], pin_memory=True)
            p[k].numpy()[...] = getattr(ch, k)
        p["faces"] = {}
        for key, u in faces.items():
            t = torch.empty(u.shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = u
            p["faces"][key] = t
        pinned.append(p)
    h2d = sum(pinned[1][k].numel() * pinned[1][k].element_size() for k in keys) + \
        sum(u.numel() * 8 for u in pinned[1]["faces"].values())
    d2h = 4 * 8
    dev = [{k: torch.empty_like(pinned[1][k], device="cuda") for k in keys} for _ in range(2)]
    for d in dev:
        d["faces"] = {key: torch.empty_like(u, device="cuda") for key, u in pinned[1]["faces"].items()}
    copy = torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    for e in free:
        e.record(lat.stream)

    def upload(k, slot):
        p = pinned[1 + k % args.snapshots]
        with torch.cuda.stream(copy):
            copy.wait_event(free[slot])
            for name in keys:
                dev[slot][name].copy_(p[name], non_blocking=True)
            for key, u in p["faces"].items():
                dev[slot]["faces"][key].copy_(u, non_blocking=True)
            ready[slot].record(copy)

    def run(k0, count):
        upload(k0, k0 % 2)
        for k in range(k0, k0 + count):
            slot = k % 2
            if k + 1 < k0 + count:
                upload(k + 1, 1 - slot)
            lat.stream.wait_event(ready[slot])
            d = dev[slot]
            if mixed:
                lat.update_metric_mixed(d["g6"], d["dg18"], d["J9"])
            else:
                lat.update_metric(d["g6"], d["dg18"], d["J9"])
            for (a, s), u in d["faces"].items():
                lat.set_boundary_velocity(a, s, u)
            free[slot].record(lat.stream)
            lat.step(STEPS_PER_CYCLE)
            lat.total_mass()
            lat.wall_force(0, 1)

    run(0, 2)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    run(2, args.steps)
    torch.cuda.synchronize()
    t_e2e = reduce_max(time.perf_counter() - t0, world)
    barrier(world)
    return {"value": world * N * STEPS_PER_CYCLE * args.steps / t_e2e / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "note": "inputs copied host -> device on a second stream, double-buffered, overlapping the previous "
                    "cycle's steps" + ("; metric FP64, its derivatives and the Jacobian FP32 "
                                       "(cslbm_update_metric_mixed, the same state as FP64 inputs)" if mixed else "")}


if __name__ == "__main__":
    main()
