"""Benchmark of the Oregonator time-stepper (GCUPS and fraction of HBM roofline).

Workload (one bench step = one pass of the whole hot path over one input):
  8192 x 8192 grid, Table 1 kinetics, uniform phi = 0.054 plus 200 seeded
  u = 0.8 disks (radius U{4..10}, centres uniform, PCG64 seed 3), FP32 compute
  and storage: stimulate the 200 disks, advance 10000 explicit Euler steps
  with the single-step kernel, run the health check.  The state (1.34 GB)
  is far larger than L2 (129 MB), so no flush is needed between steps.

The JSON line also reports temporal blocking (k steps per launch) and the
reduced-storage modes as effective GCUPS on the same grid, the end-to-end
rate through the C ABI with host buffers (phi in, state out, every step),
the 512-grid parameter sweep (batched kernels, one CUDA graph), the
64-session serving workload (p50/p99 frame latency) and its loaded variant
(all 64 sessions live, each asking 60 frames per second), the colour map's rate,
and the FP64 oracle timed on the host cores as a baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs its own independent copy of the
workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rdc_inputs as ri  # noqa: E402

W = H = 8192
EULER_STEPS = 10000
N_DISKS = 200
DISK_SEED = 3
BYTES_PER_CELL = {"f32": 20, "bf16": 12, "f16": 12, "f64": 40}
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth
STORAGE_TYPE = {"f32": "float", "f64": "double", "bf16": "__nv_bfloat16", "f16": "__half"}
METRIC = "GCUPS (cell-updates/s)"


# Sources that define the single-step kernel; a traffic figure measured on
# other sources is stale.
KERNEL_SOURCES = ["paper_1901_06535_gb300/csrc/rdc_device.cuh",
                  "paper_1901_06535_gb300/csrc/rdc_step_impl.cuh"]


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic(kernel: str, cells: int):
    """DRAM bytes (read + write) per launch from the recorded ncu capture, or
    None when there is none or the kernel changed since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("sources_sha256") != kernel_sources_sha256():
        return None
    return rec["bytes_per_cell"] * cells


def record_traffic(csv_path: str) -> dict:
    """The traffic record of the single-step FP32 kernel from an ncu CSV log of
    `dram__bytes_read.sum`, `dram__bytes_write.sum` and `gpu__time_duration.sum`
    over launches of k_step1<float> on the default grid, keyed to the SHA-256
    of the kernel's sources as they are when this runs (right after the
    capture, on the same tree)."""
    import csv
    rows = []
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        if "k_step1<float" in r.get("Kernel Name", ""):
            rows.append(r)
    by_id = {}
    for r in rows:
        val = float(r["Metric Value"].replace(",", ""))
        unit = r.get("Metric Unit", "")
        scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(unit, 1.0)
        by_id.setdefault(r["ID"], {})[r["Metric Name"]] = val * scale
    launches = [m for m in by_id.values()
                if "dram__bytes_read.sum" in m and "dram__bytes_write.sum" in m]
    if not launches:
        raise SystemExit(f"no k_step1<float> launches with DRAM counters in {csv_path}")
    rd = float(np.mean([m["dram__bytes_read.sum"] for m in launches]))
    wr = float(np.mean([m["dram__bytes_write.sum"] for m in launches]))
    return {"k_step1<float>": {
        "bytes_per_cell": (rd + wr) / (W * H),
        "dram_bytes_read_per_launch": rd, "dram_bytes_write_per_launch": wr,
        "launches": len(launches), "grid": [W, H],
        "command": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,"
                   "gpu__time_duration.sum --clock-control none -k regex:k_step1 -s 5 -c 2 "
                   "--csv --log-file <csv> python bench.py --steps 1 --warmup 3 "
                   "--no-cpu-baseline --no-extras --euler-steps 50; "
                   "python bench.py --record-traffic <csv>",
        "sources_sha256": kernel_sources_sha256(),
        "note": "mean over the captured launches (both sweep directions); ncu flushes "
                "the caches before each launch"}}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------

def dist_setup(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(cells_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job GCUPS: every rank advanced its own copy of the workload, the
    job took as long as the slowest rank."""
    return world * cells_per_rank / t_max / 1e9


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_gcups(target_s: float = 15.0, steps: int | None = None):
    """Times the FP64 oracle on the host cores on the 8192^2 workload for a
    bounded number of Euler steps; returns (gcups, threads, steps)."""
    import oracle
    orc = oracle.load()
    threads = os.cpu_count() or 1
    phi = np.full((H, W), ri.PHI_ACTIVE)
    us = orc.rest_state(ri.PHI_ACTIVE)
    u = np.full((H, W), us)
    v = u.copy()
    for (cx, cy, r) in ri.random_disks(DISK_SEED, N_DISKS, W, H):
        orc.seed_disk(u, cx, cy, r, ri.SEED_VALUE)
    if steps is None:
        t0 = time.perf_counter()
        orc.run(phi, u, v, 1, nthreads=threads)
        one = time.perf_counter() - t0
        steps = max(1, int(target_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    orc.run(phi, u, v, steps, nthreads=threads)
    dt = time.perf_counter() - t0
    return W * H * steps / dt / 1e9, threads, steps


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each "step" of the reference arm: the oracle on the full grid for a
    # bounded number of Euler steps (sized so the whole run stays short)
    gc, threads, steps = oracle_gcups(target_s=8.0)
    vals = []
    for i in range(args.warmup + args.steps):
        g, _, _ = oracle_gcups(steps=steps)
        if i >= args.warmup:
            vals.append(g)
    value = float(np.median(vals)) if vals else gc
    sample = f"FP64 oracle, {W}x{H} grid, {steps} Euler steps per bench step, {threads} threads"
    line = {"metric": METRIC, "value": value, "unit": "GCUPS", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"oregonator_{W}x{H}_phi0.054_200disks", "grid": [W, H],
                       "euler_steps_per_bench_step": steps, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--euler-steps", type=int, default=EULER_STEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the temporal-blocking / storage-mode / e2e lines")
    ap.add_argument("--kblock", type=int, default=1,
                    help="Euler steps per launch of the timed kernel (1 = single-step kernel)")
    ap.add_argument("--grid", type=int, default=None,
                    help="square grid size (default 8192); smaller sizes are for profiling")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "bf16", "f16"],
                    help="storage of the timed run (default f32; the others are for profiling)")
    ap.add_argument("--stoch", action="store_true",
                    help="stochastic rounding of the 16-bit storage (profiling)")
    ap.add_argument("--only", default=None, choices=["batch", "render", "serve"],
                    help="profiling: run one extra alone and print its JSON (batch: "
                         "--batch-grids grids of the sweep, --euler-steps steps at the "
                         "fixed shape k=6, rows=16, krows=256, no autotuning; render: "
                         "the colour map of the --grid state; serve: both serving "
                         "workloads)")
    ap.add_argument("--batch-grids", type=int, default=512,
                    help="grids in the sweep of --only batch")
    ap.add_argument("--record-traffic", default=None, metavar="CSV",
                    help="print the traffic record (profiles/traffic.json) computed from "
                         "the ncu CSV log of a capture of k_step1<float>, keyed to the "
                         "current kernel sources, and exit")
    args = ap.parse_args()
    if args.record_traffic:
        print(json.dumps(record_traffic(args.record_traffic), indent=1))
        return 0
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.grid:
        global W, H
        W = H = int(args.grid)
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)

    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    import paper_1901_06535_gb300 as pkg
    pkg.lib()

    # a dedicated stream: the simulation and the CUDA events share it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    p = pkg.rdc_params_default(precision=args.precision, k_block=args.kblock,
                               flags=4 if args.stoch else 0)
    h = pkg.rdc_create(W, H, p, None, stream.cuda_stream)
    disks = ri.random_disks(DISK_SEED, N_DISKS, W, H)
    nE = args.euler_steps

    def one_step(ev=None):
        for (cx, cy, r) in disks:
            pkg.rdc_seed(h, cx, cy, r, ri.SEED_VALUE)
        if ev is not None:
            ev[0].record(stream)
        pkg.rdc_step(h, nE)
        if ev is not None:
            ev[1].record(stream)
        rc, _ = pkg.rdc_check(h)
        return rc

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    launches0 = pkg.rdc_get_view(h).launches

    clocks = ClockSampler(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    statuses = [one_step(evs[i]) for i in range(args.steps)]
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    step_kernel_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    launches = pkg.rdc_get_view(h).launches - launches0
    t_max = max_over_ranks(elapsed, world)

    cells = W * H * nE * args.steps
    value = weak_scaling_value(cells, world, t_max)
    ms_per_step = t_max / args.steps * 1e3
    peak, peak_kind = _peaks()
    per_launch_s = step_kernel_s / launches
    # one launch moves the state once whatever k is (k Euler steps per launch)
    bytes_per_launch = BYTES_PER_CELL[args.precision] * W * H
    achieved = bytes_per_launch / per_launch_s / 1e9

    # end to end through the C ABI right after the timed region, on the same
    # handle and under the same conditions (before the compute-heavy extras)
    e2e = None
    if not args.no_extras:
        e2e_clocks = ClockSampler(local)
        e2e_clocks.start()
        e2e = _e2e(pkg, stream, h, disks, nE, args)
        e2e["clocks"] = e2e_clocks.stop()

    extras = {}
    if rank == 0 and not args.no_extras:
        # temporal blocking and storage modes: effective GCUPS on the same grid
        tb = {"1": _mode_gcups(pkg, stream, "f32", 1, 1000)}
        for k in (2, 3, 4, 5, 6, 7, 8):
            tb[str(k)] = max(_mode_gcups(pkg, stream, "f32", k, 960 // k * k, krows=kr)
                             for kr in (64, 128))
        tuned = _tuned(pkg, stream, "f32")
        modes = {m: _mode_gcups(pkg, stream, m, 1, 1000) for m in ("bf16", "f16")}
        modes["bf16_tuned"] = _tuned(pkg, stream, "bf16")
        modes["f16_tuned"] = _tuned(pkg, stream, "f16")
        modes["f64"] = _mode_gcups(pkg, stream, "f64", 1, 100)
        # stochastic rounding to the 16-bit storage (RDC_STOCH_ROUND = 4)
        modes["bf16_stoch"] = _mode_gcups(pkg, stream, "bf16", 1, 1000, flags=4)
        modes["bf16_stoch_tuned"] = _tuned(pkg, stream, "bf16", flags=4)
        extras = {"temporal_blocking_gcups": tb, "tuned_f32": tuned, "storage_modes_gcups": modes,
                  "batch_sweep": _batch_sweep(pkg, stream), "serving": _serving(pkg),
                  "serving_loaded": _serving_loaded(pkg),
                  "render": _render(pkg, stream, h)}
    pkg.rdc_destroy(h)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, threads, steps = oracle_gcups(target_s=15.0)
        cpu = {"value": g, "unit": "GCUPS", "cores": threads, "kind": "oracle",
               "sample": f"FP64 oracle on the same {W}x{H} workload, {steps} Euler steps, "
                         f"{threads} host threads"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.precision, "data": "synthetic",
                "config": {"workload": f"oregonator_{W}x{H}_phi0.054_200disks",
                           "grid": [W, H], "euler_steps_per_bench_step": nE,
                           "kernel": ("single-step (k=1)" if args.kblock == 1 else
                                      f"temporally blocked (k={args.kblock})"),
                           "precision": args.precision,
                           "l2": "inputs larger than L2 (1.34 GB state), no flush"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak,
                             "peak_kind": peak_kind,
                             "nominal_peak": NOMINAL_HBM_GBS,
                             "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                             "traffic": (_traffic("k_step1<float>", W * H)
                                         if args.kblock == 1 and args.precision == "f32" else None),
                             "kernel": f"{'k_step1' if args.kblock == 1 else 'k_stepk_stream'}"
                                       f"<{STORAGE_TYPE[args.precision]}>",
                             "bytes_per_cell_update": BYTES_PER_CELL[args.precision],
                             "launch_us": per_launch_s * 1e6},
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": int(launches + args.steps * (N_DISKS + 1)),
                "health": [int(s) for s in statuses]}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _tuned(pkg, stream, mode, n=960, flags=0):
    """Autotuned shape on the 8192^2 grid and its GCUPS over n steps."""
    import torch
    prec = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3}[mode]
    h = pkg.rdc_create(W, H, pkg.rdc_params_default(precision=prec, flags=flags), None,
                       stream.cuda_stream)
    try:
        pkg.rdc_seed(h, W / 2, H / 2, 10.0, 0.8)
        shape, est = pkg.rdc_tune(h, 3)
        pkg.rdc_step(h, 3 * shape["k"])
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        pkg.rdc_step(h, n)
        b.record(stream)
        torch.cuda.synchronize()
        return {"gcups": W * H * n / (a.elapsed_time(b) / 1e3) / 1e9, "k": shape["k"],
                "variant": shape["variant"], "krows": shape["krows"], "rows": shape["rows"]}
    finally:
        pkg.rdc_destroy(h)


def _mode_gcups(pkg, stream, mode, k, n, krows=None, flags=0):
    import torch
    prec = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3}[mode]
    p = pkg.rdc_params_default(precision=prec, k_block=k, flags=flags)
    h = pkg.rdc_create(W, H, p, None, stream.cuda_stream)
    try:
        if krows is not None:
            s = pkg.rdc_get_shape(h)
            pkg.rdc_set_shape(h, s.bx, s.rows, s.tx, s.ty, s.nthreads, k, 0, krows)
        pkg.rdc_seed(h, W / 2, H / 2, 10.0, 0.8)
        pkg.rdc_step(h, 3 * k)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        pkg.rdc_step(h, n)
        b.record(stream)
        torch.cuda.synchronize()
        return W * H * n / (a.elapsed_time(b) / 1e3) / 1e9
    finally:
        pkg.rdc_destroy(h)


def _render(pkg, stream, h, reps=20):
    """Colour map of the bench grid into a device RGBA8 buffer (reads u, v and
    phi, 12 B per pixel in FP32, writes 4 B): pixels per second and the
    fraction of the measured copy peak."""
    import torch
    out = torch.empty((H, W, 4), dtype=torch.uint8, device="cuda")
    pkg.rdc_render(h, out=out)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        pkg.rdc_render(h, out=out)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3 / reps
    peak, kind = _peaks()
    gbs = 16.0 * W * H / sec / 1e9
    return {"gpix_per_s": W * H / sec / 1e9, "ms_per_frame": sec * 1e3, "gb_s": gbs,
            "frac": gbs / peak, "peak_kind": kind, "bytes_per_pixel": 16}


def _batch_sweep(pkg, stream, steps=5000, n_grids=512, shape=None):
    """Parameter sweep: 512 grids of sizes U{128, 256, 512, 1024}^2, phi ~
    U[0.05, 0.08], eps ~ U[0.02, 0.03], 1-8 disks each (PCG64 seed 4); the
    autotuner picks the launch shape (or `shape` = (k, rows, krows) fixes
    it), then `steps` Euler steps run as one CUDA graph of persistent
    launches over all grids."""
    import torch
    spec = ri.sweep_batch(seed=4, n_grids=n_grids)
    grids = [(n, n) for n in spec.sizes]
    params = [pkg.rdc_params_default(precision=0, eps=e) for e in spec.eps]
    phis = [np.full((n, n), ph, dtype=np.float32) for n, ph in zip(spec.sizes, spec.phi)]
    b = pkg.rdc_batch_create(grids, params, phis, stream=stream.cuda_stream)
    try:
        for i, disks in enumerate(spec.disks):
            for (cx, cy, r) in disks:
                pkg.rdc_batch_seed(b, i, cx, cy, r, ri.SEED_VALUE)
        t0 = time.perf_counter()
        if shape is None:
            info = pkg.rdc_batch_tune(b, 3)
        else:
            pkg.rdc_batch_set_config(b, *shape, True)
            info = pkg.rdc_batch_get_info(b)
        tune_s = time.perf_counter() - t0
        pkg.rdc_batch_step(b, None, steps)          # captures the graph (and warms up)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pkg.rdc_batch_step(b, None, steps)          # graph replay
        z.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(z) / 1e3
        bad = [i for i in range(len(grids)) if pkg.rdc_batch_check(b, i)[0] != 0]
        cells = float(sum(n * n for n in spec.sizes))
        healthy = cells - float(sum(spec.sizes[i] ** 2 for i in bad))
    finally:
        pkg.rdc_batch_destroy(b)
    # the grids that crossed the pole (u + q <= 0), replayed alone up to the
    # first step whose state fails the health check (same bits as in the batch)
    first_bad = {}
    for i in bad:
        first_bad[str(i)] = _first_bad_step(pkg, stream, spec, i, 2 * steps)
    return {"gcups": cells * steps / sec / 1e9, "seconds": sec, "grids": len(grids),
            "cells": cells, "steps": steps, "k": info.k, "rows": info.rows,
            "krows": info.krows, "tuned_gcups": info.tuned_gcups,
            "tune_seconds": tune_s, "unhealthy_grids": bad,
            "gcups_healthy_grids_only": healthy * steps / sec / 1e9,
            "first_bad": first_bad}


def _first_bad_step(pkg, stream, spec, i, steps):
    """Step index and flat cell of the first unhealthy state of sweep grid i
    run alone (FP32, single steps, a health check after each), or None."""
    n = spec.sizes[i]
    p = pkg.rdc_params_default(precision=0, eps=spec.eps[i], k_block=1)
    phi = np.full((n, n), spec.phi[i], dtype=np.float32)
    h = pkg.rdc_create(n, n, p, phi, stream.cuda_stream)
    try:
        for (cx, cy, r) in spec.disks[i]:
            pkg.rdc_seed(h, cx, cy, r, ri.SEED_VALUE)
        for s in range(1, steps + 1):
            pkg.rdc_step(h, 1)
            rc, cell = pkg.rdc_check(h)
            if rc != 0:
                return {"step": s, "cell": int(cell)}
        return None
    finally:
        pkg.rdc_destroy(h)


def run_only(args):
    """One extra alone, for profiling its kernel on a small case."""
    import torch
    torch.cuda.set_device(0)
    import paper_1901_06535_gb300 as pkg
    pkg.lib()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.only == "batch":
        out = _batch_sweep(pkg, stream, steps=args.euler_steps, n_grids=args.batch_grids,
                           shape=(6, 16, 256))
    elif args.only == "serve":
        out = {"serving": _serving(pkg), "serving_loaded": _serving_loaded(pkg)}
    else:
        h = pkg.rdc_create(W, H, pkg.rdc_params_default(precision=args.precision), None,
                           stream.cuda_stream)
        try:
            for (cx, cy, r) in ri.random_disks(DISK_SEED, N_DISKS, W, H):
                pkg.rdc_seed(h, cx, cy, r, ri.SEED_VALUE)
            pkg.rdc_step(h, args.euler_steps)
            out = _render(pkg, stream, h, reps=args.steps)
        finally:
            pkg.rdc_destroy(h)
    print(json.dumps({"only": args.only, **out}))


def _serving(pkg, frames=100, steps_per_frame=50):
    """Interactive serving: 64 sessions arriving Poisson at 20/s (seed 5),
    grids U{512, 1024, 2048}^2 with diode maps at random positions and
    orientations, each requesting `frames` frames of `steps_per_frame` steps
    with a u = 0.8 touch before each; continuous batching, one batch and
    stream per size class."""
    from paper_1901_06535_gb300 import serve
    specs = ri.diode_sessions(seed=5, n=64, frames=frames)
    sessions = [serve.Session(s.sid, s.size, s.size, phi=s.phi, frames=frames,
                              touches=s.touches) for s in specs]
    srv = serve.Server(precision=0, k_block=6, steps_per_frame=steps_per_frame)
    try:
        wall, st = serve.run_workload(sessions, [s.arrival for s in specs], srv)
    finally:
        srv.close()
    st["wall_seconds"] = wall
    st["gcups"] = st["cells_stepped"] / wall / 1e9
    st["sessions"] = len(sessions)
    st["frames_per_session"] = frames
    st["steps_per_frame"] = steps_per_frame
    return st


def _serving_loaded(pkg, fps=60.0, seconds=3.0, steps_per_frame=50, rate=64.0):
    """Interactive serving with every session live at once: the 64 diode
    sessions of the serving workload (same sizes, maps and touches), arriving
    Poisson at 64/s, each client asking for a frame at a fixed `fps` for
    `seconds` (a frame due while its previous one is still on the GPU waits,
    and its latency counts from its due time); continuous batching, one batch
    and stream per size class."""
    from paper_1901_06535_gb300 import serve
    frames = int(round(fps * seconds))
    specs = ri.diode_sessions(seed=5, n=64, frames=frames, rate=rate)
    sessions = [serve.Session(s.sid, s.size, s.size, phi=s.phi, frames=frames,
                              touches=s.touches, frame_period=1.0 / fps) for s in specs]
    srv = serve.Server(precision=0, k_block=6, steps_per_frame=steps_per_frame)
    try:
        wall, st = serve.run_workload(sessions, [s.arrival for s in specs], srv)
    finally:
        srv.close()
    st["wall_seconds"] = wall
    st["gcups"] = st["cells_stepped"] / wall / 1e9
    st["sessions"] = len(sessions)
    st["frames_per_session"] = frames
    st["frames_per_second_per_session"] = fps
    st["steps_per_frame"] = steps_per_frame
    st["arrival_rate_per_s"] = rate
    return st


def _e2e(pkg, stream, h, disks, nE, args):
    """Same metric through the C ABI with host buffers: each step uploads the
    phi map (pinned host memory; the library resets to the rest state),
    stimulates, steps, and reads u and v back into pinned host memory."""
    import torch
    phi = torch.full((H, W), ri.PHI_ACTIVE, dtype=torch.float32).pin_memory()
    uo = torch.empty((H, W), dtype=torch.float32).pin_memory()
    vo = torch.empty((H, W), dtype=torch.float32).pin_memory()
    steps = max(1, min(args.steps, 3))
    times = []
    for i in range(1 + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg.rdc_set_phi(h, phi)
        for (cx, cy, r) in disks:
            pkg.rdc_seed(h, cx, cy, r, ri.SEED_VALUE)
        pkg.rdc_step(h, nE)
        pkg.rdc_read(h, uo, vo)
        times.append(time.perf_counter() - t0)
    t = float(np.median(times[1:]))
    return {"value": W * H * nE / t / 1e9, "unit": "GCUPS",
            "h2d_bytes_per_step": W * H * 4 + 0, "d2h_bytes_per_step": 2 * W * H * 4,
            "steps": steps}


if __name__ == "__main__":
    sys.exit(main())
