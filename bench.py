"""Benchmark of the representative-particle coagulation step on GB300.

One step = one pass of the whole hot path over the disk: equal-count regrid,
per-cell Zsom & Dullemond collision chain to t + dt, transport over dt.
Metric: collision events per second (and simulated years per second), mixed
precision (FP32 rates, FP64 masses/clock/row sums) beside the plain FP64 path
on the same state.

Workload: the paper's Benchmark-table disk at 256 radial x 16 vertical cells x
200 particles (819,200 particles, 4,096 cells), dt = 1 yr, starting from a
synthetic growth/fragmentation-balance state (workloads.midrun_state).  The
working set (about 100 MB) is below the 129 MB L2, so a 512 MB buffer is
written between timed steps and each step is timed alone with CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent disk (seed + rank): the work
shards by disk with no data-path collective (weak scaling); the collective is
used only for the barrier and the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "collision events/s & sim-yr/s on 1 GB300, FP32-mixed vs FP64 at fixed error"
UNIT = "events/s"
FLOPS_PER_ENTRY = 60          # FP32 flops of one kernel entry + rate weight (FMA = 2, div/sqrt = 1)
REGRID_BYTES = 92             # algorithmic bytes per particle per regrid
TRANSPORT_BYTES = 44          # algorithmic bytes per particle per transport
SMS, FP32_LANES = 152, 128


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), float(mp.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region: the sampler
    starts first and the region waits (up to 3 s) for its first sample; only
    samples stamped between start() and stop() count (the nearest one when
    the region is shorter than the sampling period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.perf_counter() + 3.0
            while not self.rows and time.perf_counter() < deadline:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        self.t0 = time.perf_counter()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def __exit__(self, *a):
        self.t1 = time.perf_counter()
        if self.proc:
            time.sleep(2e-3 * self.PERIOD_MS)  # one more sample past the end
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [r for t, r in self.rows if self.t0 is not None and self.t0 <= t <= self.t1]
        if not rows and self.rows and self.t0 is not None:  # region shorter than the period: the nearest sample
            rows = [min(self.rows, key=lambda tr: abs(tr[0] - 0.5 * (self.t0 + self.t1)))[1]]
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows if len(r) > 8 for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm),
                "window_ms": 1e3 * (self.t1 - self.t0) if self.t0 is not None and self.t1 else None}


def measured_traffic(name: str):
    """DRAM bytes per launch recorded from an ncu capture (profiles/traffic.json),
    or None when the kernel's source changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[name]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != rec["sha1"]:
                return None
        return float(rec["bytes_per_launch"])
    except Exception:
        return None


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def aggregate(total_ms: float, events: int, device=None):
    """Whole-job numbers over ranks: the slowest rank's time and the summed
    events.  A timing reduction only; the disks share no data."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, events
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    e = torch.tensor([float(events)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t[0]), int(e[0])


def rank_seed(base: int, rank: int) -> int:
    """Each rank simulates its own disk: same physics, its own random stream."""
    return base + rank


def workload(args):
    from paper_2507_21239_gb300 import workloads as W
    wl = W.WORKLOADS[args.workload]
    grid = (wl["n_r"], wl["n_z"], wl["per_cell"])
    return W, wl, wl["params"], grid


def make_state(args, ctx_or_none, rank):
    """Synthetic mid-run state: m, r, z from the recipe; M, id from the initial state."""
    W, wl, P, grid = workload(args)
    N = grid[0] * grid[1] * grid[2]
    m, r, z = W.midrun_state(P, N, seed=rank_seed(wl["seed"], rank))
    return P, grid, N, m, r, z


def cpu_model() -> str:
    """The host CPU: lscpu's model name, else /proc/cpuinfo's, else the architecture."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def cpu_oracle_steps(P, grid, state, seed, step0, dt, budget_s, max_steps, min_steps=1, cores=None):
    """Time full oracle steps (regrid, collide, transport) on the host cores
    (all of them unless cores is given)."""
    import oracle
    s = oracle.DiskState(*[np.copy(a) for a in state])
    cores = cores or os.cpu_count() or 1
    steps, ev0, t0 = 0, 0, time.perf_counter()
    elapsed = 0.0
    while steps < max_steps and (steps < min_steps or elapsed < budget_s):
        oracle.run(P, grid[0], grid[1], s, step0 * dt, dt, step0, 1, seed, nthreads=cores)
        step0 += 1
        steps += 1
        elapsed = time.perf_counter() - t0
    return s.events - ev0, elapsed, steps, cores


def run_reference(args):
    """The oracle on the host cores, on this arm's workload and metric."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    W, wl, P, grid = workload(args)
    N = grid[0] * grid[1] * grid[2]
    s0 = oracle.init_disk(P, N, seed=wl["seed"])
    m, r, z = W.midrun_state(P, N, seed=wl["seed"])
    state = (m, s0.M, r, z, s0.id)
    dt = args.dt_yr * W.YR
    # warm-up steps (untimed), then K timed steps, each one full disk step
    import oracle as O
    s = O.DiskState(*state)
    cores = os.cpu_count() or 1
    for k in range(args.warmup):
        O.run(P, grid[0], grid[1], s, k * dt, dt, k, 1, wl["seed"], nthreads=cores)
    ev0 = s.events
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.run(P, grid[0], grid[1], s, (args.warmup + k) * dt, dt, args.warmup + k, 1, wl["seed"], nthreads=cores)
    el = time.perf_counter() - t0
    ev = s.events - ev0
    value = ev / el if el > 0 else 0.0
    sample = f"{args.steps} full oracle steps (dt = {args.dt_yr} yr) of the {N:,}-particle disk from the mid-run state"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "sim_yr_per_s": args.steps * args.dt_yr / el if el > 0 else 0.0,
            "config": {"workload": args.workload, "particles": N, "cells": grid[0] * grid[1], "dt_yr": args.dt_yr,
                       "state": "synthetic growth/fragmentation-balance state (workloads.midrun_state)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(mcd, d, dt, K, stream, flush, trace=True):
    """K steps, each timed alone with CUDA events after an L2 flush."""
    import torch
    times, phases = [], []
    for k in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mcd.mcd_step(d.ctx, dt)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        if trace:
            phases.append(mcd.mcd_trace_read(d.ctx))
    return np.array(times), np.array(phases) if phases else None


def run_ours(args):
    import torch
    from paper_2507_21239_gb300 import build as B, mcd
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    B.build()
    W, wl, P, grid = workload(args)
    N = grid[0] * grid[1] * grid[2]
    seed = rank_seed(wl["seed"], rank)
    dt = args.dt_yr * W.YR
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(max(args.flush_mb, 1) << 20, dtype=torch.uint8, device=dev)
    _, _, _, m, r, z = make_state(args, None, rank)

    def fresh(prec):
        d = mcd.Disk(P, grid, seed=seed, prec=prec, stream=stream)
        p = d.particles()
        mcd.mcd_set_particles(d.ctx, 0, m, p["M"], r, z, p["id"])
        return d, p

    # ---- mixed precision, device-resident inputs ---------------------------
    d, p0 = fresh("mixed")
    mcd.mcd_trace(d.ctx, True)
    for _ in range(args.warmup):
        mcd.mcd_step(d.ctx, dt)
    torch.cuda.synchronize()
    st0 = mcd.mcd_get_stats(d.ctx, 0)
    l0 = mcd.mcd_get_launch_count(d.ctx)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and vis.split(",")[0].strip().isdigit():
        gpu_index = int(vis.split(",")[local].strip())
    with ClockSampler(gpu_index) as clk:
        times, phases = timed_steps(mcd, d, dt, args.steps, stream, flush)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    st1 = mcd.mcd_get_stats(d.ctx, 0)
    launches = mcd.mcd_get_launch_count(d.ctx) - l0
    status = mcd.mcd_sync(d.ctx)
    events = st1.events - st0.events
    total_ms = float(times.sum())
    total_ms, events = aggregate(total_ms, events, device=dev)
    value = events / (total_ms * 1e-3)
    yr_per_s = args.steps * args.dt_yr / (total_ms * 1e-3)
    # cell populations for the algorithmic flop count of the collide kernel
    off = np.zeros(grid[0] * grid[1] + 1, np.int64)
    mcd.mcd_get_cells(d.ctx, 0, off, None, None)
    n_c = np.diff(off).astype(np.float64)
    ev_step = (st1.events - st0.events) / args.steps
    ph = phases.mean(axis=0)  # regrid, order, collide, transport [ms]
    hbm, mhz, src = peaks()
    fp32_peak = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12  # TFLOP/s
    entries = float(np.sum(n_c * (n_c + 1) / 2) + n_c.mean() * ev_step)
    coll = {"bound": "alu", "achieved": entries * FLOPS_PER_ENTRY / (ph[2] * 1e-3) / 1e12, "peak": fp32_peak,
            "unit": "TFLOP/s", "traffic": measured_traffic("k_collide<float>"), "kernel": "k_collide<float>"}
    reg = {"bound": "hbm", "achieved": REGRID_BYTES * N / (ph[0] * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
           "traffic": measured_traffic("regrid"), "kernel": "regrid (k_regrid_keys, k_radix_*, k_zone)"}
    tra = {"bound": "hbm", "achieved": TRANSPORT_BYTES * N / (ph[3] * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
           "traffic": measured_traffic("k_transport<true>"), "kernel": "k_transport<true>"}
    for x in (coll, reg, tra):
        x["frac"] = x["achieved"] / x["peak"]
        x["peak_source"] = src
    dom = max(((ph[2], coll), (ph[0], reg), (ph[3], tra)), key=lambda a: a[0])[1]
    d.close()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
           "sim_yr_per_s": yr_per_s, "status": mcd.mcd_strerror(status),
           "config": {"workload": args.workload, "particles_per_gpu": N, "cells_per_gpu": grid[0] * grid[1],
                      "dt_yr": args.dt_yr, "precision": "mixed",
                      "state": "synthetic growth/fragmentation-balance state (workloads.midrun_state)",
                      "l2": f"{args.flush_mb} MB buffer written between timed steps; each step timed alone",
                      "graph": "step replayed as one CUDA graph", "parallelism": f"{world} independent disks"},
           "phases_ms": {"regrid": ph[0], "order": ph[1], "collide": ph[2], "transport": ph[3]},
           "roofline": dom, "roofline_all": {"collide": coll, "regrid": reg, "transport": tra},
           "gpu_launches": int(launches), "events_per_step": ev_step}

    if rank == 0 and not args.no_fp64:
        # ---- plain FP64 path on the same state --------------------------------
        d64, _ = fresh("fp64")
        mcd.mcd_trace(d64.ctx, True)
        for _ in range(min(args.warmup, 2)):
            mcd.mcd_step(d64.ctx, dt)
        torch.cuda.synchronize()
        s0 = mcd.mcd_get_stats(d64.ctx, 0)
        k64 = max(1, min(args.steps, args.fp64_steps))
        t64, ph64 = timed_steps(mcd, d64, dt, k64, stream, flush)
        s1 = mcd.mcd_get_stats(d64.ctx, 0)
        v64 = (s1.events - s0.events) / (t64.sum() * 1e-3)
        out["fp64"] = {"value": v64, "unit": UNIT, "steps": k64, "ms_per_step": float(t64.mean()),
                       "sim_yr_per_s": k64 * args.dt_yr / (t64.sum() * 1e-3),
                       "phases_ms": dict(zip(("regrid", "order", "collide", "transport"), ph64.mean(axis=0).tolist())),
                       "mixed_over_fp64_events_per_s": value / world / v64 if v64 > 0 else None}
        d64.close()

    if rank == 0 and not args.no_e2e:
        # ---- end to end through the C ABI with pinned host buffers -----------
        de, pe = fresh("mixed")
        for _ in range(args.warmup):
            mcd.mcd_step(de.ctx, dt)
        hm = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
        hM = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
        hr = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
        hz = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
        hid = torch.empty(N, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
        mcd.mcd_get_particles(de.ctx, 0, hm, hM, hr, hz, hid, mcd.MCD_HOST)
        s0 = mcd.mcd_get_stats(de.ctx, 0)
        ke = max(1, min(args.steps, args.e2e_steps))
        wall = 0.0
        for k in range(ke):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mcd.mcd_set_particles(de.ctx, 0, hm, hM, hr, hz, hid, mcd.MCD_HOST)
            mcd.mcd_step(de.ctx, dt)
            mcd.mcd_get_particles(de.ctx, 0, hm, hM, hr, hz, hid, mcd.MCD_HOST)
            wall += time.perf_counter() - t0
        s1 = mcd.mcd_get_stats(de.ctx, 0)
        out["e2e"] = {"value": (s1.events - s0.events) / wall, "unit": UNIT, "h2d_bytes_per_step": 36 * N,
                      "d2h_bytes_per_step": 36 * N, "steps": ke, "ms_per_step": 1e3 * wall / ke}
        de.close()

    if rank == 0 and not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        s = oracle.init_disk(P, N, seed)
        ev, el, steps, cores = cpu_oracle_steps(P, grid, (m, s.M, r, z, s.id), seed, 0, dt,
                                                budget_s=args.cpu_budget_s, max_steps=50)
        ev1, el1, steps1, _ = cpu_oracle_steps(P, grid, (m, s.M, r, z, s.id), seed, 0, dt,
                                               budget_s=0.2 * args.cpu_budget_s, max_steps=10, cores=1)
        out["cpu_baseline"] = {"value": ev / el, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{steps} full oracle step(s) (dt = {args.dt_yr} yr) of the same "
                                         f"{N:,}-particle mid-run disk, {el:.1f} s",
                               "cpu": cpu_model(),
                               "single_core": {"value": ev1 / el1, "unit": UNIT, "cores": 1,
                                               "sample": f"{steps1} full oracle step(s), {el1:.1f} s"}}
    out["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batched(args):
    """The 64-disk batch (workloads.batched_disks) in one context: mixed path,
    one mid-run state per disk, whole-batch events/s over timed steps.  A
    measurement of that configuration, not the benchmark line."""
    import torch
    from paper_2507_21239_gb300 import build as B, mcd, workloads as W
    torch.cuda.set_device(0)
    B.build()
    disks = W.batched_disks()
    params = [x["params"] for x in disks]
    grids = [(x["n_r"], x["n_z"], x["per_cell"]) for x in disks]
    stream = torch.cuda.Stream()
    flush = torch.empty(max(args.flush_mb, 1) << 20, dtype=torch.uint8, device="cuda")
    d = mcd.Disk(params, grids, seed=0, prec="mixed", stream=stream)
    for k, g in enumerate(grids):
        m, r, z = W.midrun_state(params[k], g[0] * g[1] * g[2], seed=k)
        p = d.particles(k)
        mcd.mcd_set_particles(d.ctx, k, m, p["M"], r, z, p["id"])
    dt = args.dt_yr * W.YR
    mcd.mcd_trace(d.ctx, True)
    for _ in range(args.warmup):
        mcd.mcd_step(d.ctx, dt)
    torch.cuda.synchronize()
    events = lambda: sum(d.stats(k).events for k in range(len(disks)))
    ev0, l0 = events(), mcd.mcd_get_launch_count(d.ctx)
    with ClockSampler(0) as clk:
        times, phases = timed_steps(mcd, d, dt, args.steps, stream, flush)
    torch.cuda.synchronize()
    ev = events() - ev0
    launches = mcd.mcd_get_launch_count(d.ctx) - l0
    status = mcd.mcd_sync(d.ctx)
    total_ms = float(times.sum())
    ph = phases.mean(axis=0)
    n = sum(g[0] * g[1] * g[2] for g in grids)
    out = {"metric": METRIC, "value": ev / (total_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "dtype": "f32+f64 (mixed)", "data": "synthetic", "status": mcd.mcd_strerror(status),
           "config": {"workload": "batched64", "disks": len(disks), "particles": n,
                      "cells": sum(g[0] * g[1] for g in grids), "dt_yr": args.dt_yr,
                      "state": "workloads.midrun_state per disk (seed = disk)"},
           "events_per_step": ev / args.steps,
           "phases_ms": {"regrid": ph[0], "order": ph[1], "collide": ph[2], "transport": ph[3]},
           "gpu_launches": launches, "clocks": clk.summary()}
    d.close()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="disk2d_256x16x200",
                    help="a workloads.WORKLOADS name, or batched64 (the 64-disk batch, mixed path only)")
    ap.add_argument("--dt-yr", dest="dt_yr", type=float, default=1.0)
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--flush-mb", type=int, default=512, help="L2 flush buffer written between timed steps")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
