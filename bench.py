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

The same line carries the other configurations of the metric as records
beside the benchmark number: "batched64" (64 independent disks in one
context, 28.5 M particles), "stress" (1024 x 32 cells x 400 particles,
alpha = 1e-2, v_frag = 1 m/s), both from mid-run states, and "full_run" (the
benchmark disk evolved from its all-monomer initial state for 1e4 yr).  The
collide kernel is reported against the FP32 ALU peak and against the
shared-memory bandwidth measured in the same run (mcd_probe_peaks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-extra] [--full-run-yr Y] [--peaks]

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
SMEM_BYTES_PER_EVENT_SWARM = 60   # shared-memory bytes per event and swarm of the cell (two scans, row/column i)
SMEM_BYTES_PER_ENTRY = 52         # shared-memory bytes per rate-matrix entry of a build (48-B swarm cache + 4-B dv)


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


def probe_peaks(stream=None) -> dict:
    """This GPU's shared-memory read bandwidth and FP32/FP64 FMA throughput,
    measured by the library's microbenchmarks (mcd_probe_peaks)."""
    from paper_2507_21239_gb300 import mcd
    return mcd.mcd_probe_peaks(stream)


def collide_smem_bytes(n_c, ev_c) -> float:
    """Algorithmic shared-memory bytes of one collide over cells of n_c swarms
    with ev_c events each: every rate-matrix entry of a full build reads one
    swarm cache and one dv (SMEM_BYTES_PER_ENTRY); a build at the start and
    one every 4 n events; and per event ~60 n bytes (the two scans over the row
    sums and row i, row i read, the new row and column written, the row-sum
    updates and the caches read)."""
    n = np.asarray(n_c, np.float64)
    ev = np.asarray(ev_c, np.float64)
    live = n > 0
    builds = 1.0 + np.floor(ev[live] / (4.0 * n[live]))
    return float(np.sum(SMEM_BYTES_PER_ENTRY * n[live] ** 2 * builds + SMEM_BYTES_PER_EVENT_SWARM * n[live] * ev[live]))


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


def smi_index(local: int) -> int:
    """nvidia-smi's index of this process's GPU (CUDA_VISIBLE_DEVICES mapped)."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and vis.split(",")[0].strip().isdigit():
        return int(vis.split(",")[local].strip())
    return local


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


def pin_variant(mcd, d, spec: str):
    """Pin the mixed collide's variant instead of the timed trial's choice
    (for profiling one kernel): "S,store" (swarms per thread 1 or 2; dv store
    0 recompute, 1 shared memory, 2 workspace) or "cw,store" (control warp)."""
    shape, store = spec.split(",")
    if shape == "cw":
        mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_CONTROL_WARP, 1)
    else:
        mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_SWARMS_PER_THREAD, int(shape))
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DV_MATRIX, int(store))


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


def timed_steps(mcd, d, dt, K, stream, flush, trace=True, on_step=None):
    """K steps, each timed alone with CUDA events after an L2 flush; on_step(k),
    if given, runs after step k has finished, outside its timed interval."""
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
        if on_step is not None:
            on_step(k)
    return np.array(times), np.array(phases) if phases else None


def cell_loads(mcd, d, grids):
    """Every cell's swarm count and events in the last collide, over all disks."""
    ns, evs = [], []
    for k, g in enumerate(grids):
        C = g[0] * g[1]
        off = np.zeros(C + 1, np.int64)
        mcd.mcd_get_cells(d.ctx, k, off, None, None)
        ev = np.zeros(C, np.int64)
        mcd.mcd_get_cell_events(d.ctx, k, ev)
        ns.append(np.diff(off))
        evs.append(ev)
    return np.concatenate(ns), np.concatenate(evs)


def collide_rooflines(n_c, ev_c, n_steps, collide_ms, pk, fp32_unit_peak):
    """The collide kernel against the FP32 ALU peak (unit counts x clock) and
    against the measured shared-memory bandwidth; n_c, ev_c per cell and step
    (arrays of shape steps x cells), collide_ms the mean phase time."""
    entries = float(np.sum(n_c * (n_c + 1) / 2 + n_c * ev_c)) / n_steps
    sm_bytes = sum(collide_smem_bytes(n_c[k], ev_c[k]) for k in range(n_steps)) / n_steps
    t = collide_ms * 1e-3
    alu = {"bound": "alu", "achieved": entries * FLOPS_PER_ENTRY / t / 1e12, "peak": fp32_unit_peak,
           "unit": "TFLOP/s", "traffic": measured_traffic("k_collide<float>"), "kernel": "k_collide<float>",
           "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock (MEASURED_PEAKS.json)",
           "work": f"{FLOPS_PER_ENTRY} flop x {entries:.4g} kernel entries per step"}
    smem = {"bound": "smem", "achieved": sm_bytes / t / 1e9, "peak": pk["smem_gbs"], "unit": "GB/s",
            "traffic": None, "kernel": "k_collide<float>",
            "peak_source": "measured in this run (mcd_probe_peaks shared-memory read loop)",
            "work": f"{sm_bytes:.4g} algorithmic shared-memory bytes per step"}
    for x in (alu, smem):
        x["frac"] = x["achieved"] / x["peak"] if x["peak"] else None
    return alu, smem


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
        if prec == "mixed" and args.collide_variant:
            pin_variant(mcd, d, args.collide_variant)
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
    gpu_index = smi_index(local)
    loads = []  # (swarms, events) per cell of every timed step: the collide's algorithmic work
    with ClockSampler(gpu_index) as clk:
        times, phases = timed_steps(mcd, d, dt, args.steps, stream, flush,
                                    on_step=lambda k: loads.append(cell_loads(mcd, d, [grid])))
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
    ev_step = (st1.events - st0.events) / args.steps
    ph = phases.mean(axis=0)  # regrid, order, collide, transport [ms]
    hbm, mhz, src = peaks()
    pk = probe_peaks(stream)
    fp32_peak = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12  # TFLOP/s
    n_c = np.array([x[0] for x in loads], np.float64)
    ev_c = np.array([x[1] for x in loads], np.float64)
    coll, coll_smem = collide_rooflines(n_c, ev_c, args.steps, ph[2], pk, fp32_peak)
    reg = {"bound": "hbm", "achieved": REGRID_BYTES * N / (ph[0] * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
           "traffic": measured_traffic("regrid"), "kernel": "regrid (k_regrid_keys, k_radix_*, k_zone)",
           "peak_source": src}
    tra = {"bound": "hbm", "achieved": TRANSPORT_BYTES * N / (ph[3] * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
           "traffic": measured_traffic("k_transport<true>"), "kernel": "k_transport<true>", "peak_source": src}
    for x in (reg, tra):
        x["frac"] = x["achieved"] / x["peak"]
    dom = max(((ph[2], coll), (ph[0], reg), (ph[3], tra)), key=lambda a: a[0])[1]
    classes = mcd.mcd_get_collide_classes(d.ctx)
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
           "roofline": dom,
           "roofline_all": {"collide": coll, "collide_smem": coll_smem, "regrid": reg, "transport": tra},
           "peaks_probe": {k: pk[k] for k in ("smem_gbs", "fp32_tflops", "fp64_tflops", "sm_count", "sm_clock_mhz",
                                              "l2_bytes", "smem_per_sm_bytes")},
           "collide_classes": [{k: c[k] for k in ("n_lo", "n_hi", "cells", "threads", "swarms_per_thread", "store",
                                                  "control_warp", "persistent", "trials")} for c in classes],
           "gpu_launches": int(launches), "events_per_step": ev_step,
           "heaviest_cell_events": int(ev_c.max(axis=1).mean()) if ev_c.size else 0}

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
    if rank == 0 and world == 1 and not args.no_extra:
        # the other configurations of the metric, each in its own context:
        # the 64-disk batch and the stress disk (mid-run states), and the
        # benchmark disk's whole evolution from its initial state
        out["batched64"] = measure_batched(args, stream, flush, pk, fp32_peak)
        out["stress"] = measure_single(args, "stress_1024x32x400", stream, flush, pk, fp32_peak)
    if rank == 0 and world == 1 and args.full_run_yr > 0:
        out["full_run"] = measure_full_run(args, stream)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_context(name, params, grids, states, seed, args, stream, flush, pk, fp32_peak, steps, warmup):
    """One mixed-precision context of several disks (params, grids; mid-run
    states m, r, z per disk) stepped `warmup` times untimed and `steps` times
    timed (each step alone, after an L2 flush): whole-context events/s,
    phases, launches, the collide's rooflines, the tuned cell classes."""
    import torch
    from paper_2507_21239_gb300 import mcd, workloads as W
    d = mcd.Disk(params, grids, seed=seed, prec="mixed", stream=stream)
    for k, (m, r, z) in enumerate(states):
        p = d.particles(k)
        mcd.mcd_set_particles(d.ctx, k, m, p["M"], r, z, p["id"])
    dt = args.dt_yr * W.YR
    mcd.mcd_trace(d.ctx, True)
    for _ in range(warmup):
        mcd.mcd_step(d.ctx, dt)
    torch.cuda.synchronize()
    events = lambda: sum(d.stats(k).events for k in range(len(grids)))
    ev0, l0 = events(), mcd.mcd_get_launch_count(d.ctx)
    loads = []
    with ClockSampler(smi_index(0)) as clk:
        times, phases = timed_steps(mcd, d, dt, steps, stream, flush,
                                    on_step=lambda k: loads.append(cell_loads(mcd, d, grids)))
    torch.cuda.synchronize()
    ev = events() - ev0
    launches = mcd.mcd_get_launch_count(d.ctx) - l0
    status = mcd.mcd_sync(d.ctx)
    total_ms = float(times.sum())
    ph = phases.mean(axis=0)
    n_c = np.array([x[0] for x in loads], np.float64)
    ev_c = np.array([x[1] for x in loads], np.float64)
    alu, smem = collide_rooflines(n_c, ev_c, steps, ph[2], pk, fp32_peak)
    classes = mcd.mcd_get_collide_classes(d.ctx)
    n = sum(g[0] * g[1] * g[2] for g in grids)
    out = {"workload": name, "value": ev / (total_ms * 1e-3), "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": total_ms / steps, "disk_yr_per_s": len(grids) * steps * args.dt_yr / (total_ms * 1e-3),
           "status": mcd.mcd_strerror(status), "disks": len(grids), "particles": n,
           "cells": sum(g[0] * g[1] for g in grids), "dt_yr": args.dt_yr, "events_per_step": ev / steps,
           "heaviest_cell_events": int(ev_c.max(axis=1).mean()) if ev_c.size else 0,
           "phases_ms": {"regrid": ph[0], "order": ph[1], "collide": ph[2], "transport": ph[3]},
           "roofline_collide": alu, "roofline_collide_smem": smem, "gpu_launches": int(launches),
           "collide_classes": [{k: c[k] for k in ("n_lo", "n_hi", "cells", "threads", "swarms_per_thread", "store",
                                                  "control_warp", "persistent", "trials")} for c in classes],
           "state": "workloads.midrun_state per disk (seed = disk)", "clocks": clk.summary()}
    d.close()
    return out


def measure_batched(args, stream, flush, pk, fp32_peak):
    """The 64-disk batch (workloads.batched_disks: alpha x v_frag grid, 32-512
    radial zones and 50-400 particles per cell per disk, 8 vertical cells) in
    one context."""
    from paper_2507_21239_gb300 import workloads as W
    disks = W.batched_disks()
    params = [x["params"] for x in disks]
    grids = [(x["n_r"], x["n_z"], x["per_cell"]) for x in disks]
    states = [W.midrun_state(params[k], g[0] * g[1] * g[2], seed=k) for k, g in enumerate(grids)]
    return measure_context("batched64", params, grids, states, 0, args, stream, flush, pk, fp32_peak,
                           args.extra_steps, args.extra_warmup)


def measure_single(args, name, stream, flush, pk, fp32_peak):
    """One of workloads.WORKLOADS (a single disk) from its mid-run state."""
    from paper_2507_21239_gb300 import workloads as W
    wl = W.WORKLOADS[name]
    grid = (wl["n_r"], wl["n_z"], wl["per_cell"])
    state = W.midrun_state(wl["params"], grid[0] * grid[1] * grid[2], seed=wl["seed"])
    return measure_context(name, [wl["params"]], [grid], [state], wl["seed"], args, stream, flush, pk, fp32_peak,
                           args.extra_steps, args.extra_warmup)


def measure_full_run(args, stream):
    """The 819,200-particle disk evolved from its initial state (all monomers,
    z ~ N(0, H_g)) for args.full_run_yr years in 1-yr steps, mixed path, as
    one stream of graph replays: wall time, simulated years per second, events
    per step over time, and the mass bookkeeping at the end."""
    import torch
    from paper_2507_21239_gb300 import mcd, workloads as W
    wl = W.WORKLOADS["disk2d_256x16x200"]
    grid = (wl["n_r"], wl["n_z"], wl["per_cell"])
    d = mcd.Disk(wl["params"], grid, seed=wl["seed"], prec="mixed", stream=stream)
    M0 = float(d.particles()["M"].sum())
    dt = args.dt_yr * W.YR
    n_steps = int(round(args.full_run_yr / args.dt_yr))
    mark = max(1, n_steps // 10)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    trace, prev_ev, prev_k = [], 0, 0
    with ClockSampler(smi_index(0)) as clk:
        for k in range(1, n_steps + 1):
            mcd.mcd_step(d.ctx, dt)
            if k % mark == 0 or k == n_steps:
                ev = d.stats().events  # (synchronises: a few per run)
                trace.append({"yr": k * args.dt_yr, "events_per_step": (ev - prev_ev) / (k - prev_k)})
                prev_ev, prev_k = ev, k
    e1.record(stream)
    e1.synchronize()
    wall = time.perf_counter() - t0
    dev_ms = e0.elapsed_time(e1)
    st = d.stats()
    status = mcd.mcd_sync(d.ctx)
    x = d.particles()
    alive = np.isfinite(x["r"])
    mass_err = abs(float(x["M"][alive].sum()) + st.accreted_mass - M0) / M0
    m = x["m"][alive]
    out = {"workload": "disk2d_256x16x200 from the initial state", "sim_yr": n_steps * args.dt_yr,
           "steps": n_steps, "wall_s": wall, "device_s": dev_ms * 1e-3, "sim_yr_per_s": n_steps * args.dt_yr / wall,
           "events": int(st.events), "events_per_s": st.events / wall, "status": mcd.mcd_strerror(status),
           "events_per_step_trace": trace, "mass_rel_err": mass_err, "alive": int(alive.sum()),
           "m_max_g": float(m.max()) if m.size else None,
           "note": "wall time of the whole run including the host's graph launches and a few status reads",
           "clocks": clk.summary()}
    d.close()
    return out


def run_batched(args):
    """The 64-disk batch alone: one JSON line (not the benchmark line)."""
    import torch
    from paper_2507_21239_gb300 import build as B
    torch.cuda.set_device(0)
    B.build()
    stream = torch.cuda.Stream()
    flush = torch.empty(max(args.flush_mb, 1) << 20, dtype=torch.uint8, device="cuda")
    _, mhz, _ = peaks()
    out = measure_batched(args, stream, flush, probe_peaks(stream), SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12)
    out["metric"] = METRIC
    print(json.dumps(out), flush=True)


def _oracle_disk_run(job):
    """One oracle disk evolution (spawned worker, one thread): (events, seconds)."""
    workload, seed, disk, dt_yr, steps = job
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2507_21239_gb300 import workloads as W
    wl = W.WORKLOADS[workload]
    P, grid = wl["params"], (wl["n_r"], wl["n_z"], wl["per_cell"])
    s = oracle.init_disk(P, grid[0] * grid[1] * grid[2], seed=seed, disk=disk)
    t0 = time.perf_counter()
    st = oracle.run(P, grid[0], grid[1], s, 0.0, dt_yr * W.YR, 0, steps, seed=seed, disk=disk, nthreads=1)
    return int(s.events), time.perf_counter() - t0, int(st)


def run_oracle_runs(args):
    """Full runs timed end to end: the 0D constant-kernel cell (200 swarms to
    t = 100) and the 16 x 4 x 100 disk through 1e4 yr (32 seeds, 50-yr steps),
    the oracle on every host core (one disk per process) and per core, the GPU
    (mixed and FP64, the seeds batched in one context) beside it."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    from paper_2507_21239_gb300 import workloads as W
    cores = os.cpu_count() or 1
    seeds, dt_yr, steps = args.oracle_seeds, 50.0, 200
    jobs = [("disk2d_16x4x100", 7, d, dt_yr, steps) for d in range(seeds)]
    # the pool starts (spawn) before this process touches the GPU
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(cores, seeds)) as pool:
        res = pool.map(_oracle_disk_run, jobs)
    wall = time.perf_counter() - t0
    ev = sum(r[0] for r in res)
    per_core = [r[0] / r[1] for r in res]
    out = {"host": {"cpu": cpu_model(), "cores": cores}}
    out["disk2d_16x4x100_1e4yr"] = {
        "seeds": seeds, "sim_yr_per_disk": dt_yr * steps, "oracle_all_cores": {
            "wall_s": wall, "events": ev, "events_per_s": ev / wall, "disk_yr_per_s": seeds * dt_yr * steps / wall,
            "processes": min(cores, seeds), "status": sorted({r[2] for r in res})},
        "oracle_one_core": {"events_per_s_median": float(np.median(per_core)),
                            "disk_yr_per_s_median": float(np.median([dt_yr * steps / r[1] for r in res])),
                            "seconds_per_disk_median": float(np.median([r[1] for r in res]))}}
    P0 = W.constant_kernel_cell()
    t0 = time.perf_counter()
    st, m, ev0, _, _ = oracle.collide_cell(P0, 0.0, 0.0, 1.0, np.ones(200), np.full(200, 1.0 / 200), 0.0, 100.0,
                                           0, 0, 0, 0)
    el0 = time.perf_counter() - t0
    out["0d_const_200_t100"] = {"oracle_one_core": {"seconds": el0, "events": ev0, "status": st,
                                                    "mean_mass": float(m.mean())}}
    # the GPU on the same runs
    import torch
    from paper_2507_21239_gb300 import build as B, mcd
    torch.cuda.set_device(0)
    B.build()
    d = mcd.Disk(P0, (1, 1, 200), seed=0, prec="fp64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mcd.mcd_collide(d.ctx, 100.0)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    el = time.perf_counter() - t0
    out["0d_const_200_t100"]["gpu_fp64"] = {"seconds": el, "events": int(d.stats().events),
                                           "mean_mass": float(d.particles()["m"].mean())}
    d.close()
    wl = W.WORKLOADS["disk2d_16x4x100"]
    grid = (wl["n_r"], wl["n_z"], wl["per_cell"])
    for prec, nd in (("mixed", seeds), ("fp64", seeds)):
        d = mcd.Disk([wl["params"]] * nd, [grid] * nd, seed=7, prec=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            mcd.mcd_step(d.ctx, dt_yr * W.YR)
        status = mcd.mcd_sync(d.ctx)
        el = time.perf_counter() - t0
        evg = sum(d.stats(k).events for k in range(nd))
        out["disk2d_16x4x100_1e4yr"]["gpu_" + prec] = {
            "disks": nd, "wall_s": el, "events": evg, "events_per_s": evg / el, "disk_yr_per_s": nd * dt_yr * steps / el,
            "status": mcd.mcd_strerror(status)}
        d.close()
    print(json.dumps({"oracle_runs": out}), flush=True)


def run_peaks(args):
    import torch
    from paper_2507_21239_gb300 import build as B
    torch.cuda.set_device(0)
    B.build()
    print(json.dumps({"peaks_probe": probe_peaks(torch.cuda.current_stream())}), flush=True)


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
    ap.add_argument("--no-extra", action="store_true", help="skip the batched64 and stress records")
    ap.add_argument("--extra-steps", type=int, default=5, help="timed steps of the batched64 and stress records")
    ap.add_argument("--extra-warmup", type=int, default=3)
    ap.add_argument("--full-run-yr", type=float, default=1e4,
                    help="years of the full_run record (the benchmark disk from its initial state); 0 skips it")
    ap.add_argument("--peaks", action="store_true", help="print the microbenchmarked peaks only")
    ap.add_argument("--collide-variant", default=None,
                    help='pin the mixed collide variant of the main line, "S,store" or "cw,store" (profiling)')
    ap.add_argument("--oracle-runs", action="store_true",
                    help="time the oracle's full runs (0D cell; the 16 x 4 x 100 disk through 1e4 yr) and the GPU beside it")
    ap.add_argument("--oracle-seeds", type=int, default=32)
    args = ap.parse_args()
    if args.oracle_runs:
        run_oracle_runs(args)
    elif args.peaks:
        run_peaks(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
