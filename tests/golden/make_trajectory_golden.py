"""Write the oracle's statistics of whole disk evolutions for the trajectory
parity tests (tests/test_gpu_trajectory_bar.py).  It calls only the oracle
and the seeded workload recipes; nothing here comes from the CUDA path.

Two fixtures, each a JSON file beside this script:

* trajectory_16x4x100_1e4yr.json -- the Benchmark-table disk at 16 x 4 cells
  x 100 particles, 32 disks (seed 7, disk 0..31, the oracle's keyed initial
  draw), 200 steps of 50 yr (1e4 yr);
* trajectory_256x16x200_20yr.json -- the same physics at 256 x 16 x 200
  (819,200 particles), 8 disks (seed 11, disk 0..7), 20 steps of 1 yr from
  the initial state.

Per disk: the per-bin sums (sum M, M m, M m^2, M m^3, count) over 16
logarithmic radial bins of [r_in, r_out], the per-bin histogram of log10 m
(0.2 dex bins over [-12, 6]), the accreted mass, the initial swarm mass and
the event count.  Per bin: the quantiles (levels 0, 0.001, ..., 1) of
log10 m pooled over the disks' particles in the bin, to 5 decimals.

  python tests/golden/make_trajectory_golden.py [--workers N]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CASES = {
    "trajectory_16x4x100_1e4yr.json": dict(workload="disk2d_16x4x100", seed=7, disks=32, dt_yr=50.0, steps=200),
    "trajectory_256x16x200_20yr.json": dict(workload="disk2d_256x16x200", seed=11, disks=8, dt_yr=1.0, steps=20),
}
LEVELS = np.linspace(0.0, 1.0, 1001)
HIST_EDGES = np.linspace(-12.0, 6.0, 91)  # log10 m [g], 0.2 dex; values outside fall in the end bins


def _edges(P):
    return P["r_in"] * np.geomspace(1.0, P["r_out"] / P["r_in"], 17)


def log10m_hist(m, r, edges):
    """Per radial bin: counts of log10 m on HIST_EDGES (the end bins take what
    lies beyond)."""
    ok = np.isfinite(r) & (r >= edges[0]) & (r < edges[-1])
    b = np.searchsorted(edges, r[ok], side="right") - 1
    lm = np.clip(np.log10(m[ok]), HIST_EDGES[0], np.nextafter(HIST_EDGES[-1], -np.inf))
    return [np.histogram(lm[b == q], bins=HIST_EDGES)[0].tolist() for q in range(edges.size - 1)]


def evolve(workload, seed, disk, dt_yr, steps):
    import oracle
    from paper_2507_21239_gb300 import workloads as W
    wl = W.WORKLOADS[workload]
    P, grid = wl["params"], (wl["n_r"], wl["n_z"], wl["per_cell"])
    N = grid[0] * grid[1] * grid[2]
    s = oracle.init_disk(P, N, seed=seed, disk=disk)
    M0 = float(s.M.sum())
    t0 = time.perf_counter()
    st = oracle.run(P, grid[0], grid[1], s, 0.0, dt_yr * W.YR, 0, steps, seed=seed, disk=disk, nthreads=1)
    el = time.perf_counter() - t0
    if st != 0:
        raise RuntimeError(f"oracle status {st} for disk {disk}")
    mom = oracle.moments(s.m, s.M, s.r, _edges(P))
    return dict(disk=disk, sums=mom.tolist(), accreted=s.accreted, M0=M0, events=int(s.events), seconds=el,
                hist=log10m_hist(s.m, s.r, _edges(P)), m=s.m, r=s.r)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default=None)
    args = ap.parse_args()
    import oracle
    from paper_2507_21239_gb300 import workloads as W
    oracle.build()
    for name, c in CASES.items():
        if args.only and args.only != name:
            continue
        P = W.WORKLOADS[c["workload"]]["params"]
        edges = _edges(P)
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(min(args.workers, c["disks"])) as pool:
            runs = pool.starmap(evolve, [(c["workload"], c["seed"], k, c["dt_yr"], c["steps"])
                                         for k in range(c["disks"])])
        pooled = [[] for _ in range(edges.size - 1)]
        for x in runs:
            ok = np.isfinite(x["r"]) & (x["r"] >= edges[0]) & (x["r"] < edges[-1])
            b = np.searchsorted(edges, x["r"][ok], side="right") - 1
            lm = np.log10(x["m"][ok])
            for q in range(edges.size - 1):
                pooled[q].append(lm[b == q])
        pooled = [np.concatenate(v) for v in pooled]
        out = dict(case=c, edges=edges.tolist(), levels=LEVELS.tolist(),
                   hist_edges=HIST_EDGES.tolist(),
                   disks=[{k: x[k] for k in ("disk", "sums", "accreted", "M0", "events", "seconds", "hist")}
                          for x in runs],
                   log10m_count=[int(v.size) for v in pooled],
                   log10m_quantiles=[np.round(np.quantile(v, LEVELS), 5).tolist() if v.size else [] for v in pooled],
                   wall_seconds=time.perf_counter() - t0, workers=min(args.workers, c["disks"]),
                   cpu=os.uname().machine)
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(out, f)
        print(name, f"{out['wall_seconds']:.0f} s", sum(x["events"] for x in runs), "events", flush=True)


if __name__ == "__main__":
    main()
