"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times: mixed path, step graph, one collide CTA per SM, stored dv
matrix.  Sampled outputs are checked one by one against the oracle; the rest by
properties that hold at any size.

* 819,200-particle disk:
  - the regrid of the benchmark's mid-run state, bit-exact;
  - FP64 collide: sampled cells' event counts and masses equal the oracle's
    for the same cell inputs;
  - mixed collide: sampled cells' incremental row sums equal the oracle's
    O(n^2) recomputation from the masses the GPU reached;
  - a graph-replayed step conserves mass.
* The largest zone of each zone-sort path (4,096 radix, 14,336 bitonic),
  bit-exact.
* 64 batched disks (28.5 M particles): a sampled disk's regrid bit-exact, and
  every disk conserves mass over a step.
* The 13.1 M-particle stress disk: one zone's (z, id) order, cell counts and
  vertical bounds equal the oracle's regrid of that zone alone; mass is
  conserved.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_21239_gb300 import mcd, workloads as W

pytestmark = pytest.mark.gpu

AU, YR = W.AU, W.YR


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))) if a.size else 0.0


def _cells(d, disk, ncell):
    off = np.zeros(ncell + 1, np.int64)
    b = np.zeros((ncell, 6))
    V = np.zeros(ncell)
    mcd.mcd_get_cells(d.ctx, disk, off, b, V)
    return off, b, V


def _with_state(P, grid, prec, m, r, z, seed=0):
    d = mcd.Disk(P, grid, seed=seed, prec=prec)
    p = d.particles()
    mcd.mcd_set_particles(d.ctx, 0, m, p["M"], r, z, p["id"])
    return d, p


@pytest.fixture(scope="module")
def disk819k():
    wl = W.WORKLOADS["disk2d_256x16x200"]
    P, grid = wl["params"], (wl["n_r"], wl["n_z"], wl["per_cell"])
    N = grid[0] * grid[1] * grid[2]
    m, r, z = W.midrun_state(P, N, seed=wl["seed"])
    return P, grid, N, m, r, z


def _check_regrid(d, disk, P, grid, state):
    """The context's regrid of one disk against the oracle's of the same state."""
    ncell = grid[0] * grid[1]
    x = d.particles(disk)
    off, b, V = _cells(d, disk, ncell)
    s = oracle.DiskState(*state)
    st, _, coff, cb, cv, na = oracle.regrid(P, grid[0], grid[1], s)
    assert st == 0
    for key in ("id", "m", "M", "r", "z"):
        assert np.array_equal(x[key], getattr(s, key)), key
    assert np.array_equal(off, coff)
    assert np.array_equal(b[:, :4], cb[:, :4]) and np.array_equal(V, cv)
    return x, off, b, V


def test_fullsize_regrid_bit_exact(disk819k):
    P, grid, N, m, r, z = disk819k
    d, p = _with_state(P, grid, mcd.MCD_MIXED, m, r, z)
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    _check_regrid(d, 0, P, grid, (m, p["M"], r, z, p["id"]))
    d.close()


# the innermost (heaviest) cells, a few in the middle, the outermost
SAMPLE = [0, 1, 7, 15, 16, 300, 1000, 2047, 3000, 4095]


def test_fullsize_fp64_sampled_cells(disk819k):
    P, grid, N, m, r, z = disk819k
    d, _ = _with_state(P, grid, mcd.MCD_FP64, m, r, z)
    mcd.mcd_regrid(d.ctx)
    x = d.particles()
    off, b, V = _cells(d, 0, grid[0] * grid[1])
    mcd.mcd_collide(d.ctx, YR)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    y = d.particles()
    ce = np.zeros(grid[0] * grid[1], np.int64)
    mcd.mcd_get_cell_events(d.ctx, 0, ce)
    assert ce[:16].max() > 500  # the sample includes long event chains
    for c in SAMPLE:
        lo, hi = off[c], off[c + 1]
        st, m_o, ev_o, _, _ = oracle.collide_cell(P, b[c, 4], b[c, 5], V[c], x["m"][lo:hi], x["M"][lo:hi], 0.0, YR,
                                                  0, 0, 0, c)
        assert st == 0 and ce[c] == ev_o, c
        assert rel(y["m"][lo:hi], m_o) < 1e-12, c
    d.close()


def test_fullsize_mixed_row_sums_and_step(disk819k):
    P, grid, N, m, r, z = disk819k
    d, p = _with_state(P, grid, mcd.MCD_MIXED, m, r, z)
    M0 = p["M"].sum()
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DUMP_R, 1)
    mcd.mcd_regrid(d.ctx)
    off, b, V = _cells(d, 0, grid[0] * grid[1])
    mcd.mcd_collide(d.ctx, YR)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    y = d.particles()
    R = np.zeros(N)
    mcd.mcd_get_rates(d.ctx, 0, R)
    for c in SAMPLE:
        lo, hi = off[c], off[c + 1]
        _, Ro = oracle.rate_matrix(P, b[c, 4], b[c, 5], V[c], y["m"][lo:hi], y["M"][lo:hi])
        assert rel(R[lo:hi], Ro) < 1e-5, c
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DUMP_R, 0)
    for _ in range(2):
        d.step(YR)  # graph replay
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    x, st = d.particles(), d.stats()
    alive = np.isfinite(x["r"])
    assert abs(x["M"][alive].sum() + st.accreted_mass - M0) <= 1e-12 * M0
    assert st.events > 100_000
    d.close()


@pytest.mark.parametrize("grid", [(4, 16, 256), (2, 28, 512)], ids=["zone4096_radix", "zone14336_bitonic"])
def test_largest_zones_bit_exact(grid):
    P = W.benchmark_disk()
    N = grid[0] * grid[1] * grid[2]
    m, r, z = W.midrun_state(P, N, seed=5)
    z[1::2] = z[0:N - 1:2]  # every other particle repeats its neighbour's height: ties broken by id
    d, p = _with_state(P, grid, mcd.MCD_MIXED, m, r, z)
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    _check_regrid(d, 0, P, grid, (m, p["M"], r, z, p["id"]))
    d.close()


def test_batched_fullsize_regrid_and_mass():
    disks = W.batched_disks()
    params = [x["params"] for x in disks]
    grids = [(x["n_r"], x["n_z"], x["per_cell"]) for x in disks]
    q = int(np.argmax([g[0] * g[1] * g[2] for g in grids]))  # the largest disk
    d = mcd.Disk(params, grids, seed=0, prec=mcd.MCD_MIXED)
    Nq = grids[q][0] * grids[q][1] * grids[q][2]
    m, r, z = W.midrun_state(params[q], Nq, seed=q)
    p = d.particles(q)
    mcd.mcd_set_particles(d.ctx, q, m, p["M"], r, z, p["id"])
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    _check_regrid(d, q, params[q], grids[q], (m, p["M"], r, z, p["id"]))
    M0 = [d.particles(k)["M"].sum() for k in range(len(disks))]
    d.step(YR)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    for k in range(len(disks)):
        x, st = d.particles(k), d.stats(k)
        alive = np.isfinite(x["r"])
        assert abs(x["M"][alive].sum() + st.accreted_mass - M0[k]) <= 1e-12 * M0[k], k
    d.close()


def test_stress_fullsize_zone_and_mass():
    wl = W.WORKLOADS["stress_1024x32x400"]
    P, grid = wl["params"], (wl["n_r"], wl["n_z"], wl["per_cell"])
    N = grid[0] * grid[1] * grid[2]
    d = mcd.Disk(P, grid, seed=0, prec=mcd.MCD_MIXED)
    M0 = d.particles()["M"].sum()
    d.step(YR)
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    x = d.particles()
    off, b, V = _cells(d, 0, grid[0] * grid[1])
    alive = np.isfinite(x["r"])
    assert abs(x["M"][alive].sum() + d.stats().accreted_mass - M0) <= 1e-12 * M0
    # one zone (the 300th): its particles regridded alone by the oracle into
    # 1 x n_z cells give the same (z, id) order, counts and vertical bounds
    k = 300
    lo, hi = off[k * grid[1]], off[(k + 1) * grid[1]]
    s = oracle.DiskState(x["m"][lo:hi], x["M"][lo:hi], x["r"][lo:hi], x["z"][lo:hi], x["id"][lo:hi])
    # ids must be a permutation of 0..n-1 for the oracle: rank them
    s.id = np.argsort(np.argsort(s.id)).astype(np.uint32)
    ids_sorted = np.sort(x["id"][lo:hi])
    st, _, coff, cb, _, _ = oracle.regrid(P, 1, grid[1], s)
    assert st == 0
    assert np.array_equal(ids_sorted[s.id], x["id"][lo:hi])
    assert np.array_equal(coff, off[k * grid[1]:(k + 1) * grid[1] + 1] - lo)
    assert np.array_equal(cb[:, 2:4], b[k * grid[1]:(k + 1) * grid[1], 2:4])
    d.close()
