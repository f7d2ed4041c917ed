"""The collide's launch variants against each other and against the oracle.

The collide runs cells in classes by particles per cell, each class with its
own launch (and stream), threads per cell, swarms per thread and dv-matrix
store; a timed trial picks the swarms per thread and the store per class;
persistent CTAs may take the cells by atomic ticket instead of one CTA per
cell; and the mixed path's total rate is a compensated FP32 sum.  Here:

* every disk of a batch that spans all five classes follows the oracle event
  for event (FP64), so the classes' concurrent launches change nothing;
* persistent CTAs give the bits of one CTA per cell on the 64-disk batch;
* the trial records its candidates and keeps the fastest;
* the total rate that sets the waiting time is, by default, the block scan's
  plain FP32 sum (bit for bit the host's sum in the kernel's order, within
  10 ulp of the exact total) and, with MCD_OPT_EXACT_TOTAL, a compensated sum
  within 2e-9 of the exact total of the kernel's own row sums, a bound the
  plain sum misses; both equal the oracle's FP64 total to 1e-5.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
from paper_2507_21239_gb300 import mcd, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
AU, YR = W.AU, W.YR


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21239_gb300 import build
    build.build()
    oracle.build()


def _squeezed_midrun(P, N, seed):
    """A mid-run state squeezed to 1..6 AU: many events per cell and year."""
    m, r, z = W.midrun_state(P, N, seed=seed)
    r2 = P["r_in"] + (r - P["r_in"]) * (5.0 * AU / (P["r_out"] - P["r_in"]))
    return m, r2, z * (r2 / r) ** 1.25


def test_five_classes_follow_the_oracle_event_for_event():
    """FP64: disks of 40, 100, 200, 300 and 450 particles per cell (one in each
    class, each class its own launch on its own stream) take the oracle's
    event counts and masses through two steps."""
    P = W.benchmark_disk(dust_to_gas=0.3)
    ppcs = (40, 100, 200, 300, 450)
    grids = [(2, 1, n) for n in ppcs]
    d = mcd.Disk([P] * len(grids), grids, seed=9, prec="fp64")
    cls = mcd.mcd_get_collide_classes(d.ctx)
    assert [(k["n_lo"], k["n_hi"], k["cells"]) for k in cls] == [(n, n, 2) for n in ppcs]
    states = []
    for k, g in enumerate(grids):
        N = g[0] * g[1] * g[2]
        m, r, z = _squeezed_midrun(P, N, seed=20 + k)
        p = d.particles(k)
        mcd.mcd_set_particles(d.ctx, k, m, p["M"], r, z, p["id"])
        states.append(oracle.DiskState(m, p["M"], r, z, p["id"]))
    for _ in range(2):
        d.step(YR)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    for k, g in enumerate(grids):
        s = states[k]
        oracle.run(P, g[0], g[1], s, 0.0, YR, 0, 2, seed=9, disk=k)
        got = d.particles(k)
        assert d.stats(k).events == s.events and s.events > 1000, (k, d.stats(k).events, s.events)
        go, so = np.argsort(got["id"]), np.argsort(s.id)
        for key in ("m", "r", "z"):
            a, b = got[key][go], getattr(s, key)[so]
            fin = np.isfinite(b)
            assert np.array_equal(np.isfinite(a), fin)
            assert np.max(np.abs(a[fin] / b[fin] - 1)) < 1e-10, (k, key)
    d.close()


@pytest.mark.parametrize("control_warp", [0, 1])
def test_persistent_ctas_equal_one_cta_per_cell_on_the_64_disk_batch(control_warp):
    """Mixed path, the 64-disk batch (28.5 M particles, classes from 50 to 400
    particles per cell): one step from each disk's mid-run state with
    persistent CTAs gives the masses, row sums and event counts of one CTA per
    cell, bit for bit (the random numbers are keyed by disk, cell and event,
    not by the CTA that runs the cell); for the block variants and for the
    control-warp variant."""
    disks = W.batched_disks()
    params = [x["params"] for x in disks]
    grids = [(x["n_r"], x["n_z"], x["per_cell"]) for x in disks]
    states = [W.midrun_state(params[k], g[0] * g[1] * g[2], seed=k) for k, g in enumerate(grids)]
    out = []
    shape = ((mcd.MCD_OPT_CONTROL_WARP, 1),) if control_warp else ((mcd.MCD_OPT_SWARMS_PER_THREAD, 1),)
    for persistent in (0, 1):
        d = mcd.Disk(params, grids, seed=0, prec="mixed")
        for key, v in ((mcd.MCD_OPT_PERSISTENT, persistent), (mcd.MCD_OPT_DV_MATRIX, 1),
                       (mcd.MCD_OPT_DUMP_R, 1)) + shape:
            mcd.mcd_set_option(d.ctx, key, v)
        for k, (m, r, z) in enumerate(states):
            p = d.particles(k)
            mcd.mcd_set_particles(d.ctx, k, m, p["M"], r, z, p["id"])
        d.step(YR)
        assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
        assert all(k["control_warp"] == control_warp for k in mcd.mcd_get_collide_classes(d.ctx))
        res = []
        for k in (0, 17, 40, 63):
            R = np.zeros(grids[k][0] * grids[k][1] * grids[k][2])
            mcd.mcd_get_rates(d.ctx, k, R)
            res.append((d.particles(k)["m"], R, d.stats(k).events))
        out.append((res, sum(d.stats(k).events for k in range(len(disks)))))
        d.close()
    (ra, ea), (rb, eb) = out
    assert ea == eb and ea > 10**6
    for (ma, Ra, xa), (mb, Rb, xb) in zip(ra, rb):
        assert xa == xb
        assert np.array_equal(ma, mb) and np.array_equal(Ra, Rb)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_timed_trial_keeps_the_fastest_candidate(prec):
    """Before the first collide each class times its candidates (mixed: one or
    two swarms per thread, or the control warp, x shared or no matrix; FP64:
    workspace or no matrix) and runs the fastest; the step then conserves
    mass."""
    P = W.benchmark_disk()
    grid = (8, 4, 200)
    d = mcd.Disk(P, grid, seed=1, prec=prec)
    m, r, z = _squeezed_midrun(P, 8 * 4 * 200, seed=5)
    p = d.particles()
    mcd.mcd_set_particles(d.ctx, 0, m, p["M"], r, z, p["id"])
    d.step(YR)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    (k,) = mcd.mcd_get_collide_classes(d.ctx)
    assert k["tuned"] == 1
    want = ({(1, 1, 0), (1, 0, 0), (2, 1, 0), (2, 0, 0), (1, 1, 1), (1, 0, 1)} if prec == "mixed"
            else {(1, 2, 0), (1, 0, 0)})
    got = {(t["swarms_per_thread"], t["store"], t["control_warp"]) for t in k["trials"]}
    assert got == want
    best = min(k["trials"], key=lambda t: t["us_per_event"])
    assert all(t["us_per_event"] > 0 for t in k["trials"])
    assert (k["swarms_per_thread"], k["store"], k["control_warp"]) == (
        best["swarms_per_thread"], best["store"], best["control_warp"])
    # one thread per swarm, per two, or a control warp and one worker thread per swarm
    assert k["threads"] == (256 if k["control_warp"] else 224 if k["swarms_per_thread"] == 1 else 128)
    x = d.particles()
    alive = np.isfinite(x["r"])
    M0 = p["M"].sum()
    assert abs(x["M"][alive].sum() + d.stats().accreted_mass - M0) <= 1e-12 * M0
    d.close()


def _plain_scan_total(x, spt):
    """The plain FP32 total of the kernel's choice scan over x (float32): each
    thread's swarms summed in order, a Kogge-Stone scan over the 32 lanes of
    each warp, then one over the warp totals (lane 31's prefix)."""
    x = np.asarray(x, np.float32)
    nthr = max(32, ((len(x) + spt - 1) // spt + 31) // 32 * 32)
    v = np.zeros(nthr * spt, np.float32)
    v[:len(x)] = x
    t = v.reshape(nthr, spt)
    thr = t[:, 0].copy()
    for s in range(1, spt):
        thr = (thr + t[:, s]).astype(np.float32)
    wt = []
    for w in range(nthr // 32):
        a = thr[32 * w:32 * w + 32].copy()
        o = 1
        while o < 32:
            b = a.copy()
            b[o:] = (a[o:] + a[:-o]).astype(np.float32)
            a = b
            o *= 2
        wt.append(a[31])
    a = np.array(wt, np.float32)
    o = 1
    while o < len(a):
        b = a.copy()
        b[o:] = (a[o:] + a[:-o]).astype(np.float32)
        a = b
        o *= 2
    return float(a[-1])


@pytest.mark.parametrize("spt", [1, 2, 0])
def test_total_rate_plain_and_compensated(spt):
    """Cells of 400 swarms whose masses span 1e-12 .. 1 g (row sums over ~12
    decades), mixed path, stopped after the rebuild.  By default the total
    rate is the block scan's plain FP32 sum of the row sums' leading parts: it
    equals, bit for bit, that sum formed on the host in the kernel's order
    (thread sums, a Kogge-Stone scan over each warp's lanes, then over the warp
    totals), and lies within 10 ulp of the exact total.  With
    MCD_OPT_EXACT_TOTAL it is the compensated sum: within 2e-9 of the exact
    (fsum) total of the kernel's own row sums in every cell, a bound that the
    plain sum misses in most cells.  Both equal the oracle's FP64 total of the
    same cell to 1e-5.  spt 0: the control-warp variant, whose plain total is
    the one warp's scan of 16 row sums per lane (the exact total then runs the
    block variant with its helper warp).  The two runs' row sums agree bit for
    bit when one kernel forms them and to 1e-6 across kernels (the compiler
    may fuse a product into a sum in one kernel and not in another): each
    total is checked against its own run's row sums."""
    P = W.benchmark_disk()
    grid = (2, 4, 400)
    N = grid[0] * grid[1] * grid[2]
    rng = np.random.default_rng(77)
    m = 10.0 ** rng.uniform(-12, 0, N)
    r = rng.uniform(1.0, 3.0, N) * AU
    z = rng.normal(0, 1, N) * 0.03 * r
    out = {}
    for exact in (0, 1):
        d = mcd.Disk(P, grid, seed=2, prec="mixed")
        p = d.particles()
        mcd.mcd_set_particles(d.ctx, 0, m, p["M"], r, z, p["id"])
        mcd.mcd_regrid(d.ctx)
        shape = ((mcd.MCD_OPT_SWARMS_PER_THREAD, spt),) if spt else ((mcd.MCD_OPT_CONTROL_WARP, -1 if exact else 1),)
        # (the row sums are formed from recomputed entries in every run: the
        # stored-matrix build rounds a few entries differently, and a timed
        # trial left free to pick the store would make the runs' rows differ)
        for key, v in ((mcd.MCD_OPT_MAX_EVENTS, 0), (mcd.MCD_OPT_CAP_STOPS, 1), (mcd.MCD_OPT_DUMP_R, 1),
                       (mcd.MCD_OPT_EXACT_TOTAL, exact), (mcd.MCD_OPT_DV_MATRIX, 0)) + shape:
            mcd.mcd_set_option(d.ctx, key, v)
        mcd.mcd_collide(d.ctx, 1.0)
        assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
        R = np.zeros(N)
        mcd.mcd_get_rates(d.ctx, 0, R)
        Rt = np.zeros(grid[0] * grid[1])
        mcd.mcd_get_total_rates(d.ctx, 0, Rt)
        off = np.zeros(grid[0] * grid[1] + 1, np.int64)
        cb = np.zeros((grid[0] * grid[1], 6))
        V = np.zeros(grid[0] * grid[1])
        mcd.mcd_get_cells(d.ctx, 0, off, cb, V)
        out[exact] = (R, Rt, off, cb, V, d.particles())
        d.close()
    R, _, off, cb, V, x = out[1]
    plain_misses = 0
    for c in range(grid[0] * grid[1]):
        Rc = R[off[c]:off[c + 1]]
        R0 = out[0][0][off[c]:off[c + 1]]
        assert len(Rc) == 400
        if spt:
            assert np.array_equal(Rc, R0)
        else:
            assert np.max(np.abs(Rc / R0 - 1)) <= 1e-6
        exact, exact0 = math.fsum(Rc), math.fsum(R0)
        plain = _plain_scan_total(R0, spt if spt else 16)
        assert out[0][1][c] == plain, (c, out[0][1][c], plain)  # the kernel's plain sum, bit for bit
        assert abs(plain / exact0 - 1) <= 10 * 2.0**-24
        assert abs(out[1][1][c] / exact - 1) <= 2e-9, (c, out[1][1][c], exact)
        plain_misses += abs(plain / exact0 - 1) > 2e-9
        sl = slice(off[c], off[c + 1])
        _, Ro = oracle.rate_matrix(P, cb[c, 4], cb[c, 5], V[c], x["m"][sl], x["M"][sl])
        assert abs(out[1][1][c] / math.fsum(Ro) - 1) < 1e-5
        assert np.max(np.abs(Rc / Ro - 1)) < 1e-5
    assert plain_misses >= 6, plain_misses
