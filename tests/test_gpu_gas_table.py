"""A gas disk tabulated in radius (mcd_set_gas_table) against the oracle's
tabulated gas, through the C ABI.

The table is the gap-and-bump profile of the workloads module (a stand-in for
an azimuthally averaged hydrodynamic snapshot), with knots from 1.5 to 80 AU
so that particles of the 1-100 AU disk also meet both extended end segments.
Tolerances are those of the power-law parity tests: FP64 1e-12 relative on
displacements (event sequences identical), mixed 1e-5, regrid bounds to the
ulp level.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
from paper_2507_21239_gb300 import mcd, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
AU, YR = W.AU, W.YR
TOL = {mcd.MCD_FP64: 1e-12, mcd.MCD_MIXED: 1e-5}
PRECS = [mcd.MCD_FP64, mcd.MCD_MIXED]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21239_gb300 import build
    build.build()
    oracle.build()


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    d = np.abs(a - b)
    s = np.abs(b)
    out = np.where(s > 0, d / np.where(s > 0, s, 1), d)
    return float(out.max()) if out.size else 0.0


def _tabled(noise=0.01, **over):
    P = W.benchmark_disk(**over)
    return dict(P, gas_table=W.gap_bump_gas_table(P, noise=noise, seed=3))


def _transport_case(P, prec, seed=9):
    grid = (8, 4, 250)
    N = 8 * 4 * 250
    d = mcd.Disk(P, grid, seed=seed, prec=prec)
    rng = np.random.default_rng(4)
    r = AU * np.geomspace(1.0, 100.0, N) * (1 + rng.uniform(-1e-3, 1e-3, N))
    r = np.clip(r, P["r_in"] * (1 + 1e-9), P["r_out"] * (1 - 1e-9))
    r[:50] = P["r_in"] * (1 + rng.uniform(0, 1e-3, 50))  # some leave through the inner edge
    r[50:100] = P["r_out"] * (1 - rng.uniform(0, 1e-3, 50))  # some are reflected
    H = oracle.gas(P, r, np.zeros(N))["H"]
    z = rng.normal(0, 1, N) * H
    m = W.random_masses(N, seed=5, lo=1e-12, hi=1e4)
    M = np.full(N, 3e26)
    ids = rng.permutation(N).astype(np.uint32)
    mcd.mcd_set_particles(d.ctx, 0, m, M, r, z, ids)
    return d, (m, M, r, z, ids)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("flags", [3, 1 | 4, 2 | 4])
def test_transport_with_table(prec, flags):
    P = _tabled(tr_flags=flags)
    d, (m, M, r, z, ids) = _transport_case(P, prec)
    dt = 30 * YR
    mcd.mcd_transport(d.ctx, dt)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    got = d.particles()
    s = oracle.DiskState(m, M, r, z, ids)
    oracle.transport(P, s, dt, seed=9, disk=0, step=0)
    gone = ~np.isfinite(s.r)
    assert np.array_equal(gone, ~np.isfinite(got["r"]))
    keep = ~gone
    g = oracle.gas(P, r[keep], z[keep])
    sig = np.sqrt(2 * g["D"] * dt)
    tol = TOL[prec]
    assert np.all(np.abs(got["r"][keep] - s.r[keep]) <= tol * (np.abs(s.r[keep] - r[keep]) + sig) + 1e-15 * r[keep])
    assert np.all(np.abs(got["z"][keep] - s.z[keep]) <= tol * (np.abs(s.z[keep] - z[keep]) + sig)
                  + 1e-15 * np.abs(z[keep]))
    # the table matters here: the power-law oracle misses the GPU's radial steps
    if flags & 1:
        s0 = oracle.DiskState(m, M, r, z, ids)
        oracle.transport(W.benchmark_disk(tr_flags=flags), s0, dt, seed=9, disk=0, step=0)
        k2 = keep & np.isfinite(s0.r)
        assert np.max(np.abs(s0.r[k2] - s.r[k2]) / (np.abs(s.r[k2] - r[k2]) + 1e-300)) > 0.1
    d.close()


@pytest.mark.parametrize("knots", [2, 17])
def test_power_law_table_equals_power_laws(knots):
    """A table sampled from the disk's own power laws (two knots: one segment
    extended both ways) gives the power-law disk's steps: same events,
    positions and masses to 1e-10 (FP64, three steps of event chains)."""
    P = W.benchmark_disk(dust_to_gas=0.5, v_frag=300.0)
    rk = AU * np.geomspace(0.5, 200.0, knots) if knots > 2 else AU * np.array([3.0, 30.0])
    tab = np.c_[rk, P["sigma0"] * (rk / AU) ** -P["p"], P["T0"] * (rk / AU) ** -P["q"]]
    grid, seed, dt = (6, 3, 20), 4, 100 * YR
    a = mcd.Disk(P, grid, seed=seed, prec=mcd.MCD_FP64)
    b = mcd.Disk(dict(P, gas_table=tab), grid, seed=seed, prec=mcd.MCD_FP64)
    for _ in range(3):
        a.step(dt)
        b.step(dt)
    assert mcd.mcd_sync(a.ctx) == mcd.MCD_OK and mcd.mcd_sync(b.ctx) == mcd.MCD_OK
    x, y = a.particles(), b.particles()
    assert a.stats().events == b.stats().events > 100_000
    assert np.array_equal(x["id"], y["id"])
    fin = np.isfinite(x["r"])
    assert np.array_equal(fin, np.isfinite(y["r"]))
    for k in ("m", "r", "z"):
        assert rel(y[k][fin], x[k][fin]) < 1e-10, k
    a.close()
    b.close()


def test_steps_fp64_with_table_match_oracle():
    """Three full FP64 steps (regrid, collide with cell constants from the
    table, transport) of a small disk with the same keys: the oracle's event
    count and every particle's r, z, m."""
    P = _tabled(dust_to_gas=0.5, v_frag=300.0)
    grid, seed, dt = (6, 3, 20), 4, 100 * YR
    d = mcd.Disk(P, grid, seed=seed, prec=mcd.MCD_FP64)
    s = oracle.init_disk(P, 6 * 3 * 20, seed)
    for _ in range(3):
        d.step(dt)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    oracle.run(P, 6, 3, s, 0.0, dt, 0, 3, seed)
    got = d.particles()
    go, so = np.argsort(got["id"]), np.argsort(s.id)
    assert s.events > 100_000
    assert mcd.mcd_get_stats(d.ctx, 0).events == s.events
    for key in ("m", "r", "z"):
        a, b = got[key][go], getattr(s, key)[so]
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin)
        assert rel(a[fin], b[fin]) < 1e-10, key
    d.close()


@pytest.mark.parametrize("prec", PRECS)
def test_cell_rates_with_table(prec):
    """After a regrid of a mid-run state, every cell's row sums from the
    GPU's table-derived cell constants equal the oracle's O(n^2) rates in the
    same tabulated disk."""
    P = _tabled()
    grid = (16, 4, 40)
    N = 16 * 4 * 40
    d = mcd.Disk(P, grid, seed=2, prec=prec)
    m, r, z = W.midrun_state(P, N, seed=7)
    p = d.particles()
    mcd.mcd_set_particles(d.ctx, 0, m, p["M"], r, z, p["id"])
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DUMP_R, 1)
    mcd.mcd_regrid(d.ctx)
    off = np.zeros(grid[0] * grid[1] + 1, np.int64)
    b = np.zeros((grid[0] * grid[1], 6))
    V = np.zeros(grid[0] * grid[1])
    mcd.mcd_get_cells(d.ctx, 0, off, b, V)
    mcd.mcd_collide(d.ctx, 1e-30)  # no event fits: the row sums of the regridded state
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    x = d.particles()
    R = np.zeros(N)
    mcd.mcd_get_rates(d.ctx, 0, R)
    P0 = W.benchmark_disk()
    differs = 0
    for c in range(grid[0] * grid[1]):
        lo, hi = off[c], off[c + 1]
        _, Ro = oracle.rate_matrix(P, b[c, 4], b[c, 5], V[c], x["m"][lo:hi], x["M"][lo:hi])
        assert rel(R[lo:hi], Ro) < TOL[prec], c
        _, Rp = oracle.rate_matrix(P0, b[c, 4], b[c, 5], V[c], x["m"][lo:hi], x["M"][lo:hi])
        differs += rel(Rp, Ro) > 1e-3
    assert differs > grid[0]  # the table changes the rates of many cells
    d.close()


@pytest.mark.parametrize("grid,dead", [((5, 7, 3), 100), ((4, 3, 5), 59)])
def test_regrid_single_particle_bounds_with_table(grid, dead):
    """A zone holding one particle spans H_g of the tabulated gas vertically;
    a disk holding one particle, radially too."""
    P = _tabled()
    N = grid[0] * grid[1] * grid[2]
    d = mcd.Disk(P, grid, seed=0, prec=mcd.MCD_FP64)
    rng = np.random.default_rng(11)
    r = rng.uniform(2 * AU, 60 * AU, N)
    z = rng.normal(0, 1, N) * 0.03 * r
    r[rng.choice(N, dead, replace=False)] = np.inf
    m = W.random_masses(N, seed=12, lo=1e-11, hi=1e-2)
    M = np.full(N, 1e26)
    ids = rng.permutation(N).astype(np.uint32)
    mcd.mcd_set_particles(d.ctx, 0, m, M, r, z, ids)
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    s = oracle.DiskState(m, M, r, z, ids)
    st, _, off, cb, cv, na = oracle.regrid(P, grid[0], grid[1], s)
    assert st == 0
    goff = np.zeros(grid[0] * grid[1] + 1, np.int64)
    gb = np.zeros((grid[0] * grid[1], 6))
    gv = np.zeros(grid[0] * grid[1])
    mcd.mcd_get_cells(d.ctx, 0, goff, gb, gv)
    assert np.array_equal(goff, off)
    assert np.any(np.diff(off) == 1)
    assert rel(gb, cb) < 1e-14 and rel(gv, cv) < 1e-13
    # the power-law H would give other bounds
    _, _, _, cb0, _, _ = oracle.regrid(W.benchmark_disk(), grid[0], grid[1], oracle.DiskState(m, M, r, z, ids))
    assert rel(cb0, cb) > 1e-3
    d.close()


def test_table_set_after_graph_capture_and_reset():
    """The step graph reads the table in place: setting it after the graph
    was captured, then clearing it, gives the results of direct launches."""
    P = W.benchmark_disk(dust_to_gas=0.5, v_frag=300.0)
    tab = W.gap_bump_gas_table(P, noise=0.01, seed=3)
    grid, dt = (6, 3, 20), 50 * YR
    out = []
    for graph in (1, 0):
        d = mcd.Disk(P, grid, seed=6, prec=mcd.MCD_MIXED)
        mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_USE_GRAPH, graph)
        d.step(dt)
        d.set_gas_table(tab)
        d.step(dt)
        d.step(dt)
        d.set_gas_table(None)
        d.step(dt)
        assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
        out.append((d.particles(), d.stats().events))
        d.close()
    (x, ex), (y, ey) = out
    assert ex == ey
    for k in ("m", "M", "r", "z", "id"):
        assert np.array_equal(x[k], y[k]), k


def test_bad_tables_rejected_and_previous_kept():
    P = _tabled(tr_flags=3)
    good = P["gas_table"]
    d, (m, M, r, z, ids) = _transport_case(P, mcd.MCD_FP64)
    bad = [good[:1], np.r_[good[:5], good[3:4]], np.tile(good[:1], (2, 1))]
    for k, col in ((1, 1), (2, 2)):
        t = good.copy()
        t[7, col] = -1.0 if k == 1 else np.nan
        bad.append(t)
    t = good.copy()
    t[0, 0] = np.inf
    bad.append(t)
    bad.append(np.c_[AU * np.geomspace(1, 100, mcd.MCD_MAX_GAS_KNOTS + 1), np.ones((mcd.MCD_MAX_GAS_KNOTS + 1, 2))])
    for t in bad:
        with pytest.raises(mcd.McdError) as e:
            d.set_gas_table(t)
        assert e.value.code == mcd.MCD_EINVAL
    with pytest.raises(mcd.McdError):
        mcd.mcd_set_gas_table(d.ctx, 1, good)  # no such disk
    # the table set at creation is still in force
    dt = 30 * YR
    mcd.mcd_transport(d.ctx, dt)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    s = oracle.DiskState(m, M, r, z, ids)
    oracle.transport(P, s, dt, seed=9, disk=0, step=0)
    got = d.particles()
    keep = np.isfinite(s.r)
    assert np.array_equal(keep, np.isfinite(got["r"]))
    assert rel(got["r"][keep], s.r[keep]) < 1e-13
    # the largest table is accepted
    n = mcd.MCD_MAX_GAS_KNOTS
    rk = AU * np.geomspace(1, 100, n)
    d.set_gas_table(np.c_[rk, 1000 * (rk / AU) ** -1.0, 280 * (rk / AU) ** -0.5])
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    d.close()


def test_mixed_steps_with_table_conserve_mass():
    P = _tabled()
    grid = (16, 4, 100)
    d = mcd.Disk([P] * 4, [grid] * 4, seed=1, prec=mcd.MCD_MIXED)
    M0 = [d.particles(k)["M"].sum() for k in range(4)]
    for _ in range(10):
        d.step(50 * YR)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    for k in range(4):
        x, st = d.particles(k), d.stats(k)
        alive = np.isfinite(x["r"])
        assert np.all(np.isfinite(x["m"][alive])) and np.all(np.isfinite(x["z"][alive]))
        assert abs(x["M"][alive].sum() + st.accreted_mass - M0[k]) <= 1e-12 * M0[k]
    d.close()
