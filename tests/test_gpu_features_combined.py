"""The features together, against the oracle: a fragmentation ramp, the tracer,
a gas table and the adaptive step in one FP64 run (three steps, the oracle's
event count, tracer and positions); and a mixed batched context whose disks
each use a different subset (mass conserved per disk, tracer in range)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
from paper_2507_21239_gb300 import mcd, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
YR = W.YR


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


def test_ramp_tracer_table_adaptive_fp64_match_oracle():
    P = W.benchmark_disk(frag_ramp=0.4, v_frag=300.0, frag_xi=1.6, erosion_chi=2.0)
    P = dict(P, gas_table=W.gap_bump_gas_table(P, noise=0.01, seed=5))
    grid, seed, dt_max = (20, 2, 10), 4, 1e4 * YR
    n = grid[0] * grid[1] * grid[2]
    m, r, z = W.midrun_state(P, n, seed=8)
    M = np.full(n, 1e26)
    ids = np.arange(n, dtype=np.uint32)
    q = 0.1 + 0.8 * (ids % 5) / 4.0
    d = mcd.Disk(P, grid, seed=seed, prec=mcd.MCD_FP64)
    mcd.mcd_set_particles(d.ctx, 0, m, M, r, z, ids)
    d.set_tracer(q)
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DT_MAX, dt_max)
    for _ in range(3):
        d.step(0.0)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    s = oracle.DiskState(m.copy(), M.copy(), r.copy(), z.copy(), ids.copy())
    s.q = q.copy()
    dts = np.zeros(3)
    assert oracle.run(P, grid[0], grid[1], s, 0.0, 0.0, 0, 3, seed, dt_max=dt_max, dts=dts) == 0
    assert s.events > 1000 and np.all(dts < dt_max)
    assert rel(d.stats().t, dts.sum()) < 1e-12
    assert d.stats().events == s.events
    x, tq = d.particles(), d.tracer()
    go, so = np.argsort(x["id"]), np.argsort(s.id)
    for key in ("m", "r", "z"):
        a, b = x[key][go], getattr(s, key)[so]
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin)
        assert rel(a[fin], b[fin]) < 1e-10, key
    assert rel(tq[go], s.q[so]) < 1e-10
    assert not np.array_equal(tq[go], q[so])
    d.close()


def test_mixed_batched_feature_subsets():
    base = W.benchmark_disk()
    Ps = [base,
          W.benchmark_disk(frag_ramp=0.3),
          dict(base, gas_table=W.gap_bump_gas_table(base, noise=0.02, seed=1)),
          dict(W.benchmark_disk(frag_ramp=0.2, v_frag=300.0), gas_table=W.gap_bump_gas_table(base, seed=2))]
    grids = [(16, 4, 50), (8, 4, 60), (16, 2, 40), (12, 3, 30)]
    d = mcd.Disk(Ps, grids, seed=3, prec=mcd.MCD_MIXED)
    m0 = []
    for k, g in enumerate(grids):
        p = d.particles(k)
        m0.append(p["M"].sum())
        d.set_tracer(np.where(p["id"] % 2 == 0, 0.0, 1.0), k)
    for _ in range(6):
        d.step(0.0)
    for _ in range(4):
        d.step(20 * YR)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    for k in range(len(grids)):
        x, st, tq = d.particles(k), d.stats(k), d.tracer(k)
        alive = np.isfinite(x["r"])
        assert abs(x["M"][alive].sum() + st.accreted_mass - m0[k]) <= 1e-12 * m0[k], k
        assert np.all((tq >= -1e-12) & (tq <= 1 + 1e-12)), k
        assert 0.0 < (x["M"][alive] * tq[alive]).sum() / x["M"][alive].sum() < 1.0
    d.close()


def test_emptied_disk_latches_eempty_while_others_step():
    """A disk whose particles are all removed latches MCD_EEMPTY at the next
    regrid; the other disk of the context keeps stepping and conserving mass,
    with the adaptive step too (the empty disk asks for nothing)."""
    P = W.benchmark_disk()
    grids = [(8, 2, 20), (4, 2, 10)]
    d = mcd.Disk([P, P], grids, seed=1, prec=mcd.MCD_MIXED)
    p = d.particles(1)
    mcd.mcd_set_particles(d.ctx, 1, p["m"], p["M"], np.full(p["r"].size, np.inf), p["z"], p["id"])
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_EEMPTY
    assert d.stats(1).n_alive == 0 and d.stats(1).status == mcd.MCD_EEMPTY
    m0 = d.particles(0)["M"].sum()
    m, r, z = W.midrun_state(P, 8 * 2 * 20, seed=2)
    q = d.particles(0)
    mcd.mcd_set_particles(d.ctx, 0, m, q["M"], r, z, q["id"])
    for dt in (YR, 0.0, 0.0):
        d.step(dt)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_EEMPTY  # latched
    x, st = d.particles(0), d.stats(0)
    alive = np.isfinite(x["r"])
    assert st.events > 0 and st.n_alive == alive.sum() > 0
    assert abs(x["M"][alive].sum() + st.accreted_mass - m0) <= 1e-12 * m0
    assert d.stats(1).events == 0 and d.stats(1).accreted_mass == 0.0
    d.close()


def test_particles_as_device_tensors():
    """Disk.particles_device gives the host copy's values as CUDA tensors, on a
    private stream too."""
    P = W.benchmark_disk()
    for stream in (None, torch.cuda.Stream()):
        d = mcd.Disk(P, (8, 2, 25), seed=2, prec=mcd.MCD_MIXED, stream=stream)
        d.step(YR)
        x, t = d.particles(), d.particles_device()
        for k in ("m", "M", "r", "z"):
            assert t[k].is_cuda and np.array_equal(t[k].cpu().numpy(), x[k]), k
        assert np.array_equal(t["id"].cpu().numpy().view(np.uint32), x["id"])
        d.close()
