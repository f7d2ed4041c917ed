"""The adaptive step of mcd_step(dt <= 0) against the oracle's, through the C
ABI: dt = min(dt_max, C min_c dr_c / max_i |v_r,i|) chosen on the device after
the regrid, the smallest over the disks of a context.

Tolerances: FP64 steps 1e-12 relative (the regrid is bit-exact, |v_r| differs
from the oracle's at the ulp level), then the same event counts and r, z, m to
1e-10 over three steps; mixed path (|v_r| in FP32) 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
from paper_2507_21239_gb300 import mcd, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
AU, YR = W.AU, W.YR
GRID = (20, 2, 10)
N = GRID[0] * GRID[1] * GRID[2]


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


def _drifting(P, seed=8, grid=GRID):
    """A context holding a mid-run state (grains that drift), and that state."""
    n = grid[0] * grid[1] * grid[2]
    m, r, z = W.midrun_state(P, n, seed=seed)
    M = np.full(n, 1e26)
    ids = np.arange(n, dtype=np.uint32)
    return m, M, r, z, ids


def _ctx(P, prec, state, grid=GRID, seed=4):
    d = mcd.Disk(P, grid, seed=seed, prec=prec)
    mcd.mcd_set_particles(d.ctx, 0, *state)
    return d


def _adaptive_steps(d, k):
    """k adaptive steps; returns each step's dt read from the device clock."""
    t, out = d.stats().t, []
    for _ in range(k):
        d.step(0.0)
        t1 = d.stats().t
        out.append(t1 - t)
        t = t1
    return np.array(out)


def _oracle_dt(P, state, grid=GRID, dt_max=YR, courant=0.5):
    s = oracle.DiskState(*[np.copy(a) for a in state])
    st, _, off, cb, _, _ = oracle.regrid(P, grid[0], grid[1], s)
    assert st == 0
    return oracle.adaptive_dt(P, off, cb, s, dt_max, courant)


@pytest.mark.parametrize("flags", [W.TR_RADIAL | W.TR_VERTICAL, W.TR_RADIAL | W.TR_ST_MIDPLANE])
def test_adaptive_steps_fp64_match_oracle(flags):
    P = W.benchmark_disk(tr_flags=flags)
    state = _drifting(P)
    dt_max = 1e4 * YR
    d = _ctx(P, mcd.MCD_FP64, state)
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DT_MAX, dt_max)
    got = _adaptive_steps(d, 3)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    s = oracle.DiskState(*[np.copy(a) for a in state])
    dts = np.zeros(3)
    assert oracle.run(P, GRID[0], GRID[1], s, 0.0, 0.0, 0, 3, 4, dt_max=dt_max, dts=dts) == 0
    assert np.all(dts < dt_max) and s.events > 1000
    assert rel(got, dts) < 1e-12
    x = d.particles()
    assert d.stats().events == s.events
    go, so = np.argsort(x["id"]), np.argsort(s.id)
    for key in ("m", "r", "z"):
        a, b = x[key][go], getattr(s, key)[so]
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin)
        assert rel(a[fin], b[fin]) < 1e-10, key
    d.close()


def test_adaptive_step_mixed_and_options():
    """Mixed path: the first step's dt is the oracle's for the same state to
    1e-5; halving C halves it exactly; a small dt_max caps it exactly."""
    P = W.benchmark_disk()
    state = _drifting(P)
    ref = _oracle_dt(P, state, dt_max=1e30)
    out = []
    for courant, dt_max in ((0.5, 1e30), (0.25, 1e30), (0.5, 0.1 * ref)):
        d = _ctx(P, mcd.MCD_MIXED, state)
        mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_COURANT, courant)
        mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DT_MAX, dt_max)
        out.append(_adaptive_steps(d, 1)[0])
        assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
        d.close()
    assert rel(out[0], ref) < 1e-5
    assert out[1] == out[0] / 2
    assert out[2] == 0.1 * ref


def test_batched_disks_share_the_smallest_step():
    """Three disks in one context: the step is the smallest of the disks' own
    steps; a disk without radial transport asks for dt_max."""
    Ps = [W.benchmark_disk(), W.benchmark_disk(alpha=1e-2, v_frag=300.0), W.benchmark_disk(tr_flags=W.TR_VERTICAL)]
    grids = [GRID, (12, 3, 15), (8, 2, 10)]
    states = [_drifting(P, seed=20 + k, grid=g) for k, (P, g) in enumerate(zip(Ps, grids))]
    d = mcd.Disk(Ps, grids, seed=1, prec=mcd.MCD_FP64)
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DT_MAX, 1e5 * YR)
    for k, st in enumerate(states):
        mcd.mcd_set_particles(d.ctx, k, *st)
    got = _adaptive_steps(d, 1)[0]
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    refs = [_oracle_dt(P, st, grid=g, dt_max=1e5 * YR) for P, st, g in zip(Ps, states, grids)]
    assert refs[2] == 1e5 * YR and min(refs) < 1e5 * YR
    assert rel(got, min(refs)) < 1e-12
    d.close()


def test_adaptive_graph_equals_direct_and_mode_switches():
    """Graph replay equals direct launches in the adaptive mode, switching
    between fixed and adaptive steps included; mcd_collide after adaptive
    steps reads the device clock."""
    P = W.benchmark_disk()
    state = _drifting(P)
    res = []
    for graph in (1, 0):
        d = _ctx(P, mcd.MCD_MIXED, state)
        mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_USE_GRAPH, graph)
        d.step(0.0)
        d.step(10 * YR)
        d.step(0.0)
        d.step(-1.0)
        assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
        t = d.stats().t
        mcd.mcd_regrid(d.ctx)
        with pytest.raises(mcd.McdError):
            mcd.mcd_collide(d.ctx, 0.5 * t)  # behind the clock
        mcd.mcd_collide(d.ctx, t + YR)
        assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
        assert d.stats().t == t + YR
        res.append((d.particles(), t, d.stats().events))
        d.close()
    (x, tx, ex), (y, ty, ey) = res
    assert tx == ty and ex == ey and tx > 10 * YR
    for k in ("m", "r", "z", "id"):
        assert np.array_equal(x[k], y[k]), k


def test_adaptive_step_with_gas_table_fp64():
    P = W.benchmark_disk()
    P = dict(P, gas_table=W.gap_bump_gas_table(P, noise=0.01, seed=3))
    state = _drifting(P)
    d = _ctx(P, mcd.MCD_FP64, state)
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_DT_MAX, 1e5 * YR)
    got = _adaptive_steps(d, 1)[0]
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    ref = _oracle_dt(P, state, dt_max=1e5 * YR)
    assert rel(got, ref) < 1e-12
    assert rel(ref, _oracle_dt(W.benchmark_disk(), state, dt_max=1e5 * YR)) > 1e-3  # the table matters
    d.close()


def test_bad_steps_and_options_rejected():
    d = mcd.Disk(W.benchmark_disk(), (4, 2, 10), seed=0, prec=mcd.MCD_MIXED)
    for dt in (np.nan, np.inf, -np.inf):
        with pytest.raises(mcd.McdError):
            d.step(dt)
    for key in (mcd.MCD_OPT_DT_MAX, mcd.MCD_OPT_COURANT):
        for v in (0.0, -1.0, np.inf, np.nan):
            with pytest.raises(mcd.McdError):
                mcd.mcd_set_option(d.ctx, key, v)
    d.step(0.0)  # the all-monomer start barely drifts: dt_max
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    assert d.stats().t == YR
    d.close()
