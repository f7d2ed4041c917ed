"""Checkpoint and resume through the C ABI: a context stepped 3 years, then
checkpointed (particles, tracer, clock, step, counters read with
mcd_get_particles / mcd_get_tracer / mcd_get_stats), restored into a new
context and stepped 3 more years, equals the same context stepped 6 years
without interruption, bit for bit: particles, tracer, event counts, accreted
mass, clock and step.  Both precisions, two disks of a batch, the mixed path
with its collide variant pinned."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2507_21239_gb300 import mcd, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
YR = W.YR


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21239_gb300 import build
    build.build()


def _start(prec, params, grids, states):
    d = mcd.Disk(params, grids, seed=11, prec=prec)
    if prec == "mixed":
        mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_SWARMS_PER_THREAD, 1)
    for k, (m, r, z) in enumerate(states):
        p = d.particles(k)
        mcd.mcd_set_particles(d.ctx, k, m, p["M"], r, z, p["id"])
        N = m.size
        d.set_tracer(np.linspace(0.0, 1.0, N), k)
    return d


def _snapshot(d, nd):
    out = []
    for k in range(nd):
        st = d.stats(k)
        out.append(dict(d.particles(k), q=d.tracer(k), t=st.t, step=st.step, events=st.events,
                        accreted=st.accreted_mass))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resume_equals_uninterrupted_run(prec):
    P = W.benchmark_disk()
    params = [P, W.benchmark_disk(alpha=1e-2, v_frag=300.0)]
    grids = [(8, 4, 100), (4, 4, 60)]
    states = []
    for k, g in enumerate(grids):
        N = g[0] * g[1] * g[2]
        states.append(W.midrun_state(params[k], N, seed=30 + k))
    # the uninterrupted run
    a = _start(prec, params, grids, states)
    for _ in range(6):
        a.step(YR)
    assert mcd.mcd_sync(a.ctx) == mcd.MCD_OK
    ref = _snapshot(a, 2)
    a.close()
    # 3 years, checkpoint, a new context restored, 3 more years
    b = _start(prec, params, grids, states)
    for _ in range(3):
        b.step(YR)
    assert mcd.mcd_sync(b.ctx) == mcd.MCD_OK
    ck = _snapshot(b, 2)
    b.close()
    assert ck[0]["step"] == 3 and ck[0]["events"] > 0
    c = mcd.Disk(params, grids, seed=11, prec=prec)
    if prec == "mixed":
        mcd.mcd_set_option(c.ctx, mcd.MCD_OPT_SWARMS_PER_THREAD, 1)
    for k in range(2):
        x = ck[k]
        mcd.mcd_set_particles(c.ctx, k, x["m"], x["M"], x["r"], x["z"], x["id"])
        c.set_tracer(x["q"], k)
        mcd.mcd_set_counters(c.ctx, k, x["events"], x["accreted"])
    mcd.mcd_set_clock(c.ctx, ck[0]["t"], ck[0]["step"])
    for _ in range(3):
        c.step(YR)
    assert mcd.mcd_sync(c.ctx) == mcd.MCD_OK
    got = _snapshot(c, 2)
    c.close()
    for k in range(2):
        for key in ("m", "M", "r", "z", "q"):
            assert np.array_equal(got[k][key].view(np.uint64), ref[k][key].view(np.uint64)), (k, key)
        assert np.array_equal(got[k]["id"], ref[k]["id"])
        for key in ("t", "step", "events", "accreted"):
            assert got[k][key] == ref[k][key], (k, key, got[k][key], ref[k][key])


def test_restore_rejects_bad_values():
    d = mcd.Disk(W.benchmark_disk(), (2, 2, 10), seed=0, prec="fp64")
    for args in ((float("nan"), 0), (-1.0, 0), (0.0, -1)):
        with pytest.raises(mcd.McdError):
            mcd.mcd_set_clock(d.ctx, *args)
    for args in ((0, -1, 0.0), (0, 0, -1.0), (5, 0, 0.0)):
        with pytest.raises(mcd.McdError):
            mcd.mcd_set_counters(d.ctx, *args)
    d.close()
