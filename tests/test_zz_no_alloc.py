"""The regrid entry point that allocates nothing, against mcd_regrid and the oracle.

mcd_regrid_noalloc serves callers that cannot call cudaMalloc (code inside
another framework's memory pool, a real-time loop where an allocation would
stall, or a fixed memory budget): it keeps its scratch in one fixed device
array shared by every call.  Here it must give exactly what the context-based
mcd_regrid gives for the same particles, and what the oracle's regrid gives,
on several calls in a row with different disks (so nothing of a previous call
leaks into the next); report bad input through its status word and recover on
the next clean call; and leave a larger context able to step.  This file is
collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
from paper_2507_21239_gb300 import mcd, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
AU = W.AU


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21239_gb300 import build
    build.build()
    oracle.build()


def _state(grid, seed, dead):
    n_r, n_z, ppc = grid
    N = n_r * n_z * ppc
    P = W.benchmark_disk()
    rng = np.random.default_rng(seed)
    r = rng.uniform(P["r_in"], 0.3 * P["r_out"], N)
    z = rng.normal(0, 1, N) * 0.03 * r
    r[1] = r[0]
    z[3] = z[2]
    z[4] = -0.0
    z[6] = 0.0
    r[rng.choice(N, dead, replace=False)] = np.inf
    m = W.random_masses(N, seed=seed + 1, lo=1e-11, hi=1e-2)
    M = np.full(N, 1e26)
    ids = rng.permutation(N).astype(np.uint32)
    return P, (m, M, r, z, ids)


def _with_context(P, grid, st):
    d = mcd.Disk(P, grid, seed=0, prec="fp64")
    mcd.mcd_set_particles(d.ctx, 0, *st)
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    ncell = grid[0] * grid[1]
    off = np.zeros(ncell + 1, np.int64)
    b = np.zeros((ncell, 6))
    V = np.zeros(ncell)
    mcd.mcd_get_cells(d.ctx, 0, off, b, V)
    out = dict(d.particles(), off=off, b=b, V=V, n_alive=mcd.mcd_get_stats(d.ctx, 0).n_alive)
    d.close()
    return out


def _without_allocation(P, grid, st):
    N = len(st[0])
    ncell = grid[0] * grid[1]
    dev = "cuda"
    m, M, r, z, ids = st
    inp = [torch.tensor(a, device=dev) for a in (m, M, r, z)] + [torch.tensor(ids.view(np.int32), device=dev)]
    outs = [torch.empty(N, dtype=torch.float64, device=dev) for _ in range(4)]
    outs.append(torch.empty(N, dtype=torch.int32, device=dev))
    cs = torch.empty(ncell, dtype=torch.int64, device=dev)
    cn = torch.empty(ncell, dtype=torch.int32, device=dev)
    b = torch.empty((ncell, 6), dtype=torch.float64, device=dev)
    V = torch.empty(ncell, dtype=torch.float64, device=dev)
    na = torch.empty(1, dtype=torch.int64, device=dev)
    status = torch.full((1,), 99, dtype=torch.int32, device=dev)
    mcd.mcd_regrid_noalloc(P, grid, inp, outs + [cs, cn, b, V, na, status])
    torch.cuda.synchronize()
    off = np.append(cs.cpu().numpy(), cs.cpu().numpy()[-1] + cn.cpu().numpy()[-1])
    res = {k: t.cpu().numpy() for k, t in zip(("m", "M", "r", "z"), outs[:4])}
    res.update(id=outs[4].cpu().numpy().view(np.uint32), off=off, b=b.cpu().numpy(), V=V.cpu().numpy(),
               n_alive=int(na.cpu()[0]), status=int(status.cpu()[0]))
    return res


def test_noalloc_regrid_matches_context_regrid_on_consecutive_calls():
    cases = [((16, 4, 100), 11, 37), ((7, 3, 9), 12, 5), ((64, 16, 12), 13, 100), ((16, 4, 100), 11, 37)]
    for grid, seed, dead in cases:
        P, st = _state(grid, seed, dead)
        ref = _with_context(P, grid, st)
        got = _without_allocation(P, grid, st)
        assert got["status"] == mcd.MCD_OK
        _same(got, ref)


def test_noalloc_regrid_rejects_sizes_beyond_its_scratch():
    P = W.benchmark_disk()
    t = torch.empty(1, dtype=torch.float64, device="cuda")
    args = [t] * 5 + [t] * 5 + [t] * 6
    with pytest.raises(mcd.McdError) as e:
        mcd.mcd_regrid_noalloc(P, (512, 16, 16), args[:5], args[5:])  # 131,072 > 65,536 particles
    assert e.value.code == mcd.MCD_EINVAL


def _same(got, ref):
    assert got["n_alive"] == ref["n_alive"]
    assert np.array_equal(got["id"], ref["id"])
    for key in ("m", "M", "r", "z", "b", "V"):
        assert np.array_equal(np.asarray(got[key]).view(np.uint64), np.asarray(ref[key]).view(np.uint64)), key
    assert np.array_equal(got["off"], ref["off"])


def test_noalloc_regrid_matches_the_oracle():
    """Ids, reordered columns, offsets, bounds and volumes equal the oracle's
    regrid of the same particles bit for bit (a disk without single-particle
    cells, whose bounds come from the gas functions)."""
    grid = (16, 4, 100)
    P, st = _state(grid, 31, 20)
    got = _without_allocation(P, grid, st)
    assert got["status"] == mcd.MCD_OK
    s = oracle.DiskState(*st)
    rc, perm, off, cb, cv, na = oracle.regrid(P, grid[0], grid[1], s)
    assert rc == oracle.OK
    ref = {"m": s.m, "M": s.M, "r": s.r, "z": s.z, "id": s.id, "off": off, "b": cb, "V": cv, "n_alive": na}
    assert np.all(np.diff(off) != 1)
    _same(got, ref)


@pytest.mark.parametrize("fault", ["nan_z", "bad_id", "all_removed"])
def test_noalloc_status_codes_then_a_clean_call(fault):
    """A NaN height latches MCD_ENAN, an id outside 0..count-1 MCD_EINVAL and a
    disk whose particles are all removed MCD_EEMPTY; the kernels' own checks
    keep every access in bounds.  The next call with clean input reports
    MCD_OK and equals the context regrid: no status bit survives a call."""
    grid = (8, 4, 50)
    P, st = _state(grid, 41, 3)
    m, M, r, z, ids = (np.copy(a) for a in st)
    if fault == "nan_z":
        z[17] = np.nan
        want = mcd.MCD_ENAN
    elif fault == "bad_id":
        ids[5] = len(ids) + 3
        want = mcd.MCD_EINVAL
    else:
        r[:] = np.inf
        want = mcd.MCD_EEMPTY
    bad = _without_allocation(P, grid, (m, M, r, z, ids))
    assert bad["status"] == want
    clean = _without_allocation(P, grid, st)
    assert clean["status"] == mcd.MCD_OK
    _same(clean, _with_context(P, grid, st))


def test_a_larger_context_steps_after_noalloc_calls():
    """The zone sort's shared-memory limit belongs to the kernel, not to one
    caller: a context with 3,200-particle zones, created first, still regrids
    and steps after a no-allocation call on a disk with 400-particle zones and
    after a smaller context has been created."""
    P = W.benchmark_disk()
    big = mcd.Disk(P, (64, 16, 200), seed=5, prec="mixed")
    big.step(W.YR)
    assert mcd.mcd_sync(big.ctx) == mcd.MCD_OK
    grid = (16, 4, 100)
    Ps, st = _state(grid, 51, 0)
    assert _without_allocation(Ps, grid, st)["status"] == mcd.MCD_OK
    small = mcd.Disk(P, (4, 2, 10), seed=6, prec="mixed")
    small.step(W.YR)
    for _ in range(2):
        big.step(W.YR)
        mcd.mcd_regrid(big.ctx)
    assert mcd.mcd_sync(big.ctx) == mcd.MCD_OK
    assert mcd.mcd_sync(small.ctx) == mcd.MCD_OK
    small.close()
    big.close()
