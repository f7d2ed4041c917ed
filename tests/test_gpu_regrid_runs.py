"""The radial sort's fix-up against the oracle's regrid.

The regrid sorts the radial keys by their upper 32 bits (sign, exponent and
20 mantissa bits) and then puts every run of equal upper words in (r, id)
order: short runs in place, long ones by one CTA each in shared memory, the
longest in global memory; a run whose radii are all equal is already in id
order.  Here radii are built from their bit patterns so that every path runs:
runs of 2..64 positions, of 65..14,336, one of 16,000, one long run of equal
radii, ties inside runs, removed particles (+inf) and the heights and masses
of an ordinary disk.  The id order, the reordered columns, the cell offsets,
bounds and volumes must equal the oracle's bit for bit, with the graph and
with direct launches."""
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


def _radii(rng, sizes, P, equal_run=0):
    """Radii in runs of equal upper words: one run per entry of sizes (its
    upper word from a random radius of the disk, its lower words random, with
    a few exact repeats), then equal_run copies of one radius."""
    out = []
    for L in sizes:
        base = np.array([rng.uniform(P["r_in"], P["r_out"])]).view(np.uint64)[0]
        hi = int(base) & 0xFFFFFFFF00000000
        lo = rng.integers(0, 2**32, L, dtype=np.uint64)
        if L > 4:
            lo[rng.integers(0, L, L // 4)] = lo[0]  # ties inside the run
        out.append((np.uint64(hi) | lo).view(np.float64))
    if equal_run:
        out.append(np.full(equal_run, rng.uniform(P["r_in"], P["r_out"])))
    return np.concatenate(out)


CASES = {
    "short_runs": dict(grid=(16, 4, 50), sizes="short", seed=1),
    "smem_runs": dict(grid=(16, 4, 320), sizes=[65, 300, 1000, 2500, 14336], equal_run=700, seed=2),
    "global_run": dict(grid=(16, 4, 300), sizes=[16000, 90, 3], equal_run=1500, seed=3),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("graph", [0, 1])
def test_radial_runs_match_the_oracle(case, graph):
    spec = CASES[case]
    P = W.benchmark_disk()
    grid = spec["grid"]
    N = grid[0] * grid[1] * grid[2]
    rng = np.random.default_rng(spec["seed"])
    if spec["sizes"] == "short":
        sizes = []
        while sum(sizes) < N - 400:
            sizes.append(int(rng.integers(2, 65)))
        r = _radii(rng, sizes, P)
    else:
        r = _radii(rng, spec["sizes"], P, spec.get("equal_run", 0))
    fill = N - r.size
    assert fill >= 0
    r = np.concatenate([r, rng.uniform(P["r_in"], P["r_out"], fill)])
    r[rng.choice(N, 37, replace=False)] = np.inf  # removed particles
    r = r[rng.permutation(N)]
    z = rng.normal(0, 1, N) * 0.03 * r
    z[~np.isfinite(z)] = 0.0
    m = W.random_masses(N, seed=5, lo=1e-11, hi=1e-2)
    M = np.full(N, 1e26)
    ids = rng.permutation(N).astype(np.uint32)
    # no transport and no events: a step's graph then moves particles only by its regrid
    d = mcd.Disk(dict(P, tr_flags=0), grid, seed=0, prec="fp64")
    for key, v in ((mcd.MCD_OPT_MAX_EVENTS, 0), (mcd.MCD_OPT_CAP_STOPS, 1), (mcd.MCD_OPT_USE_GRAPH, graph)):
        mcd.mcd_set_option(d.ctx, key, v)
    mcd.mcd_set_particles(d.ctx, 0, m, M, r, z, ids)
    if graph:
        d.step(1.0)
    else:
        mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    s = oracle.DiskState(m, M, r, z, ids)
    st, _, off, cb, cv, na = oracle.regrid(P, grid[0], grid[1], s)
    assert st == 0
    got = d.particles()
    assert np.array_equal(got["id"], s.id)
    for key in ("m", "M", "r", "z"):
        assert np.array_equal(got[key].view(np.uint64), getattr(s, key).view(np.uint64)), key
    goff = np.zeros(grid[0] * grid[1] + 1, np.int64)
    gb = np.zeros((grid[0] * grid[1], 6))
    gv = np.zeros(grid[0] * grid[1])
    mcd.mcd_get_cells(d.ctx, 0, goff, gb, gv)
    assert np.array_equal(goff, off)
    exact = np.diff(off) != 1
    assert np.array_equal(gb[exact].view(np.uint64), cb[exact].view(np.uint64))
    assert np.array_equal(gv[exact].view(np.uint64), cv[exact].view(np.uint64))
    assert d.stats().n_alive == na
    d.close()
