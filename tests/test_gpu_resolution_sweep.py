"""A particles-per-cell resolution sweep in one batched launch.

The Benchmark section notes that a Monte Carlo run leaves the regions of the
(mass, distance) plane that hold little of the dust mass unsampled, and that
more representative particles fill them.  The Benchmark-table disk on 16 x 4
cells runs at 25, 50, 100, 200 and 400 particles per cell (4 seeds each, all
20 disks in one context) for 1,000 yr:

* every disk conserves its mass (alive plus accreted) to 1e-12;
* the sigma_d(m, r) map (16 log radial bins x 48 log mass bins) covers more
  bins, on average over the seeds, at every doubling of the resolution;
* the two highest resolutions agree per radial bin: the across-seed mean bin
  mass within max(5 %, 4 sigma) and the mass-weighted mean log10 m within
  max(0.1 dex, 4 sigma).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2507_21239_gb300 import mcd, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
YR = W.YR
PPCS = (25, 50, 100, 200, 400)
SEEDS = 4
DT, STEPS = 50 * YR, 20


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21239_gb300 import build
    build.build()


def test_resolution_sweep_batched():
    params, grids, res = W.ppc_sweep(PPCS, seeds=SEEDS)
    nd = len(params)
    d = mcd.Disk(params, grids, seed=11, prec=mcd.MCD_MIXED)
    m0 = [d.particles(k)["M"].sum() for k in range(nd)]
    for _ in range(STEPS):
        d.step(DT)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    P = params[0]
    r_edges = P["r_in"] * np.geomspace(1.0, P["r_out"] / P["r_in"], 17)
    m_edges = np.geomspace(1e-12, 1e4, 49)
    cover = np.zeros(nd)
    mass = np.zeros((nd, 16))
    logm = np.full((nd, 16), np.nan)
    for k in range(nd):
        x, st = d.particles(k), d.stats(k)
        alive = np.isfinite(x["r"])
        assert abs(x["M"][alive].sum() + st.accreted_mass - m0[k]) <= 1e-12 * m0[k], k
        sig = d.sigma_map(r_edges, m_edges, k)
        cover[k] = np.count_nonzero(sig)
        mass[k] = sig.sum(axis=1)
        b = np.searchsorted(r_edges, x["r"][alive], side="right") - 1
        lm, M = np.log10(x["m"][alive]), x["M"][alive]
        for q in range(16):
            sel = b == q
            if sel.any():
                logm[k, q] = (M[sel] * lm[sel]).sum() / M[sel].sum()
    ev = [sum(d.stats(k).events for k in np.flatnonzero(res == p)) for p in PPCS]
    d.close()
    cov = [cover[res == p].mean() for p in PPCS]
    assert all(b > a for a, b in zip(cov, cov[1:])), cov
    hi, lo = res == PPCS[-1], res == PPCS[-2]
    for q in range(16):
        x, y = mass[hi, q], mass[lo, q]
        sig = np.sqrt(x.var(ddof=1) / x.size + y.var(ddof=1) / y.size)
        assert abs(x.mean() - y.mean()) <= max(0.05 * y.mean(), 4 * sig), ("mass", q)
        x, y = logm[hi, q], logm[lo, q]
        if np.all(np.isfinite(x)) and np.all(np.isfinite(y)):
            sig = np.sqrt(x.var(ddof=1) / x.size + y.var(ddof=1) / y.size)
            assert abs(x.mean() - y.mean()) <= max(0.1, 4 * sig), ("log m", q, x.mean(), y.mean(), sig)
    print("sigma_d map bins covered per resolution:", dict(zip(PPCS, np.round(cov, 1))), "events:", dict(zip(PPCS, ev)))
