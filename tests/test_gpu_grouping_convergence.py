"""Convergence in the grouping ratio dm of the Zsom & Dullemond rates.

Grouping (a swarm meets dm m_i / m_j particles of a much lighter swarm in one
event, at a rate divided by that number) is the reading that makes disk runs
feasible; its pin is that the outcome no longer depends on dm.  On the
16 x 4 x 100 Benchmark-table disk, 16 seeds evolve for 2,000 yr (growth and
fragmentation) with dm = 1e-3 and with dm / 4 in one batched mixed-path
context each.  Per logarithmic radial bin:

* the across-seed mean of the bin's swarm mass agrees within max(2 %, 4 sigma);
* the across-seed mean of the swarm-mass-weighted mean of log10 m agrees within
  max(0.05 dex, 4 sigma).

sigma is the standard error of the difference of the two across-seed means:
the seeds are the independent samples.  The particles of one run are not (a
fragmentation front moves as a whole from seed to seed), so a KS test on log m
pooled over seeds overstates its sample size; measured, its p-values do not
order with dm, and it is not used.  The mass-weighted moments of m itself are
not compared either: each is dominated by the bin's largest grain, and over
16 seeds their relative scatter reaches order one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2507_21239_gb300 import mcd, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
YR = W.YR
SEEDS = 16
DT, STEPS = 50 * YR, 40


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_21239_gb300 import build
    build.build()


def _evolve(dm):
    wl = W.WORKLOADS["disk2d_16x4x100"]
    P = dict(wl["params"], dm_group=dm)
    grid = (wl["n_r"], wl["n_z"], wl["per_cell"])
    edges = P["r_in"] * np.geomspace(1.0, P["r_out"] / P["r_in"], 17)
    d = mcd.Disk([P] * SEEDS, [grid] * SEEDS, seed=7, prec=mcd.MCD_MIXED)
    m0 = [d.particles(k)["M"].sum() for k in range(SEEDS)]
    for _ in range(STEPS):
        d.step(DT)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    nb = edges.size - 1
    mass = np.zeros((SEEDS, nb))
    logm = np.full((SEEDS, nb), np.nan)
    for k in range(SEEDS):
        x = d.particles(k)
        alive = np.isfinite(x["r"])
        assert abs(x["M"][alive].sum() + d.stats(k).accreted_mass - m0[k]) <= 1e-12 * m0[k]
        b = np.searchsorted(edges, x["r"][alive], side="right") - 1
        lm, M = np.log10(x["m"][alive]), x["M"][alive]
        for q in range(nb):
            sel = b == q
            mass[k, q] = M[sel].sum()
            if sel.any():
                logm[k, q] = (M[sel] * lm[sel]).sum() / M[sel].sum()
    ev = sum(d.stats(k).events for k in range(SEEDS))
    d.close()
    return mass, logm, ev


def test_disk_outcome_converged_in_dm():
    ma, la, ev_a = _evolve(1e-3)
    mb, lb, ev_b = _evolve(2.5e-4)
    assert ev_b > ev_a  # finer grouping takes more events
    tested = [q for q in range(ma.shape[1]) if np.all(np.isfinite(la[:, q])) and np.all(np.isfinite(lb[:, q]))]
    assert len(tested) >= 12
    worst_mass = worst_log = 0.0
    for q in tested:
        x, y = ma[:, q], mb[:, q]
        diff, sig = abs(x.mean() - y.mean()), np.sqrt(x.var(ddof=1) / SEEDS + y.var(ddof=1) / SEEDS)
        assert diff <= max(0.02 * y.mean(), 4 * sig), ("mass", q, x.mean(), y.mean(), sig)
        worst_mass = max(worst_mass, diff / y.mean())
        x, y = la[:, q], lb[:, q]
        diff, sig = abs(x.mean() - y.mean()), np.sqrt(x.var(ddof=1) / SEEDS + y.var(ddof=1) / SEEDS)
        assert diff <= max(0.05, 4 * sig), ("log m", q, x.mean(), y.mean(), sig)
        worst_log = max(worst_log, diff)
    print(f"grouping dm 1e-3 vs 2.5e-4 over {len(tested)} bins: bin mass within {worst_mass:.3g}, "
          f"mean log10 m within {worst_log:.3g} dex; events {ev_a} vs {ev_b}")
