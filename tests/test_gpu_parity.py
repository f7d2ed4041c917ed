"""GPU path against the CPU oracle, through the C ABI.

Tolerances: FP64 path 1e-12 relative on kernel entries, rates, row sums and
displacements; mixed path 1e-5; regrid permutations, counts, bounds and
volumes bit-exact; stochastic trajectories with identical keys event by
event (FP64) and by moments (mixed).
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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    d = np.abs(a - b)
    s = np.abs(b)
    out = np.where(s > 0, d / np.where(s > 0, s, 1), d)
    return float(out.max()) if out.size else 0.0


# ------------------------------------------------------------ kernel entries ---
PAIR_CASES = [
    ("all", W.benchmark_disk(), 1.0, 0.0),
    ("all_z", W.benchmark_disk(), 2.5, 1.3),
    ("outer", W.benchmark_disk(), 70.0, 0.4),
    ("settle_form1", W.benchmark_disk(settle_form=1), 3.0, 2.0),
    ("bm_only", W.benchmark_disk(dv_flags=1), 1.0, 0.2),
    ("turb_only", W.benchmark_disk(dv_flags=2), 1.0, 0.2),
    ("rad_only", W.benchmark_disk(dv_flags=4), 5.0, 0.0),
    ("phi_only", W.benchmark_disk(dv_flags=8), 5.0, 0.0),
    ("set_only", W.benchmark_disk(dv_flags=16), 5.0, 1.0),
    ("alpha1e-2", W.benchmark_disk(alpha=1e-2), 1.0, 0.5),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,P,r_au,zH", PAIR_CASES, ids=[c[0] for c in PAIR_CASES])
def test_pair_entries(prec, name, P, r_au, zH):
    rc = r_au * AU
    zc = zH * oracle.gas(P, rc, 0.0)["H"][0]
    m = W.random_masses(40_000, seed=hash(name) % 1000, lo=1e-12, hi=1e8)
    mi, mj = m[:20_000], m[20_000:]
    # the drag-law switch and the turbulence-regime edges, approached from both sides
    g = oracle.gas(P, rc, zc)
    msw = 4 / 3 * np.pi * P["rho_s"] * g["asw"][0] ** 3
    edge = msw * (1 + np.array([-1e-3, -1e-6, 1e-6, 1e-3]))
    mi = np.concatenate([mi, edge, edge[::-1], mi[:4]])
    mj = np.concatenate([mj, edge[::-1], edge * 1.5, mi[:4]])
    ref = oracle.pairs(P, rc, zc, mi, mj)
    ti, tj = dev(mi), dev(mj)
    dv, K = torch.empty_like(ti), torch.empty_like(ti)
    mcd.mcd_pair_probe(P, prec, rc, zc, ti, tj, dv, K)
    torch.cuda.synchronize()
    eps = _conditioning(P, rc, zc, mi, mj, ref)
    for got, want in ((K.cpu().numpy(), ref["K"]), (dv.cpu().numpy(), ref["dv"])):
        err = np.abs(got - want)
        assert np.all(err <= (TOL[prec] + 10 * eps) * np.abs(want)), float(np.max(err / np.maximum(np.abs(want), 1e-300)))
    # the allowance is confined to the ill-conditioned pairs
    assert np.mean(eps > TOL[prec]) < 0.01


def _conditioning(P, rc, zc, mi, mj, ref):
    """Relative uncertainty of dv that FP64 itself leaves: |St_i - St_j| of a
    pair straddling the drag-law switch carries the ulp of the switch mass
    (4e-16 St / dSt), and 1 - St_i St_j carries 4e-16 St_i St_j / |1 - St_i St_j|;
    each enters dv through the share of the terms it multiplies."""
    _, Si, ki = oracle.particle(P, rc, zc, mi)
    _, Sj, kj = oracle.particle(P, rc, zc, mj)
    D, t = ref["dst"], ref["terms"]
    T = t.sum(axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        c_sw = np.where((ki != kj) & (D > 0), 4e-16 * np.maximum(Si, Sj) / np.where(D > 0, D, 1.0), 0.0)
        c_om = 4e-16 * Si * Sj / np.maximum(np.abs(1.0 - Si * Sj), 1e-300)
        eps = np.where(T > 0, ((t[:, 1] + t[:, 2] + t[:, 3] + t[:, 4]) * c_sw + t[:, 2] * c_om) / np.where(T > 0, T, 1.0),
                       0.0)
    return eps


# --------------------------------------------------------------- rate matrix ---
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,dm,mode", [(1, 1e-3, 0), (2, 0.0, 0), (37, 1e-3, 0), (200, 1e-2, 0), (333, 0.0, 0),
                                       (1024, 1e-3, 0), (64, 0.0, 1)])
def test_rate_matrix(prec, n, dm, mode):
    P = W.benchmark_disk(dm_group=dm) if mode == 0 else W.constant_kernel_cell()
    rng = np.random.default_rng(n)
    m = W.random_masses(n, seed=n + 7, lo=1e-12, hi=1e3) if mode == 0 else rng.integers(1, 50, n).astype(float)
    M = rng.uniform(1e25, 1e27, n) if mode == 0 else np.full(n, 1.0 / n)
    rc, zc, V = 1.7 * AU, 2e11, 3e39
    rate_o, R_o = oracle.rate_matrix(P, rc, zc, V, m, M)
    rate = torch.empty((n, n), dtype=torch.float64, device="cuda")
    R = torch.empty(n, dtype=torch.float64, device="cuda")
    mcd.mcd_rate_probe(P, prec, rc, zc, V, dev(m), dev(M), rate, R)
    torch.cuda.synchronize()
    assert rel(rate.cpu().numpy(), rate_o) < TOL[prec]
    assert rel(R.cpu().numpy(), R_o) < TOL[prec]


# -------------------------------------------------------------------- regrid ---
def _make_ctx(params, grids, seed=0, prec=mcd.MCD_FP64):
    return mcd.Disk(params, grids, seed=seed, prec=prec)


def _state(N, seed, P, dead=0, ties=True):
    rng = np.random.default_rng(seed)
    r = rng.uniform(P["r_in"], 0.3 * P["r_out"], N)
    z = rng.normal(0, 1, N) * 0.03 * r
    if ties and N > 6:
        r[1] = r[0]
        r[5] = r[4]
        z[3] = z[2]
        z[4] = -0.0
        z[6] = 0.0
    if dead:
        r[rng.choice(N, dead, replace=False)] = np.inf
    m = W.random_masses(N, seed=seed + 1, lo=1e-11, hi=1e-2)
    M = np.full(N, 1e26)
    ids = rng.permutation(N).astype(np.uint32)
    return m, M, r, z, ids


@pytest.mark.parametrize("grids,dead", [([(4, 3, 5)], 0), ([(4, 3, 5)], 7), ([(1, 1, 9)], 0),
                                        ([(16, 4, 100), (3, 5, 7), (7, 1, 13)], 11), ([(5, 7, 3)], 90),
                                        ([(64, 16, 12)], 100)])
def test_regrid_bit_exact(grids, dead):
    P = W.benchmark_disk()
    d = _make_ctx([P] * len(grids), grids)
    states = []
    for k, g in enumerate(grids):
        N = g[0] * g[1] * g[2]
        st = _state(N, 100 + k, P, dead=min(dead, N - 1))
        states.append(st)
        mcd.mcd_set_particles(d.ctx, k, *st)
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    for k, g in enumerate(grids):
        nr, nz = g[0], g[1]
        s = oracle.DiskState(*states[k])
        st, perm, off, cb, cv, na = oracle.regrid(P, nr, nz, s)
        got = d.particles(k)
        assert np.array_equal(got["id"], s.id)
        for key in ("m", "M", "r", "z"):
            assert np.array_equal(got[key].view(np.uint64), getattr(s, key).view(np.uint64)), key
        goff = np.zeros(nr * nz + 1, np.int64)
        gb = np.zeros((nr * nz, 6))
        gv = np.zeros(nr * nz)
        mcd.mcd_get_cells(d.ctx, k, goff, gb, gv)
        assert np.array_equal(goff, off)
        # single-particle zones/cells take +-H/2 from the gas functions (ulp-level); all others bit-exact
        n_cell = np.diff(off)
        exact = n_cell != 1
        assert np.array_equal(gb[exact].view(np.uint64), cb[exact].view(np.uint64))
        assert np.array_equal(gv[exact].view(np.uint64), cv[exact].view(np.uint64))
        assert rel(gb, cb) < 1e-14 and rel(gv, cv) < 1e-13
        assert mcd.mcd_get_stats(d.ctx, k).n_alive == na
    d.close()


@pytest.mark.parametrize("kind", ["all_equal", "three_levels", "short_runs"])
def test_regrid_equal_heights_bit_exact(kind):
    """Heights that repeat within a zone: every height equal, three distinct
    heights (runs longer than the in-place tie fix-up takes), and heights
    rounded so that runs of equal heights stay short.  The cells' (z, id)
    order, counts and bounds equal the oracle's."""
    P = W.benchmark_disk()
    grid = (4, 8, 100)
    N = grid[0] * grid[1] * grid[2]
    rng = np.random.default_rng(21)
    r = rng.uniform(P["r_in"], 0.3 * P["r_out"], N)
    if kind == "all_equal":
        z = np.zeros(N)
    elif kind == "three_levels":
        z = rng.choice([-1e11, 0.0, 2e11], N)
    else:
        z = np.round(rng.normal(0, 1, N) * 30) * 1e10  # ~60 distinct heights per zone of 800
    z[::97 if kind == "short_runs" else 7] = -0.0  # negative zero orders with +0 (short_runs: runs stay short)
    m = W.random_masses(N, seed=22, lo=1e-11, hi=1e-2)
    M = np.full(N, 1e26)
    ids = rng.permutation(N).astype(np.uint32)
    d = _make_ctx(P, grid)
    mcd.mcd_set_particles(d.ctx, 0, m, M, r, z, ids)
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
    mcd.mcd_get_cells(d.ctx, 0, goff, gb, None)
    assert np.array_equal(goff, off)
    n_cell = np.diff(off)
    exact = n_cell != 1
    assert np.array_equal(gb[exact].view(np.uint64), cb[exact].view(np.uint64))
    d.close()


# ----------------------------------------------------------------- transport ---
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("flags", [3, 1, 2, 2 | 4])
def test_transport(prec, flags):
    P = W.benchmark_disk(tr_flags=flags)
    grid = (8, 4, 250)
    N = 8 * 4 * 250
    d = _make_ctx(P, grid, seed=9, prec=prec)
    rng = np.random.default_rng(4)
    r = rng.uniform(P["r_in"], P["r_out"], N)
    r[:50] = P["r_in"] * (1 + rng.uniform(0, 1e-3, 50))  # some leave through the inner edge
    r[50:100] = P["r_out"] * (1 - rng.uniform(0, 1e-3, 50))  # some are reflected
    H = oracle.gas(P, r, np.zeros(N))["H"]
    z = rng.normal(0, 1, N) * H
    m = W.random_masses(N, seed=5, lo=1e-12, hi=1e4)
    M = np.full(N, 3e26)
    ids = rng.permutation(N).astype(np.uint32)
    mcd.mcd_set_particles(d.ctx, 0, m, M, r, z, ids)
    dt = 30 * YR
    mcd.mcd_transport(d.ctx, dt)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    got = d.particles()
    s = oracle.DiskState(m, M, r, z, ids)
    oracle.transport(P, s, dt, seed=9, disk=0, step=0)
    gone_o = ~np.isfinite(s.r)
    gone_g = ~np.isfinite(got["r"])
    if flags & 1:
        assert gone_o.sum() > 0
    assert np.array_equal(gone_o, gone_g)
    keep = ~gone_o
    g = oracle.gas(P, r[keep], z[keep])
    sig = np.sqrt(2 * g["D"] * dt)
    tol = TOL[prec]
    assert np.all(np.abs(got["r"][keep] - s.r[keep]) <= tol * (np.abs(s.r[keep] - r[keep]) + sig) + 1e-15 * r[keep])
    assert np.all(np.abs(got["z"][keep] - s.z[keep]) <= tol * (np.abs(s.z[keep] - z[keep]) + sig) + 1e-15 * np.abs(z[keep]))
    acc = mcd.mcd_get_stats(d.ctx, 0).accreted_mass
    assert acc == pytest.approx(s.accreted, rel=1e-12)
    d.close()


# ----------------------------------------------------------------- collide ---
def _one_cell(P, n, seed, prec, masses, r_au=1.3, M=None):
    d = _make_ctx(P, (1, 1, n), seed=seed, prec=prec)
    rng = np.random.default_rng(seed)
    r = r_au * AU * (1 + rng.uniform(-0.05, 0.05, n))
    z = rng.normal(0, 1, n) * 2e11
    M = np.full(n, 2e26) if M is None else M
    ids = np.arange(n, dtype=np.uint32)
    mcd.mcd_set_particles(d.ctx, 0, masses, M, r, z, ids)
    mcd.mcd_regrid(d.ctx)
    off = np.zeros(2, np.int64)
    b = np.zeros((1, 6))
    V = np.zeros(1)
    mcd.mcd_get_cells(d.ctx, 0, off, b, V)
    cell = d.particles()
    return d, cell, b[0], V[0]


@pytest.mark.parametrize("mode,n,vfrag,dm,extra", [
    ("phys", 50, 300.0, 1e-3, {}), ("phys", 200, 1000.0, 1e-2, {}), ("phys", 96, 30.0, 0.0, {}),
    ("const", 200, 0, 0, {}),
    # outcome variants: a fragmentation ramp, another fragment slope xi, another erosion efficiency chi
    ("phys", 120, 100.0, 1e-3, {"frag_ramp": 0.6}),
    ("phys", 120, 60.0, 1e-3, {"frag_ramp": 0.3, "frag_xi": 1.5, "erosion_chi": 0.5}),
], ids=["vf300", "vf1000", "vf30", "const", "ramp", "ramp_xi_chi"])
def test_event_sequence_fp64(mode, n, vfrag, dm, extra):
    """Same keys, FP64: the GPU event chain is the oracle's, event by event."""
    seed = 21
    if mode == "const":
        P = W.constant_kernel_cell()
        masses = np.ones(n)
    else:
        P = W.benchmark_disk(v_frag=vfrag, dm_group=dm, **extra)
        masses = W.random_masses(n, seed=3, lo=1e-11, hi=1e-1, ties=0.2)
    d, cell, b, V = _one_cell(P, n, seed, mcd.MCD_FP64, masses, M=np.full(n, 1.0 / n) if mode == "const" else None)
    Vo = V if mode == "phys" else 1.0
    R = oracle.rate_matrix(P, b[4], b[5], Vo, cell["m"], cell["M"])[1]
    t_end = (10.0 if mode == "const" else 600.0 / R.sum())
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_LOG_CELL, 0)
    mcd.mcd_collide(d.ctx, t_end)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    ijo, t, mnew, nlog = mcd.mcd_get_event_log(d.ctx, 100000)
    st, m_o, ev_o, _, lg = oracle.collide_cell(P, b[4], b[5], Vo, cell["m"], cell["M"], 0.0, t_end, seed, 0, 0, 0,
                                               log_cap=100000)
    assert ev_o > 100 and nlog == ev_o
    assert np.array_equal(ijo[:, 0], lg["i"]) and np.array_equal(ijo[:, 1], lg["j"])
    assert np.array_equal(ijo[:, 2], lg["outcome"])
    assert rel(t, lg["t"]) < 1e-12
    assert rel(mnew, lg["m_new"]) < 1e-12
    got = d.particles()
    assert rel(got["m"], m_o) < 1e-12
    ce = np.zeros(1, np.int64)
    mcd.mcd_get_cell_events(d.ctx, 0, ce)
    assert ce[0] == ev_o
    d.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,k", [(8, 40), (64, 300), (250, 500)])
def test_row_sums_after_events(prec, n, k):
    """After k events the incrementally kept R_i equal an O(n^2) recomputation
    (oracle) from the masses the GPU reached."""
    P = W.benchmark_disk(v_frag=100.0, dm_group=1e-3)
    masses = W.random_masses(n, seed=n, lo=1e-11, hi=1e1)
    d, cell, b, V = _one_cell(P, n, 5, prec, masses)
    for key, v in ((mcd.MCD_OPT_MAX_EVENTS, k), (mcd.MCD_OPT_CAP_STOPS, 1), (mcd.MCD_OPT_DUMP_R, 1),
                   (mcd.MCD_OPT_REBUILD_EVERY, 10**9)):
        mcd.mcd_set_option(d.ctx, key, v)
    mcd.mcd_collide(d.ctx, 1e30)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    ce = np.zeros(1, np.int64)
    mcd.mcd_get_cell_events(d.ctx, 0, ce)
    assert ce[0] == k
    got = d.particles()
    R = np.zeros(n)
    mcd.mcd_get_rates(d.ctx, 0, R)
    _, Rb = oracle.rate_matrix(P, b[4], b[5], V, got["m"], got["M"])
    assert rel(R, Rb) < TOL[prec]
    d.close()


def test_event_cap_latches_timeout():
    P = W.constant_kernel_cell()
    d = _make_ctx(P, (1, 1, 64))
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_MAX_EVENTS, 10)
    mcd.mcd_collide(d.ctx, 100.0)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_ETIMEOUT
    d.close()


def test_nan_position_latches_enan():
    P = W.benchmark_disk()
    d = _make_ctx(P, (2, 2, 4))
    p = d.particles()
    p["r"][3] = np.nan
    mcd.mcd_set_particles(d.ctx, 0, p["m"], p["M"], p["r"], p["z"], p["id"])
    mcd.mcd_regrid(d.ctx)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_ENAN
    d.close()


def test_out_of_order_and_bad_ids_rejected():
    P = W.benchmark_disk()
    d = _make_ctx(P, (2, 2, 4))
    mcd.mcd_transport(d.ctx, YR)
    with pytest.raises(mcd.McdError) as e:
        mcd.mcd_collide(d.ctx, 10 * YR)
    assert e.value.code == mcd.MCD_ESTATE
    p = d.particles()
    before = d.particles()
    p["id"][0] = p["id"][1]
    with pytest.raises(mcd.McdError):
        mcd.mcd_set_particles(d.ctx, 0, p["m"], p["M"], p["r"], p["z"], p["id"])
    after = d.particles()
    for key in before:  # a rejected replacement leaves the live state as it was
        assert np.array_equal(before[key], after[key]), key
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    d.close()


def test_set_particles_from_device_checks_ids():
    """Device arrays: bad ids (a repeat, one out of range) latch MCD_EINVAL and
    leave the state as it was; a permutation replaces it."""
    P = W.benchmark_disk()
    d = _make_ctx(P, (2, 2, 4))
    before = d.particles()
    n = before["id"].size
    cols = {k: dev(before[k]) for k in ("m", "M", "r", "z")}
    for bad in (np.r_[before["id"][1], before["id"][1:]], np.r_[n + 3, before["id"][1:]]):
        idd = torch.tensor(bad.astype(np.int64), dtype=torch.int32, device="cuda")
        mcd.mcd_set_particles(d.ctx, 0, cols["m"], cols["M"], cols["r"], cols["z"], idd, mcd.MCD_DEVICE)
        assert mcd.mcd_sync(d.ctx) == mcd.MCD_EINVAL
        after = d.particles()
        for key in before:
            assert np.array_equal(before[key], after[key]), key
        d.close()
        d = _make_ctx(P, (2, 2, 4))
        before = d.particles()
    perm = np.random.default_rng(0).permutation(n).astype(np.int32)
    new_m = before["m"] * 2.0
    mcd.mcd_set_particles(d.ctx, 0, dev(new_m), cols["M"], cols["r"], cols["z"],
                          torch.tensor(perm, device="cuda"), mcd.MCD_DEVICE)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    got = d.particles()
    assert np.array_equal(got["m"], new_m) and np.array_equal(got["id"], perm.astype(np.uint32))
    d.close()


# -------------------------------------------------- constant kernel, batched ---
def test_constant_kernel_batched_matches_oracle_and_smoluchowski():
    """32 independent 0D cells in one context: every disk's final masses equal
    the oracle's bit for bit (integer sticking), and the pooled moments match
    the analytic Smoluchowski solution."""
    P = W.constant_kernel_cell()
    nd, n, t_end, seed = 32, 200, 100.0, 0
    d = _make_ctx([P] * nd, [(1, 1, n)] * nd, seed=seed)
    mcd.mcd_collide(d.ctx, t_end)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    means, sq = [], []
    for k in range(nd):
        got = d.particles(k)
        s = oracle.init_disk(P, n, seed, disk=k)
        oracle.regrid(P, 1, 1, s)  # the cell order the GPU path also reached
        st, m_o, ev, _, _ = oracle.collide_cell(P, 0.0, 0.0, 1.0, s.m, s.M, 0.0, t_end, seed, k, 0, 0)
        assert np.array_equal(got["m"][np.argsort(got["id"])], m_o[np.argsort(s.id)])
        means.append(got["m"].mean())
        sq.append((got["m"] ** 2).mean())
    for vals, ref in ((means, 1 + t_end), (sq, 1 + 3 * t_end + 1.5 * t_end**2)):
        v = np.array(vals)
        err = abs(v.mean() / ref - 1)
        assert err < max(0.02, 3 * v.std(ddof=1) / np.sqrt(nd) / ref)
    d.close()


# ------------------------------------------------------------ whole steps ---
def test_steps_fp64_match_oracle():
    """Three full steps (regrid, collide, transport) of a small disk with the
    same keys, about 6e5 events: the same event count and every particle's
    r, z, m as the oracle's."""
    P = W.benchmark_disk(dust_to_gas=0.5, v_frag=300.0)
    grid, seed, dt = (6, 3, 20), 4, 100 * YR
    d = _make_ctx(P, grid, seed=seed)
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


def test_batched_disk_equals_same_disk_in_other_batch():
    P = W.benchmark_disk(dust_to_gas=0.3)
    Q = W.benchmark_disk(alpha=1e-2, v_frag=100.0, dust_to_gas=0.3)
    a = _make_ctx([P, Q, P], [(5, 2, 11), (7, 3, 9), (2, 2, 5)], seed=8)
    b = _make_ctx([P, Q], [(3, 3, 3), (7, 3, 9)], seed=8)
    for _ in range(3):
        a.step(50 * YR)
        b.step(50 * YR)
    x, y = a.particles(1), b.particles(1)
    for key in ("m", "M", "r", "z", "id"):
        assert np.array_equal(x[key], y[key]), key
    a.close()
    b.close()


@pytest.mark.parametrize("prec", PRECS)
def test_graph_replay_equals_direct_launches(prec):
    P = W.benchmark_disk(dust_to_gas=0.3)
    a = _make_ctx(P, (8, 4, 30), seed=2, prec=prec)
    b = _make_ctx(P, (8, 4, 30), seed=2, prec=prec)
    mcd.mcd_set_option(b.ctx, mcd.MCD_OPT_USE_GRAPH, 0)
    for _ in range(5):
        a.step(40 * YR)
        b.step(40 * YR)
    x, y = a.particles(), b.particles()
    for key in ("m", "r", "z", "id"):
        assert np.array_equal(x[key], y[key]), key
    sa, sb = a.stats(), b.stats()
    assert sa.events == sb.events and sa.step == sb.step == 5 and sa.t == sb.t
    a.close()
    b.close()


DV_CASES = [(mcd.MCD_FP64, 1), (mcd.MCD_MIXED, 1), (mcd.MCD_MIXED, 2), (mcd.MCD_MIXED, 0)]


@pytest.mark.parametrize("prec,spt", DV_CASES, ids=["fp64", "mixed_s1", "mixed_s2", "mixed_control_warp"])
@pytest.mark.parametrize("grid,reb", [((8, 4, 30), 0), ((4, 2, 57), 7), ((1, 1, 200), 0), ((2, 2, 224), 13),
                                      ((1, 2, 312), 0), ((2, 1, 400), 11)])
def test_dv_matrix_equals_recompute(grid, reb, prec, spt):
    """Collide with each cell's symmetric dv matrix kept (circulant half form:
    mixed in shared memory up to ~314 swarms and in the workspace above, FP64
    in the workspace) reaches the same bits as the path that recomputes row i
    at every event, for one and two swarms per thread.  Mid-run state, so
    sticking, erosion and fragmentation all occur; reb > 0 also runs the full
    rebuilds from stored entries; 312 swarms is a class whose matrix just fits
    in shared memory, 400 one that takes the workspace matrix.  spt 0 runs the
    control-warp variant (one warp holds the row sums and chooses, one worker
    thread per swarm)."""
    P = W.benchmark_disk()
    N = grid[0] * grid[1] * grid[2]
    m, r, z = W.midrun_state(P, N, seed=3)
    # squeezed to 1..6 AU: ~10^3..10^4 events per cell and year
    r2 = P["r_in"] + (r - P["r_in"]) * (5.0 * AU / (P["r_out"] - P["r_in"]))
    r, z = r2, z * (r2 / r) ** 1.25
    out = []
    for mat in (1, 2, 0):
        d = _make_ctx(P, grid, seed=4, prec=prec)
        p = d.particles()
        mcd.mcd_set_particles(d.ctx, 0, m, p["M"], r, z, p["id"])
        opts = [(mcd.MCD_OPT_DV_MATRIX, mat), (mcd.MCD_OPT_REBUILD_EVERY, reb), (mcd.MCD_OPT_DUMP_R, 1)]
        opts += [(mcd.MCD_OPT_SWARMS_PER_THREAD, spt)] if spt else [(mcd.MCD_OPT_CONTROL_WARP, 1)]
        for key, v in opts:
            mcd.mcd_set_option(d.ctx, key, v)
        for _ in range(2):
            d.step(YR)
        assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
        k0 = mcd.mcd_get_collide_classes(d.ctx)[0]
        assert k0["control_warp"] == (spt == 0)
        store = k0["store"]
        R = np.zeros(N)
        mcd.mcd_get_rates(d.ctx, 0, R)
        out.append((d.particles(), d.stats().events, R, store))
        d.close()
    (x, ea, Ra, sa), (y, eb, Rb, sb), (w, ec, Rc, sc) = out
    assert sc == 0 and sa in (1, 2) and sb in (0, 2)  # the stored paths ran where a matrix exists
    if prec == mcd.MCD_FP64 or grid[2] > 314:
        assert sa == 2 and sb == 2
    assert ea == eb == ec and ea > 50
    for key in ("m", "r", "z", "id"):
        assert np.array_equal(x[key], w[key]), key
        assert np.array_equal(y[key], w[key]), key
    assert np.array_equal(Ra, Rc) and np.array_equal(Rb, Rc)


@pytest.mark.parametrize("prec", PRECS)
def test_moments_match_oracle(prec):
    """Diagnostics on the device equal the oracle's sums over the particles the
    GPU holds: counts exactly, sums to a few ulp (both compensated); edges that
    coincide with particle radii; the same bits on a repeated call."""
    P = W.benchmark_disk(dust_to_gas=0.1)
    d = _make_ctx(P, (8, 4, 50), seed=3, prec=prec)
    for _ in range(3):
        d.step(10 * YR)
    x = d.particles()
    edges = AU * np.geomspace(1.0, 100.0, 17)
    alive = np.sort(x["r"][np.isfinite(x["r"])])
    edges2 = np.concatenate([[0.0], alive[::97], [np.inf]])  # edges on particle radii
    for e in (edges, edges2):
        got = d.moments(e)
        want = oracle.moments(x["m"], x["M"], x["r"], e)
        assert np.array_equal(got[:, 4], want[:, 4])
        assert np.allclose(got, want, rtol=1e-14, atol=0.0)
        assert np.array_equal(d.moments(e), got)
    assert d.moments(edges2)[:, 4].sum() == alive.size
    with pytest.raises(mcd.McdError):
        d.moments(edges[::-1])
    with pytest.raises(mcd.McdError):
        d.moments(np.array([AU, np.nan, 2 * AU]))
    d.close()


@pytest.mark.parametrize("prec", PRECS)
def test_sigma_map_matches_oracle(prec):
    """The sigma_d(m, r) map on the device equals the oracle's on the particles
    the GPU holds (each M rounded to 2^-61 of the disk's mass at most; empty
    bins exactly zero); repeated calls give the same bits; bad edges rejected."""
    P = W.benchmark_disk(dust_to_gas=0.1)
    d = _make_ctx(P, (8, 4, 50), seed=5, prec=prec)
    for _ in range(3):
        d.step(10 * YR)
    x = d.particles()
    r_edges = AU * np.geomspace(1.0, 100.0, 25)
    m_edges = np.geomspace(1e-12, 1e6, 37)
    got = d.sigma_map(r_edges, m_edges)
    want = oracle.sigma_map(x["m"], x["M"], x["r"], r_edges, m_edges)
    assert np.array_equal(got == 0, want == 0)
    assert np.allclose(got, want, rtol=1e-12, atol=0.0)
    assert np.array_equal(d.sigma_map(r_edges, m_edges), got)
    alive = np.isfinite(x["r"])
    assert np.isclose(got.sum(), x["M"][alive].sum(), rtol=1e-12)
    with pytest.raises(mcd.McdError):
        d.sigma_map(r_edges[::-1], m_edges)
    with pytest.raises(mcd.McdError):
        d.sigma_map(r_edges, np.geomspace(1e-12, 1e6, 5000))
    d.close()


# ------------------------------------------------------------------- tracer ---
def test_tracer_event_chain_fp64_matches_oracle():
    """FP64, same keys: one cell's event chain leaves the tracer column the
    oracle's, for a chain with sticking, fragmentation and erosion."""
    P = W.benchmark_disk(v_frag=30.0, dm_group=1e-3)
    n = 60
    masses = W.random_masses(n, seed=9, lo=1e-6, hi=1e-2)
    d, cell, b, V = _one_cell(P, n, 21, mcd.MCD_FP64, masses)
    q0 = np.random.default_rng(4).uniform(0.1, 0.9, n)
    d.set_tracer(q0)
    R = oracle.rate_matrix(P, b[4], b[5], V, cell["m"], cell["M"])[1]
    t_end = 3000.0 / R.sum()
    mcd.mcd_collide(d.ctx, t_end)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    st, m_o, q_o, ev_o, _, _ = oracle.collide_cell_q(P, b[4], b[5], V, cell["m"], cell["M"], q0, 0.0, t_end, 21, 0,
                                                     0, 0)
    assert ev_o > 1000 and d.stats().events == ev_o
    assert rel(d.particles()["m"], m_o) < 1e-12
    assert rel(d.tracer(), q_o) < 1e-12
    d.close()


def test_tracer_steps_fp64_match_oracle():
    """Three full FP64 steps with the tracer a function of the id on both
    sides: every particle's tracer equals the oracle's."""
    P = W.benchmark_disk(dust_to_gas=0.5, v_frag=300.0)
    grid, seed, dt = (6, 3, 20), 4, 100 * YR
    d = _make_ctx(P, grid, seed=seed)
    f = lambda ids: 0.1 + 0.8 * (ids.astype(float) % 7) / 6.0
    d.set_tracer(f(d.particles()["id"]))
    s = oracle.init_disk(P, 6 * 3 * 20, seed)
    s.q = f(s.id)
    for _ in range(3):
        d.step(dt)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK
    oracle.run(P, 6, 3, s, 0.0, dt, 0, 3, seed)
    got, q = d.particles(), d.tracer()
    go, so = np.argsort(got["id"]), np.argsort(s.id)
    assert mcd.mcd_get_stats(d.ctx, 0).events == s.events > 100_000
    assert rel(q[go], s.q[so]) < 1e-10
    assert not np.array_equal(q[go], f(got["id"][go]))  # the tracer did change
    d.close()


def test_tracer_mixed_invariants_regrid_and_switch_off():
    """Mixed path: a uniform tracer stays uniform and a spread one stays in its
    range over full steps; the tracer follows its particle through a regrid;
    get/set round trip; switching the tracer off clears it."""
    P = W.benchmark_disk(dust_to_gas=0.3)
    d = _make_ctx(P, (8, 4, 30), seed=2, prec=mcd.MCD_MIXED)
    d.set_tracer(np.full(8 * 4 * 30, 0.25))
    for _ in range(3):
        d.step(40 * YR)
    assert mcd.mcd_sync(d.ctx) == mcd.MCD_OK and d.stats().events > 1000
    assert np.allclose(d.tracer(), 0.25, rtol=1e-14, atol=0)
    ids = d.particles()["id"]
    q0 = 0.2 + 0.6 * (ids % 11) / 10.0
    d.set_tracer(q0)
    assert np.array_equal(d.tracer(), q0)
    mcd.mcd_regrid(d.ctx)
    x = d.particles()
    assert np.array_equal(d.tracer(), 0.2 + 0.6 * (x["id"] % 11) / 10.0)
    for _ in range(3):
        d.step(40 * YR)
    q = d.tracer()
    assert q.min() >= 0.2 * (1 - 1e-12) and q.max() <= 0.8 * (1 + 1e-12)
    mcd.mcd_set_option(d.ctx, mcd.MCD_OPT_TRACER, 0)
    assert np.array_equal(d.tracer(), np.zeros_like(q))
    d.close()
