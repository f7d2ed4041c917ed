"""Workload definitions and seeded synthetic inputs.

This module is shared by the tests, the benchmark and the smoke check.  It
holds parameter tables and random-input recipes only: none of the method's
arithmetic.  It imports neither the CUDA binding nor the oracle.

The disk parameters are the paper's Benchmark table (gas surface density and
temperature at 1 AU, alpha, v_frag, erosion mass ratio, p, q); everything the
paper does not give (dust-to-gas ratio, radial extent, monomer size and
density, stellar mass, molecular constants, grouping and fragment-slope
parameters) is a stated reading.
"""
from __future__ import annotations

import numpy as np

AU = 1.495978707e13  # cm
YR = 3.15576e7       # s (Julian year)

# relative-velocity term switches and transport switches (shared numbering)
DV_ALL = 31
TR_RADIAL, TR_VERTICAL, TR_ST_MIDPLANE = 1, 2, 4


def benchmark_disk(**over) -> dict:
    """The paper's Benchmark-table disk (CGS), with the readings filled in."""
    d = dict(
        sigma0=1000.0, p=1.0, T0=280.0, q=0.5, alpha=1e-3, v_frag=1000.0, erosion_ratio=10.0,
        dust_to_gas=0.01, r_in=1.0 * AU, r_out=100.0 * AU, m_star=1.0, rho_s=1.6, a_mono=1e-4,
        mu=2.34, sigma_h2=2e-15, dm_group=1e-3, frag_xi=11.0 / 6.0, erosion_chi=1.0,
        K_const=1.0, V_const=1.0, m_init=0.0, M_total=0.0, frag_ramp=0.0,
        kernel_mode=0, settle_form=0, dv_flags=DV_ALL, tr_flags=TR_RADIAL | TR_VERTICAL,
    )
    d.update(over)
    return d


def constant_kernel_cell(**over) -> dict:
    """0D well-mixed cell, constant kernel K = 1, V = 1, monomers of mass 1,
    total mass 1 (so the initial monomer number density is 1)."""
    d = benchmark_disk(kernel_mode=1, K_const=1.0, V_const=1.0, m_init=1.0, M_total=1.0, dm_group=0.0,
                       tr_flags=0)
    d.update(over)
    return d


# ---- the five workloads -------------------------------------------------
WORKLOADS = {
    "0d_const_200": dict(params=constant_kernel_cell(), n_r=1, n_z=1, per_cell=200, t_end=100.0, seed=0),
    "disk2d_16x4x100": dict(params=benchmark_disk(), n_r=16, n_z=4, per_cell=100, t_end=1e4 * YR, seed=0),
    "disk2d_256x16x200": dict(params=benchmark_disk(), n_r=256, n_z=16, per_cell=200, t_end=1e4 * YR, seed=0),
    "stress_1024x32x400": dict(params=benchmark_disk(alpha=1e-2, v_frag=100.0), n_r=1024, n_z=32, per_cell=400,
                               t_end=1e3 * YR, seed=0),
}


def batched_disks(n_disks: int = 64, key=(2507, 0xB47C)):
    """64 independent disks: alpha in {1e-4,1e-3,1e-2}, v_frag in {1,3,10,30} m/s,
    radial zones uniform in 32..512 and particles per cell uniform in 50..400
    (drawn from numpy's Philox with the stated key), 8 vertical cells."""
    rng = np.random.Generator(np.random.Philox(key=list(key)))
    alphas = (1e-4, 1e-3, 1e-2)
    vfr = (100.0, 300.0, 1000.0, 3000.0)
    n_r = rng.integers(32, 513, size=n_disks)
    ppc = rng.integers(50, 401, size=n_disks)
    disks = []
    for d in range(n_disks):
        disks.append(dict(params=benchmark_disk(alpha=alphas[d % 3], v_frag=vfr[(d // 3) % 4]),
                          n_r=int(n_r[d]), n_z=8, per_cell=int(ppc[d]), seed=d))
    return disks


def ppc_sweep(ppcs=(25, 50, 100, 200, 400), seeds: int = 4, n_r: int = 16, n_z: int = 4, **over):
    """A resolution sweep for one batched launch: the Benchmark-table disk at
    every particles-per-cell value in ppcs, `seeds` disks of each (seed k of a
    resolution is disk k of that resolution's block), n_r x n_z cells.
    Returns (params list, grid list, ppc of each disk)."""
    P = benchmark_disk(**over)
    params, grids, res = [], [], []
    for ppc in ppcs:
        for _ in range(seeds):
            params.append(dict(P))
            grids.append((n_r, n_z, int(ppc)))
            res.append(int(ppc))
    return params, grids, np.array(res)


# ---- random inputs for the unit-level parity tests ----------------------
def random_masses(n: int, seed: int, lo: float = 1e-12, hi: float = 1e4, ties: float = 0.1) -> np.ndarray:
    """Log-uniform masses over [lo, hi] with a fraction of exact repeats and of
    near-repeats (relative offsets 1e-9..1e-3), so that equal and nearly equal
    pairs occur."""
    rng = np.random.default_rng(seed)
    m = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    k = int(ties * n)
    if k and n > 2:
        src = rng.integers(0, n, k)
        dst = rng.integers(0, n, k)
        m[dst] = m[src]
        dst2 = rng.integers(0, n, k)
        m[dst2] = m[rng.integers(0, n, k)] * (1.0 + np.exp(rng.uniform(np.log(1e-9), np.log(1e-3), k)))
    return m


def random_cell_positions(n: int, seed: int, params: dict) -> tuple[np.ndarray, np.ndarray]:
    """Random (r, z) inside the disk; z scaled by a rough aspect ratio 0.05 r."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(params["r_in"], params["r_out"], n)
    z = rng.normal(0.0, 1.0, n) * 0.05 * r
    return r, z


def midrun_state(params: dict, N: int, seed: int, a_max_1au: float = 10.0, a_slope: float = -1.0,
                 settle_a: float = 1e-2):
    """Synthetic particle state shaped like a disk in growth/fragmentation
    balance, for timing steps away from the all-monomer start.

    Recipe (numpy, seeded): r uniform on [r_in, r_out] (the dust-mass
    distribution of a p = 1 disk); radii from a mass-weighted n(a) ~ a^-3.5
    between a_mono and a_max(r) = a_max_1au (r/AU)^a_slope (at least a_mono);
    z ~ N(0, h) with h = 0.0334 AU (r/AU)^1.25 / sqrt(1 + a/settle_a), a
    flared scale height that shrinks for large grains.  Returns (m, r, z) for
    ids 0..N-1; swarm masses and ids come from the initial state."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x5EED]))
    r = rng.uniform(params["r_in"], params["r_out"], N)
    a0 = params["a_mono"]
    amax = np.maximum(a0, a_max_1au * (r / AU) ** a_slope)
    u = rng.uniform(size=N)
    a = (np.sqrt(a0) + u * (np.sqrt(amax) - np.sqrt(a0))) ** 2
    m = 4.0 / 3.0 * np.pi * params["rho_s"] * a**3
    h = 0.0334 * AU * (r / AU) ** 1.25 / np.sqrt(1.0 + a / settle_a)
    z = rng.normal(size=N) * h
    return m, r, z


# ---- a gas disk tabulated in radius -------------------------------------
def gap_bump_gas_table(params: dict, n: int = 64, r_lo_au: float = 1.5, r_hi_au: float = 80.0,
                       noise: float = 0.0, seed: int = 0) -> np.ndarray:
    """Knots (r, Sigma_g, T), an (n, 3) array: a synthetic stand-in for the
    azimuthally averaged profile of a hydrodynamic snapshot (no snapshot data
    is at hand).  The disk's power laws with a gap at 10 AU (surface density
    down by 90 %, as a planet carves one), a pressure bump at 20 AU (three
    times the background), a temperature break at 10 AU (slope q inside,
    q + 1/4 outside) and, if noise > 0, seeded relative noise of that size on
    every knot.  Knots are log-spaced over [r_lo_au, r_hi_au]."""
    x = np.geomspace(r_lo_au, r_hi_au, n)
    S = params["sigma0"] * x ** -params["p"]
    S = S * (1 - 0.9 * np.exp(-((x - 10.0) ** 2) / (2 * 1.5**2))) * (1 + 3.0 * np.exp(-((x - 20.0) ** 2) / (2 * 2.0**2)))
    q = params["q"]
    T = np.where(x < 10.0, params["T0"] * x**-q, params["T0"] * 10.0**-q * (x / 10.0) ** -(q + 0.25))
    if noise > 0:
        rng = np.random.default_rng(seed)
        S = S * (1 + noise * rng.standard_normal(n))
        T = T * (1 + noise * rng.standard_normal(n))
    return np.c_[x * AU, S, T]
