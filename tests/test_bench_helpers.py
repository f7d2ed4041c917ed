"""The benchmark's host-side arithmetic on CPU: the collide's algorithmic
shared-memory bytes and flops behind the roofline fractions, and the
profiling pin of the collide variant."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_collide_smem_bytes_counts_builds_and_events():
    # 200 swarms, 800 events: the build at the start and one rebuild after 4n = 800 events
    b = bench.collide_smem_bytes([200], [800])
    assert b == 52 * 200**2 * 2 + 60 * 200 * 800
    # 799 events: no rebuild yet; an empty cell costs nothing
    assert bench.collide_smem_bytes([200, 0], [799, 5]) == 52 * 200**2 + 60 * 200 * 799
    # cells add up
    n, e = [64, 128, 400], [0, 1000, 10]
    assert bench.collide_smem_bytes(n, e) == sum(bench.collide_smem_bytes([a], [b]) for a, b in zip(n, e))


def test_collide_rooflines_from_per_step_loads():
    n_c = np.array([[200.0, 100.0], [200.0, 100.0]])
    ev_c = np.array([[1000.0, 10.0], [500.0, 0.0]])
    pk = {"smem_gbs": 40000.0}
    alu, smem = bench.collide_rooflines(n_c, ev_c, 2, 2.0, pk, 80.0)
    entries = (2 * (200 * 201 / 2 + 100 * 101 / 2) + 200 * 1500 + 100 * 10) / 2
    assert abs(alu["achieved"] - entries * bench.FLOPS_PER_ENTRY / 2e-3 / 1e12) < 1e-9
    assert alu["bound"] == "alu" and smem["bound"] == "smem"
    bytes_step = (bench.collide_smem_bytes(n_c[0], ev_c[0]) + bench.collide_smem_bytes(n_c[1], ev_c[1])) / 2
    assert abs(smem["achieved"] - bytes_step / 2e-3 / 1e9) < 1e-9
    assert abs(smem["frac"] - smem["achieved"] / 40000.0) < 1e-15


class _FakeMcd:
    MCD_OPT_CONTROL_WARP, MCD_OPT_SWARMS_PER_THREAD, MCD_OPT_DV_MATRIX = 18, 14, 10

    def __init__(self):
        self.calls = []

    def mcd_set_option(self, ctx, key, value):
        self.calls.append((key, value))


class _FakeDisk:
    ctx = 0


def test_pin_variant_sets_the_options():
    m = _FakeMcd()
    bench.pin_variant(m, _FakeDisk(), "2,0")
    assert m.calls == [(14, 2), (10, 0)]
    m = _FakeMcd()
    bench.pin_variant(m, _FakeDisk(), "cw,1")
    assert m.calls == [(18, 1), (10, 1)]
