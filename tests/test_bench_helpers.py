"""bench.py's reporting helpers on fixed inputs (no GPU): the per-kernel rooflines from a
kernel_ms profile and the workload's sizes, and the chain's flop count."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

C3_RANKS = [1, 9, 44, 177, 480, 180, 49, 10, 1]
# per-kernel totals (ms, launches) of three bench steps on the d = 3 workload
PROF = {"apply": (1.23, 3), "domain": (9.3, 768), "mode_transform": (111.3, 24), "dgemm": (435.3, 36),
        "householder": (1665.4, 27), "jacobi": (720.1, 42), "theta_core": (53.1, 768), "chain_tc": (1287.0, 768)}


def test_kernel_rooflines_from_a_profile():
    r = bench.kernel_rooflines(PROF, 3, C3_RANKS, 3, 2, 12, 1_000_000, 6754.1, 1.25)
    # apply: 3 launches x 4 B x (1M x 177 + 1M x 180 + 2M)
    assert r["apply"]["bytes"] == pytest.approx(3 * 4.0 * (177e6 + 180e6 + 2e6))
    assert r["apply"]["achieved_gbs"] == pytest.approx(r["apply"]["bytes"] / 1.23e-3 / 1e9)
    assert r["domain"]["bytes"] == pytest.approx(768 * 4.0 * 2 * 1e6 * 3)
    assert r["mode_transform"]["bytes"] == pytest.approx(3 * 4 * 24.0 * 12.0 ** 8)
    for k in ("apply", "domain", "mode_transform"):
        assert 0.0 < r[k]["frac"] < 1.5
    # dgemm: the projections X <- G_k^T X, 2 r_k n^{D-k} r_{k-1} n flops each, 3 steps
    proj = sum(2.0 * C3_RANKS[k] * 12.0 ** (8 - k) * C3_RANKS[k - 1] * 12 for k in range(1, 8))
    assert r["dgemm"]["achieved"] == pytest.approx(3 * proj / 0.4353 / 1e12)
    assert 0.0 < r["dgemm"]["frac_lower_bound"] < 1.5
    for k in ("householder", "jacobi", "theta_core"):
        assert r[k]["frac"] is None and r[k]["note"]
    assert "chain_tc" not in r  # reported by the main roofline


def test_kernel_rooflines_skip_missing_or_empty_entries():
    r = bench.kernel_rooflines({"apply": (0.0, 0)}, 3, C3_RANKS, 3, 2, 12, 1000, 6754.1, 1.25)
    assert r == {}


def test_chain_flops_counts_both_sides():
    # 2 n N (sum over the source cores + sum over the target cores of r_{i-1} r_i)
    f = bench.chain_flops(C3_RANKS, 3, 2, 12, 1)
    src = 1 * 9 + 9 * 44 + 44 * 177
    tgt = 1 * 10 + 10 * 49 + 49 * 180
    assert f == 2.0 * 12 * (src + tgt)
    assert math.isclose(f, 196632 + 223680)
