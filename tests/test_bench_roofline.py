"""The roofline accounting of the bench line (host logic, no GPU).

The symmetric near field evaluates every unordered pair of points once (pairs
of distinct leaves, and the pairs within one leaf by the cyclic schedule), so
its algorithmic work is the number of unordered pairs times the operations of
one pair in both directions; the per-point kernel evaluates every ordered
pair.  The DRAM traffic of the symmetric kernel follows the points.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def leaf_counts():
    return np.array([61, 64, 1, 0, 33], dtype=np.int64)


def test_symmetric_kernel_counts_unordered_pairs():
    n = leaf_counts()
    self_ordered = int(np.sum(n * (n - 1)))
    cross_unordered = 1000
    pairs = self_ordered + 2 * cross_unordered  # ordered evaluations in the lists
    r = bench.roofline(True, pairs, 1.0, self_ordered, n_points=int(n.sum()), clusters=True)
    per = bench.MIXED_OPS_PER_PAIR + bench.SYM_EXTRA_OPS_PER_PAIR
    assert r["unordered_pairs"] == cross_unordered + self_ordered // 2
    assert r["unordered_pairs_within_leaves"] == self_ordered // 2
    assert r["ops_per_unordered_pair"] == per
    assert np.isclose(r["achieved"], r["unordered_pairs"] * per / 1e-3 / 1e12)
    assert np.isclose(r["frac"], r["achieved"] / r["peak"])
    assert r["traffic"] == round(bench.P2P_SYM_DRAM_BYTES_PER_POINT * n.sum())
    assert r["bound"] == "alu"


def test_symmetric_fp64_counts_unordered_pairs():
    n = leaf_counts()
    self_ordered = int(np.sum(n * (n - 1)))
    pairs = self_ordered + 2 * 777
    r = bench.roofline(False, pairs, 2.0, self_ordered)
    per = bench.FP64_FLOPS_PER_PAIR + bench.FP64_SYM_EXTRA_FLOPS
    assert r["unordered_pairs"] == 777 + self_ordered // 2
    assert np.isclose(r["achieved"], r["unordered_pairs"] * per / 2e-3 / 1e12)


def test_per_point_kernel_counts_ordered_pairs():
    r = bench.roofline(True, 5000, 0.5)
    assert np.isclose(r["achieved"], 5000 * bench.MIXED_OPS_PER_PAIR / 0.5e-3 / 1e12)
    assert r["traffic"] is None
    r = bench.roofline(False, 5000, 0.5)
    assert np.isclose(r["achieved"], 5000 * bench.FP64_FLOPS_PER_PAIR / 0.5e-3 / 1e12)


def test_traffic_only_for_the_captured_workload():
    # the per-point DRAM figure was captured on the log kernel and the cluster workload
    n = leaf_counts()
    self_ordered = int(np.sum(n * (n - 1)))
    assert bench.roofline(True, self_ordered, 1.0, self_ordered, n_points=100,
                          clusters=False)["traffic"] is None
    assert bench.roofline(True, self_ordered, 1.0, self_ordered, harmonic=True, n_points=100,
                          clusters=True)["traffic"] is None
