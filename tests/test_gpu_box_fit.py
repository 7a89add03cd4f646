"""Shrink-wrapped box geometry (option box_fit = 1) against the oracle.

The splits (and so the permutations and split rectangles) are unchanged; the
bounding rectangles of every box's points must match the oracle's bit for
bit, the lists built on them likewise, and the potentials the oracle FMM on
the same geometry (FP64 1e-12, mixed 1e-11).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

from test_gpu_parity import as_complex, check_topology, dev  # noqa: E402
from test_gpu_shortcut import check_shortcut  # noqa: E402


def gpu(src, q, p, leaf, tgt=None, precision=0, p2l_m2p=0):
    opt = G.fmm_default_options(p=p, leaf_size=leaf, precision=precision, p2l_m2p=p2l_m2p,
                                box_fit=1)
    tree = G.fmm_build_tree(dev(src), dev(tgt) if tgt is not None else None, opt)
    m = len(tgt) if tgt is not None else len(src)
    phi = torch.empty((m, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(q), phi)
    G.fmm_tree_sync(tree)
    return as_complex(phi.cpu().numpy()), tree


def oracle_fit(src, q, p, leaf, tgt=None, shortcut=False):
    L = O.levels_cap(len(src), leaf)
    tree0 = O.build_tree(src, L, tgt)
    tree = O.shrink(tree0, src, tgt)
    lists = O.connect(tree)
    sc = O.leaf_shortcut(tree, lists) if shortcut else None
    phi = O.evaluate(tree, lists, src, q, p, tgt, shortcut=sc)
    return phi, tree0, tree, lists, sc


CASES = [
    # name, dist, n, p, leaf, tgt_dist, m
    ("curve_8e3", "curve", 8_000, 20, 30, None, 0),
    ("clusters_2e4", "clusters", 20_000, 24, 32, None, 0),
    ("clusters_targets", "clusters", 6_000, 20, 25, "uniform", 4_500),
    ("uniform_ragged", "uniform", 4_099, 12, 7, None, 0),
]


@pytest.mark.parametrize("shortcut", [0, 1], ids=["plain", "shortcut"])
@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_box_fit_vs_oracle(case, precision, shortcut):
    name, dist, n, p, leaf, tgt_dist, m = case
    src, q, tgt = W.problem(dist, n, W.BASE_SEED + 300 + n, tgt_dist=tgt_dist, m=m)
    phi_o, tree0, otree, olists, sc = oracle_fit(src, q, p, leaf, tgt, bool(shortcut))
    phi_g, tree = gpu(src, q, p, leaf, tgt, precision, shortcut)
    check_topology(tree, tree0, olists)  # split rectangles unchanged, lists on the new geometry
    geo = G.fmm_tree_export_geometry(tree)
    assert np.array_equal(geo.view(np.uint64), otree.rect.view(np.uint64))
    if shortcut:
        check_shortcut(tree, otree, sc)
    err = O.normwise_error(phi_g, phi_o)
    assert err <= (1e-12 if precision == G.FMM_PREC_FP64 else 1e-11), err


def test_box_fit_degenerate_and_batched():
    rng = np.random.default_rng(9)
    src = rng.random((3000, 2))
    src[100:400] = src[5]
    src[500:900, 1] = 0.25
    q = W.complex_strengths(3000, rng)
    phi_o, _, otree, olists, _ = oracle_fit(src, q, 16, 16)
    for prec in (G.FMM_PREC_FP64, G.FMM_PREC_MIXED):
        phi_g, tree = gpu(src, q, 16, 16, precision=prec)
        assert np.all(np.isfinite(phi_g))
        assert O.normwise_error(phi_g, phi_o) <= (1e-12 if prec == G.FMM_PREC_FP64 else 1e-11)
    # a forest of instances with the fitted geometry
    inst = W.batched_instances(12, seed=7021, log_lo=2.0, log_hi=3.7)
    off = np.concatenate([[0], np.cumsum([len(s) for _, s, _ in inst])]).astype(np.int64)
    allsrc = np.concatenate([s for _, s, _ in inst])
    allq = np.concatenate([qq for _, _, qq in inst])
    opt = G.fmm_default_options(p=18, leaf_size=24, precision=G.FMM_PREC_MIXED, p2l_m2p=1,
                                box_fit=1)
    tree = G.fmm_build_batched(off, dev(allsrc), opt)
    phi = torch.empty((len(allsrc), 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(allq), phi)
    G.fmm_tree_sync(tree)
    got = as_complex(phi.cpu().numpy())
    for i, (_, s, qi) in enumerate(inst):
        ref, _, _, _, _ = oracle_fit(s, qi, 18, 24, shortcut=True)
        assert O.normwise_error(got[off[i]:off[i + 1]], ref) <= 1e-11, i


def test_box_fit_full_size_clusters_1e6_sampled():
    """The 1e6 cluster workload in the bench's configuration with box_fit:
    geometry and lists bit-exact, 256 sampled points against the oracle."""
    src, q, _ = W.make("clusters_1e6")
    L = O.levels_cap(len(src), 64)
    tree0 = O.build_tree(src, L)
    otree = O.shrink(tree0, src)
    olists = O.connect(otree)
    sc = O.leaf_shortcut(otree, olists)
    phi_g, tree = gpu(src, q, 24, 64, precision=G.FMM_PREC_MIXED, p2l_m2p=1)
    check_topology(tree, tree0, olists)
    check_shortcut(tree, otree, sc)
    sample = np.random.default_rng(0).choice(len(src), 256, replace=False)
    ref = O.evaluate(otree, olists, src, q, 24, sample=sample, shortcut=sc)
    assert O.normwise_error(phi_g[sample], ref) <= 1e-11


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_single_point_leaves_with_empty_siblings(precision):
    """Leaves of at most one point with shrink-wrapped geometry: a box holding
    one point (or only copies of one point) has radius 0, and its children
    without points keep their split rectangles.  M2M skips children without
    sources and L2L children without evaluation points, so nothing is
    translated across a radius-0 box; the potentials match the oracle."""
    src, q, _ = W.problem("uniform", 3000, 815)
    src[100:130] = src[99]
    phi_o = O.fmm(src, q, p=16, leaf=1, box_fit=True)[0]
    opt = G.fmm_default_options(p=16, leaf_size=1, precision=precision, box_fit=1)
    tree = G.fmm_build_tree(dev(src), None, opt)
    phi = torch.empty((3000, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(q), phi)
    G.fmm_tree_sync(tree)
    tree.free()
    got = as_complex(phi.cpu().numpy())
    assert np.all(np.isfinite(got))
    assert O.normwise_error(got, phi_o) <= (1e-12 if precision == 0 else 1e-11)
