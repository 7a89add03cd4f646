"""Leaf P2L / M2P shortcut (Sec. 2, option p2l_m2p = 1) against the oracle.

The near / P2L / M2P split of the leaf strong lists is bit-exact with the
oracle's.  FP64 potentials match the oracle FMM with the same shortcut
within 1e-12 normwise; the mixed path (df32 P2L, M2P and P2P) within 1e-11,
and the branch-consistent direct sum within the truncation level.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

from test_gpu_parity import as_complex, check_topology, dev, gpu_fmm  # noqa: E402

TOL_FP64 = 1e-12
TOL_MIXED = 1e-11


def check_shortcut(tree, otree, sc):
    """GPU lists (CSR over all boxes, empty above the leaves) against the
    oracle's (CSR over the leaves)."""
    ex = G.fmm_tree_export_shortcut(tree)
    base = O.n_boxes(otree.L - 1) if otree.L > 0 else 0
    nleaf = 4 ** otree.L
    for name in ("near", "p2l", "m2p"):
        off = ex[name + "_off"]
        assert np.all(off[:base + 1] == 0), name
        assert np.array_equal(off[base:base + nleaf + 1], getattr(sc, name + "_off")), name
        n = getattr(sc, name + "_off")[-1]
        assert np.array_equal(ex[name], getattr(sc, name)[:n]), name
    return ex


CASES = [
    # name, dist, n, p, leaf, real_q, tgt_dist, m
    ("uniform_1e4", "uniform", 10_000, 20, 40, False, None, 0),
    ("clusters_2e4", "clusters", 20_000, 24, 32, False, None, 0),
    ("curve_8e3_real", "curve", 8_000, 24, 30, True, None, 0),
    ("clusters_targets", "clusters", 6_000, 20, 25, False, "uniform", 4_500),
    ("ragged_4099", "uniform", 4_099, 12, 7, False, None, 0),
]


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_shortcut_vs_oracle(case, precision):
    name, dist, n, p, leaf, real_q, tgt_dist, m = case
    src, q, tgt = W.problem(dist, n, W.BASE_SEED + 100 + n, real_q=real_q, tgt_dist=tgt_dist, m=m)
    phi_o, otree, olists, sc = O.fmm(src, q, p=p, leaf=leaf, tgt=tgt, p2l_m2p=True)
    phi_g, tree = gpu_fmm(src, q, p, leaf, tgt=tgt, precision=precision, p2l_m2p=1)
    check_topology(tree, otree, olists)
    check_shortcut(tree, otree, sc)
    assert sc.p2l_off[-1] > 0 and sc.m2p_off[-1] > 0
    err = O.normwise_error(phi_g, phi_o)
    assert err <= (TOL_FP64 if precision == G.FMM_PREC_FP64 else TOL_MIXED), err


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
def test_shortcut_direct_sum_gate(precision):
    """p = 20 on 1e4 uniform points with the shortcut: against the FP64
    branch-consistent direct sum (which takes the P2L / M2P pairs on their
    expansions' branches)."""
    src, q, _ = W.make("uniform_1e4")
    phi_g, tree = gpu_fmm(src, q, 20, 40, precision=precision, p2l_m2p=1)
    otree = O.build_tree(src, O.levels_cap(len(src), 40))
    olists = O.connect(otree)
    sc = O.leaf_shortcut(otree, olists)
    ref = O.direct_branch(otree, olists, src, q, shortcut=sc)
    assert O.normwise_error(phi_g, ref) < 1e-9


@pytest.mark.parametrize("kind", ["duplicates", "collinear", "tiny_n", "all_same"])
def test_shortcut_degenerate_inputs(kind):
    rng = np.random.default_rng(7)
    if kind == "duplicates":
        src = rng.random((3000, 2))
        src[100:400] = src[5]
        src[500:900, 1] = 0.25
        leaf = 16
    elif kind == "collinear":
        src = np.stack([np.full(2000, 0.5), rng.random(2000)], 1)
        leaf = 16
    elif kind == "tiny_n":
        src = rng.random((5, 2))
        leaf = 1
    else:
        src = np.tile([[0.3, 0.7]], (200, 1))
        leaf = 8
    q = W.complex_strengths(src.shape[0], rng)
    phi_o, otree, olists, sc = O.fmm(src, q, p=16, leaf=leaf, p2l_m2p=True)
    for precision, tol in ((G.FMM_PREC_FP64, TOL_FP64), (G.FMM_PREC_MIXED, TOL_MIXED)):
        phi_g, tree = gpu_fmm(src, q, 16, leaf, precision=precision, p2l_m2p=1)
        check_topology(tree, otree, olists)
        check_shortcut(tree, otree, sc)
        assert np.all(np.isfinite(phi_g))
        scale = max(np.max(np.abs(phi_o)), 1e-300)
        assert np.max(np.abs(phi_g - phi_o)) <= tol * scale + 1e-300


def test_shortcut_high_order_mixed_uses_fp64_kernels():
    """p above the df32 kernels' range (p = 40): the mixed path runs the FP64
    P2L / M2P and still matches the oracle."""
    src, q, _ = W.problem("clusters", 12_000, 91)
    phi_o, otree, olists, sc = O.fmm(src, q, p=40, leaf=32, p2l_m2p=True)
    phi_g, tree = gpu_fmm(src, q, 40, 32, precision=G.FMM_PREC_MIXED, p2l_m2p=1)
    assert O.normwise_error(phi_g, phi_o) <= TOL_MIXED


def test_shortcut_tensor_m2l():
    src, q, _ = W.problem("clusters", 20_000, 93)
    phi_o, otree, olists, sc = O.fmm(src, q, p=24, leaf=32, p2l_m2p=True)
    phi_g, tree = gpu_fmm(src, q, 24, 32, precision=G.FMM_PREC_MIXED, m2l_slices=0, p2l_m2p=1)
    assert O.normwise_error(phi_g, phi_o) <= TOL_MIXED


def test_shortcut_off_is_unchanged():
    """p2l_m2p = 0 keeps the direct near field: identical to the default."""
    src, q, _ = W.problem("clusters", 8_000, 95)
    a, _ = gpu_fmm(src, q, 18, 32)
    b, _ = gpu_fmm(src, q, 18, 32, p2l_m2p=0)
    assert np.array_equal(a, b)
    _, tree = gpu_fmm(src, q, 18, 32)
    with pytest.raises(G.FmmError):
        G.fmm_tree_export_shortcut(tree)


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
def test_shortcut_batched_and_graph(precision):
    """Forest of instances with the shortcut: every instance against the
    oracle with the shortcut, graph replay equal to direct launches."""
    inst = W.batched_instances(16, seed=7011, log_lo=2.0, log_hi=3.7)
    off = np.concatenate([[0], np.cumsum([len(s) for _, s, _ in inst])]).astype(np.int64)
    src = np.concatenate([s for _, s, _ in inst])
    q = np.concatenate([qq for _, _, qq in inst])
    p, leaf = 18, 24
    opt = G.fmm_default_options(p=p, leaf_size=leaf, precision=precision, p2l_m2p=1)
    outs = []
    for graph in (False, True):
        tree = G.fmm_build_batched(off, dev(src), opt)
        if graph:
            G.fmm_set_graph(tree, True)
        phi = torch.empty((len(src), 2), dtype=torch.float64, device="cuda")
        qd = dev(q)
        for _ in range(2 if graph else 1):
            G.fmm_evaluate(tree, qd, phi)
        G.fmm_tree_sync(tree)
        outs.append(as_complex(phi.cpu().numpy()))
    tol = TOL_FP64 if precision == G.FMM_PREC_FP64 else TOL_MIXED
    for i, (_, s, qi) in enumerate(inst):
        ref, _, _, _ = O.fmm(s, qi, p=p, leaf=leaf, p2l_m2p=True)
        assert O.normwise_error(outs[0][off[i]:off[i + 1]], ref) <= tol, i
    if precision == G.FMM_PREC_FP64:
        assert np.array_equal(outs[0], outs[1])
    else:
        assert O.normwise_error(outs[1], outs[0]) <= 1e-14


def test_shortcut_full_size_clusters_1e6_sampled():
    """The 1e6-point cluster workload (p = 24, leaf 64) in the mixed path
    with the shortcut: lists bit-exact, 512 sampled points against the
    oracle FMM with the same shortcut."""
    src, q, _ = W.make("clusters_1e6")
    L = O.levels_cap(len(src), 64)
    otree = O.build_tree(src, L)
    olists = O.connect(otree)
    sc = O.leaf_shortcut(otree, olists)
    phi_g, tree = gpu_fmm(src, q, 24, 64, precision=G.FMM_PREC_MIXED, p2l_m2p=1)
    check_topology(tree, otree, olists)
    check_shortcut(tree, otree, sc)
    sample = np.random.default_rng(0).choice(len(src), 512, replace=False)
    ref = O.evaluate(otree, olists, src, q, 24, sample=sample, shortcut=sc)
    assert O.normwise_error(phi_g[sample], ref) <= TOL_MIXED
