"""CUDA path against the CPU oracle, through the C ABI.

Topology (permutations, rectangles, box ranges, interaction lists) must be
bit-exact; FP64 potentials must match the oracle FMM within 1e-12 normwise
(max |d phi| / max |phi|), and the direct sum within the truncation level.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

TOL_FP64 = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def as_complex(a):
    a = np.asarray(a)
    return a[:, 0] + 1j * a[:, 1]


def gpu_fmm(src, q, p, leaf, tgt=None, theta=0.5, level_shift=0, precision=0, level_rule=0,
            m2l_slices=0, p2l_m2p=0):
    opt = G.fmm_default_options(p=p, leaf_size=leaf, theta=theta, level_shift=level_shift,
                                precision=precision, level_rule=level_rule,
                                m2l_slices=m2l_slices, p2l_m2p=p2l_m2p)
    s = dev(src)
    t = dev(tgt) if tgt is not None else None
    tree = G.fmm_build_tree(s, t, opt)
    m = tgt.shape[0] if tgt is not None else src.shape[0]
    phi = torch.empty((m, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(q), phi)
    G.fmm_tree_sync(tree)
    return as_complex(phi.cpu().numpy()), tree


def check_topology(tree, otree, olists):
    ex = G.fmm_tree_export(tree)
    assert ex["levels"] == otree.L
    assert np.array_equal(ex["perm"], otree.perm)
    assert np.array_equal(ex["tperm"], otree.tperm)
    assert np.array_equal(ex["rect"].view(np.uint64), otree.rect.view(np.uint64))
    assert np.array_equal(ex["box_src"], otree.box_src)
    assert np.array_equal(ex["box_tgt"], otree.box_tgt)
    assert np.array_equal(ex["weak_off"], olists.weak_off)
    assert np.array_equal(ex["strong_off"], olists.strong_off)
    assert np.array_equal(ex["weak"], olists.weak[:olists.weak_off[-1]])
    assert np.array_equal(ex["strong"], olists.strong[:olists.strong_off[-1]])


CASES = [
    # name, dist, n, p, leaf, real_q, tgt_dist, m
    ("uniform_1e4", "uniform", 10_000, 20, 40, False, None, 0),
    ("clusters_2e4", "clusters", 20_000, 24, 32, False, None, 0),
    ("curve_8e3_real", "curve", 8_000, 24, 30, True, None, 0),
    ("clusters_targets", "clusters", 6_000, 20, 25, False, "uniform", 4_500),
    ("ragged_4099", "uniform", 4_099, 12, 7, False, None, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_vs_oracle_fmm(case):
    name, dist, n, p, leaf, real_q, tgt_dist, m = case
    src, q, tgt = W.problem(dist, n, W.BASE_SEED + 100 + n, real_q=real_q, tgt_dist=tgt_dist, m=m)
    phi_o, otree, olists = O.fmm(src, q, p=p, leaf=leaf, tgt=tgt)
    phi_g, tree = gpu_fmm(src, q, p, leaf, tgt=tgt)
    check_topology(tree, otree, olists)
    err = O.normwise_error(phi_g, phi_o)
    assert err <= TOL_FP64, err


def test_direct_sum_gate_uniform_1e4():
    """p = 20, theta = 1/2, leaf 40 on 1e4 uniform points: the GPU FMM against
    the branch-consistent FP64 direct sum stays at the truncation level."""
    src, q, _ = W.make("uniform_1e4")
    phi_g, tree = gpu_fmm(src, q, 20, 40)
    otree = O.build_tree(src, O.levels_cap(len(src), 40))
    olists = O.connect(otree)
    ref = O.direct_branch(otree, olists, src, q)
    assert O.normwise_error(phi_g, ref) < 1e-9


def test_single_leaf_equals_direct_sum():
    src, q, _ = W.problem("uniform", 50, 5)
    phi_g, tree = gpu_fmm(src, q, 10, 64)
    assert G.fmm_tree_info(tree)["levels"] == 0
    ref = O.direct(src, q)
    assert O.normwise_error(phi_g, ref) < 1e-14


@pytest.mark.parametrize("kind", ["duplicates", "collinear", "tiny_n", "all_same", "two"])
def test_degenerate_inputs(kind):
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
    elif kind == "all_same":
        src = np.tile([[0.3, 0.7]], (200, 1))
        leaf = 8
    else:
        src = np.array([[0.0, 0.0], [1.0, 1.0]])
        leaf = 1
    q = W.complex_strengths(src.shape[0], rng)
    phi_o, otree, olists = O.fmm(src, q, p=16, leaf=leaf)
    phi_g, tree = gpu_fmm(src, q, 16, leaf)
    check_topology(tree, otree, olists)
    assert np.all(np.isfinite(phi_g))
    scale = max(np.max(np.abs(phi_o)), 1e-300)
    assert np.max(np.abs(phi_g - phi_o)) <= TOL_FP64 * scale + 1e-300


def test_level_shift_and_eq_rule():
    src, q, _ = W.problem("clusters", 12_000, 77)
    for kw, L in ((dict(level_shift=1), O.levels_cap(12_000, 64) + 1),
                  (dict(level_rule=1), O.levels_eq(12_000, 64))):
        phi_o, otree, olists = O.fmm(src, q, p=18, leaf=64, L=L)
        phi_g, tree = gpu_fmm(src, q, 18, 64, **kw)
        check_topology(tree, otree, olists)
        assert O.normwise_error(phi_g, phi_o) <= TOL_FP64


def test_nonfinite_rejected():
    src = np.random.default_rng(1).random((100, 2))
    src[17, 0] = np.nan
    with pytest.raises(G.FmmError) as ei:
        G.fmm_build_tree(dev(src), None, G.fmm_default_options())
    assert ei.value.status == G.FMM_ERR_NONFINITE


def test_solve_host_matches_device_path():
    src, q, tgt = W.problem("clusters", 5000, 3, tgt_dist="uniform", m=3000)
    opt = G.fmm_default_options(p=16, leaf_size=32)
    phi_h = as_complex(G.fmm_solve_host(src, q, tgt, opt))
    phi_d, _ = gpu_fmm(src, q, 16, 32, tgt=tgt)
    assert np.array_equal(phi_h, phi_d)


def test_repeat_evaluation_is_deterministic():
    src, q, _ = W.problem("clusters", 20_000, 9)
    opt = G.fmm_default_options(p=20, leaf_size=32)
    tree = G.fmm_build_tree(dev(src), None, opt)
    outs = []
    for _ in range(2):
        phi = torch.empty((20_000, 2), dtype=torch.float64, device="cuda")
        G.fmm_evaluate(tree, dev(q), phi)
        G.fmm_tree_sync(tree)
        outs.append(phi.cpu().numpy())
    a, b = as_complex(outs[0]), as_complex(outs[1])
    assert O.normwise_error(b, a) <= 1e-13
    tree.free()


@pytest.mark.parametrize("precision, tol", [(0, TOL_FP64), (1, 1e-11)], ids=["fp64", "mixed"])
def test_new_strengths_on_a_built_tree(precision, tol):
    """Sec. 3.1 splits the method into a topological phase (tree and lists,
    which depend on the points only) and a computational phase (which depends
    on the strengths): one built tree evaluated with a second, independent
    strength vector must give the oracle FMM's potentials for that vector."""
    n = 20_000
    src, q, _ = W.problem("clusters", n, 9)
    q2 = W.complex_strengths(n, np.random.default_rng(2))
    opt = G.fmm_default_options(p=20, leaf_size=32, precision=precision)
    tree = G.fmm_build_tree(dev(src), None, opt)
    for qq in (q, q2):
        phi = torch.empty((n, 2), dtype=torch.float64, device="cuda")
        G.fmm_evaluate(tree, dev(qq), phi)
        G.fmm_tree_sync(tree)
        ref, _, _ = O.fmm(src, qq, p=20, leaf=32)
        assert O.normwise_error(as_complex(phi.cpu().numpy()), ref) <= tol
    tree.free()


def test_full_size_clusters_1e6_sampled():
    """The 1e6-point cluster workload (p = 24, leaf 64): bit-exact topology and
    oracle-FMM parity on 512 sampled evaluation points."""
    src, q, _ = W.make("clusters_1e6")
    L = O.levels_cap(len(src), 64)
    otree = O.build_tree(src, L)
    olists = O.connect(otree)
    phi_g, tree = gpu_fmm(src, q, 24, 64)
    check_topology(tree, otree, olists)
    sample = np.random.default_rng(0).choice(len(src), 512, replace=False)
    ref = O.evaluate(otree, olists, src, q, 24, sample=sample)
    assert O.normwise_error(phi_g[sample], ref) <= TOL_FP64


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
def test_overlapped_far_field_matches_sequential_phases(precision):
    """Unless phase timing is on, an evaluation runs the far field (P2M .. P2L)
    on a second stream beside the near field, joined before M2P (which reads
    the multipoles) and before the combination; with timing on every phase
    runs alone.  On the 1e6-point workload with the bench's options both give
    the same potentials, over repeated evaluations: FP64 bit for bit, mixed to
    the rounding of the tensor M2L's atomic additions."""
    src, q, _ = W.make("clusters_1e6")
    opt = G.fmm_default_options(p=24, leaf_size=64, precision=precision, p2l_m2p=1, box_fit=1)
    tree = G.fmm_build_tree(dev(src), None, opt)
    outs = []
    try:
        for timing in (True, False, False):
            G.fmm_set_timing(tree, timing)
            phi = torch.empty((len(src), 2), dtype=torch.float64, device="cuda")
            G.fmm_evaluate(tree, dev(q), phi)
            G.fmm_tree_sync(tree)
            outs.append(as_complex(phi.cpu().numpy()))
    finally:
        tree.free()
    for o in outs[1:]:
        assert np.all(np.isfinite(o))
        if precision == G.FMM_PREC_FP64:
            assert np.array_equal(o, outs[0])
        else:
            assert O.normwise_error(o, outs[0]) <= 1e-13


@pytest.mark.parametrize("n, leaf, shift", [(300, 64, 6), (5000, 4, 2), (2100, 1, 0)])
def test_deep_trees_topology(n, leaf, shift):
    """Deep trees with many empty boxes: the split rounds that run in shared
    memory (capped number of rounds per block) and the global rounds before
    them must give the oracle's topology bit for bit."""
    src, q, _ = W.problem("clusters", n, 1300 + n)
    L = O.levels_cap(n, leaf) + shift
    phi_o, otree, olists = O.fmm(src, q, p=6, leaf=leaf, L=L)
    phi_g, tree = gpu_fmm(src, q, 6, leaf, level_shift=shift)
    check_topology(tree, otree, olists)
    assert O.normwise_error(phi_g, phi_o) <= TOL_FP64


def test_evaluate_on_another_stream():
    """The last build steps stay queued on the build stream; an evaluation on
    another stream waits for them and gives the same potentials (to the
    rounding of the mixed M2L's atomic additions)."""
    src, q, _ = W.problem("clusters", 30_000, 5)
    opt = G.fmm_default_options(p=20, leaf_size=32, precision=G.FMM_PREC_MIXED)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    sd, qd = dev(src), dev(q)
    torch.cuda.synchronize()
    outs = []
    for ev_stream in (s1, s2):
        tree = G.fmm_build_tree(sd, None, opt, stream=s1)
        phi = torch.zeros((30_000, 2), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        G.fmm_evaluate(tree, qd, phi, stream=ev_stream)
        G.fmm_tree_sync(tree, stream=ev_stream)
        outs.append(phi.cpu().numpy())
        tree.free()
    a, b = as_complex(outs[0]), as_complex(outs[1])
    assert O.normwise_error(b, a) <= 1e-13


def test_tree_freed_and_reused_across_streams():
    """Freeing a tree right after queueing its evaluation on another stream
    waits for that evaluation before the tree's device blocks go to the next
    build on the build stream; two evaluations of one tree queued on two
    streams (different strengths) run one after the other, since they share the
    tree's expansion buffers.  Potentials equal those of plain evaluations (to
    the rounding of the mixed M2L's atomic additions)."""
    n = 30_000
    src, q, _ = W.problem("clusters", n, 11)
    src_b, q_b, _ = W.problem("uniform", n, 12)
    opt = G.fmm_default_options(p=20, leaf_size=32, precision=G.FMM_PREC_MIXED)
    sd, qd, sd_b, qd_b = dev(src), dev(q), dev(src_b), dev(q_b)

    def plain(s_dev, q_dev):
        tree = G.fmm_build_tree(s_dev, None, opt)
        phi = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
        G.fmm_evaluate(tree, q_dev, phi)
        G.fmm_tree_sync(tree)
        tree.free()
        return as_complex(phi.cpu().numpy())

    ref_a, ref_b, ref_aq = plain(sd, qd), plain(sd_b, qd_b), plain(sd, qd_b)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    # A built on s1, evaluated on s2, freed at once; B reuses the blocks on s1
    phi_a = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    phi_b = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    tree = G.fmm_build_tree(sd, None, opt, stream=s1)
    G.fmm_evaluate(tree, qd, phi_a, stream=s2)
    tree.free()
    tree_b = G.fmm_build_tree(sd_b, None, opt, stream=s1)
    G.fmm_evaluate(tree_b, qd_b, phi_b, stream=s1)
    G.fmm_tree_sync(tree_b, stream=s1)
    tree_b.free()
    torch.cuda.synchronize()
    assert O.normwise_error(as_complex(phi_a.cpu().numpy()), ref_a) <= 1e-13
    assert O.normwise_error(as_complex(phi_b.cpu().numpy()), ref_b) <= 1e-13
    # one tree, two evaluations queued on two streams
    p1 = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    p2 = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    tree = G.fmm_build_tree(sd, None, opt, stream=s1)
    G.fmm_evaluate(tree, qd, p1, stream=s1)
    G.fmm_evaluate(tree, qd_b, p2, stream=s2)
    G.fmm_tree_sync(tree, stream=s2)
    tree.free()
    torch.cuda.synchronize()
    assert O.normwise_error(as_complex(p1.cpu().numpy()), ref_a) <= 1e-13
    assert O.normwise_error(as_complex(p2.cpu().numpy()), ref_aq) <= 1e-13


@pytest.mark.parametrize("kernel", [0, 1], ids=["log", "harmonic"])
def test_fp64_symmetric_near_field_matches_per_point_pass(kernel):
    """FP64 self-evaluation: p2p_mode 0 (each pair of distinct leaves' points
    evaluated once, the reverse term by Log(-z) = Log(z) +- i pi, or +q/z for
    the harmonic kernel) against p2p_mode 1 (one pass per point) and the
    oracle, with shared ordinates and exact duplicates across leaves."""
    rng = np.random.default_rng(23)
    src = rng.random((6000, 2))
    src[100:160] = src[7]
    src[1000:1400, 1] = np.round(src[1000:1400, 1] * 8) / 8
    q = W.complex_strengths(6000, rng)
    out = []
    for mode in (0, 1):
        opt = G.fmm_default_options(p=18, leaf_size=48, p2p_mode=mode, kernel=kernel)
        tree = G.fmm_build_tree(dev(src), None, opt)
        phi = torch.empty((6000, 2), dtype=torch.float64, device="cuda")
        G.fmm_evaluate(tree, dev(q), phi)
        G.fmm_tree_sync(tree)
        tree.free()
        out.append(as_complex(phi.cpu().numpy()))
    assert O.normwise_error(out[0], out[1]) <= 1e-13
    ref = O.fmm(src, q, p=18, leaf=48, kernel=kernel)[0]
    assert O.normwise_error(out[0], ref) <= TOL_FP64
