"""Batched form: a forest of independent instances evaluated in one pass.

FP64: every instance of the forest equals its own single-tree GPU result bit
for bit (same kernels, same per-box order) and the oracle FMM within 1e-12.
Mixed: the tensor-core M2L sums the weak pairs in runs of 128 consecutive
entries of the whole weak list and adds into the locals with atomics, so a
forest groups an instance's pair terms differently from the instance's own
tree.  Both sums are correct to the df32 rounding level (~2^-48 relative per
term, a few hundred terms per coefficient): instances agree with the
single-tree mixed result within 5e-14 and with the oracle within 1e-11.
A CUDA-graph replay reproduces the direct launches bit for bit.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

from test_gpu_parity import as_complex, dev, gpu_fmm  # noqa: E402


def make_batch(n_inst, seed, log_lo=2.0, log_hi=3.7):
    inst = W.batched_instances(n_inst, seed=seed, log_lo=log_lo, log_hi=log_hi)
    sizes = [len(s) for _, s, _ in inst]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    src = np.concatenate([s for _, s, _ in inst])
    q = np.concatenate([q for _, _, q in inst])
    return inst, off, src, q


def run_batched(off, src, q, opt, graph=False, repeat=1):
    tree = G.fmm_build_batched(off, dev(src), opt)
    if graph:
        G.fmm_set_graph(tree, True)
    phi = torch.empty((len(src), 2), dtype=torch.float64, device="cuda")
    qd = dev(q)
    for _ in range(repeat):
        G.fmm_evaluate(tree, qd, phi)
    G.fmm_tree_sync(tree)
    return as_complex(phi.cpu().numpy()), tree


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED])
def test_forest_matches_single_trees_and_oracle(precision):
    inst, off, src, q = make_batch(24, 7001)
    p, leaf = 18, 24
    opt = G.fmm_default_options(p=p, leaf_size=leaf, precision=precision)
    phi_b, tree = run_batched(off, src, q, opt)
    info = G.fmm_tree_info(tree)
    assert info["levels"] == max(O.levels_cap(len(s), leaf) for _, s, _ in inst)
    for i, (_, s, qi) in enumerate(inst):
        got = phi_b[off[i]:off[i + 1]]
        single, _ = gpu_fmm(s, qi, p, leaf, precision=precision)
        ref, _, _ = O.fmm(s, qi, p=p, leaf=leaf)
        if precision == G.FMM_PREC_FP64:
            assert np.array_equal(got, single), i
            assert O.normwise_error(got, ref) <= 1e-12, i
        else:
            assert O.normwise_error(got, single) <= 5e-14, i
            assert O.normwise_error(got, ref) <= 1e-11, i


def test_one_shot_batched_entry_point():
    inst, off, src, q = make_batch(9, 7002)
    opt = G.fmm_default_options(p=14, leaf_size=16)
    phi = torch.empty((len(src), 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate_batched(off, dev(src), dev(q), phi, opt)
    torch.cuda.synchronize()
    got = as_complex(phi.cpu().numpy())
    ref, _ = run_batched(off, src, q, opt)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED])
def test_graph_replay_matches_direct_launches(precision):
    inst, off, src, q = make_batch(12, 7003)
    opt = G.fmm_default_options(p=16, leaf_size=20, precision=precision)
    direct, _ = run_batched(off, src, q, opt)
    graphed, _ = run_batched(off, src, q, opt, graph=True, repeat=3)
    if precision == G.FMM_PREC_FP64:
        assert np.array_equal(direct, graphed)
    else:
        assert O.normwise_error(graphed, direct) <= 1e-14


def test_single_instance_graph_mode():
    src, q, _ = W.problem("clusters", 30_000, 41)
    opt = G.fmm_default_options(p=20, leaf_size=32)
    tree = G.fmm_build_tree(dev(src), None, opt)
    G.fmm_set_graph(tree, True)
    phi = torch.empty((len(src), 2), dtype=torch.float64, device="cuda")
    for _ in range(2):
        G.fmm_evaluate(tree, dev(q), phi)  # a new q buffer each time: recapture
    G.fmm_tree_sync(tree)
    direct, _ = gpu_fmm(src, q, 20, 32)
    assert np.array_equal(as_complex(phi.cpu().numpy()), direct)


def test_batched_rejects_bad_offsets():
    src = np.random.default_rng(0).random((10, 2))
    opt = G.fmm_default_options()
    with pytest.raises(G.FmmError):
        G.fmm_build_batched(np.array([0, 5, 5, 10]), dev(src), opt)  # empty instance
    with pytest.raises(G.FmmError):
        G.fmm_build_batched(np.array([1, 10]), dev(src), opt)


def test_leaf_autotuner():
    """The autotuner returns one of the candidates with a positive time for
    each, for a single problem and for a forest."""
    src, q, _ = W.problem("clusters", 50_000, 61)
    opt = G.fmm_default_options(p=16, precision=G.FMM_PREC_MIXED)
    best, trials = G.fmm_autotune_leaf(dev(src), dev(q), opt, [16, 32, 64], repeats=1)
    assert best in (16, 32, 64) and all(t > 0 for t in trials.values())
    assert trials[best] == min(trials.values())
    inst, off, bsrc, bq = make_batch(8, 7031)
    best, trials = G.fmm_autotune_leaf(dev(bsrc), dev(bq), opt, [24, 48], src_off=off,
                                       repeats=1, evaluations=2)
    assert best in (24, 48) and trials[best] == min(trials.values())


def _forest_layout(inst_sizes, leaf, level_rule=0):
    """Where every instance's boxes sit in a forest: instances grouped by their
    number of levels (groups in increasing L, roots in caller order), each
    group level-major over its R roots.  Returns per instance (group base box,
    R, root index, L)."""
    Ls = [O.levels(n, leaf, level_rule) for n in inst_sizes]
    groups = sorted(set(Ls))
    out, base = [None] * len(inst_sizes), 0
    for L in groups:
        members = [i for i, x in enumerate(Ls) if x == L]
        R = len(members)
        for r, i in enumerate(members):
            out[i] = (base, R, r, L)
        base += R * O.n_boxes(L)
    return out


def _local_ids(L, R, r):
    """Global ids (relative to the group base) of one root's boxes, in the
    single tree's level-major order."""
    ids = []
    for l in range(L + 1):
        lb = (4 ** l - 1) // 3
        ids.extend(R * lb + r * 4 ** l + np.arange(4 ** l))
    return np.array(ids, np.int64)


@pytest.mark.parametrize("box_fit", [0, 1])
def test_forest_topology_per_instance_bitexact(box_fit):
    """Instances built together (several per tree, one tree per number of
    levels) have, box for box, the oracle's rectangles, source ranges and
    weak / strong lists of their own single trees."""
    inst, off, src, q = make_batch(30, 7010, log_lo=1.0, log_hi=3.8)
    leaf = 20
    opt = G.fmm_default_options(p=10, leaf_size=leaf, box_fit=box_fit)
    tree = G.fmm_build_batched(off, dev(src), opt)
    ex = G.fmm_tree_export(tree)
    geo = G.fmm_tree_export_geometry(tree)
    lay = _forest_layout([len(s) for _, s, _ in inst], leaf)
    for i, (_, s, _) in enumerate(inst):
        base, R, r, L = lay[i]
        otree = O.build_tree(s, L)
        if box_fit:
            otree = O.shrink(otree, s)
        olists = O.connect(otree)
        ids = base + _local_ids(L, R, r)
        to_local = {int(g): k for k, g in enumerate(ids)}
        assert np.array_equal(ex["rect"][ids].view(np.uint64),
                              O.build_tree(s, L).rect.view(np.uint64)), i
        if box_fit:
            assert np.array_equal(geo[ids].view(np.uint64), otree.rect.view(np.uint64)), i
        bs = ex["box_src"][ids]
        first = bs[0, 0]
        got_src = bs.copy()
        got_src[:, 0] -= first
        assert np.array_equal(got_src, otree.box_src), i
        # the permutation of the instance's sources, in caller indices
        assert np.array_equal(ex["perm"][first:first + len(s)] - off[i], otree.perm), i
        for name, off_name, ref, ref_off in (("weak", "weak_off", olists.weak, olists.weak_off),
                                             ("strong", "strong_off", olists.strong,
                                              olists.strong_off)):
            for k, g in enumerate(ids):
                lo, hi = ex[off_name][g], ex[off_name][g + 1]
                got = [to_local[int(x)] for x in ex[name][lo:hi]]
                assert got == list(ref[ref_off[k]:ref_off[k + 1]]), (i, name, k)
    tree.free()


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED])
def test_forest_with_separate_evaluation_points(precision):
    """Eq. 2 per instance: instance i is evaluated at its own points
    tgt[tgt_off[i]:tgt_off[i+1]] (some instances have none); every block of
    the result matches the oracle FMM of that instance with those points."""
    inst, off, src, q = make_batch(14, 7020)
    rng = np.random.default_rng(7021)
    m = [int(x) for x in rng.integers(0, 700, len(inst))]
    m[3] = 0
    tgts = [W.points("uniform", k, rng) if k else np.zeros((0, 2)) for k in m]
    toff = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    tgt = np.concatenate(tgts)
    p, leaf = 16, 24
    opt = G.fmm_default_options(p=p, leaf_size=leaf, precision=precision, p2l_m2p=1)
    tree = G.fmm_build_batched(off, dev(src), opt, tgt_off=toff, tgt=dev(tgt))
    phi = torch.empty((len(tgt), 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(q), phi)
    G.fmm_tree_sync(tree)
    tree.free()
    got = as_complex(phi.cpu().numpy())
    tol = 1e-12 if precision == G.FMM_PREC_FP64 else 1e-11
    for i, (_, s, qi) in enumerate(inst):
        if m[i] == 0:
            continue
        ref = O.fmm(s, qi, p=p, leaf=leaf, tgt=tgts[i], p2l_m2p=True)[0]
        assert O.normwise_error(got[toff[i]:toff[i + 1]], ref) <= tol, i
    # the one-shot form gives the same potentials
    phi2 = torch.empty((len(tgt), 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate_batched(off, dev(src), dev(q), phi2, opt, tgt_off=toff, tgt=dev(tgt))
    torch.cuda.synchronize()
    got2 = as_complex(phi2.cpu().numpy())
    if precision == G.FMM_PREC_FP64:
        assert np.array_equal(got2, got)
    else:
        assert O.normwise_error(got2, got) <= 1e-14


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED])
def test_near_field_item_size_changes_only_rounding(precision):
    """p2p_item_sources cuts every leaf's near list into runs of at most that
    many sources (the symmetric items at the sources, the per-point items at
    separate points): any size gives the oracle's potentials."""
    src, q, tgt = W.problem("clusters", 12_000, 7041, tgt_dist="uniform", m=3000)
    tol = 1e-12 if precision == G.FMM_PREC_FP64 else 1e-11
    for t in (None, tgt):
        ref = O.fmm(src, q, p=16, leaf=48, tgt=t)[0]
        outs = []
        for items in (64, 256, 0, 65536):
            opt = G.fmm_default_options(p=16, leaf_size=48, precision=precision,
                                        p2p_item_sources=items)
            tree = G.fmm_build_tree(dev(src), dev(t) if t is not None else None, opt)
            out = torch.empty((len(t) if t is not None else len(src), 2), dtype=torch.float64,
                              device="cuda")
            G.fmm_evaluate(tree, dev(q), out)
            G.fmm_tree_sync(tree)
            tree.free()
            got = as_complex(out.cpu().numpy())
            assert O.normwise_error(got, ref) <= tol, items
            outs.append(got)
        # FP64: regrouped sums differ at the FP64 rounding level.  Mixed: the df32
        # sums span one source leaf (one tile) and are then added in FP64, so the
        # run length does not change their rounding (with one df32 sum over a whole
        # run, 2048 sources gave 1.2e-12 here against 1.8e-14 for 64)
        cross = 1e-13
        for o in outs[1:]:
            assert O.normwise_error(o, outs[0]) <= cross


def test_autotuner_of_leaf_and_item_size():
    """fmm_autotune returns the fastest of the (leaf size, item size)
    candidates in the options, for a single problem and for a forest."""
    src, q, _ = W.problem("clusters", 40_000, 7042)
    base = G.fmm_default_options(p=16, precision=G.FMM_PREC_MIXED)
    opt, trials = G.fmm_autotune(dev(src), dev(q), base, [32, 64], [256, 2048], repeats=1)
    assert set(trials) == {(32, 256), (32, 2048), (64, 256), (64, 2048)}
    assert all(v > 0 for v in trials.values())
    best = min(trials, key=trials.get)
    assert (opt.leaf_size, opt.p2p_item_sources) == best
    assert opt.p == 16 and opt.precision == G.FMM_PREC_MIXED
    inst, off, bsrc, bq = make_batch(8, 7043)
    opt, trials = G.fmm_autotune(dev(bsrc), dev(bq), base, [24, 48], [512, 4096], src_off=off,
                                 repeats=1)
    assert (opt.leaf_size, opt.p2p_item_sources) == min(trials, key=trials.get)
