"""The paper's harmonic kernel (kernel = FMM_KERNEL_HARMONIC): u(y) = sum q_j /
(x_j - y), evaluated with the same tree, lists and expansions as the log
kernel and differentiated at the points.  Against the oracle FMM with
kernel 1 (FP64 1e-12, mixed 1e-11) and against the direct sum (no branch)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

from test_gpu_parity import as_complex, dev  # noqa: E402


def gpu(src, q, p, leaf, tgt=None, precision=0, **kw):
    opt = G.fmm_default_options(p=p, leaf_size=leaf, precision=precision,
                                kernel=G.FMM_KERNEL_HARMONIC, **kw)
    tree = G.fmm_build_tree(dev(src), dev(tgt) if tgt is not None else None, opt)
    m = len(tgt) if tgt is not None else len(src)
    u = torch.empty((m, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(q), u)
    G.fmm_tree_sync(tree)
    return as_complex(u.cpu().numpy())


CASES = [
    ("uniform_1e4", "uniform", 10_000, 17, 45, None, 0),   # the paper's p and N_d
    ("clusters_2e4", "clusters", 20_000, 24, 32, None, 0),
    ("curve_targets", "curve", 8_000, 20, 30, "uniform", 5_000),
]


@pytest.mark.parametrize("opts", [dict(), dict(p2l_m2p=1), dict(p2l_m2p=1, box_fit=1)],
                         ids=["plain", "shortcut", "shortcut_fit"])
@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_harmonic_vs_oracle(case, precision, opts):
    name, dist, n, p, leaf, tgt_dist, m = case
    src, q, tgt = W.problem(dist, n, W.BASE_SEED + 500 + n, tgt_dist=tgt_dist, m=m)
    ref = O.fmm(src, q, p=p, leaf=leaf, tgt=tgt, kernel=1,
                p2l_m2p=bool(opts.get("p2l_m2p")), box_fit=bool(opts.get("box_fit")))[0]
    got = gpu(src, q, p, leaf, tgt, precision, **opts)
    err = O.normwise_error(got, ref)
    assert err <= (1e-12 if precision == G.FMM_PREC_FP64 else 1e-11), err


def test_harmonic_direct_sum_gate():
    """p = 17, theta = 1/2, N_d = 45 on 1e4 uniform points (the paper's setting):
    against the direct sum, well inside the paper's 1e-6 tolerance."""
    src, q, _ = W.make("uniform_1e4")
    ref = O.direct_harmonic(src, q)
    for prec in (G.FMM_PREC_FP64, G.FMM_PREC_MIXED):
        got = gpu(src, q, 17, 45, precision=prec)
        assert O.normwise_error(got, ref) < 1e-7


def test_harmonic_full_size_clusters_1e6_sampled():
    src, q, _ = W.make("clusters_1e6")
    got = gpu(src, q, 24, 64, precision=G.FMM_PREC_MIXED, p2l_m2p=1, box_fit=1)
    sample = np.random.default_rng(0).choice(len(src), 256, replace=False)
    L = O.levels_cap(len(src), 64)
    tree = O.shrink(O.build_tree(src, L), src)
    lists = O.connect(tree)
    sc = O.leaf_shortcut(tree, lists)
    ref = O.evaluate(tree, lists, src, q, 24, sample=sample, shortcut=sc, kernel=1)
    assert O.normwise_error(got[sample], ref) <= 1e-11
    d = O.direct_harmonic(src, q, sample=sample[:64])
    assert O.normwise_error(got[sample[:64]], d) <= 1e-9
