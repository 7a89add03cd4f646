"""The theta-criterion (Eq. 3) at values of theta other than the paper's 1/2.

theta decides which box pairs interact through expansions (weak list) and
which directly (strong list), and with the leaf shortcut which leaf pairs take
P2L / M2P; everything downstream follows from the lists.  At each theta the
GPU lists must equal the oracle's connectivity at that theta bit for bit, and
the potentials the oracle FMM with the same theta (FP64 1e-12, mixed 1e-11
normwise).  A smaller theta demands better separation: more strong pairs and
a smaller truncation error, which the direct-sum check at the end confirms.
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

TOL = {G.FMM_PREC_FP64: 1e-12, G.FMM_PREC_MIXED: 1e-11}


def gpu(src, q, p, leaf, theta, precision, shortcut, tgt=None):
    opt = G.fmm_default_options(p=p, leaf_size=leaf, theta=theta, precision=precision,
                                p2l_m2p=int(shortcut))
    tree = G.fmm_build_tree(dev(src), dev(tgt) if tgt is not None else None, opt)
    m = len(tgt) if tgt is not None else len(src)
    phi = torch.empty((m, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(q), phi)
    G.fmm_tree_sync(tree)
    return as_complex(phi.cpu().numpy()), tree


@pytest.mark.parametrize("shortcut", [False, True], ids=["plain", "shortcut"])
@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("theta", [0.3, 0.7, 0.9])
def test_theta_lists_and_potentials(theta, precision, shortcut):
    src, q, tgt = W.problem("clusters", 12_000, W.BASE_SEED + 400, tgt_dist="uniform", m=2_500)
    for t in (None, tgt):
        res = O.fmm(src, q, p=20, leaf=32, theta=theta, tgt=t, p2l_m2p=shortcut)
        phi_o, otree, olists = res[:3]
        phi_g, tree = gpu(src, q, 20, 32, theta, precision, shortcut, tgt=t)
        try:
            check_topology(tree, otree, olists)
            if shortcut:
                check_shortcut(tree, otree, res[3])
        finally:
            tree.free()
        err = O.normwise_error(phi_g, phi_o)
        assert err <= TOL[precision], (t is None, err)


def test_theta_trades_strong_pairs_for_accuracy():
    """Against the branch-consistent direct sum the truncation error shrinks
    with theta (Eq. 3: the expansions converge like theta^p), while the strong
    lists grow."""
    src, q, _ = W.problem("uniform", 8_000, W.BASE_SEED + 401)
    errs, strong = [], []
    for theta in (0.8, 0.5, 0.3):
        phi_g, tree = gpu(src, q, 12, 24, theta, G.FMM_PREC_FP64, False)
        try:
            ex = G.fmm_tree_export(tree)
        finally:
            tree.free()
        otree = O.build_tree(src, ex["levels"])
        olists = O.connect(otree, theta)
        ref = O.direct_branch(otree, olists, src, q)
        errs.append(O.normwise_error(phi_g, ref))
        strong.append(int(ex["strong_off"][-1]))
    assert errs[0] > errs[1] > errs[2], errs
    assert strong[0] < strong[1] < strong[2], strong
    assert errs[2] < 1e-9, errs
