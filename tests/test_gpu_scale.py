"""Coordinates at any scale.

For the log kernel, scaling every point by s > 0 changes each pair term by
q_j ln s (Log(s z) = Log z + ln s for real s > 0: the argument is unchanged),
so with distinct points
    Phi_s(y_i) = Phi(y_i) + ln s * sum_{j != i} q_j;
the harmonic kernel is homogeneous of degree -1: Phi_s = Phi / s.  The FMM's
decisions (median splits, the theta-criterion) are scale-free as well, so the
GPU result at scale s must equal the one at scale 1 transformed this way.
The result at scale 1 is checked against the oracle FMM (the oracle keeps raw
expansion coefficients, as the paper does, and does not reach scales like
1e25: its powers overflow).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

from test_gpu_parity import as_complex, dev  # noqa: E402

# powers of two, so that the scaled inputs are exact
SCALES = [2.0 ** e for e in (-90, -83, -28, -13, 13, 30, 83, 90)]
TOL = {G.FMM_PREC_FP64: 1e-12, G.FMM_PREC_MIXED: 1e-11}


def gpu(src, q, tgt, precision, kernel=0, shortcut=1, box_fit=1):
    opt = G.fmm_default_options(p=20, leaf_size=32, precision=precision, kernel=kernel,
                                p2l_m2p=shortcut, box_fit=box_fit)
    tree = G.fmm_build_tree(dev(src), dev(tgt) if tgt is not None else None, opt)
    m = len(tgt) if tgt is not None else len(src)
    phi = torch.empty((m, 2), dtype=torch.float64, device="cuda")
    try:
        G.fmm_evaluate(tree, dev(q), phi)
        G.fmm_tree_sync(tree)
    finally:
        tree.free()
    return as_complex(phi.cpu().numpy())


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("separate", [False, True], ids=["self", "targets"])
def test_log_kernel_at_any_scale(precision, separate):
    src, q, tgt = W.problem("clusters", 8_000, W.BASE_SEED + 500, tgt_dist="uniform", m=2_000)
    t = tgt if separate else None
    qc = q[:, 0] + 1j * q[:, 1]
    base = gpu(src, q, t, precision)
    ref = O.fmm(src, q, p=20, leaf=32, tgt=t, p2l_m2p=True, box_fit=True)[0]
    assert O.normwise_error(base, ref) <= TOL[precision]
    # sum over j != i of q_j (self-evaluation; the points are distinct)
    qsum = qc.sum() - (qc if t is None else 0.0)
    for s in SCALES:
        got = gpu(src * s, q, None if t is None else t * s, precision)
        pred = base + qsum * np.log(s)
        assert np.all(np.isfinite(got)), s
        err = np.max(np.abs(got - pred)) / max(np.max(np.abs(pred)), np.max(np.abs(base)))
        assert err <= TOL[precision], (s, err)


@pytest.mark.parametrize("precision", [G.FMM_PREC_FP64, G.FMM_PREC_MIXED], ids=["fp64", "mixed"])
def test_harmonic_kernel_at_any_scale(precision):
    src, q, _ = W.problem("uniform", 6_000, W.BASE_SEED + 501)
    base = gpu(src, q, None, precision, kernel=G.FMM_KERNEL_HARMONIC)
    for s in SCALES:
        got = gpu(src * s, q, None, precision, kernel=G.FMM_KERNEL_HARMONIC)
        assert np.all(np.isfinite(got)), s
        err = O.normwise_error(got * s, base)
        assert err <= TOL[precision], (s, err)
