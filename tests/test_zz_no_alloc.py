"""fmm_direct_noalloc: the direct sum for callers that cannot allocate device
memory, on two calls in a row, against the library's allocating path (an
L = 0 tree, whose P2P is the same direct sum) and against the oracle's FP64
direct sum of Eq. (1) / Eq. (2).  Collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

TOL = 1e-12  # FP64 tolerance of the parity tests


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def _reference(src, q, tgt=None):
    """The allocating entry points: one leaf holding every source (L = 0)."""
    n = src.shape[0]
    opt = G.fmm_default_options(p=4, leaf_size=n)
    tree = G.fmm_build_tree(_dev(src), _dev(tgt) if tgt is not None else None, opt)
    assert G.fmm_tree_info(tree)["levels"] == 0
    m = tgt.shape[0] if tgt is not None else n
    phi = torch.empty((m, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, _dev(q), phi)
    G.fmm_tree_sync(tree)
    tree.free()
    return phi.cpu().numpy()


def _noalloc(src, q, tgt=None):
    m = tgt.shape[0] if tgt is not None else src.shape[0]
    phi = torch.empty((m, 2), dtype=torch.float64, device="cuda")
    G.fmm_direct_noalloc(_dev(src), _dev(q), phi, _dev(tgt) if tgt is not None else None)
    torch.cuda.synchronize()
    return phi.cpu().numpy()


def _c(a):
    a = np.asarray(a)
    return a[:, 0] + 1j * a[:, 1] if a.ndim == 2 else a


def _pairs(z):
    return np.stack([z.real, z.imag], 1)


def _err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_noalloc_matches_allocating_path_twice():
    # first call: self-evaluation with duplicates, several source runs
    src, q, _ = W.problem("clusters", 5000, 901)
    src[10:20] = src[3]
    ref1 = _reference(src, q)
    got1 = _noalloc(src, q)
    assert _err(got1, ref1) <= TOL
    assert _err(got1, _pairs(O.direct(src, _c(q)))) <= TOL
    # second call in a row: separate evaluation points, fewer sources (the
    # static scratch still holds the first call's partial sums)
    src2, q2, tgt2 = W.problem("curve", 3000, 902, tgt_dist="uniform", m=1700)
    ref2 = _reference(src2, q2, tgt2)
    got2 = _noalloc(src2, q2, tgt2)
    assert _err(got2, ref2) <= TOL
    assert _err(got2, _pairs(O.direct(src2, _c(q2), tgt2))) <= TOL


def test_noalloc_rejects_oversized_call():
    src = np.random.default_rng(0).random((2049, 2))  # 2 source runs
    tgt = np.random.default_rng(1).random((64 * 2048 + 1, 2))  # 2049 chunks
    q = np.ones((2049, 2))
    phi = torch.empty((tgt.shape[0], 2), dtype=torch.float64, device="cuda")
    with pytest.raises(G.FmmError) as ei:
        G.fmm_direct_noalloc(_dev(src), _dev(q), phi, _dev(tgt))
    assert ei.value.status == G.FMM_ERR_ARG
    assert "static scratch" in G.fmm_last_error()
