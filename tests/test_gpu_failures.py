"""Error paths, exercised without any GPU fault: an injected device
allocation failure (host-side) must give FMM_ERR_NOMEM and release every
block the call held; an injected status bit (host-side) must map to its
status code in fmm_tree_sync.  No device wait is made to expire."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

from test_gpu_parity import dev  # noqa: E402


def _build(src, opt):
    return G.fmm_build_tree(dev(src), None, opt)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_allocation_failure_gives_nomem_and_no_leak(precision):
    src, q, _ = W.problem("clusters", 20_000, 61)
    opt = G.fmm_default_options(p=20, leaf_size=32, precision=precision, p2l_m2p=1, box_fit=1)
    torch.cuda.synchronize()
    base = G.fmm_memory_info()["in_use"]
    failed = 0
    try:
        for k in (0, 1, 2, 5, 9, 17, 33, 65):
            G.fmm_debug_inject(G.FMM_INJECT_ALLOC_FAILURE, k)
            try:
                tree = _build(src, opt)
            except G.FmmError as e:
                assert e.status == G.FMM_ERR_NOMEM, e
                failed += 1
            else:
                tree.free()  # the build needed fewer allocations than k
            G.fmm_debug_inject(G.FMM_INJECT_ALLOC_FAILURE, -1)
            assert G.fmm_memory_info()["in_use"] == base, k
    finally:
        G.fmm_debug_inject(G.FMM_INJECT_ALLOC_FAILURE, -1)
    assert failed >= 5
    # the library still works afterwards
    tree = _build(src, opt)
    phi = torch.empty((20_000, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(q), phi)
    G.fmm_tree_sync(tree)
    tree.free()
    assert G.fmm_memory_info()["in_use"] == base
    assert np.all(np.isfinite(phi.cpu().numpy()))


@pytest.mark.parametrize("bits, status", [(4, "FMM_ERR_TIMEOUT"), (1, "FMM_ERR_NONFINITE"),
                                          (8, "FMM_ERR_CUDA")])
def test_status_word_maps_to_status_code(bits, status):
    src, q, _ = W.problem("uniform", 5000, 62)
    tree = _build(src, G.fmm_default_options(p=12, leaf_size=32))
    phi = torch.empty((5000, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, dev(q), phi)
    G.fmm_debug_inject(G.FMM_INJECT_STATUS, bits)
    with pytest.raises(G.FmmError) as ei:
        G.fmm_tree_sync(tree)
    assert ei.value.status == getattr(G, status)
    G.fmm_tree_sync(tree)  # one-shot: the next synchronisation is clean
    tree.free()


def test_memory_info_counts_a_tree():
    src, _, _ = W.problem("clusters", 50_000, 63)
    torch.cuda.synchronize()
    before = G.fmm_memory_info(reset_peak=True)
    tree = _build(src, G.fmm_default_options(p=20, leaf_size=64, precision=1))
    held = G.fmm_memory_info()
    assert held["in_use"] > before["in_use"] + 50_000 * 16  # at least the permuted points
    assert held["peak"] >= held["in_use"]
    tree.free()
    assert G.fmm_memory_info()["in_use"] == before["in_use"]
