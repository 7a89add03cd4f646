"""The C-ABI library builds, loads and exports every entry point declared in
include/gbfmm.h; host-side argument checks answer without a GPU."""
import ctypes as C
import os
import re

import pytest

import paper_1205_4611_gb300 as G
from paper_1205_4611_gb300 import binding as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "gbfmm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = G.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_default_options():
    o = G.fmm_default_options()
    assert (o.p, o.theta, o.leaf_size, o.level_rule, o.level_shift, o.precision) == (
        20, 0.5, 64, 0, 0, 0)
    assert o.p2l_m2p == 0


@pytest.mark.parametrize("field,value", [("p", 0), ("p", 65), ("theta", 0.0), ("theta", 1.0),
                                         ("leaf_size", 0), ("level_rule", 7),
                                         ("level_shift", -1), ("precision", 9),
                                         ("p2l_m2p", 2), ("p2l_m2p", -1), ("m2l_slices", 6),
                                         ("m2l_slices", -2), ("p2p_mode", 2), ("box_fit", 2),
                                         ("kernel", 2), ("p2p_item_sources", 63),
                                         ("p2p_item_sources", 65537)])
def test_bad_options_rejected_on_host(field, value):
    lib = G.load()
    o = G.fmm_default_options(**{field: value})
    h = C.c_void_p()
    st = lib.fmm_build_tree(C.c_void_p(16), 10, None, 0, C.byref(o), None, C.byref(h))
    assert st == G.FMM_ERR_ARG
    assert h.value is None
    assert len(G.fmm_last_error()) > 0


def test_null_arguments_rejected_on_host():
    lib = G.load()
    o = G.fmm_default_options()
    h = C.c_void_p()
    assert lib.fmm_build_tree(None, 10, None, 0, C.byref(o), None, C.byref(h)) == G.FMM_ERR_ARG
    assert lib.fmm_build_tree(C.c_void_p(16), 0, None, 0, C.byref(o), None,
                              C.byref(h)) == G.FMM_ERR_ARG
    assert lib.fmm_build_tree(C.c_void_p(16), 10, None, 0, C.byref(o), None, None) == G.FMM_ERR_ARG
    assert lib.fmm_evaluate(None, None, None, None) == G.FMM_ERR_ARG
    assert lib.fmm_tree_info(None, None, None, None, None) == G.FMM_ERR_ARG
    lib.fmm_tree_free(None)  # no-op


CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1205_4611_gb300", "csrc")


def test_every_kernel_waits_for_its_predecessor_first():
    """Kernels are launched with programmatic stream serialisation (their
    launch overlaps the end of the previous kernel), so each one must begin
    with pdl_wait() before touching memory, and no launch may bypass the
    helper that counts launches."""
    n_kernels = 0
    for name in sorted(os.listdir(CSRC)):
        if not name.endswith(".cu"):
            continue
        text = open(os.path.join(CSRC, name)).read()
        code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", text, flags=re.S))
        assert "<<<" not in code, f"{name}: launch outside launch_k"
        for m in re.finditer(r"__global__", code):
            depth, i = 0, m.end()
            while True:
                c = code[i]
                if c == "(":
                    depth += 1
                elif c == ")":
                    depth -= 1
                elif depth == 0 and c in ";{":
                    break
                i += 1
            if code[i] == ";":
                continue  # declaration
            body = code[i + 1:].lstrip()
            assert body.startswith("pdl_wait();"), f"{name}: kernel at {m.start()} starts with {body[:40]!r}"
            n_kernels += 1
    assert n_kernels >= 70


class _Rows:
    """Stands in for a device tensor: only its row count is read before the
    binding refuses the call."""

    def __init__(self, n):
        self.shape = (n, 2)


def test_binding_refuses_mismatched_lengths_before_any_launch():
    import numpy as np
    n0 = G.fmm_launch_count()
    tree = B.FmmTree(None, 100, 80)
    with pytest.raises(ValueError, match="q has 99 rows"):
        G.fmm_evaluate(tree, _Rows(99), _Rows(80))
    with pytest.raises(ValueError, match="phi has 79 rows"):
        G.fmm_evaluate(tree, _Rows(100), _Rows(79))
    with pytest.raises(ValueError, match="q has 9 rows"):
        G.fmm_direct_noalloc(_Rows(10), _Rows(9), _Rows(10))
    with pytest.raises(ValueError, match="phi has 6 rows"):
        G.fmm_direct_noalloc(_Rows(10), _Rows(10), _Rows(6), tgt=_Rows(7))
    off = np.array([0, 5, 12])
    with pytest.raises(ValueError, match="src has 11 rows"):
        G.fmm_build_batched(off, _Rows(11), G.fmm_default_options())
    with pytest.raises(ValueError, match="phi has 13 rows"):
        G.fmm_evaluate_batched(off, _Rows(12), _Rows(12), _Rows(13), G.fmm_default_options())
    src = np.zeros((10, 2))
    with pytest.raises(ValueError, match="q has 9 rows"):
        G.fmm_solve_host(src, np.zeros((9, 2)), opt=G.fmm_default_options())
    with pytest.raises(ValueError, match="out has 10 rows, expected 4"):
        G.fmm_solve_host(src, np.zeros((10, 2)), np.zeros((4, 2)), G.fmm_default_options(),
                         out=np.zeros((10, 2)))
    tree.handle = None
    assert G.fmm_launch_count() == n0
