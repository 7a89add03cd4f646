"""Thin ctypes binding of libgbfmm.so (include/gbfmm.h): argument marshalling
only.  Every step of the method runs in the library's CUDA kernels; there is
no fallback.  Device arrays are torch CUDA tensors (float64, C-contiguous,
points shaped [n, 2], complex values shaped [n, 2] as (re, im)); streams are
torch CUDA streams (default: the current stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FMM_OK = 0
FMM_ERR_ARG = -1
FMM_ERR_NOMEM = -2
FMM_ERR_CUDA = -3
FMM_ERR_TIMEOUT = -4
FMM_ERR_NONFINITE = -5

FMM_PREC_FP64 = 0
FMM_PREC_MIXED = 1
FMM_KERNEL_LOG = 0
FMM_KERNEL_HARMONIC = 1
FMM_LEVELS_CAP = 0
FMM_LEVELS_EQ = 1

# names declared in include/gbfmm.h
EXPORTS = (
    "fmm_default_options", "fmm_build_tree", "fmm_evaluate", "fmm_tree_sync", "fmm_solve_host",
    "fmm_evaluate_batched", "fmm_tree_info", "fmm_tree_export", "fmm_get_timings",
    "fmm_set_timing", "fmm_tree_free", "fmm_launch_count", "fmm_last_error",
    "fmm_build_batched", "fmm_set_graph", "fmm_direct_noalloc", "fmm_tree_shortcut_info",
    "fmm_tree_export_shortcut", "fmm_tree_export_geometry", "fmm_autotune_leaf",
    "fmm_memory_info", "fmm_debug_inject", "fmm_autotune",
)
FMM_INJECT_ALLOC_FAILURE = 1
FMM_INJECT_STATUS = 2


class FmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gbfmm status {status}: {msg}")
        self.status = status


class fmm_options(C.Structure):
    _fields_ = [("p", C.c_int), ("theta", C.c_double), ("leaf_size", C.c_int),
                ("level_rule", C.c_int), ("level_shift", C.c_int), ("precision", C.c_int),
                ("m2l_slices", C.c_int), ("p2p_mode", C.c_int), ("p2l_m2p", C.c_int),
                ("box_fit", C.c_int), ("kernel", C.c_int), ("p2p_item_sources", C.c_int)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load the CUDA library; raises if it is missing or cannot be built."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise FmmError(FMM_ERR_ARG, f"CUDA library not built: {path}")
            path = _build.build()
        L = C.CDLL(path)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        L.fmm_default_options.argtypes = [C.POINTER(fmm_options)]
        L.fmm_default_options.restype = None
        L.fmm_build_tree.argtypes = [vp, i64, vp, i64, C.POINTER(fmm_options), vp, C.POINTER(vp)]
        L.fmm_evaluate.argtypes = [vp, vp, vp, vp]
        L.fmm_tree_sync.argtypes = [vp, vp]
        L.fmm_solve_host.argtypes = [vp, i64, vp, i64, vp, vp, C.POINTER(fmm_options), vp]
        L.fmm_evaluate_batched.argtypes = [i32, vp, vp, vp, vp, vp, vp, C.POINTER(fmm_options),
                                           vp]
        L.fmm_tree_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i64),
                                    C.POINTER(i64)]
        L.fmm_tree_export.argtypes = [vp] * 10
        L.fmm_tree_shortcut_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        L.fmm_tree_export_shortcut.argtypes = [vp] * 7
        L.fmm_tree_export_geometry.argtypes = [vp, vp]
        L.fmm_autotune_leaf.argtypes = [vp, i64, vp, i64, i32, vp, vp, C.POINTER(fmm_options),
                                        vp, i32, i32, i32, vp, C.POINTER(i32), vp]
        L.fmm_autotune.argtypes = [vp, i64, vp, i64, i32, vp, vp, C.POINTER(fmm_options), vp, i32,
                                   vp, i32, i32, i32, vp, vp]
        L.fmm_autotune.restype = i32
        L.fmm_get_timings.argtypes = [vp, C.POINTER(C.c_float), i32]
        L.fmm_set_timing.argtypes = [vp, i32]
        L.fmm_tree_free.argtypes = [vp]
        L.fmm_tree_free.restype = None
        L.fmm_build_batched.argtypes = [i32, vp, vp, vp, vp, C.POINTER(fmm_options), vp,
                                        C.POINTER(vp)]
        L.fmm_build_batched.restype = i32
        L.fmm_set_graph.argtypes = [vp, i32]
        L.fmm_set_graph.restype = i32
        L.fmm_direct_noalloc.argtypes = [vp, i64, vp, vp, i64, vp, vp]
        L.fmm_direct_noalloc.restype = i32
        L.fmm_memory_info.argtypes = [C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), i32]
        L.fmm_memory_info.restype = i32
        L.fmm_debug_inject.argtypes = [i32, i64]
        L.fmm_debug_inject.restype = i32
        L.fmm_launch_count.argtypes = []
        L.fmm_launch_count.restype = C.c_int64
        L.fmm_last_error.argtypes = []
        L.fmm_last_error.restype = C.c_char_p
        for f in ("fmm_build_tree", "fmm_evaluate", "fmm_tree_sync", "fmm_solve_host",
                  "fmm_evaluate_batched", "fmm_tree_info", "fmm_tree_export", "fmm_get_timings",
                  "fmm_set_timing", "fmm_tree_shortcut_info", "fmm_tree_export_shortcut",
                  "fmm_tree_export_geometry", "fmm_autotune_leaf"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


def fmm_launch_count() -> int:
    return int(load().fmm_launch_count())


def fmm_memory_info(reset_peak: bool = False) -> dict:
    """Bytes of device memory held through the library's block cache."""
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().fmm_memory_info(C.byref(a), C.byref(b), C.byref(c), int(reset_peak)))
    return dict(in_use=a.value, peak=b.value, cached=c.value)


def fmm_debug_inject(what: int, arg: int):
    """Host-side fault injection (testing hook, see include/gbfmm.h)."""
    _check(load().fmm_debug_inject(int(what), int(arg)))


def fmm_last_error() -> str:
    return load().fmm_last_error().decode()


def _check(st: int):
    if st != FMM_OK:
        raise FmmError(st, fmm_last_error())


def fmm_default_options(**kw) -> fmm_options:
    o = fmm_options()
    load().fmm_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and t.dim() == 2 and t.shape[1] == 2):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor of shape [n, 2]")
    return C.c_void_p(t.data_ptr())


def _rows(t) -> int:
    return int(t.shape[0])


def _need_rows(t, n, name):
    """Refuse a buffer whose row count differs from what the library will
    read or write (a short buffer would be accessed out of bounds on the
    device)."""
    if t is not None and _rows(t) != n:
        raise ValueError(f"{name} has {_rows(t)} rows, expected {n}")


class FmmTree:
    """Owns an fmm_tree handle."""

    def __init__(self, handle, n_src, n_tgt):
        self.handle = handle
        self.n_src = n_src
        self.n_tgt = n_tgt

    def free(self):
        if self.handle:
            load().fmm_tree_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fmm_build_tree(src, tgt=None, opt: fmm_options | None = None, stream=None) -> FmmTree:
    L = load()
    opt = opt or fmm_default_options()
    h = C.c_void_p()
    n = src.shape[0]
    m = tgt.shape[0] if tgt is not None else 0
    st = L.fmm_build_tree(_dev_ptr(src, "src"), n, _dev_ptr(tgt, "tgt"), m, C.byref(opt),
                          _stream_ptr(stream), C.byref(h))
    _check(st)
    return FmmTree(h, n, m if tgt is not None else n)


def fmm_evaluate(tree: FmmTree, q, phi, stream=None):
    _need_rows(q, tree.n_src, "q")
    _need_rows(phi, tree.n_tgt, "phi")
    _check(load().fmm_evaluate(tree.handle, _dev_ptr(q, "q"), _dev_ptr(phi, "phi"),
                               _stream_ptr(stream)))


def fmm_tree_sync(tree: FmmTree, stream=None):
    _check(load().fmm_tree_sync(tree.handle, _stream_ptr(stream)))


def fmm_solve_host(src: np.ndarray, q: np.ndarray, tgt: np.ndarray | None = None,
                   opt: fmm_options | None = None, stream=None, out: np.ndarray | None = None):
    """One FMM from host arrays (copies in and out inside the call)."""
    opt = opt or fmm_default_options()
    src = np.ascontiguousarray(src, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    m = tgt.shape[0] if tgt is not None else src.shape[0]
    if out is None:
        out = np.empty((m, 2), np.float64)
    for a, n, name in ((src, None, "src"), (q, src.shape[0], "q"), (out, m, "out"),
                       (tgt, None, "tgt")):
        if a is None:
            continue
        if a.ndim != 2 or a.shape[1] != 2:
            raise ValueError(f"{name} must have shape [n, 2]")
        if n is not None and a.shape[0] != n:
            raise ValueError(f"{name} has {a.shape[0]} rows, expected {n}")
    if not (out.dtype == np.float64 and out.flags.c_contiguous):
        raise ValueError("out must be a C-contiguous float64 array")
    tp = None
    if tgt is not None:
        tgt = np.ascontiguousarray(tgt, np.float64)
        tp = tgt.ctypes.data_as(C.c_void_p)
    sp = _stream_ptr(stream) if stream is not None else C.c_void_p(0)
    _check(load().fmm_solve_host(src.ctypes.data_as(C.c_void_p), src.shape[0], tp,
                                 tgt.shape[0] if tgt is not None else 0,
                                 q.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p),
                                 C.byref(opt), sp))
    return out


def _offsets(off, name):
    off = np.ascontiguousarray(off, np.int64)
    if off.ndim != 1 or len(off) < 2:
        raise ValueError(f"{name} must hold n_inst + 1 offsets")
    return off


def fmm_evaluate_batched(src_off: np.ndarray, src, q, phi, opt: fmm_options | None = None,
                         stream=None, tgt_off: np.ndarray | None = None, tgt=None):
    """One-shot batched evaluation; with `tgt` / `tgt_off`, instance i is
    evaluated at tgt[tgt_off[i]:tgt_off[i+1]] (Eq. 2), else at its sources."""
    opt = opt or fmm_default_options()
    off = _offsets(src_off, "src_off")
    toff = None
    _need_rows(src, int(off[-1]), "src")
    _need_rows(q, int(off[-1]), "q")
    if tgt is not None:
        toff = _offsets(tgt_off, "tgt_off")
        if len(toff) != len(off):
            raise ValueError("src_off and tgt_off must have the same length")
        _need_rows(tgt, int(toff[-1]), "tgt")
        _need_rows(phi, int(toff[-1]), "phi")
    else:
        _need_rows(phi, int(off[-1]), "phi")
    _check(load().fmm_evaluate_batched(
        len(off) - 1, off.ctypes.data_as(C.c_void_p),
        toff.ctypes.data_as(C.c_void_p) if toff is not None else None, _dev_ptr(src, "src"),
        _dev_ptr(tgt, "tgt"), _dev_ptr(q, "q"), _dev_ptr(phi, "phi"), C.byref(opt),
        _stream_ptr(stream)))


def fmm_build_batched(src_off: np.ndarray, src, opt: fmm_options | None = None,
                      stream=None, tgt_off: np.ndarray | None = None, tgt=None) -> FmmTree:
    """Forest of independent instances (instance i = sources src_off[i]:src_off[i+1],
    evaluated at its sources, or at tgt[tgt_off[i]:tgt_off[i+1]] when given)."""
    opt = opt or fmm_default_options()
    off = _offsets(src_off, "src_off")
    _need_rows(src, int(off[-1]), "src")
    toff = None
    if tgt is not None:
        toff = _offsets(tgt_off, "tgt_off")
        if len(toff) != len(off):
            raise ValueError("src_off and tgt_off must have the same length")
        _need_rows(tgt, int(toff[-1]), "tgt")
    h = C.c_void_p()
    _check(load().fmm_build_batched(len(off) - 1, off.ctypes.data_as(C.c_void_p),
                                    _dev_ptr(src, "src"),
                                    toff.ctypes.data_as(C.c_void_p) if toff is not None else None,
                                    _dev_ptr(tgt, "tgt"), C.byref(opt), _stream_ptr(stream),
                                    C.byref(h)))
    m = int(toff[-1]) if toff is not None else int(off[-1])
    return FmmTree(h, int(off[-1]), m)


def fmm_set_graph(tree: FmmTree, enable: bool = True):
    _check(load().fmm_set_graph(tree.handle, int(enable)))


def fmm_direct_noalloc(src, q, phi, tgt=None, stream=None):
    """Direct sum without device allocation (static scratch in the library)."""
    m = tgt.shape[0] if tgt is not None else 0
    _need_rows(q, _rows(src), "q")
    _need_rows(phi, m if tgt is not None else _rows(src), "phi")
    _check(load().fmm_direct_noalloc(_dev_ptr(src, "src"), src.shape[0], _dev_ptr(q, "q"),
                                     _dev_ptr(tgt, "tgt"), m, _dev_ptr(phi, "phi"),
                                     _stream_ptr(stream)))


def fmm_tree_info(tree: FmmTree) -> dict:
    lv = C.c_int()
    nb, nw, ns = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().fmm_tree_info(tree.handle, C.byref(lv), C.byref(nb), C.byref(nw), C.byref(ns)))
    return dict(levels=lv.value, n_boxes=nb.value, n_weak=nw.value, n_strong=ns.value)


def fmm_tree_export(tree: FmmTree) -> dict:
    info = fmm_tree_info(tree)
    nb = info["n_boxes"]
    out = dict(
        perm=np.zeros(tree.n_src, np.uint32), tperm=np.zeros(tree.n_tgt, np.uint32),
        rect=np.zeros((nb, 4)), box_src=np.zeros((nb, 2), np.int64),
        box_tgt=np.zeros((nb, 2), np.int64), weak_off=np.zeros(nb + 1, np.int64),
        weak=np.zeros(max(info["n_weak"], 1), np.int32), strong_off=np.zeros(nb + 1, np.int64),
        strong=np.zeros(max(info["n_strong"], 1), np.int32))
    order = ("perm", "tperm", "rect", "box_src", "box_tgt", "weak_off", "weak", "strong_off",
             "strong")
    _check(load().fmm_tree_export(tree.handle, *[out[k].ctypes.data_as(C.c_void_p) for k in order]))
    out["weak"] = out["weak"][:info["n_weak"]]
    out["strong"] = out["strong"][:info["n_strong"]]
    out.update(info)
    return out


def fmm_autotune_leaf(src, q, opt: fmm_options, candidates, tgt=None, src_off=None,
                      repeats: int = 2, evaluations: int = 1, stream=None):
    """Fastest leaf size among `candidates` for this problem (single, or
    batched with `src_off`); returns (best_leaf, {candidate: ms})."""
    cand = np.ascontiguousarray(candidates, np.int32)
    ms = np.zeros(len(cand), np.float32)
    best = C.c_int()
    off = None if src_off is None else np.ascontiguousarray(src_off, np.int64)
    _check(load().fmm_autotune_leaf(
        _dev_ptr(src, "src"), src.shape[0], _dev_ptr(tgt, "tgt"),
        tgt.shape[0] if tgt is not None else 0, (len(off) - 1) if off is not None else 0,
        off.ctypes.data_as(C.c_void_p) if off is not None else None, _dev_ptr(q, "q"),
        C.byref(opt), cand.ctypes.data_as(C.c_void_p), len(cand), repeats, evaluations,
        _stream_ptr(stream), C.byref(best), ms.ctypes.data_as(C.c_void_p)))
    return int(best.value), {int(c): float(t) for c, t in zip(cand, ms)}


def fmm_autotune(src, q, opt: fmm_options, leaf_candidates, item_candidates, tgt=None,
                 src_off=None, repeats: int = 2, evaluations: int = 1, stream=None):
    """Fastest (leaf size, near-field item size) among the candidates; returns
    (options with both set, {(leaf, items): ms})."""
    lc = np.ascontiguousarray(leaf_candidates, np.int32)
    ic = np.ascontiguousarray(item_candidates, np.int32)
    ms = np.zeros(len(lc) * len(ic), np.float32)
    off = None if src_off is None else np.ascontiguousarray(src_off, np.int64)
    o = fmm_options.from_buffer_copy(opt)
    _check(load().fmm_autotune(
        _dev_ptr(src, "src"), src.shape[0], _dev_ptr(tgt, "tgt"),
        tgt.shape[0] if tgt is not None else 0, (len(off) - 1) if off is not None else 0,
        off.ctypes.data_as(C.c_void_p) if off is not None else None, _dev_ptr(q, "q"),
        C.byref(o), lc.ctypes.data_as(C.c_void_p), len(lc), ic.ctypes.data_as(C.c_void_p),
        len(ic), repeats, evaluations, _stream_ptr(stream), ms.ctypes.data_as(C.c_void_p)))
    trials = {(int(a), int(b)): float(ms[i * len(ic) + j])
              for i, a in enumerate(lc) for j, b in enumerate(ic)}
    return o, trials


def fmm_tree_export_geometry(tree: FmmTree) -> np.ndarray:
    """Rectangles the box geometry comes from (split or shrink-wrapped)."""
    out = np.zeros((fmm_tree_info(tree)["n_boxes"], 4))
    _check(load().fmm_tree_export_geometry(tree.handle, out.ctypes.data_as(C.c_void_p)))
    return out


def fmm_tree_export_shortcut(tree: FmmTree) -> dict:
    """Leaf shortcut lists (near / P2L / M2P) of a tree built with p2l_m2p=1."""
    nn, npl, nm = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().fmm_tree_shortcut_info(tree.handle, C.byref(nn), C.byref(npl), C.byref(nm)))
    nb = fmm_tree_info(tree)["n_boxes"]
    out = dict(near_off=np.zeros(nb + 1, np.int64), near=np.zeros(max(nn.value, 1), np.int32),
               p2l_off=np.zeros(nb + 1, np.int64), p2l=np.zeros(max(npl.value, 1), np.int32),
               m2p_off=np.zeros(nb + 1, np.int64), m2p=np.zeros(max(nm.value, 1), np.int32))
    order = ("near_off", "near", "p2l_off", "p2l", "m2p_off", "m2p")
    _check(load().fmm_tree_export_shortcut(tree.handle,
                                           *[out[k].ctypes.data_as(C.c_void_p) for k in order]))
    out["near"] = out["near"][:nn.value]
    out["p2l"] = out["p2l"][:npl.value]
    out["m2p"] = out["m2p"][:nm.value]
    return out


def fmm_set_timing(tree: FmmTree, enable: bool = True):
    _check(load().fmm_set_timing(tree.handle, int(enable)))


TIMING_NAMES = ("tree", "connect", "p2m", "m2m", "m2l", "l2l", "l2p_p2p", "permute", "p2l", "p2p",
                "m2p_l2p")


def fmm_get_timings(tree: FmmTree) -> dict:
    buf = (C.c_float * len(TIMING_NAMES))()
    _check(load().fmm_get_timings(tree.handle, buf, len(TIMING_NAMES)))
    return dict(zip(TIMING_NAMES, list(buf)))
