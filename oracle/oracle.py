"""ctypes front end of the C oracle (test infrastructure only).

Arrays in and out are numpy float64 / int arrays; complex values are numpy
complex128 (stored as (re, im) pairs, which is the C layout).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i64, i32, d = C.c_int64, C.c_int, C.c_double
        vp = C.c_void_p
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_set_threads.restype = None
        L.oracle_n_boxes.argtypes = [i32]
        L.oracle_n_boxes.restype = i64
        L.oracle_levels_cap.argtypes = [i64, i32]
        L.oracle_levels_cap.restype = i32
        L.oracle_levels_eq.argtypes = [i64, i32]
        L.oracle_levels_eq.restype = i32
        L.oracle_direct.argtypes = [i64, _dp, _dp, i64, _dp, _dp]
        L.oracle_direct.restype = None
        L.oracle_direct_sample.argtypes = [i64, _dp, _dp, _dp, i64, _i64p, _dp]
        L.oracle_direct_sample.restype = None
        L.oracle_p2m.argtypes = [i32, d, d, i64, _dp, _dp, _dp]
        L.oracle_m2p.argtypes = [i32, d, d, _dp, d, d, _dp]
        L.oracle_m2m.argtypes = [i32, d, d, d, d, _dp, _dp]
        L.oracle_m2l.argtypes = [i32, d, d, d, d, _dp, _dp]
        L.oracle_l2l.argtypes = [i32, d, d, d, d, _dp, _dp]
        L.oracle_l2p.argtypes = [i32, d, d, _dp, d, d, _dp]
        L.oracle_p2l.argtypes = [i32, d, d, i64, _dp, _dp, _dp]
        for f in ("oracle_p2l", "oracle_p2m", "oracle_m2p", "oracle_m2m", "oracle_m2l", "oracle_l2l", "oracle_l2p"):
            getattr(L, f).restype = None
        L.oracle_build_tree.argtypes = [i64, _dp, i64, vp, i32, _u32p, _dp, _i64p, _i8p, _dp,
                                        _u32p, _i64p]
        L.oracle_build_tree.restype = i32
        L.oracle_well_separated.argtypes = [_dp, _dp, d]
        L.oracle_well_separated.restype = i32
        L.oracle_connect.argtypes = [i32, _dp, d, _i64p, vp, i64, _i64p, vp, i64,
                                     C.POINTER(i64), C.POINTER(i64)]
        L.oracle_connect.restype = i32
        L.oracle_fmm_evaluate.argtypes = [i32, i32, _dp, _i64p, _i64p, _u32p, _u32p, _i64p,
                                          _i32p, _i64p, _i32p, i64, _dp, _dp, i64, _dp, i64,
                                          vp, _dp, vp, vp, vp, vp, vp, vp, vp, i32]
        L.oracle_fmm_evaluate.restype = i32
        L.oracle_direct_harmonic.argtypes = [i64, _dp, _dp, i64, _dp, i64, vp, _dp]
        L.oracle_direct_harmonic.restype = None
        L.oracle_l2p_deriv.argtypes = [i32, d, d, _dp, d, d, _dp]
        L.oracle_l2p_deriv.restype = None
        L.oracle_m2p_deriv.argtypes = [i32, d, d, _dp, d, d, _dp]
        L.oracle_m2p_deriv.restype = None
        L.oracle_direct_branch.argtypes = [i32, _dp, _i64p, _i64p, _u32p, _u32p, _i64p, _i32p,
                                           _i64p, _i32p, _dp, _dp, i64, _dp, i64, vp, _dp,
                                           vp, vp, vp, vp, vp, vp]
        L.oracle_direct_branch.restype = i32
        L.oracle_leaf_shortcut.argtypes = [i32, _dp, d, _i64p, _i32p, _i64p, _i32p, _i64p,
                                           _i32p, _i64p, _i32p]
        L.oracle_leaf_shortcut.restype = i32
        L.oracle_tight_rects.argtypes = [i32, _dp, _i64p, _u32p, _dp, _i64p, _u32p, vp, _dp]
        L.oracle_tight_rects.restype = None
        _lib = L
    return _lib


def _xy(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(-1, 2)


def _cplx_in(q) -> np.ndarray:
    q = np.asarray(q)
    if np.iscomplexobj(q):
        return np.ascontiguousarray(np.stack([q.real, q.imag], axis=-1), dtype=np.float64)
    return _xy(q)


def _cplx_out(buf: np.ndarray) -> np.ndarray:
    buf = buf.reshape(-1, 2)
    return buf[:, 0] + 1j * buf[:, 1]


def set_threads(n: int) -> None:
    """Threads for the FMM's independent per-target loops (1 = serial)."""
    lib().oracle_set_threads(int(n))


# ---------------------------------------------------------------- levels

def n_boxes(L: int) -> int:
    return int(lib().oracle_n_boxes(L))


def levels_cap(n: int, leaf: int) -> int:
    return int(lib().oracle_levels_cap(n, leaf))


def levels_eq(n: int, nd: int) -> int:
    return int(lib().oracle_levels_eq(n, nd))


# ---------------------------------------------------------------- direct sums

def direct(src, q, tgt=None) -> np.ndarray:
    src = _xy(src)
    q = _cplx_in(q)
    tgt = src if tgt is None else _xy(tgt)
    out = np.zeros((tgt.shape[0], 2))
    lib().oracle_direct(src.shape[0], src, q, tgt.shape[0], tgt, out)
    return _cplx_out(out)


def direct_sample(src, q, tgt, sample) -> np.ndarray:
    src = _xy(src)
    q = _cplx_in(q)
    tgt = src if tgt is None else _xy(tgt)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    out = np.zeros((sample.size, 2))
    lib().oracle_direct_sample(src.shape[0], src, q, tgt, sample.size, sample, out)
    return _cplx_out(out)


def direct_harmonic(src, q, tgt=None, sample=None) -> np.ndarray:
    """u(y_i) = sum_{x_j != y_i} q_j / (x_j - y_i): the paper's harmonic kernel."""
    src = _xy(src)
    q = _cplx_in(q)
    tgt = src if tgt is None else _xy(tgt)
    ns, sp, keep = _sample_arg(sample)
    out = np.zeros((ns if sample is not None else tgt.shape[0], 2))
    lib().oracle_direct_harmonic(src.shape[0], src, q, tgt.shape[0], tgt, ns, sp, out)
    del keep
    return _cplx_out(out)


# ---------------------------------------------------------------- operators

def _coef(a, p):
    a = _cplx_in(a)
    assert a.shape[0] == p + 1
    return a


def p2m(p, c, xy, q) -> np.ndarray:
    xy = _xy(xy)
    q = _cplx_in(q)
    a = np.zeros((p + 1, 2))
    lib().oracle_p2m(p, c.real, c.imag, xy.shape[0], xy, q, a)
    return _cplx_out(a)


def m2p(p, c, a, z) -> complex:
    out = np.zeros(2)
    lib().oracle_m2p(p, c.real, c.imag, _coef(a, p), z.real, z.imag, out)
    return complex(out[0], out[1])


def m2m(p, zc, zp, a) -> np.ndarray:
    out = np.zeros((p + 1, 2))
    lib().oracle_m2m(p, zc.real, zc.imag, zp.real, zp.imag, _coef(a, p), out)
    return _cplx_out(out)


def m2l(p, zs, zt, a) -> np.ndarray:
    out = np.zeros((p + 1, 2))
    lib().oracle_m2l(p, zs.real, zs.imag, zt.real, zt.imag, _coef(a, p), out)
    return _cplx_out(out)


def l2l(p, zp, zc, b) -> np.ndarray:
    out = np.zeros((p + 1, 2))
    lib().oracle_l2l(p, zp.real, zp.imag, zc.real, zc.imag, _coef(b, p), out)
    return _cplx_out(out)


def p2l(p, c, xy, q) -> np.ndarray:
    xy = _xy(xy)
    q = _cplx_in(q)
    b = np.zeros((p + 1, 2))
    lib().oracle_p2l(p, c.real, c.imag, xy.shape[0], xy, q, b)
    return _cplx_out(b)


def l2p_deriv(p, c, b, z) -> complex:
    out = np.zeros(2)
    lib().oracle_l2p_deriv(p, c.real, c.imag, _coef(b, p), z.real, z.imag, out)
    return complex(out[0], out[1])


def m2p_deriv(p, c, a, z) -> complex:
    out = np.zeros(2)
    lib().oracle_m2p_deriv(p, c.real, c.imag, _coef(a, p), z.real, z.imag, out)
    return complex(out[0], out[1])


def l2p(p, c, b, z) -> complex:
    out = np.zeros(2)
    lib().oracle_l2p(p, c.real, c.imag, _coef(b, p), z.real, z.imag, out)
    return complex(out[0], out[1])


# ---------------------------------------------------------------- tree

@dataclass
class Tree:
    L: int
    perm: np.ndarray        # uint32[N]   tree position -> source index
    rect: np.ndarray        # float64[nb, 4]  x0, x1, y0, y1
    box_src: np.ndarray     # int64[nb, 2]    start, count
    split_axis: np.ndarray  # int8[nb_internal, 3]
    split_line: np.ndarray  # float64[nb_internal, 3]
    tperm: np.ndarray       # uint32[M]
    box_tgt: np.ndarray     # int64[nb, 2]
    separate: bool

    @property
    def n_boxes(self) -> int:
        return self.rect.shape[0]

    def centres(self) -> np.ndarray:
        return 0.5 * (self.rect[:, 0] + self.rect[:, 1]) + 1j * 0.5 * (self.rect[:, 2] + self.rect[:, 3])


@dataclass
class Lists:
    weak_off: np.ndarray
    weak: np.ndarray
    strong_off: np.ndarray
    strong: np.ndarray


def build_tree(src, L: int, tgt=None) -> Tree:
    src = _xy(src)
    n = src.shape[0]
    nb = n_boxes(L)
    nbi = n_boxes(L - 1) if L > 0 else 0
    perm = np.zeros(n, np.uint32)
    rect = np.zeros((nb, 4))
    box_src = np.zeros((nb, 2), np.int64)
    sa = np.zeros((max(nbi, 1), 3), np.int8)
    sl = np.zeros((max(nbi, 1), 3))
    if tgt is None:
        m = n
        tptr = None
        tgt_arr = None
    else:
        tgt_arr = _xy(tgt)
        m = tgt_arr.shape[0]
        tptr = tgt_arr.ctypes.data_as(C.c_void_p)
    tperm = np.zeros(max(m, 1), np.uint32)
    box_tgt = np.zeros((nb, 2), np.int64)
    rc = lib().oracle_build_tree(n, src, m, tptr, L, perm, rect, box_src, sa, sl, tperm, box_tgt)
    if rc != 0:
        raise RuntimeError(f"oracle_build_tree failed: {rc}")
    return Tree(L, perm, rect, box_src, sa[:nbi], sl[:nbi], tperm[:m], box_tgt, tgt is not None)


def tight_rects(tree: Tree, src, tgt=None) -> np.ndarray:
    """Bounding rectangles of every box's points (sources, and evaluation
    points when separate); empty boxes keep their split rectangles."""
    src = _xy(src)
    out = np.zeros((tree.n_boxes, 4))
    tgt_arr = _xy(tgt) if tgt is not None else None
    tperm = tree.tperm if tgt is not None else tree.perm
    box_tgt = tree.box_tgt if tgt is not None else tree.box_src
    lib().oracle_tight_rects(tree.L, np.ascontiguousarray(tree.rect), tree.box_src, tree.perm, src,
                             box_tgt, np.ascontiguousarray(tperm, np.uint32),
                             tgt_arr.ctypes.data_as(C.c_void_p) if tgt_arr is not None else None,
                             out)
    return out


def shrink(tree: Tree, src, tgt=None) -> Tree:
    """The same tree with the shrink-wrapped geometry (its `rect` replaced by
    the tight rectangles); connect / evaluate / direct_branch then use it."""
    import dataclasses
    return dataclasses.replace(tree, rect=tight_rects(tree, src, tgt))


def well_separated(rect_b, rect_c, theta=0.5) -> bool:
    return bool(lib().oracle_well_separated(np.ascontiguousarray(rect_b, np.float64),
                                            np.ascontiguousarray(rect_c, np.float64), theta))


def connect(tree: Tree, theta: float = 0.5) -> Lists:
    nb = tree.n_boxes
    wo = np.zeros(nb + 1, np.int64)
    so = np.zeros(nb + 1, np.int64)
    nw, ns = C.c_int64(0), C.c_int64(0)
    rect = np.ascontiguousarray(tree.rect)
    lib().oracle_connect(tree.L, rect, theta, wo, None, 0, so, None, 0, C.byref(nw), C.byref(ns))
    weak = np.zeros(max(nw.value, 1), np.int32)
    strong = np.zeros(max(ns.value, 1), np.int32)
    lib().oracle_connect(tree.L, rect, theta, wo, weak.ctypes.data_as(C.c_void_p), weak.size,
                         so, strong.ctypes.data_as(C.c_void_p), strong.size, C.byref(nw),
                         C.byref(ns))
    return Lists(wo, weak, so, strong)


@dataclass
class Shortcut:
    """Leaf-level split of the strong lists (Sec. 2): offsets over the 4^L
    leaves, entries are global box ids."""
    near_off: np.ndarray
    near: np.ndarray
    p2l_off: np.ndarray
    p2l: np.ndarray
    m2p_off: np.ndarray
    m2p: np.ndarray

    def ptrs(self):
        return [a.ctypes.data_as(C.c_void_p) for a in
                (self.near_off, self.near, self.p2l_off, self.p2l, self.m2p_off, self.m2p)]


def leaf_shortcut(tree: Tree, lists: Lists, theta: float = 0.5) -> Shortcut:
    nleaf = 1 << (2 * tree.L)
    base = n_boxes(tree.L - 1) if tree.L > 0 else 0
    cap = max(int(lists.strong_off[base + nleaf] - lists.strong_off[base]), 1)
    no, po, mo = (np.zeros(nleaf + 1, np.int64) for _ in range(3))
    nl, pl, ml = (np.zeros(cap, np.int32) for _ in range(3))
    strong = np.ascontiguousarray(lists.strong, np.int32)
    rc = lib().oracle_leaf_shortcut(tree.L, np.ascontiguousarray(tree.rect), theta,
                                    lists.strong_off, strong, no, nl, po, pl, mo, ml)
    if rc != 0:
        raise RuntimeError(f"oracle_leaf_shortcut failed: {rc}")
    return Shortcut(no, nl[:max(no[-1], 1)], po, pl[:max(po[-1], 1)], mo, ml[:max(mo[-1], 1)])


def _short_args(sc: Shortcut | None):
    return [None] * 6 if sc is None else sc.ptrs()


def _sample_arg(sample):
    if sample is None:
        return 0, None, None
    s = np.ascontiguousarray(sample, dtype=np.int64)
    return s.size, s.ctypes.data_as(C.c_void_p), s


def evaluate(tree: Tree, lists: Lists, src, q, p: int, tgt=None, sample=None,
             seconds: np.ndarray | None = None, shortcut: Shortcut | None = None,
             kernel: int = 0) -> np.ndarray:
    """Oracle FMM at all evaluation points (or a sample of them).  `seconds`
    (float64[2], optional) receives the time of the expansion phases and of
    the per-point L2P + P2P phase.  With `shortcut`, the leaf-level P2L / M2P
    lists replace the corresponding direct interactions.  kernel 1: the
    harmonic kernel u = sum q_j / (x_j - y) (the same expansions, differentiated)."""
    src = _xy(src)
    q = _cplx_in(q)
    tgt_arr = src if tgt is None else _xy(tgt)
    ns, sp, keep = _sample_arg(sample)
    n_out = ns if sample is not None else tgt_arr.shape[0]
    out = np.zeros((n_out, 2))
    rc = lib().oracle_fmm_evaluate(
        tree.L, p, np.ascontiguousarray(tree.rect), tree.box_src, tree.box_tgt, tree.perm,
        tree.tperm, lists.weak_off, lists.weak, lists.strong_off, lists.strong, src.shape[0],
        src, q, tgt_arr.shape[0], tgt_arr, ns, sp, out,
        seconds.ctypes.data_as(C.c_void_p) if seconds is not None else None,
        *_short_args(shortcut), kernel)
    if rc != 0:
        raise RuntimeError(f"oracle_fmm_evaluate failed: {rc}")
    del keep
    return _cplx_out(out)


def direct_branch(tree: Tree, lists: Lists, src, q, tgt=None, sample=None,
                  shortcut: Shortcut | None = None) -> np.ndarray:
    """FP64 direct sum taking, for every pair, the branch of the logarithm
    that the FMM's expansion for that pair sums (with `shortcut`, also for the
    P2L and M2P pairs)."""
    src = _xy(src)
    q = _cplx_in(q)
    tgt_arr = src if tgt is None else _xy(tgt)
    ns, sp, keep = _sample_arg(sample)
    n_out = ns if sample is not None else tgt_arr.shape[0]
    out = np.zeros((n_out, 2))
    rc = lib().oracle_direct_branch(
        tree.L, np.ascontiguousarray(tree.rect), tree.box_src, tree.box_tgt, tree.perm,
        tree.tperm, lists.weak_off, lists.weak, lists.strong_off, lists.strong, src, q,
        tgt_arr.shape[0], tgt_arr, ns, sp, out, *_short_args(shortcut))
    if rc != 0:
        raise RuntimeError(f"oracle_direct_branch failed: {rc}")
    del keep
    return _cplx_out(out)


def levels(n: int, leaf: int, level_rule: int = 0) -> int:
    return levels_cap(n, leaf) if level_rule == 0 else levels_eq(n, leaf)


def fmm(src, q, p: int, leaf: int, theta: float = 0.5, tgt=None, level_rule: int = 0,
        sample=None, L: int | None = None, p2l_m2p: bool = False, box_fit: bool = False,
        kernel: int = 0):
    """Whole oracle FMM; returns (phi, tree, lists), and the leaf shortcut
    lists as a fourth element when `p2l_m2p`.  With `box_fit` the returned
    tree carries the shrink-wrapped rectangles."""
    src = _xy(src)
    if L is None:
        L = levels(src.shape[0], leaf, level_rule)
    tree = build_tree(src, L, tgt)
    if box_fit:
        tree = shrink(tree, src, tgt)
    lists = connect(tree, theta)
    sc = leaf_shortcut(tree, lists, theta) if p2l_m2p else None
    phi = evaluate(tree, lists, src, q, p, tgt, sample, shortcut=sc, kernel=kernel)
    if p2l_m2p:
        return phi, tree, lists, sc
    return phi, tree, lists


def normwise_error(phi, ref) -> float:
    """max_i |phi_i - ref_i| / max_i |ref_i| (the gate's error measure)."""
    ref = np.asarray(ref)
    return float(np.max(np.abs(np.asarray(phi) - ref)) / max(np.max(np.abs(ref)), 1e-300))
