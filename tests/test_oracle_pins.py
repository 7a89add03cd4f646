"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics (closed forms, exact identities, the paper's own algorithms,
truncation bounds, brute force).  CPU only.

Each test names what it pins.  A plausible slip in the oracle (a dropped
term, a wrong sign, a wrong index, a swapped operand) fails at least one.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def crandn(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


# --------------------------------------------------------------- levels

def test_levels_eq_golden():
    """Eq. (Nlevels) with N_d = 45 gives 8 levels exactly for
    N in (18*2^16, 72*2^16] (Sec. 5.1, discussion of the time table)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "levels_eq_nd45.txt"), dtype=np.int64)
    for n, nl in rows:
        assert O.levels_eq(int(n), 45) == nl, (n, nl)


def test_levels_cap_closed_form():
    # ceil(N / 4^L) <= leaf with L minimal
    assert O.levels_cap(10_000, 40) == 4      # 10000/256 = 39.06 -> 40; 10000/64 -> 157
    assert O.levels_cap(1_000_000, 64) == 7   # 1e6/16384 = 61.04 -> 62; 1e6/4096 -> 245
    assert O.levels_cap(16_000_000, 64) == 9
    assert O.levels_cap(40, 40) == 0
    assert O.levels_cap(41, 40) == 1
    assert O.n_boxes(0) == 1 and O.n_boxes(1) == 5 and O.n_boxes(2) == 21


# --------------------------------------------------------------- direct sum (Eq. 1, Eq. 2)

@pytest.mark.parametrize("n", [3, 7, 16])
def test_direct_roots_of_unity(n):
    """prod_{j != i} (z_i - z_j) = n z_i^(n-1) for the n-th roots of unity, so
    with q_j = 1: Re Phi_i = ln n and Im Phi_i = (n-1) arg z_i (mod 2 pi)."""
    th = 2 * np.pi * np.arange(n) / n
    xy = np.stack([np.cos(th), np.sin(th)], axis=1)
    q = np.ones(n, complex)
    phi = O.direct(xy, q)
    assert np.allclose(phi.real, np.log(n), rtol=0, atol=1e-13)
    k = (phi.imag - (n - 1) * th) / (2 * np.pi)
    assert np.allclose(k, np.round(k), atol=1e-12)
    # complex strength c scales everything by c
    c = 0.3 - 1.7j
    phi_c = O.direct(xy, q * c)
    assert np.allclose(phi_c, c * phi, atol=1e-13)


def test_direct_two_points_and_coincident():
    xy = np.array([[0.0, 0.0], [3.0, 4.0], [3.0, 4.0]])  # a duplicate point
    q = np.array([1.0 + 0j, 2.0 + 0.5j, -1.0 + 0j])
    phi = O.direct(xy, q)
    # point 0 sees both others at distance 5, angle atan2(-4,-3)
    l = math.log(5.0) + 1j * math.atan2(-4.0, -3.0)
    assert abs(phi[0] - (q[1] + q[2]) * l) < 1e-14
    # points 1 and 2 coincide: they skip each other, see only point 0
    l1 = math.log(5.0) + 1j * math.atan2(4.0, 3.0)
    assert abs(phi[1] - q[0] * l1) < 1e-14 and abs(phi[2] - q[0] * l1) < 1e-14
    # separate evaluation point on top of a source skips that source only
    t = np.array([[3.0, 4.0]])
    assert abs(O.direct(xy, q, t)[0] - q[0] * l1) < 1e-14


# --------------------------------------------------------------- expansions (Eq. 4, Eq. 5)

@pytest.mark.parametrize("p", [4, 10, 20, 30])
def test_p2m_single_source_truncation_bound(p):
    """Single source at offset s from the centre, evaluated at |z - c| = R:
    |M(z) - q Log(z - x)| <= |q| (|s|/R)^(p+1) / ((p+1)(1 - |s|/R))."""
    rng = np.random.default_rng(p)
    c = 0.2 + 0.1j
    for _ in range(20):
        s = 0.3 * np.exp(2j * np.pi * rng.random()) * rng.random()
        z = c + 1.0 * np.exp(2j * np.pi * rng.random())
        x = c + s
        q = complex(*rng.uniform(-1, 1, 2))
        a = O.p2m(p, c, np.array([[x.real, x.imag]]), np.array([q]))
        assert abs(a[0] - q) == 0.0
        val = O.m2p(p, c, a, z)
        exact = q * (np.log(z - c) + np.log(1 - s / (z - c)))  # same branch as the series
        ratio = abs(s) / abs(z - c)
        bound = abs(q) * ratio ** (p + 1) / ((p + 1) * (1 - ratio))
        assert abs(val - exact) <= bound * 1.0001 + 4e-15 * max(1.0, abs(exact))


def test_p2m_coefficients_closed_form():
    """a_k = -sum q (x - c)^k / k: the sign and 1/k are pinned by a source
    whose offset is 1 (all powers 1) and by one at offset 2i."""
    p = 6
    a = O.p2m(p, 0j, np.array([[1.0, 0.0]]), np.array([2.0 + 0j]))
    assert np.allclose(a, [2.0] + [-2.0 / k for k in range(1, p + 1)], atol=1e-15)
    a = O.p2m(p, 1j, np.array([[0.0, 3.0]]), np.array([1.0 + 0j]))
    assert np.allclose(a[1:], [-(2j) ** k / k for k in range(1, p + 1)], atol=1e-13)


def test_m2m_exact_identity():
    """P2M about the child centre followed by M2M equals P2M about the
    parent centre (exact: the shifted a'_l uses only a_k, k <= l)."""
    rng = np.random.default_rng(3)
    p = 24
    zc, zp = 0.3 + 0.2j, 0.1 - 0.05j
    xy = np.stack([zc.real + 0.05 * rng.uniform(-1, 1, 40), zc.imag + 0.05 * rng.uniform(-1, 1, 40)], 1)
    q = crandn(rng, 40)
    ref = O.p2m(p, zp, xy, q)
    got = O.m2m(p, zc, zp, O.p2m(p, zc, xy, q))
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-13 * scale


def test_l2p_horner_closed_form():
    p = 3
    b = np.array([1.0, 2.0 - 1j, 0.5j, -3.0])
    c, z = 0.5 + 0.5j, 1.25 - 0.5j
    w = z - c
    assert abs(O.l2p(p, c, b, z) - (b[0] + b[1] * w + b[2] * w ** 2 + b[3] * w ** 3)) < 1e-14


def test_l2l_exact_identity():
    """The re-centred local expansion is the same polynomial."""
    rng = np.random.default_rng(4)
    p = 20
    zp, zc = 0.0 + 0.0j, 0.2 - 0.1j
    b = crandn(rng, p + 1) / (2.0 ** np.arange(p + 1))
    bc = O.l2l(p, zp, zc, b)
    for _ in range(10):
        z = zc + 0.1 * (rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1))
        v0, v1 = O.l2p(p, zp, b, z), O.l2p(p, zc, bc, z)
        assert abs(v0 - v1) <= 1e-14 * max(1.0, abs(v0))


@pytest.mark.parametrize("p", [8, 16, 24])
def test_m2l_converges_to_exact_log(p):
    """P2M -> M2L -> L2P against the exact potential of sources in a
    well-separated box (same branch: Log(c_t - c_s) + Log(1 + u)); the error
    is bounded by the geometric truncation rate and decays with p."""
    rng = np.random.default_rng(5)
    zs, zt = 0.0 + 0.0j, 1.5 + 0.9j
    rs = rt = 0.25
    n = 30
    xs = zs + rs * np.sqrt(rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
    q = crandn(rng, n)
    a = O.p2m(p, zs, np.stack([xs.real, xs.imag], 1), q)
    b = O.m2l(p, zs, zt, a)
    D = zt - zs
    ratio = (rs + rt) / abs(D)
    err = 0.0
    for _ in range(10):
        y = zt + rt * np.sqrt(rng.random()) * np.exp(2j * np.pi * rng.random())
        u = ((y - zt) - (xs - zs)) / D
        exact = np.sum(q * (np.log(D) + np.log(1 + u)))
        err = max(err, abs(O.l2p(p, zt, b, y) - exact))
    bound = np.sum(np.abs(q)) * 2 * ratio ** (p + 1) / ((p + 1) * (1 - ratio))
    assert err <= bound, (err, bound)


def _paper_m2l(p, a, zs, zt):
    """The M2L shift with prescaling, two summation sweeps and postscaling
    (Alg. "Multipole to local translation"), in the reading that reproduces
    the exact expansion: r = z_s - z_t, the first sweep adds, and the a_0
    term carries Log(z_t - z_s)."""
    r = zs - zt
    b = np.zeros(p + 1, complex)
    for j in range(1, p + 1):
        b[j - 1] = (-1) ** j * a[j] / r ** j
    for k in range(2, p + 1):
        for j in range(p - k, p):
            b[j] += b[j + 1]
    for k in range(p, 0, -1):
        for j in range(k, p + 1):
            b[j] += b[j - 1]
    b[0] += a[0] * np.log(zt - zs)
    for j in range(1, p + 1):
        b[j] = (b[j] - a[0] / j) / r ** j
    return b


def _paper_m2m_scaled(p, a, zc, zp):
    """Alg. "Multipole to multipole translation" (b): scale by r^-j, repeated
    ascending prefix sweeps, then the a_0 term and r^j back."""
    a = a.copy()
    r = zc - zp
    for j in range(1, p + 1):
        a[j] /= r ** j
    for k in range(p, 1, -1):
        for j in range(k, p + 1):
            a[j] += a[j - 1]
    for j in range(1, p + 1):
        a[j] = (a[j] - a[0] / j) * r ** j
    return a


def _paper_l2l(p, b, zp, zc):
    """Alg. "Local to local translation": r = z_p - z_c, scale by r^j,
    descending difference sweeps, scale back."""
    b = b.copy()
    r = zp - zc
    for j in range(1, p + 1):
        b[j] *= r ** j
    for k in range(0, p + 1):
        for j in range(p - k, p):
            b[j] -= b[j + 1]
    for j in range(1, p + 1):
        b[j] /= r ** j
    return b


@pytest.mark.parametrize("p", [5, 17, 30])
def test_operators_match_paper_algorithms(p):
    """The oracle's closed-form operators agree with the paper's shift
    algorithms (M2M (b), L2L, and M2L in the corrected reading)."""
    rng = np.random.default_rng(p + 100)
    a = crandn(rng, p + 1)
    zs, zt = 0.1 + 0.2j, 1.3 - 0.8j
    ref = O.m2l(p, zs, zt, a)
    got = _paper_m2l(p, a, zs, zt)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    zc, zp = 0.3 + 0.1j, 0.05 - 0.02j
    ref = O.m2m(p, zc, zp, a)
    assert np.max(np.abs(_paper_m2m_scaled(p, a, zc, zp) - ref)) <= 1e-12 * np.max(np.abs(ref))
    ref = O.l2l(p, zp, zc, a)
    assert np.max(np.abs(_paper_l2l(p, a, zp, zc) - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_printed_m2l_signs_are_a_misprint():
    """With r = z_o - z_i, a subtracting first sweep and -a_0 log r, as
    printed, the M2L shift does not reproduce the expansion: the reading
    used above is needed (recorded as a reading of the paper)."""
    p = 10
    rng = np.random.default_rng(9)
    a = crandn(rng, p + 1)
    zs, zt = 0.0j, 2.0 + 1.0j
    r = zt - zs
    b = np.zeros(p + 1, complex)
    for j in range(1, p + 1):
        b[j - 1] = a[j] / r ** j * (-1) ** j
    for k in range(2, p + 1):
        for j in range(p - k, p):
            b[j] -= b[j + 1]
    for k in range(p, 0, -1):
        for j in range(k, p + 1):
            b[j] += b[j - 1]
    b[0] -= a[0] * np.log(r)
    for j in range(1, p + 1):
        b[j] = (b[j] - a[0] / j) / r ** j
    ref = O.m2l(p, zs, zt, a)
    assert np.max(np.abs(b - ref)) > 1e-3 * np.max(np.abs(ref))


# --------------------------------------------------------------- tree (Sec. 2, Sec. 3.2)

def _py_tree(xy, L):
    """Brute-force restatement of the tree rules on tiny inputs: Python
    sorted() on (coordinate, index), floor(n/2) to the left, the split line
    rules, child order 4b + 2 h1 + h2."""
    n = xy.shape[0]
    rect0 = [min(xy[:, 0]) + 0.0, max(xy[:, 0]) + 0.0, min(xy[:, 1]) + 0.0, max(xy[:, 1]) + 0.0]
    boxes = [(list(range(n)), rect0)]
    for _ in range(L):
        nxt = []
        for ids, rect in boxes:
            halves = []
            for part, rc in _py_split(xy, ids, rect):
                halves.extend(_py_split(xy, part, rc))
            nxt.extend(halves)
        boxes = nxt
    return boxes


def _py_split(xy, ids, rect):
    ax = 0 if rect[1] - rect[0] >= rect[3] - rect[2] else 1
    s = sorted(ids, key=lambda i: (xy[i, ax] + 0.0, i))
    nl = len(s) // 2
    mid = 0.5 * (rect[2 * ax] + rect[2 * ax + 1])
    if nl > 0:
        line = 0.5 * (xy[s[nl - 1], ax] + xy[s[nl], ax])
    elif s:
        line = min(mid, xy[s[0], ax] + 0.0)
    else:
        line = mid
    left, right = list(rect), list(rect)
    left[2 * ax + 1] = line
    right[2 * ax] = line
    return [(s[:nl], left), (s[nl:], right)]


@pytest.mark.parametrize("n,L,dup", [(50, 1, False), (200, 2, False), (300, 3, True), (5, 2, False)])
def test_tree_matches_bruteforce(n, L, dup):
    rng = np.random.default_rng(n)
    xy = rng.random((n, 2))
    if dup:  # duplicated points and shared coordinates exercise the (coord, index) key
        xy[10:20] = xy[0]
        xy[30:60, 0] = 0.5
    tree = O.build_tree(xy, L)
    ref = _py_tree(xy, L)
    base = O.n_boxes(L - 1) if L > 0 else 0
    for b, (ids, rect) in enumerate(ref):
        g = base + b
        lo, cnt = tree.box_src[g]
        assert cnt == len(ids)
        assert list(tree.perm[lo:lo + cnt]) == ids
        assert np.array_equal(tree.rect[g], np.array(rect))


def test_tree_invariants_clusters():
    src, q, _ = W.problem("clusters", 20_000, 7)
    L = O.levels_cap(src.shape[0], 32)
    tree = O.build_tree(src, L)
    assert sorted(tree.perm.tolist()) == list(range(src.shape[0]))
    for l in range(L):
        for b in range(4 ** l):
            g = O.n_boxes(l - 1) + b if l > 0 else 0
            n = tree.box_src[g, 1]
            ch = O.n_boxes(l) + 4 * b + np.arange(4)
            c = tree.box_src[ch, 1]
            h = [n // 2, n - n // 2]
            assert list(c) == [h[0] // 2, h[0] - h[0] // 2, h[1] // 2, h[1] - h[1] // 2]
            assert tree.box_src[ch[0], 0] == tree.box_src[g, 0]
    # every point inside its leaf rectangle
    base = O.n_boxes(L - 1)
    for b in range(4 ** L):
        lo, cnt = tree.box_src[base + b]
        pts = src[tree.perm[lo:lo + cnt]]
        r = tree.rect[base + b]
        assert np.all((pts[:, 0] >= r[0]) & (pts[:, 0] <= r[1]) & (pts[:, 1] >= r[2]) & (pts[:, 1] <= r[3]))


def test_targets_descend_split_lines():
    src, q, tgt = W.problem("clusters", 5000, 11, tgt_dist="uniform", m=3000)
    L = 3
    tree = O.build_tree(src, L, tgt)
    base = O.n_boxes(L - 1)
    assert sorted(tree.tperm.tolist()) == list(range(3000))
    for b in range(4 ** L):
        lo, cnt = tree.box_tgt[base + b]
        ids = tree.tperm[lo:lo + cnt]
        assert np.all(np.diff(ids.astype(np.int64)) > 0)  # original order inside a leaf
        r = tree.rect[base + b]
        pts = tgt[ids]
        assert np.all((pts[:, 0] >= r[0]) & (pts[:, 0] <= r[1]) & (pts[:, 1] >= r[2]) & (pts[:, 1] <= r[3]))
    # root rectangle covers sources and targets
    allp = np.vstack([src, tgt])
    assert np.array_equal(tree.rect[0], [allp[:, 0].min(), allp[:, 0].max(), allp[:, 1].min(), allp[:, 1].max()])


# --------------------------------------------------------------- connectivity (Eq. 3)

def _centre_radius(r):
    c = (0.5 * (r[0] + r[1]), 0.5 * (r[2] + r[3]))
    w, h = r[1] - r[0], r[3] - r[2]
    return c, 0.5 * math.sqrt(w * w + h * h)


def test_theta_criterion_closed_form():
    # unit squares: radius sqrt(2)/2; R + r/2 = 1.5 * 0.7071 = 1.0607 <= d/2 iff d >= 2.1213
    a = np.array([0.0, 1.0, 0.0, 1.0])
    assert not O.well_separated(a, a + np.array([2.0, 2.0, 0, 0]))      # d = 2
    assert O.well_separated(a, a + np.array([2.2, 2.2, 0, 0]))          # d = 2.2
    assert not O.well_separated(a, a)                                   # d = 0
    # unequal boxes use R = max, r = min: R + theta r <= theta d
    big = np.array([0.0, 2.0, 0.0, 2.0])                                # radius sqrt(2)
    small = np.array([3.9, 4.1, 0.9, 1.1])                              # radius 0.1414, d = 3
    R, r = math.sqrt(2), math.sqrt(0.08) / 2
    assert O.well_separated(big, small) == ((R + 0.5 * r) <= 0.5 * 3.0)
    assert O.well_separated(big, small) == O.well_separated(small, big)


def test_lists_cover_every_leaf_pair_exactly_once():
    src, q, _ = W.problem("clusters", 8000, 13)
    L = O.levels_cap(8000, 30)
    tree = O.build_tree(src, L)
    li = O.connect(tree)
    nb = tree.n_boxes
    base = O.n_boxes(L - 1)
    nleaf = 4 ** L
    cover = np.zeros((nleaf, nleaf), np.int32)
    lvl_of = np.zeros(nb, np.int64)
    for l in range(L + 1):
        lvl_of[(O.n_boxes(l - 1) if l else 0):O.n_boxes(l)] = l
    for g in range(nb):
        l = lvl_of[g]
        b = g - (O.n_boxes(l - 1) if l else 0)
        span = 4 ** (L - l)
        for s in li.weak[li.weak_off[g]:li.weak_off[g + 1]]:
            ls = lvl_of[s]
            assert ls == l
            sb = s - (O.n_boxes(ls - 1) if ls else 0)
            cover[b * span:(b + 1) * span, sb * span:(sb + 1) * span] += 1
            assert O.well_separated(tree.rect[g], tree.rect[s])
    for b in range(nleaf):
        g = base + b
        ss = li.strong[li.strong_off[g]:li.strong_off[g + 1]]
        assert g in ss
        for s in ss:
            cover[b, s - base] += 1
            assert not O.well_separated(tree.rect[g], tree.rect[s])
    assert np.all(cover == 1)


# --------------------------------------------------------------- whole FMM

def test_fmm_single_leaf_is_direct_sum_bitexact():
    """N <= leaf gives L = 0: the FMM reduces to P2P over one box, in the
    same order as the direct sum."""
    src, q, _ = W.problem("uniform", 37, 21)
    phi, tree, _ = O.fmm(src, q, p=10, leaf=40)
    assert tree.L == 0
    assert np.array_equal(phi, O.direct(src, q))


@pytest.mark.parametrize("L", [1, 2, 3])
def test_fmm_tiny_bruteforce(L):
    """Brute force on 64 points: at L = 1 all four boxes touch, so nothing is
    well separated and the FMM is the direct sum to rounding; deeper trees
    converge to the branch-consistent direct sum as p grows."""
    src, q, _ = W.problem("uniform", 64, 31 + L)
    errs = []
    for p in (6, 12, 24):
        phi, tree, li = O.fmm(src, q, p=p, leaf=64, L=L)
        ref = O.direct_branch(tree, li, src, q)
        errs.append(O.normwise_error(phi, ref))
    if L == 1:
        assert li.weak.size <= 1 and li.weak_off[-1] == 0
        assert max(errs) < 1e-15
    else:
        assert li.weak_off[-1] > 0
        assert errs[2] < 1e-9 and errs[1] < errs[0] and errs[2] < errs[1]


def test_fmm_error_decays_geometrically():
    """Truncation error falls roughly like a fixed ratio per term (p ~ log TOL / log theta)."""
    src, q, _ = W.problem("uniform", 3000, 41)
    errs = {}
    for p in (5, 10, 15, 20):
        phi, tree, li = O.fmm(src, q, p=p, leaf=20)
        ref = O.direct_branch(tree, li, src, q)
        errs[p] = O.normwise_error(phi, ref)
    assert errs[20] < 1e-8
    for a, b in ((5, 10), (10, 15), (15, 20)):
        assert errs[b] < errs[a] / 10, errs


def test_branch_direct_differs_from_principal_by_2pi_multiples():
    """For integer strengths the branch-consistent sum and the principal-log
    sum differ by 2 pi i times an integer, with identical real parts."""
    rng = np.random.default_rng(51)
    src = rng.random((1500, 2))
    q = rng.choice([-1.0, 1.0], 1500) + 0j
    _, tree, li = O.fmm(src, q, p=4, leaf=16)
    bc = O.direct_branch(tree, li, src, q)
    pr = O.direct(src, q)
    assert np.allclose(bc.real, pr.real, rtol=0, atol=1e-10)
    k = (bc.imag - pr.imag) / (2 * np.pi)
    assert np.allclose(k, np.round(k), atol=1e-8)
    assert np.any(np.round(k) != 0)  # the branch really matters


def test_fmm_real_part_vs_plain_direct_real_strengths():
    src, q, _ = W.problem("curve", 4000, 61, real_q=True)
    phi, tree, li = O.fmm(src, q, p=24, leaf=32)
    ref = O.direct(src, q)
    assert np.max(np.abs(phi.real - ref.real)) <= 1e-9 * np.max(np.abs(ref.real))


def test_fmm_separate_targets():
    src, q, tgt = W.problem("clusters", 4000, 71, tgt_dist="uniform", m=2500)
    phi, tree, li = O.fmm(src, q, p=24, leaf=32, tgt=tgt)
    ref = O.direct_branch(tree, li, src, q, tgt)
    assert O.normwise_error(phi, ref) < 1e-9
    samp = np.array([0, 7, 100, 2499])
    assert np.array_equal(O.evaluate(tree, li, src, q, 24, tgt, sample=samp), phi[samp])
    assert np.array_equal(O.direct_branch(tree, li, src, q, tgt, sample=samp), ref[samp])


# --------------------------------------------------------------- leaf shortcut (Sec. 2)

@pytest.mark.parametrize("p", [6, 14, 28])
def test_p2l_single_source_truncation_bound(p):
    """One source x at distance d from the local centre c, evaluated at
    |z - c| = rho: |L(z) - q Log(z - x)| <= |q| (rho/d)^(p+1) / ((p+1)(1 - rho/d))
    on the branch Log(c - x) + Log(1 + (z - c)/(c - x))."""
    rng = np.random.default_rng(100 + p)
    c = -0.3 + 0.4j
    for _ in range(20):
        x = c + 1.0 * np.exp(2j * np.pi * rng.random())
        z = c + 0.35 * np.sqrt(rng.random()) * np.exp(2j * np.pi * rng.random())
        q = complex(*rng.uniform(-1, 1, 2))
        b = O.p2l(p, c, np.array([[x.real, x.imag]]), np.array([q]))
        exact = q * (np.log(c - x) + np.log(1 + (z - c) / (c - x)))
        ratio = abs(z - c) / abs(x - c)
        bound = abs(q) * ratio ** (p + 1) / ((p + 1) * (1 - ratio))
        assert abs(O.l2p(p, c, b, z) - exact) <= bound * 1.0001 + 4e-15 * max(1.0, abs(exact))


def test_p2l_equals_m2l_of_a_point_multipole():
    """A source at a box centre has the multipole a_0 = q, a_k = 0, and M2L of
    that multipole is the local expansion of q Log(z - x): P2L and M2L (two
    independent formulas of the oracle) must agree term by term."""
    rng = np.random.default_rng(111)
    p = 20
    for _ in range(5):
        x = complex(*rng.uniform(-1, 1, 2))
        c = x + 3.0 * np.exp(2j * np.pi * rng.random())
        q = complex(*rng.uniform(-1, 1, 2))
        a = np.zeros(p + 1, complex)
        a[0] = q
        ref = O.m2l(p, x, c, a)
        got = O.p2l(p, c, np.array([[x.real, x.imag]]), np.array([q]))
        assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_p2l_is_linear_and_matches_sum_of_singles():
    rng = np.random.default_rng(112)
    p = 12
    c = 0.1j
    xy = np.stack([2 + rng.random(9), rng.random(9)], 1)
    q = crandn(rng, 9)
    tot = O.p2l(p, c, xy, q)
    acc = sum(O.p2l(p, c, xy[i:i + 1], q[i:i + 1]) for i in range(9))
    assert np.max(np.abs(tot - acc)) <= 1e-14 * np.max(np.abs(tot))


def _shortcut_case(n=8000, seed=13, leaf=30):
    src, q, _ = W.problem("clusters", n, seed)
    L = O.levels_cap(n, leaf)
    tree = O.build_tree(src, L)
    li = O.connect(tree)
    sc = O.leaf_shortcut(tree, li)
    return src, q, tree, li, sc


def test_leaf_shortcut_partitions_strong_lists():
    """Every leaf's strong list splits into near, P2L and M2P with nothing lost
    or repeated and its order kept; a pair moves out of near exactly when it
    meets the theta-criterion with the two radii interchanged,
    r + theta R <= theta d with r > 0, and goes to P2L when the source box is
    the larger."""
    src, q, tree, li, sc = _shortcut_case()
    L = tree.L
    base = O.n_boxes(L - 1)
    theta = 0.5
    moved = 0
    for b in range(4 ** L):
        g = base + b
        strong = list(li.strong[li.strong_off[g]:li.strong_off[g + 1]])
        near = list(sc.near[sc.near_off[b]:sc.near_off[b + 1]])
        p2l = list(sc.p2l[sc.p2l_off[b]:sc.p2l_off[b + 1]])
        m2p = list(sc.m2p[sc.m2p_off[b]:sc.m2p_off[b + 1]])
        assert sorted(near + p2l + m2p) == sorted(strong)
        for sub in (near, p2l, m2p):  # order of strong(t) kept
            pos = [strong.index(s) for s in sub]
            assert pos == sorted(pos)
        assert g in near
        (ct, rt) = _centre_radius(tree.rect[g])
        for s in strong:
            (cs, rs) = _centre_radius(tree.rect[s])
            d = math.hypot(ct[0] - cs[0], ct[1] - cs[1])
            swapped = (s != g and min(rt, rs) > 0
                       and (min(rt, rs) + theta * max(rt, rs)) <= theta * d)
            if s in near:
                assert not swapped
            else:
                assert swapped
                assert (s in p2l) == (rs > rt)
                moved += 1
    assert moved > 0 and sc.p2l_off[-1] > 0 and sc.m2p_off[-1] > 0


def test_fmm_with_shortcut_converges_to_branch_sum():
    """With P2L / M2P the FMM still converges to the branch-consistent direct
    sum (which takes each shortcut pair on its own expansion's branch), the
    error decays with p, and dropping the shortcut changes the result only at
    the truncation level."""
    src, q, tree, li, sc = _shortcut_case(4000, 17, 20)
    ref = O.direct_branch(tree, li, src, q, shortcut=sc)
    errs = []
    for p in (6, 12, 24):
        phi = O.evaluate(tree, li, src, q, p, shortcut=sc)
        errs.append(O.normwise_error(phi, ref))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10 and errs[2] < 1e-9, errs
    plain = O.evaluate(tree, li, src, q, 24)
    assert O.normwise_error(plain, O.direct_branch(tree, li, src, q)) < 1e-9
    # real strengths: both agree with the plain direct sum in the real part
    qr = q.real + 0j
    phi = O.evaluate(tree, li, src, qr, 24, shortcut=sc)
    d = O.direct(src, qr)
    assert np.max(np.abs(phi.real - d.real)) <= 1e-9 * np.max(np.abs(d.real))


def test_shortcut_branch_sum_differs_by_2pi_multiples():
    rng = np.random.default_rng(121)
    src, _, tree, li, sc = _shortcut_case(3000, 19, 16)
    q = rng.choice([-1.0, 1.0], len(src)) + 0j
    bc = O.direct_branch(tree, li, src, q, shortcut=sc)
    pr = O.direct(src, q)
    assert np.allclose(bc.real, pr.real, rtol=0, atol=1e-10)
    k = (bc.imag - pr.imag) / (2 * np.pi)
    assert np.allclose(k, np.round(k), atol=1e-8)


def test_shortcut_separate_targets_and_sample():
    src, q, tgt = W.problem("clusters", 4000, 71, tgt_dist="uniform", m=2500)
    phi, tree, li, sc = O.fmm(src, q, p=24, leaf=32, tgt=tgt, p2l_m2p=True)
    ref = O.direct_branch(tree, li, src, q, tgt, shortcut=sc)
    assert O.normwise_error(phi, ref) < 1e-9
    samp = np.array([0, 7, 100, 2499])
    assert np.array_equal(O.evaluate(tree, li, src, q, 24, tgt, sample=samp, shortcut=sc), phi[samp])


def test_shortcut_zero_radius_box():
    """Leaves whose points all coincide have radius 0 and touch the corner of
    a neighbour holding more copies of the same point: such pairs stay in the
    near list (r > 0 is required), so coincident points are still skipped and
    the FMM converges to the branch-consistent direct sum."""
    rng = np.random.default_rng(131)
    src = rng.random((3000, 2))
    src[:200] = src[0]  # a cluster of identical points: zero-radius leaves
    q = crandn(rng, 3000)
    L = O.levels_cap(3000, 16)
    tree = O.build_tree(src, L)
    li = O.connect(tree)
    sc = O.leaf_shortcut(tree, li)
    base = O.n_boxes(L - 1)
    radii = np.array([_centre_radius(r)[1] for r in tree.rect])
    zero = [b for b in range(4 ** L) if radii[base + b] == 0.0 and tree.box_src[base + b, 1] > 0]
    assert zero
    for b in zero:
        g = base + b
        for s in np.concatenate([sc.p2l[sc.p2l_off[b]:sc.p2l_off[b + 1]],
                                 sc.m2p[sc.m2p_off[b]:sc.m2p_off[b + 1]]]):
            raise AssertionError(f"zero-radius leaf {g} in a shortcut pair with {s}")
    ref = O.direct_branch(tree, li, src, q, shortcut=sc)
    phi = O.evaluate(tree, li, src, q, 24, shortcut=sc)
    assert np.all(np.isfinite(phi))
    assert O.normwise_error(phi, ref) < 1e-9


# --------------------------------------------------------------- shrink-wrapped boxes

@pytest.mark.parametrize("separate", [False, True])
def test_tight_rects_are_the_bounding_rectangles(separate):
    """Every point lies in its box's tight rectangle, every side is attained by
    a point, the tight rectangle lies in the split rectangle and in the
    parent's tight rectangle; boxes without points keep the split rectangle."""
    if separate:
        src, q, tgt = W.problem("clusters", 3000, 141, tgt_dist="uniform", m=1500)
    else:
        src, q, tgt = W.problem("curve", 3000, 141)
    L = O.levels_cap(3000, 16)
    tree = O.build_tree(src, L, tgt)
    tr = O.tight_rects(tree, src, tgt)
    pts_s = src[tree.perm]
    pts_t = (tgt[tree.tperm] if tgt is not None else None)
    for g in range(tree.n_boxes):
        pts = [pts_s[tree.box_src[g, 0]:tree.box_src[g, 0] + tree.box_src[g, 1]]]
        if tgt is not None:
            pts.append(pts_t[tree.box_tgt[g, 0]:tree.box_tgt[g, 0] + tree.box_tgt[g, 1]])
        pts = np.concatenate(pts)
        r = tr[g]
        if len(pts) == 0:
            assert np.array_equal(r, tree.rect[g])
            continue
        assert r[0] == pts[:, 0].min() and r[1] == pts[:, 0].max()
        assert r[2] == pts[:, 1].min() and r[3] == pts[:, 1].max()
        R = tree.rect[g]
        assert R[0] <= r[0] <= r[1] <= R[1] and R[2] <= r[2] <= r[3] <= R[3]
    for l in range(1, L + 1):
        for b in range(4 ** l):
            g = O.n_boxes(l - 1) + b
            par = O.n_boxes(l - 2) + b // 4 if l > 1 else 0
            if tree.box_src[g, 1] + (tree.box_tgt[g, 1] if tgt is not None else 0) == 0:
                continue
            P, r = tr[par], tr[g]
            assert P[0] <= r[0] and r[1] <= P[1] and P[2] <= r[2] and r[3] <= P[3]


def test_tight_lists_cover_every_leaf_pair_exactly_once():
    src, q, _ = W.problem("curve", 8000, 143)
    L = O.levels_cap(8000, 30)
    tree = O.shrink(O.build_tree(src, L), src)
    li = O.connect(tree)
    base = O.n_boxes(L - 1)
    nleaf = 4 ** L
    cover = np.zeros((nleaf, nleaf), np.int32)
    lvl_of = np.zeros(tree.n_boxes, np.int64)
    for l in range(L + 1):
        lvl_of[(O.n_boxes(l - 1) if l else 0):O.n_boxes(l)] = l
    for g in range(tree.n_boxes):
        l = lvl_of[g]
        b = g - (O.n_boxes(l - 1) if l else 0)
        span = 4 ** (L - l)
        for s in li.weak[li.weak_off[g]:li.weak_off[g + 1]]:
            sb = s - (O.n_boxes(l - 1) if l else 0)
            cover[b * span:(b + 1) * span, sb * span:(sb + 1) * span] += 1
            assert O.well_separated(tree.rect[g], tree.rect[s])
    for b in range(nleaf):
        g = base + b
        for s in li.strong[li.strong_off[g]:li.strong_off[g + 1]]:
            cover[b, s - base] += 1
    assert np.all(cover == 1)


@pytest.mark.parametrize("shortcut", [False, True])
def test_fmm_tight_boxes_converge(shortcut):
    """Shrink-wrapped geometry: the FMM converges to the branch-consistent
    direct sum (error falling with p), the real part to the plain direct sum,
    and on a curve it needs far fewer near pairs than the split rectangles."""
    src, q, _ = W.problem("curve", 6000, 145)
    L = O.levels_cap(6000, 24)
    tree0 = O.build_tree(src, L)
    tree = O.shrink(tree0, src)
    li = O.connect(tree)
    sc = O.leaf_shortcut(tree, li) if shortcut else None
    ref = O.direct_branch(tree, li, src, q, shortcut=sc)
    errs = [O.normwise_error(O.evaluate(tree, li, src, q, p, shortcut=sc), ref) for p in (6, 12, 24)]
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10 and errs[2] < 1e-9, errs
    qr = q.real + 0j  # real strengths: the real part has no branch
    d = O.direct(src, qr)
    phi = O.evaluate(tree, li, src, qr, 24, shortcut=sc)
    assert np.max(np.abs(phi.real - d.real)) <= 1e-9 * np.max(np.abs(d.real))
    near = lambda lists: np.diff(lists.strong_off)[O.n_boxes(L - 1):].sum()
    assert near(li) < 0.6 * near(O.connect(tree0))


# --------------------------------------------------------------- harmonic kernel (Sec. 5)

@pytest.mark.parametrize("n", [3, 7, 16])
def test_harmonic_direct_roots_of_unity(n):
    """Unit strengths at the n-th roots of unity: sum_j 1/(w^j - y)
    = -n y^(n-1) / (y^n - 1) (the log-derivative of y^n - 1), and 0 at y = 0."""
    w = np.exp(2j * np.pi * np.arange(n) / n)
    src = np.stack([w.real, w.imag], 1)
    q = np.ones(n) + 0j
    ys = np.array([0.3 + 0.2j, -1.7 + 0.4j, 2.5 - 3.0j, 0.0j])
    tgt = np.stack([ys.real, ys.imag], 1)
    got = O.direct_harmonic(src, q, tgt)
    ref = -n * ys ** (n - 1) / (ys ** n - 1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_harmonic_direct_is_minus_derivative_of_log_sum():
    """Central differences of the log direct sum along x (away from any branch
    cut: all points to the left of the sources' convex hull's far side) give
    -u up to O(h^2)."""
    rng = np.random.default_rng(151)
    src = rng.random((40, 2))
    q = crandn(rng, 40)
    y = np.array([[2.0, 0.37], [1.6, 0.81]])  # to the right of every source
    h = 1e-5
    d = (O.direct(src, q, y + [h, 0]) - O.direct(src, q, y - [h, 0])) / (2 * h)
    u = O.direct_harmonic(src, q, y)
    assert np.max(np.abs(d + u)) <= 1e-7 * np.max(np.abs(u))


def test_l2p_and_m2p_derivatives():
    """l2p_deriv is the derivative of a known polynomial; m2p_deriv of a
    single source's multipole approaches -1 / (x - z) = 1/(z - x) within the
    series' tail bound."""
    p = 3
    b = np.array([1.0, 2.0 - 1j, 0.5j, -3.0])
    c, z = 0.5 + 0.5j, 1.25 - 0.5j
    w = z - c
    assert abs(O.l2p_deriv(p, c, b, z) - (b[1] + 2 * b[2] * w + 3 * b[3] * w ** 2)) < 1e-14
    rng = np.random.default_rng(153)
    for p in (6, 14, 28):
        c = 0.1 - 0.2j
        for _ in range(10):
            s = 0.3 * rng.random() * np.exp(2j * np.pi * rng.random())
            z = c + np.exp(2j * np.pi * rng.random())
            qv = complex(*rng.uniform(-1, 1, 2))
            a = O.p2m(p, c, np.array([[(c + s).real, (c + s).imag]]), np.array([qv]))
            exact = qv / (z - (c + s))  # d/dz q log(z - x)
            r = abs(s) / abs(z - c)
            bound = abs(qv) * r ** (p + 1) / (abs(z - c) * (1 - r)) * (p + 2)
            assert abs(O.m2p_deriv(p, c, a, z) - exact) <= bound + 1e-14 * abs(exact)


@pytest.mark.parametrize("variant", ["plain", "shortcut", "box_fit"])
def test_harmonic_fmm_converges_to_direct(variant):
    """The harmonic FMM (same tree, lists and expansions, differentiated) has
    no branch: it converges to the plain direct sum, the error falling with p;
    N <= leaf is the direct sum bit for bit."""
    src, q, tgt = W.problem("clusters", 4000, 155, tgt_dist="uniform", m=1500) \
        if variant == "plain" else W.problem("curve", 4000, 157)
    ref = O.direct_harmonic(src, q, tgt)
    errs = []
    for p in (6, 12, 24):
        phi = O.fmm(src, q, p=p, leaf=24, tgt=tgt, kernel=1, p2l_m2p=(variant == "shortcut"),
                    box_fit=(variant == "box_fit"))[0]
        errs.append(O.normwise_error(phi, ref))
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10 and errs[2] < 1e-9, errs
    small, _, _ = W.problem("uniform", 30, 159)
    qs = crandn(np.random.default_rng(1), 30)
    phi, tree, _ = O.fmm(small, qs, p=10, leaf=40, kernel=1)
    assert tree.L == 0 and np.array_equal(phi, O.direct_harmonic(small, qs))


@pytest.mark.parametrize("shortcut", [False, True])
def test_fmm_thread_count_changes_nothing(shortcut):
    """The per-target loops that may run on several threads (M2L per target
    box, L2P + P2P per evaluation point) keep every sum's order, so the FMM is
    bit-identical with 1 and 4 threads."""
    src, q, _ = W.problem("clusters", 6000, 4321)
    outs = []
    for th in (1, 4):
        O.set_threads(th)
        try:
            outs.append(O.fmm(src, q, p=14, leaf=20, p2l_m2p=shortcut)[0])
        finally:
            O.set_threads(1)
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
