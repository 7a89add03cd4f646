"""Mixed-precision path (double-float near field) against the CPU oracle.

The near field runs in df32 (about 48 significant bits per pair), so the
potentials are not bit-comparable with the FP64 oracle; the bound used here
is 1e-11 normwise against the oracle FMM (each pair's log is accurate to
~2^-42 absolute, see df32.cuh), which leaves room under the 1e-10 target for
the truncation error.  Topology is the same as in FP64 mode: bit-exact.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

from test_gpu_parity import as_complex, check_topology, dev, gpu_fmm  # noqa: E402

TOL_MIXED = 1e-11

CASES = [
    ("uniform_1e4", "uniform", 10_000, 20, 40, False, None, 0),
    ("clusters_2e4", "clusters", 20_000, 24, 32, False, None, 0),
    ("curve_8e3_real", "curve", 8_000, 24, 30, True, None, 0),
    ("clusters_targets", "clusters", 6_000, 20, 25, False, "uniform", 4_500),
    ("ragged_4099", "uniform", 4_099, 12, 7, False, None, 0),
]


@pytest.mark.parametrize("m2l", [0, -1], ids=["m2l_tensor", "m2l_sweeps"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_mixed_vs_oracle_fmm(case, m2l):
    name, dist, n, p, leaf, real_q, tgt_dist, m = case
    src, q, tgt = W.problem(dist, n, W.BASE_SEED + 100 + n, real_q=real_q, tgt_dist=tgt_dist, m=m)
    phi_o, otree, olists = O.fmm(src, q, p=p, leaf=leaf, tgt=tgt)
    phi_g, tree = gpu_fmm(src, q, p, leaf, tgt=tgt, precision=G.FMM_PREC_MIXED, m2l_slices=m2l)
    check_topology(tree, otree, olists)
    err = O.normwise_error(phi_g, phi_o)
    assert err <= TOL_MIXED, err


def test_symmetric_near_field_matches_per_point_pass():
    """p2p_mode 0 (each pair of distinct leaves' points once, reverse term by
    Log(-z) = Log(z) +- i pi) against p2p_mode 1 (one pass per point), with
    shared ordinates and exact duplicates across leaves, and with leaves of
    exactly 64 points."""
    rng = np.random.default_rng(17)
    src = rng.random((4096, 2))
    src[100:160] = src[7]                      # duplicates spread over leaves
    src[1000:1400, 1] = np.round(src[1000:1400, 1] * 8) / 8  # shared ordinates
    q = W.complex_strengths(4096, rng)
    out = []
    for mode in (0, 1):
        opt = G.fmm_default_options(p=20, leaf_size=64, precision=G.FMM_PREC_MIXED,
                                    p2p_mode=mode)
        tree = G.fmm_build_tree(dev(src), None, opt)
        phi = torch.empty((4096, 2), dtype=torch.float64, device="cuda")
        G.fmm_evaluate(tree, dev(q), phi)
        G.fmm_tree_sync(tree)
        out.append(as_complex(phi.cpu().numpy()))
    assert G.fmm_tree_info(tree)["levels"] == 3  # 64 leaves of exactly 64 points
    # the two passes round differently (the reverse term is formed in the other
    # leaf's frame): both carry double-float rounding, ~2^-44 per pair
    assert O.normwise_error(out[0], out[1]) <= 2e-12
    phi_o, _, _ = O.fmm(src, q, p=20, leaf=64)
    assert O.normwise_error(out[0], phi_o) <= TOL_MIXED


def test_mixed_single_leaf_direct_sum():
    """L = 0: the mixed path is the df32 direct sum; against the FP64 sum.

    Each pair log is within 2^-42 absolute per component (df32.cuh), so point
    i is off by at most sum_j |q_j| (2^-41 + 2^-46 |Log z_ij|) (the log plus
    the df32 product and sum roundings).  With independent errors at the
    measured ~2^-44 the normwise error is the root-sum-square of the terms,
    1.1e-13 on these 60 points; 3e-13 leaves room for the spread of so few.
    """
    src, q, _ = W.problem("clusters", 60, 11)
    phi_g, tree = gpu_fmm(src, q, 8, 64, precision=G.FMM_PREC_MIXED)
    assert G.fmm_tree_info(tree)["levels"] == 0
    ref = O.direct(src, q)
    z = src[:, 0] + 1j * src[:, 1]
    d = z[:, None] - z[None, :]
    np.fill_diagonal(d, 1.0)
    qa = np.abs(q[:, 0] + 1j * q[:, 1])
    off = ~np.eye(len(z), dtype=bool)
    bound = (off * qa[None, :] * (2.0 ** -41 + 2.0 ** -46 * np.abs(np.log(d)))).sum(1)
    assert np.all(np.abs(phi_g - ref) <= bound)
    assert O.normwise_error(phi_g, ref) < 3e-13


@pytest.mark.parametrize("kind", ["duplicates", "grid", "all_same"])
def test_mixed_shared_coordinates_and_duplicates(kind):
    """Exactly shared ordinates must land on the same side of the log's branch
    cut as in FP64 (+0, arg = +pi) and exact duplicates must be skipped, also
    when the two points sit in different leaves."""
    rng = np.random.default_rng(3)
    if kind == "duplicates":
        src = rng.random((3000, 2))
        src[100:400] = src[5]
        src[500:900, 1] = 0.25
    elif kind == "grid":
        g = np.arange(40) / 40.0
        src = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)
    else:
        src = np.tile([[0.3, 0.7]], (200, 1))
    q = W.complex_strengths(src.shape[0], rng)
    phi_o, otree, olists = O.fmm(src, q, p=20, leaf=16)
    phi_g, tree = gpu_fmm(src, q, 20, 16, precision=G.FMM_PREC_MIXED)
    check_topology(tree, otree, olists)
    scale = max(np.max(np.abs(phi_o)), 1e-300)
    assert np.max(np.abs(phi_g - phi_o)) <= TOL_MIXED * scale


def test_mixed_full_size_clusters_1e6_sampled():
    src, q, _ = W.make("clusters_1e6")
    L = O.levels_cap(len(src), 64)
    otree = O.build_tree(src, L)
    olists = O.connect(otree)
    phi_g, tree = gpu_fmm(src, q, 24, 64, precision=G.FMM_PREC_MIXED)
    sample = np.random.default_rng(1).choice(len(src), 512, replace=False)
    ref = O.evaluate(otree, olists, src, q, 24, sample=sample)
    assert O.normwise_error(phi_g[sample], ref) <= TOL_MIXED
    ref_d = O.direct_branch(otree, olists, src, q, sample=sample[:32])
    assert O.normwise_error(phi_g[sample[:32]], ref_d) <= 1e-10


@pytest.mark.parametrize("p", [5, 12, 31, 40])
def test_mixed_orders(p):
    """df32 M2L sweeps for every register width (p <= 32) and the FP64 M2L
    that mixed mode uses above that."""
    src, q, _ = W.problem("clusters", 9000, 500 + p)
    phi_o, otree, olists = O.fmm(src, q, p=p, leaf=20)
    phi_g, tree = gpu_fmm(src, q, p, 20, precision=G.FMM_PREC_MIXED)
    assert O.normwise_error(phi_g, phi_o) <= TOL_MIXED
