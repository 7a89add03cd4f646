"""M2L on the tensor cores (tcgen05, exact fp16 digit slices, FP32 TMEM
accumulation, one GEMM row per weak pair) in the mixed path, against the CPU
oracle.

With s digit slices the operator and the pair data carry 8 + 9(s-1) bits, so
the error falls by ~2^-9 per slice until the double-float floor; s = 5 (the
default) meets the same 1e-11 bound as the double-float sweeps.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1205_4611_gb300 as G  # noqa: E402

from test_gpu_parity import check_topology, gpu_fmm  # noqa: E402

MIXED = G.FMM_PREC_MIXED


@pytest.mark.parametrize("p", [5, 12, 20, 24, 31])
def test_tensor_m2l_vs_oracle(p):
    src, q, _ = W.problem("clusters", 12_000, 800 + p)
    phi_o, otree, olists = O.fmm(src, q, p=p, leaf=24)
    phi_g, tree = gpu_fmm(src, q, p, 24, precision=MIXED, m2l_slices=0)
    check_topology(tree, otree, olists)
    assert O.normwise_error(phi_g, phi_o) <= 1e-11


def test_tensor_m2l_error_falls_with_slices():
    src, q, _ = W.problem("uniform", 8_000, 811)
    phi_o, _, _ = O.fmm(src, q, p=20, leaf=16)
    errs = []
    for s in (1, 2, 3, 4, 5):
        phi_g, _ = gpu_fmm(src, q, 20, 16, precision=MIXED, m2l_slices=s)
        errs.append(O.normwise_error(phi_g, phi_o))
    assert errs[-1] <= 1e-11
    for a, b in zip(errs[:3], errs[1:4]):
        assert b < a / 64, errs


def test_tensor_m2l_matches_sweeps():
    src, q, tgt = W.problem("curve", 10_000, 812, tgt_dist="uniform", m=6000)
    sw, _ = gpu_fmm(src, q, 24, 30, tgt=tgt, precision=MIXED, m2l_slices=-1)
    tc, _ = gpu_fmm(src, q, 24, 30, tgt=tgt, precision=MIXED, m2l_slices=0)
    assert O.normwise_error(tc, sw) <= 1e-12


def test_tensor_m2l_batched():
    from test_gpu_batched import make_batch, run_batched
    inst, off, src, q = make_batch(16, 813)
    opt = G.fmm_default_options(p=18, leaf_size=24, precision=MIXED, m2l_slices=0)
    phi_b, _ = run_batched(off, src, q, opt)
    for i, (_, s, qi) in enumerate(inst):
        ref, _, _ = O.fmm(s, qi, p=18, leaf=24)
        assert O.normwise_error(phi_b[off[i]:off[i + 1]], ref) <= 1e-11, i


@pytest.mark.parametrize("box_fit", [0, 1])
def test_tensor_m2l_point_like_boxes(box_fit):
    """Leaves of one point (and, with shrink-wrapped geometry, of radius 0)
    far apart: the pair scaling keeps |D / 2^e0|^2 in the float range and the
    potentials stay finite and match the oracle."""
    src, q, _ = W.problem("uniform", 3000, 815)
    src[100:130] = src[99]  # a box whose points coincide
    phi_o = O.fmm(src, q, p=16, leaf=1, box_fit=bool(box_fit))[0]
    opt = G.fmm_default_options(p=16, leaf_size=1, precision=MIXED, box_fit=box_fit)
    tree = G.fmm_build_tree(torch.from_numpy(src).cuda(), None, opt)
    phi = torch.empty((3000, 2), dtype=torch.float64, device="cuda")
    G.fmm_evaluate(tree, torch.from_numpy(q).cuda(), phi)
    G.fmm_tree_sync(tree)
    tree.free()
    got = phi.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert O.normwise_error(got[:, 0] + 1j * got[:, 1], phi_o) <= 1e-11
