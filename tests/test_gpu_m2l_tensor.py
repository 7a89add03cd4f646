"""M2L on the tensor cores (tcgen05, exact bf16 digit slices, FP32 TMEM
accumulation) in the mixed path, against the CPU oracle.

With s digit slices the operator and the pair data carry 7 + 8(s-1) bits, so
the error falls by ~2^-8 per slice until the double-float floor; s = 6 meets
the same 1e-11 bound as the double-float sweeps.
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
    phi_g, tree = gpu_fmm(src, q, p, 24, precision=MIXED, m2l_slices=6)
    check_topology(tree, otree, olists)
    assert O.normwise_error(phi_g, phi_o) <= 1e-11


def test_tensor_m2l_error_falls_with_slices():
    src, q, _ = W.problem("uniform", 8_000, 811)
    phi_o, _, _ = O.fmm(src, q, p=20, leaf=16)
    errs = []
    for s in (1, 2, 3, 4, 6):
        phi_g, _ = gpu_fmm(src, q, 20, 16, precision=MIXED, m2l_slices=s)
        errs.append(O.normwise_error(phi_g, phi_o))
    assert errs[-1] <= 1e-11
    for a, b in zip(errs[:3], errs[1:4]):
        assert b < a / 16, errs


def test_tensor_m2l_matches_sweeps():
    src, q, tgt = W.problem("curve", 10_000, 812, tgt_dist="uniform", m=6000)
    sw, _ = gpu_fmm(src, q, 24, 30, tgt=tgt, precision=MIXED, m2l_slices=-1)
    tc, _ = gpu_fmm(src, q, 24, 30, tgt=tgt, precision=MIXED, m2l_slices=6)
    assert O.normwise_error(tc, sw) <= 1e-12


def test_tensor_m2l_batched():
    from test_gpu_batched import make_batch, run_batched
    inst, off, src, q = make_batch(16, 813)
    opt = G.fmm_default_options(p=18, leaf_size=24, precision=MIXED, m2l_slices=6)
    phi_b, _ = run_batched(off, src, q, opt)
    for i, (_, s, qi) in enumerate(inst):
        ref, _, _ = O.fmm(s, qi, p=18, leaf=24)
        assert O.normwise_error(phi_b[off[i]:off[i + 1]], ref) <= 1e-11, i
