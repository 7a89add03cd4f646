"""The p-study of the paper's Sec. 5 (Fig. "pspeedup") as sweeps.py runs it,
at N = 2e4, checked against the oracle: its reference sum and its reported
errors agree with the oracle's FP64 direct sum of the harmonic kernel, and
the error falls with p as the truncation bound says."""
import argparse

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import sweeps  # noqa: E402


def test_p_study_errors_against_the_oracle():
    torch_, G = sweeps.setup()
    args = argparse.Namespace(precision=["mixed", "fp64"], p_list=[5, 9, 13, 17], n_list=None)
    seen = {}

    def oracle_ref(src, q, sample):
        ref = O.direct_harmonic(src, q, sample=sample)
        own = sweeps.direct_harmonic_sample(torch_, src, q, sample)
        assert O.normwise_error(own, ref) <= 1e-13  # the script's own reference sum
        seen["src"], seen["q"], seen["sample"], seen["ref"] = src, q, sample, ref
        return ref

    rows = sweeps.study_p(torch_, G, args, n=20_000, n_sample=256, reference=oracle_ref)
    assert len(rows) == 8
    for prec in ("mixed", "fp64"):
        errs = [r["error"] for r in rows if r["precision"] == prec]
        assert all(b < a for a, b in zip(errs, errs[1:])), errs
        assert errs[-1] < 1e-6  # p = 17: the paper's TOL ~ 1e-6 (Sec. 5.1)
        assert errs[0] > 1e-4   # p = 5 is far from it
