"""The double-float primitives of the mixed path, built for the host.

`df32.cuh` compiles as plain C++ (its float operations through volatile
temporaries and std::fmaf, so every step rounds once, as on the GPU; the host
reciprocal is the correctly rounded 1/x where the GPU uses rcp.approx, which
the Newton steps absorb).  `df32_host_check.cpp` measures the maximum errors
against long double on seeded random inputs; the bounds below are the
accuracy the mixed path is built on:

* ln and atan2: absolute error below 2^-42 for arguments of order one (the
  target stated in df32.cuh; the table values carry 2^-48, the reduction is
  exact, the series truncation is below 2^-49, and about six roundings of
  order 2^-48 remain), and below 2^-42 |ln s| for large |ln s|, also with
  the exponent shift of pair units;
* the reciprocal: relative error below 2^-45 (one rounding of the Newton
  residual and one of the correction, each below 2^-47, plus e^2 <= 2^-46);
* a b + c d (df_dot2, df_dot2_lz): below 2^-43 of |a b| + |c d| (six
  roundings of low-order terms below 2^-46 each);
* a p = 24 Horner chain of df_horner_step: below (p + 1) 2^-46 of
  sum_k |b_k| |w|^k.

A dropped correction in the arctangent's reduced argument (its cubic term
formed from an unnormalised pair) measures 2^-39 here and fails the bound.
"""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1205_4611_gb300", "csrc")


@pytest.fixture(scope="module")
def errors(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("df32") / "df32_host_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "df32_host_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe, "200000"], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_log(errors):
    assert errors["log_small_abs"] < 2.0 ** -42
    assert errors["log_rel"] < 2.0 ** -42
    assert errors["log_shift_rel"] < 2.0 ** -42


def test_atan2(errors):
    assert errors["atan_abs"] < 2.0 ** -42


def test_reciprocal(errors):
    assert errors["recip_rel"] < 2.0 ** -45


def test_dot_products(errors):
    assert errors["dot2_rel"] < 2.0 ** -43
    assert errors["dot2_lz_rel"] < 2.0 ** -43


def test_horner_chain(errors):
    assert errors["horner_rel"] < 25 * 2.0 ** -46
