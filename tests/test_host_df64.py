"""The double-float arithmetic of the stage-5 kernels (``csrc/df64.cuh``), built for the host and
checked against long double: Tang's exponential over the kernels' argument range, the exact head
difference of grid-form coordinates, the fused sum of three squares, and the square root from an
approximate reciprocal-square-root seed.  The kernels run the
same header on the GPU; the GPU parity tests check the whole product."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2011_13861_gb300", "csrc")


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("df64") / "df64_host_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "df64_host_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_exponential_is_double_float_accurate(report):
    # 48-bit arithmetic on arguments up to 44: a few units of 2^-48 relative
    assert report["exp_rel"] < 3e-14
    assert report["exp_abs"] < 1e-14
    assert report["exp_unnormalised"] == 0


def test_grid_form_heads_subtract_exactly(report):
    assert report["inexact_heads"] == 0
    # two float tails of at most q/2 = 2^-21: the difference rounds at 2^-45 at worst
    assert report["diff_abs"] <= 2.0 ** -44


def test_sum_of_three_squares(report):
    assert report["sum_sq_rel"] < 5e-14


def test_square_root_from_an_approximate_seed(report):
    # one float Newton step leaves the seed good to about 2^-22.4 (its own roundings); the
    # double-float Heron correction is about 2^-22 of the root and carries that relative error,
    # so the root is good to about 2^-44.5 (4e-14), not to the 2^-48 of the representation
    assert report["sqrt_rel"] < 6e-14


def test_float64_split_by_bit_operations(report):
    # head: x truncated to 24 significant bits; head + tail within 2^-47 of x for magnitudes from
    # 2^-72 to 2^127 (below and above, the float conversion)
    assert report["split_head_wrong"] == 0
    assert report["split_rel"] <= 2.0 ** -47
    assert report["split_edges_ok"] == 1
