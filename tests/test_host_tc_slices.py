"""The exact slicing of the tensor-core stage 5 (``csrc/tc_slices.cuh``, the code the kernels
run), built for the host: bfloat16-exact slices with bounded digits, level sums over a
128-column drain block that are exact in float32 for the four leading levels, and the drained
double-float row sums against long double for both precision classes."""
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
    exe = str(tmp_path_factory.mktemp("tcs") / "tc_slices_host_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-Wno-unknown-pragmas", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "tc_slices_host_check.cpp"), "-o", exe], check=True)
    return json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)


def test_slices_are_bfloat16_with_bounded_digits(report):
    assert report["not_bf16"] == 0
    assert report["big_digits"] == 0
    # six 8-bit digits keep about 48 bits: the dropped remainder and the tail's rounding
    assert report["slice_remainder"] < 2.0 ** -47


def test_leading_levels_are_exact_in_float32(report):
    assert report["inexact_levels"] == 0


def test_row_sums_reach_their_precision_class(report):
    # relative to sum |g u| over 2048 columns drained every 128
    assert report["rel_err_float64_class"] < 2e-14
    assert report["rel_err_float32_class"] < 3e-7
