"""The float64 stage-5 kernel's own exponential and square root (``csrc/fp64_math.cuh``), built
for the host and checked against long double.  The device runs the same code; only the square
root's seed differs (an approximate reciprocal square root there, a perturbed exact one here)."""
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
    exe = str(tmp_path_factory.mktemp("fp64") / "fp64_host_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "fp64_host_check.cpp"),
                    "-o", exe], check=True)
    return json.loads(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)


def test_exponential_relative_error(report):
    # Tang's method with 1024 subintervals and a degree-3 polynomial: a few ulp down to -37,
    # also when the index comes from a float copy of the argument that is off by 1e-6
    assert report["exp_rel"] < 5e-15
    assert report["exp_rel_float_index"] < 5e-15


def test_exponential_tail(report):
    # below -37 the values are under 1e-16 of the diagonal; absolute error tiny, 0 below -700
    assert report["exp_abs_tail"] < 1e-29
    assert report["exp_not_zero_below_700"] == 0


def test_square_root(report):
    # the float64 Heron correction carries the refined seed's error squared
    assert report["sqrt_rel"] < 1.2e-14
    assert report["sqrt_float_rel"] < 2e-7
