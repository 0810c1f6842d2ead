"""The C-ABI library builds, loads and exports every entry point include/kl.h declares.

No CUDA call is made: loading the shared object does not need a GPU.
"""
import ctypes
import os
import re

from paper_2011_13861_gb300 import _binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "kl.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kl_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("kl_create", "kl_apply", "kl_eigs", "kl_destroy", "kl_last_error", "kl_covmv"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for every entry point of the header
    assert sorted(_binding.SIGNATURES) == declared_entry_points()


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2011_13861_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_build_tracks_every_header():
    # libkl.so is stale when any source or header changes, including the .cuh arithmetic headers
    deps = set(build.dependencies())
    for d in (os.path.join(ROOT, "paper_2011_13861_gb300", "csrc"), os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cpp", ".h", ".cuh")):
                assert os.path.join(d, f) in deps, f
