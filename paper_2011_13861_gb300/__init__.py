"""GB300-native matrix-free isogeometric Karhunen-Loeve operator and eigensolver.

Thin Python binding over the C ABI declared in ``include/kl.h`` (library ``libkl.so``
built in-tree by :mod:`paper_2011_13861_gb300.build`).  The binding only marshals
arguments: device memory and streams come from PyTorch tensors, every compute step runs
in the library's CUDA kernels, and there is no CPU fallback -- loading fails loudly when
the library is missing.
"""
from ._binding import (  # noqa: F401
    KL_GEOM_BOX, KL_GEOM_NURBS, KL_K_EXP, KL_K_GAUSS, KL_K_EXP_SEPARABLE, KL_K_POLY_TEST, KL_P_FP64, KL_P_FP32, KL_P_DF64, KL_P_TC32, KL_P_TC64,
    KLError, KLProblem, load, library_path, exported_symbols, KERNEL_KINDS, kernel_launches,
    apply_batched, eigs_batched, MLP, prolong, wait_selftest, df2_selftest, pipe_rates, set_sym_slot_limit, set_tc_symmetric, direction_factors, mapped_points, prolongation_factor, STATUS,
)
