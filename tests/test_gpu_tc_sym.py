"""The symmetric tensor-core float64-class stage 5 (each kernel value used for both (k, l) and
(l, k); column sums read the same bfloat16 value slices transposed; an option, off by default
because it measured slower than the full evaluation) against the oracle and against the
full-evaluation schedule.

Sizes span one to many 128-point row blocks, ragged tails, a size that is a multiple of 128,
all four kernel kinds (the polynomial test kernel exercises the value scaling) and 1 to 33
vectors (two vector groups).  The bar is the float64 matvec bar, 1e-12 relative to the largest
output; the two schedules differ only in the order of additions (and the column sums' atomic
additions), far below it.
"""
import numpy as np
import pytest

from oracle import ibq
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12

CASES = [
    # dim, p, ne, kernel, L ; Greville points
    (1, 2, 298, "exp", 0.3),            # 300 points: 3 row blocks
    (2, [2, 3], [23, 17], "gauss", 0.4),  # 500 points, ragged
    (2, 2, 32, "exp_sep", 0.8),         # 1,156 points
    (3, 3, 13, "gauss", 0.3),           # 4,096 points: a multiple of 128
    (3, 2, 15, "exp", 0.5),             # 4,913 points
    (3, 2, [4, 5, 3], "poly", 2),       # 336 points, polynomial test kernel
]


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%s" % (c[0], c[3]))
@pytest.mark.parametrize("nvec", [1, 5, 32, 33])
def test_symmetric_tc64_matches_oracle_and_full_schedule(kl, case, nvec):
    import torch
    dim, p, ne, kern, L = case
    lo, hi = ([0.0] * dim, [1.5, 1.0, 2.0][:dim]) if kern == "poly" else (None, None)
    P = ibq.Problem(dim, p, ne, kernel=kern, L=L, sigma=1.2, lo=lo, hi=hi)
    G = kl.KLProblem(dim, p, ne, kernel=kern, L=L, sigma=1.2, lo=lo, hi=hi)
    X, _ = P.points_and_J()
    u = inputs.random_block(P.Nt, nvec, seed=60 + nvec)
    ud = torch.from_numpy(u.T.copy()).cuda()
    kl.set_tc_symmetric(True)
    try:
        zs = G.covmv(ud, precision=kl.KL_P_TC64)
    finally:
        kl.set_tc_symmetric(False)
    zf = G.covmv(ud, precision=kl.KL_P_TC64)
    ref = P.stage5(X, u)
    assert rel(zs.cpu().numpy().T, ref) < FP64_TOL
    assert rel(zf.cpu().numpy().T, ref) < FP64_TOL
    assert float((zs - zf).abs().max() / zf.abs().max()) < 1e-13


def test_symmetric_tc64_vector_spanning_many_scales(kl):
    """A right-hand side whose entries span e^25 (the per-vector scale and six u digits) and a
    zero vector, through the symmetric schedule."""
    import torch
    P = ibq.Problem(3, 2, [9, 10, 11], kernel="exp", L=0.5)
    G = kl.KLProblem(3, 2, [9, 10, 11], kernel="exp", L=0.5)
    X, _ = P.points_and_J()
    rng = np.random.default_rng(17)
    u = np.stack([rng.uniform(-1, 1, P.Nt) * np.exp(rng.uniform(-25, 0, P.Nt)), np.zeros(P.Nt)], axis=1)
    kl.set_tc_symmetric(True)
    try:
        z = G.covmv(torch.from_numpy(u.T.copy()).cuda(), precision=kl.KL_P_TC64).cpu().numpy().T
    finally:
        kl.set_tc_symmetric(False)
    ref = P.stage5(X, u)
    assert rel(z[:, 0], ref[:, 0]) < FP64_TOL
    assert np.all(z[:, 1] == 0.0)
