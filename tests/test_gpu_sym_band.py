"""The banded schedule of the symmetric stage-5 kernels (bounded workspace) against the oracle.

kl_set_sym_slot_limit(0) forces the banded schedule at sizes the oracle finishes in seconds:
tile counts T odd and even (the band d = T/2 pairs each tile once), T = 2 and 3 (one launch,
idle CTAs), T large enough for several band launches (T/2 + 1 > 16 bands), ragged tails, and
1 to 8 vectors, for the float64, float32 and double-float kernels.  Each product is compared
element by element with the oracle's stage 5, and with the one-launch (triangular) schedule;
the workspace of the banded schedule is checked to be the fixed 20 slots.
"""
import numpy as np
import pytest

from oracle import ibq
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5

# (dim, p, ne, kernel, L): Greville points 300 (T = 2), 700 (T = 3), 34^2 = 1,156 (T = 5),
# 40^2 = 1,600 (T = 7), 100^2 = 10,000 (T = 40: 21 bands, two band launches), 17^3 = 4,913 (T = 20)
CASES = [
    (1, 2, 298, "exp", 0.3),
    (1, 3, 697, "gauss", 0.2),
    (2, 2, 32, "exp", 0.5),
    (2, 3, 37, "gauss", 0.4),
    (2, 2, 98, "exp", 0.4),
    (3, 2, 15, "gauss", 0.5),
]


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


@pytest.fixture
def band(kl):
    kl.set_sym_slot_limit(0)
    yield
    kl.set_sym_slot_limit(512 << 20)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%d-%s" % (c[0], c[2], c[3]))
@pytest.mark.parametrize("nvec", [1, 3, 4, 8])
def test_band_schedule_matches_oracle(kl, band, case, nvec):
    import torch
    dim, p, ne, kern, L = case
    P = ibq.Problem(dim, p, ne, kernel=kern, L=L, sigma=1.1)
    G = kl.KLProblem(dim, p, ne, kernel=kern, L=L, sigma=1.1)
    X, _ = P.points_and_J()
    u = inputs.random_block(P.Nt, nvec, seed=40 + nvec)
    ref = P.stage5(X, u)
    ud = torch.from_numpy(u.T.copy()).cuda()
    for prec, tol in ((kl.KL_P_FP64, FP64_TOL), (kl.KL_P_DF64, FP64_TOL), (kl.KL_P_FP32, FP32_TOL)):
        z = G.covmv(ud, precision=prec).cpu().numpy().T
        assert rel(z, ref) < tol, (prec, rel(z, ref))


def test_band_and_triangular_schedules_agree(kl):
    """Same products from both schedules up to the order of the additions, including an even
    tile count (T = 8: the band d = 4 pairs each tile once).  Reordering a sum of Ntilde ~ 2,000
    terms moves it by up to about Ntilde 2^-53 times the sum of the terms' magnitudes, a few
    1e-14 of the largest output here; 1e-13 is the bar (both schedules also meet the 1e-12
    oracle bar above)."""
    import torch
    G = kl.KLProblem(2, 2, [40, 49], kernel="exp", L=0.5)     # 42 x 51 = 2,142 points: T = 9
    G2 = kl.KLProblem(2, 2, [40, 38], kernel="gauss", L=0.5)  # 42 x 40 = 1,680 points: T = 7
    G3 = kl.KLProblem(1, 2, 1934, kernel="exp", L=0.1)        # 1,936 points: T = 8
    for H in (G, G2, G3):
        u = torch.from_numpy(inputs.random_block(H.Nt, 4, seed=3).T.copy()).cuda()
        tri = [H.covmv(u, precision=pr) for pr in (kl.KL_P_FP64, kl.KL_P_DF64)]
        kl.set_sym_slot_limit(0)
        try:
            bnd = [H.covmv(u, precision=pr) for pr in (kl.KL_P_FP64, kl.KL_P_DF64)]
        finally:
            kl.set_sym_slot_limit(512 << 20)
        for a, b in zip(tri, bnd):
            assert float((a - b).abs().max() / b.abs().max()) < 1e-13


def test_band_eigensolve_matches_oracle(kl, band):
    """A whole float64 block-Lanczos solve with the banded schedule against the dense oracle."""
    P = ibq.Problem(3, 2, 10, kernel="exp", L=0.5)
    G = kl.KLProblem(3, 2, 10, kernel="exp", L=0.5)
    lam, _ = ibq.standard_eigs(P.dense_operator(), 8)
    ev, _, info = G.eigs(8, 1e-9, method=0, block=4)
    assert np.abs(ev - lam).max() / lam[0] < 1e-10
