"""The NURBS geometry path (quarter annulus, Sec. 2.4) through the C ABI against the oracle:
mapped points and J = sqrt(det DF) (now varying from point to point), the operator in every
precision, and eigenpairs."""
import numpy as np
import pytest

from oracle import ibq, nurbs
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5

CASES = [
    # dim, p, ne, kernel, L
    (2, 2, [7, 9], "exp", 0.4),
    (3, 2, [5, 6, 4], "gauss", 0.6),
    (3, [3, 2, 2], [4, 5, 3], "exp", 1.5),
]


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def make(kl, case):
    dim, p, ne, kern, L = case
    net = inputs.quarter_annulus_net(dim=dim)
    F = nurbs.NURBSMap(net["deg"], net["knots"], net["ctrl"], net["weights"])
    P = ibq.Problem(dim, p, ne, kernel=kern, L=L, sigma=1.1, geom=F)
    G = kl.KLProblem(dim, p, ne, kernel=kern, L=L, sigma=1.1, nurbs=net)
    return P, G


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%s" % (c[0], c[3]))
def test_points_and_jacobian(kl, case):
    P, G = make(kl, case)
    X, J = G.points()
    Xo, Jo = P.points_and_J()
    assert np.abs(X[:, :P.dim] - Xo).max() < 1e-14 * np.abs(Xo).max()
    assert rel(J, Jo) < 1e-14
    assert np.ptp(Jo) > 0.1 * Jo.max()        # J really varies on the curved map


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%s" % (c[0], c[3]))
def test_operator_all_precisions(kl, case):
    import torch
    P, G = make(kl, case)
    v = inputs.random_block(P.N, 5, seed=21)
    vd = torch.from_numpy(v.T.copy()).cuda()
    ref = P.dense_operator() @ v
    for prec in (kl.KL_P_FP64, kl.KL_P_DF64, kl.KL_P_TC64):
        assert rel(G.apply(vd, precision=prec).cpu().numpy().T, ref) < FP64_TOL, prec
    for prec in (kl.KL_P_FP32, kl.KL_P_TC32):
        assert rel(G.apply(vd, precision=prec).cpu().numpy().T, ref) < FP32_TOL, prec


def test_eigenpairs_on_the_annulus(kl):
    import torch
    P, G = make(kl, CASES[1])
    lam = np.linalg.eigvalsh(P.dense_operator())[::-1][:10]
    start = torch.from_numpy(inputs.random_block(G.N, 4, seed=2).T.copy()).cuda()
    ev, _, info = G.eigs(10, 1e-8, method=0, block=4, start=start)
    assert np.abs(ev - lam).max() / lam[0] < 1e-10
    ev2, _, info2 = G.eigs(10, 1e-8, method=1, block=4, start=start, precision=kl.KL_P_TC64)
    assert np.abs(ev2 - lam).max() / lam[0] < 1e-10
    assert max(info["resid"]) <= 1e-8 and max(info2["resid"]) <= 1e-8


def test_rejects_bad_maps(kl):
    net = inputs.quarter_annulus_net(dim=2)
    bad = dict(net)
    bad["weights"] = -net["weights"]
    with pytest.raises(kl.KLError):
        kl.KLProblem(2, 2, 4, nurbs=bad)
    flipped = dict(net)                       # mirror one direction: det DF < 0
    flipped["ctrl"] = net["ctrl"][:, ::-1].copy()
    flipped["weights"] = net["weights"][:, ::-1].copy()
    with pytest.raises(kl.KLError):
        kl.KLProblem(2, 2, 4, nurbs=flipped)
    shifted = dict(net)
    shifted["knots"] = [np.array([0.0, 0.0, 0.0, 2.0, 2.0, 2.0])] * 2
    with pytest.raises(kl.KLError):
        kl.KLProblem(2, 2, 4, nurbs=shifted)
