"""Multipatch domains (Sec. 3.6) through the C ABI against the oracle: trial spaces that are C^0
and interpolation spaces that are C^{-1} at patch interfaces (Sec. 6.2, Example 1-1; Sec. 6.3),
one-sided Greville points and det DF there, the operator in every precision, and eigenpairs."""
import numpy as np
import pytest

from oracle import ibq, nurbs
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5
S = 1.0 / 3.0

CASES = [
    # name, dim, p, ne, pt, net, kernel, L, interfaces
    ("bar2d-poly", 2, 2, [6, 2], None, None, "poly", 2, [[S], []]),
    ("annulus2d-exp", 2, [2, 2], [3, 6], None, None, "exp", 0.5, [[], [S]]),
    ("annulus3d-gauss", 3, [2, 2, 2], [2, 6, 2], [3, 2, 2], [2, 3, 3], "gauss", 0.8, [[], [S], []]),
    ("annulus3d-two-interfaces", 3, [3, 2, 1], [2, 6, 2], None, None, "exp", 1.2, [[], [S, 2 * S], []]),
]


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def make(kl, case):
    name, dim, p, ne, pt, net_, kern, L, itf = case
    if name.startswith("bar"):
        net = inputs.two_patch_bar_net(a=0.6, split=S, dim=dim)
    elif "two-interfaces" in name:
        net = inputs.quarter_annulus_net(dim=dim)       # smooth map, interfaces only in the spaces
    else:
        net = inputs.two_patch_annulus_net(dim=dim, split=S)
    F = nurbs.NURBSMap(net["deg"], net["knots"], net["ctrl"], net["weights"])
    P = ibq.Problem(dim, p, ne, kernel=kern, L=L, sigma=1.1, pt=pt, net=net_, geom=F, interfaces=itf)
    G = kl.KLProblem(dim, p, ne, kernel=kern, L=L, sigma=1.1, pt=pt, net=net_, nurbs=net, interfaces=itf)
    return P, G


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_sizes_points_and_one_sided_jacobian(kl, case):
    P, G = make(kl, case)
    assert (G.N, G.Nt) == (P.N, P.Nt)
    X, J = G.points()
    Xo, Jo = P.points_and_J()
    assert np.abs(X[:, :P.dim] - Xo).max() < 1e-14 * np.abs(Xo).max()
    assert rel(J, Jo) < 1e-14
    # duplicated Greville abscissae at every C^{-1} interface, each with its own one-sided J
    xh, sd = P.parametric_points(sides=True)
    assert (sd < 0).any()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_factors_match_oracle(kl, case):
    P, G = make(kl, case)
    for k, d in enumerate(P.dirs):
        Ck = G.factor(k)
        ref = np.linalg.solve(d.Bt.T, d.M @ np.linalg.inv(d.L).T)
        assert rel(Ck, ref) < 1e-12


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_operator_all_precisions(kl, case):
    import torch
    P, G = make(kl, case)
    v = inputs.random_block(P.N, 5, seed=31)
    vd = torch.from_numpy(v.T.copy()).cuda()
    ref = P.dense_operator() @ v
    for prec in (kl.KL_P_FP64, kl.KL_P_DF64, kl.KL_P_TC64):
        assert rel(G.apply(vd, precision=prec).cpu().numpy().T, ref) < FP64_TOL, prec
    for prec in (kl.KL_P_FP32, kl.KL_P_TC32):
        assert rel(G.apply(vd, precision=prec).cpu().numpy().T, ref) < FP32_TOL, prec


def test_eigenpairs_on_the_two_patch_annulus(kl):
    import torch
    P, G = make(kl, CASES[2])
    lam = np.linalg.eigvalsh(P.dense_operator())[::-1][:10]
    start = torch.from_numpy(inputs.random_block(G.N, 4, seed=3).T.copy()).cuda()
    ev, _, info = G.eigs(10, 1e-8, method=0, block=4, start=start)
    assert np.abs(ev - lam).max() / lam[0] < 1e-10
    ev2, _, info2 = G.eigs(10, 1e-8, method=1, block=4, start=start, precision=kl.KL_P_TC64)
    assert np.abs(ev2 - lam).max() / lam[0] < 1e-10
    assert max(info["resid"]) <= 1e-8 and max(info2["resid"]) <= 1e-8


def test_rejects_interfaces_off_the_mesh(kl):
    net = inputs.two_patch_annulus_net(dim=2, split=S)
    with pytest.raises(kl.KLError):
        kl.KLProblem(2, 2, [3, 4], nurbs=net, interfaces=[[], [S]])      # 1/3 is no breakpoint of 4 elements
    with pytest.raises(kl.KLError):
        kl.KLProblem(2, 2, [3, 6], nurbs=net, interfaces=[[], [1.0]])    # not interior
    C = kl.KLProblem(2, 2, [3, 6], nurbs=net, interfaces=[[], [S]])
    F = kl.KLProblem(2, 2, [6, 12], nurbs=net, interfaces=[[], [S]])
    import torch
    with pytest.raises(kl.KLError):
        kl.prolong(C, F, torch.zeros((1, C.N), dtype=torch.float64, device="cuda"))
