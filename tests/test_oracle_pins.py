"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a textbook closed form, a
brute-force computation by an independent route, an exactness property stated
by the paper, or an invariant of the mathematics.  No GPU is used.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.special import comb

from oracle import bspline, closed_form, galerkin, ibq, kernels, nurbs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# Univariate B-splines (Sec. 2.3) -- textbook special cases
# ---------------------------------------------------------------------------------------
def test_knots_and_greville_textbook():
    t = bspline.open_uniform_knots(2, 2)
    assert np.array_equal(t, [0, 0, 0, 0.5, 1, 1, 1])
    # Greville abscissae of quadratic splines on knots (0,0,0,.5,1,1,1): 0, 1/4, 3/4, 1
    assert np.allclose(bspline.greville(t, 2), [0.0, 0.25, 0.75, 1.0], atol=0, rtol=0)
    assert bspline.dimension(bspline.open_uniform_knots(3, 48), 3) == 51


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_single_element_basis_is_bernstein(p):
    """With one element the B-splines are the Bernstein polynomials C(p,i) x^i (1-x)^(p-i)."""
    t = bspline.open_uniform_knots(p, 1)
    x = np.linspace(0.0, 1.0, 17)
    B = bspline.basis_matrix(t, p, x)
    ref = np.stack([comb(p, i) * x ** i * (1 - x) ** (p - i) for i in range(p + 1)], axis=1)
    assert np.abs(B - ref).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_bernstein_mass_matrix_closed_form(p):
    """Bernstein Gram matrix: int B_i B_j = C(p,i) C(p,j) / ((2p+1) C(2p, i+j))."""
    Z = bspline.gramian(bspline.open_uniform_knots(p, 1), p)
    ref = np.array([[comb(p, i) * comb(p, j) / ((2 * p + 1) * comb(2 * p, i + j))
                     for j in range(p + 1)] for i in range(p + 1)])
    assert np.abs(Z - ref).max() < 1e-15


def test_linear_mass_matrix_textbook():
    """Hat functions on a uniform mesh: h/6 * tridiag(1, 4, 1) with 2 at both ends."""
    ne = 6
    h = 1.0 / ne
    Z = bspline.gramian(bspline.open_uniform_knots(1, ne), 1)
    ref = np.diag([4.0] * (ne + 1)) + np.diag([1.0] * ne, 1) + np.diag([1.0] * ne, -1)
    ref[0, 0] = ref[-1, -1] = 2.0
    assert np.abs(Z - h / 6.0 * ref).max() < 1e-15


@pytest.mark.parametrize("p,ne", [(2, 7), (3, 5), (4, 9)])
def test_spline_identities(p, ne):
    t = bspline.open_uniform_knots(p, ne)
    n = bspline.dimension(t, p)
    x = np.linspace(0, 1, 101)
    B = bspline.basis_matrix(t, p, x)
    assert np.abs(B.sum(axis=1) - 1.0).max() < 1e-14          # partition of unity
    assert B.min() >= 0.0
    xi = bspline.greville(t, p)
    assert np.abs(B @ xi - x).max() < 1e-14                   # linear precision of Greville abscissae
    Z = bspline.gramian(t, p)
    integrals = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(n)])
    assert np.abs(Z.sum(axis=1) - integrals).max() < 1e-15   # int B_i = (t_{i+p+1}-t_i)/(p+1)
    assert np.abs(Z - Z.T).max() < 1e-16
    assert np.linalg.eigvalsh(Z).min() > 0
    Bt = bspline.collocation_matrix(t, p)
    assert np.abs(Bt.sum(axis=1) - 1.0).max() < 1e-14
    assert np.abs(Bt @ xi - xi).max() < 1e-14


def test_mixed_mass_matrix():
    """M_k = int B~_i B_j: equals Z when the spaces coincide; sums to |[0,1]| = 1 in general."""
    t = bspline.open_uniform_knots(2, 6)
    assert np.abs(bspline.mass_matrix(t, 2, t, 2) - bspline.gramian(t, 2)).max() < 1e-16
    tt = bspline.open_uniform_knots(3, 9)
    M = bspline.mass_matrix(tt, 3, t, 2)
    assert abs(M.sum() - 1.0) < 1e-14
    # row i integrates B~_i against sum_j B_j = 1
    assert np.abs(M.sum(axis=1) - [(tt[i + 4] - tt[i]) / 4 for i in range(M.shape[0])]).max() < 1e-15


def test_galerkin_gramian_matches_kron():
    """Two independent quadrature codes: tensor Gauss over all elements vs Kronecker of 1D Z_k."""
    P = ibq.Problem(2, [2, 3], [3, 2], kernel="gauss", L=0.5)
    _, Zg = galerkin.galerkin_matrices(P, q=4)
    assert np.abs(Zg - P.kron("Z")).max() < 1e-15


# ---------------------------------------------------------------------------------------
# Closed-form 1D spectrum (Remark in Sec. 6.1) pinned by a brute-force Nystrom solve
# ---------------------------------------------------------------------------------------
def nystrom_exp_1d(num, ell, panels=400, q=8):
    x, w = [], []
    for a in range(panels):
        xg, wg = bspline.gauss_legendre(q, a / panels, (a + 1) / panels)
        x.append(xg)
        w.append(wg)
    x, w = np.concatenate(x), np.concatenate(w)
    K = np.exp(-np.abs(x[:, None] - x[None, :]) / ell)
    sw = np.sqrt(w)
    vals = np.linalg.eigvalsh(sw[:, None] * K * sw[None, :])
    return vals[::-1][:num]


@pytest.mark.parametrize("ell", [1.0, 0.3])
def test_closed_form_matches_nystrom(ell):
    lam = closed_form.exp_kernel_1d(10, ell)
    ny = nystrom_exp_1d(10, ell)
    assert np.abs(lam - ny).max() / lam[0] < 2e-6
    assert np.all(np.diff(lam) < 0)
    assert lam.sum() < 1.0  # sum of all eigenvalues equals sigma^2 |D| = 1


def test_closed_form_golden():
    with open(os.path.join(GOLDEN, "exp_kernel_closed_form.json")) as f:
        g = json.load(f)
    lam = closed_form.exp_kernel_1d(len(g["unit_interval_ell1"]), 1.0)
    assert np.abs(lam - np.array(g["unit_interval_ell1"])).max() < 1e-15
    prod = closed_form.exp_separable_box(len(g["unit_square_ell1"]), 1.0, [1.0, 1.0])
    assert np.abs(prod - np.array(g["unit_square_ell1"])).max() < 1e-15


# ---------------------------------------------------------------------------------------
# IBQ machinery (Sec. 4.2-4.3): exact on its target space
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,p,ne,pt,net,m,lo,hi", [
    (1, 2, 5, None, None, 2, [0.0], [1.0]),
    (1, 3, 4, 3, 6, 3, [-1.0], [2.0]),
    (2, [2, 1], [3, 4], None, None, 1, [0.0, 0.0], [1.0, 1.0]),
    (2, 2, [3, 2], [3, 2], [4, 3], 2, [0.5, -1.0], [2.0, 1.5]),
])
def test_ibq_exact_for_kernel_in_target_space(dim, p, ne, pt, net, m, lo, hi):
    """A kernel whose pull-back G lies in B~ (x) B~ is integrated exactly (Sec. 4.2, end of Sec. 4.3).

    The polynomial kernel prod_k (1 + x_k x'_k)^m with m <= p~ and an affine map is such a kernel,
    so the IBQ matrix A~ must equal the brute-force Gauss Galerkin matrix A."""
    P = ibq.Problem(dim, p, ne, kernel="poly", L=m, pt=pt, net=net, lo=lo, hi=hi)
    At = P.dense()["At"]
    pmax = max(d.p for d in P.dirs)
    A, _ = galerkin.galerkin_matrices(P, q=pmax + m + 1)
    assert np.abs(At - A).max() / np.abs(A).max() < 1e-12


def test_ibq_error_decreases_for_gaussian():
    """Outside the target space IBQ is an approximation that converges under refinement."""
    errs = []
    for net in (2, 4, 8):
        P = ibq.Problem(1, 2, 3, kernel="gauss", L=0.5, pt=3, net=net)
        At = P.dense()["At"]
        A, _ = galerkin.galerkin_matrices(P, q=12)
        errs.append(np.linalg.norm(At - A, 2) / np.linalg.norm(A, 2))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4


# ---------------------------------------------------------------------------------------
# Reformulation (Sec. 4.1) and the Kronecker structure (Sec. 2.2)
# ---------------------------------------------------------------------------------------
def test_generalized_equals_standard():
    P = ibq.Problem(2, 2, [4, 6], kernel="exp", L=0.7)
    D = P.dense()
    wg, Vg = ibq.generalized_eigs(D["At"], D["Z"])
    ws, Vs = ibq.standard_eigs(0.5 * (D["Ap"] + D["Ap"].T))
    assert np.abs(wg - ws).max() / ws[0] < 1e-13
    # v' = L^T v maps Z-orthonormal generalized vectors to orthonormal standard ones
    Vp = D["L"].T @ Vg
    assert np.abs(Vp.T @ Vp - np.eye(P.N)).max() < 1e-11


def test_separable_kernel_gives_kronecker_spectrum_2d():
    """Identity map + separable kernel: A~' = A~'_2 (x) A~'_1, so the 2D spectrum is all 1D products.

    Different meshes per direction make a transposed Kronecker order fail."""
    P = ibq.Problem(2, [2, 3], [5, 7], kernel="exp_sep", L=0.8)
    w2 = np.linalg.eigvalsh(P.dense_operator())[::-1]
    w_1 = np.linalg.eigvalsh(ibq.Problem(1, 2, 5, kernel="exp", L=0.8).dense_operator())
    w_2 = np.linalg.eigvalsh(ibq.Problem(1, 3, 7, kernel="exp", L=0.8).dense_operator())
    prods = np.sort(np.outer(w_2, w_1).ravel())[::-1]
    assert np.abs(w2 - prods).max() / w2[0] < 1e-13


def test_separable_gaussian_3d_kronecker_spectrum():
    P = ibq.Problem(3, 2, [2, 3, 4], kernel="gauss", L=0.6)
    w3 = np.linalg.eigvalsh(P.dense_operator())[::-1]
    ws = [np.linalg.eigvalsh(ibq.Problem(1, 2, ne, kernel="gauss", L=0.6).dense_operator()) for ne in (2, 3, 4)]
    prods = np.sort(np.einsum("i,j,k->ijk", ws[2], ws[1], ws[0]).ravel())[::-1]
    assert np.abs(w3 - prods).max() / w3[0] < 1e-13


def test_matrix_free_algorithm_matches_dense():
    """Algorithm 1 stage by stage (mode contractions, triangular/LU solves, on-the-fly Gamma)."""
    P = ibq.Problem(3, [2, 2, 3], [3, 4, 2], kernel="exp", L=0.5, pt=[3, 2, 3], net=[4, 4, 3],
                    lo=[0, 0, 0], hi=[1.0, 2.0, 0.5])
    Ap = P.dense()["Ap"]
    v = np.random.default_rng(3).standard_normal((P.N, 3))
    y = P.apply(v, stage5_rows=37)
    ref = Ap @ v
    assert np.abs(y - ref).max() / np.abs(ref).max() < 1e-12
    y2 = P.backward(P.stage5(P.points_and_J()[0], P.forward(v)))
    assert np.abs(y2 - ref).max() / np.abs(ref).max() < 1e-12


# ---------------------------------------------------------------------------------------
# Convergence to the closed form and invariants
# ---------------------------------------------------------------------------------------
def test_convergence_to_closed_form_1d():
    """Discrete IBQ eigenvalues approach the analytic ones under h-refinement (Sec. 6.1)."""
    ref = closed_form.exp_kernel_1d(5, 1.0)
    errs = []
    for ne in (10, 20, 40, 80):
        w = np.linalg.eigvalsh(ibq.Problem(1, 2, ne, kernel="exp", L=1.0).dense_operator())[::-1][:5]
        errs.append(np.abs(w - ref).max() / ref[0])
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 5e-5
    # the observed order is at least that of the h^{3/2} interpolation estimate (caption of Fig. 3b)
    assert math.log2(errs[-2] / errs[-1]) > 1.4


def test_unit_square_config_against_closed_form():
    """The 2D unit-square, p=2, 20x20, separable exponential (sigma=L=1) top-10 vs 1D-product closed form."""
    P = ibq.Problem(2, 2, 20, kernel="exp_sep", L=1.0)
    w = np.linalg.eigvalsh(P.dense_operator())[::-1][:10]
    ref = closed_form.exp_separable_box(10, 1.0, [1.0, 1.0])
    assert np.abs(w - ref).max() / ref[0] < 2e-3   # IBQ eigenvalue error at h = 1/20 is ~1e-3


def test_invariants():
    P = ibq.Problem(2, 2, [6, 5], kernel="exp", L=0.5)
    Ap = P.dense()["Ap"]
    assert np.abs(Ap - Ap.T).max() / np.abs(Ap).max() < 1e-14        # symmetric
    w = np.linalg.eigvalsh(0.5 * (Ap + Ap.T))
    assert w.min() > -1e-14 * w.max()                                  # PSD (congruence with Gamma)
    assert w[::-1][:20].sum() <= 1.0 * (1 + 1e-6)                      # sum_k lambda_k <= sigma^2 |D|
    # trace of A~' is the discrete total variance; it tends to int Gamma(x, x) dx = sigma^2 |D| = 1
    errs = [abs(np.trace(ibq.Problem(1, 2, ne, kernel="exp", L=0.5).dense_operator()) - 1.0)
            for ne in (5, 10, 20, 40)]
    assert all(a > b for a, b in zip(errs, errs[1:])) and errs[-1] < 0.01


def test_similarity_scaling():
    """Scaling the box and L by s scales every eigenvalue by s^d exactly (J = s^{d/2})."""
    s = 2.0
    P1 = ibq.Problem(2, 2, [4, 3], kernel="exp", L=0.5)
    Ps = ibq.Problem(2, 2, [4, 3], kernel="exp", L=0.5 * s, lo=[0, 0], hi=[s, s])
    w1 = np.linalg.eigvalsh(P1.dense_operator())
    ws = np.linalg.eigvalsh(Ps.dense_operator())
    assert np.abs(ws - s ** 2 * w1).max() / ws.max() < 1e-13


def test_cube_symmetry_multiplicities():
    """Euclidean exponential kernel on the unit cube: eigenvalue clusters of size 1, 2 or 3 from cube symmetry."""
    P = ibq.Problem(3, 2, 3, kernel="exp", L=0.5)
    w = np.linalg.eigvalsh(P.dense_operator())[::-1][:10]
    assert abs(w[1] - w[2]) / w[0] < 1e-13 and abs(w[2] - w[3]) / w[0] < 1e-13


def test_kernel_values_at_pythagorean_offsets():
    """Kernel values at point pairs whose Euclidean distance is known exactly: offsets
    (3, 4)/5, (3, 4, 12)/13 and (2, 3, 6)/7 have length 1 (Pythagorean triples and quadruples),
    scaled by s.  exp must give e^{-s/L}, gauss e^{-s^2/L^2} and exp_sep e^{-s |o|_1/L}; an L1
    or maximum norm, or a distance without the square root, fails the first two."""
    for off in ([3.0, 4.0], [3.0, 4.0, 12.0], [2.0, 3.0, 6.0]):
        off = np.array(off) / np.linalg.norm(off)
        for s, L in ((0.5, 0.7), (1.3, 0.4), (2.0, 3.0)):
            x0 = np.linspace(-0.3, 0.4, len(off))
            X1, X2 = x0[None, :], (x0 + s * off)[None, :]
            assert abs(kernels.kernel_matrix(X1, X2, "exp", 1.5, L)[0, 0] - 2.25 * math.exp(-s / L)) < 1e-15
            assert abs(kernels.kernel_matrix(X2, X1, "gauss", 1.0, L)[0, 0] - math.exp(-(s / L) ** 2)) < 1e-15
            l1 = s * np.abs(off).sum()
            assert abs(kernels.kernel_matrix(X1, X2, "exp_sep", 1.0, L)[0, 0] - math.exp(-l1 / L)) < 1e-15


def rotated_box_map(dim, lx, ly, lz=1.0, angle=math.pi / 6):
    """The box [0,lx] x [0,ly] (x [0,lz]) rotated by `angle` in the x-y plane, written as a
    degree-1 NURBS map with unit weights (an affine map, det DF = lx ly lz everywhere)."""
    c, s = math.cos(angle), math.sin(angle)
    t = np.array([0.0, 0.0, 1.0, 1.0])
    if dim == 2:
        ctrl = np.zeros((2, 2, 2))
        for j in range(2):
            for i in range(2):
                x, y = lx * i, ly * j
                ctrl[j, i] = [c * x - s * y, s * x + c * y]
        return nurbs.NURBSMap([1, 1], [t, t], ctrl, np.ones((2, 2)))
    ctrl = np.zeros((2, 2, 2, 3))
    for k in range(2):
        for j in range(2):
            for i in range(2):
                x, y = lx * i, ly * j
                ctrl[k, j, i] = [c * x - s * y, s * x + c * y, lz * k]
    return nurbs.NURBSMap([1, 1, 1], [t, t, t], ctrl, np.ones((2, 2, 2)))


@pytest.mark.parametrize("dim,p,ne", [(2, 2, [5, 4]), (3, 2, [3, 3, 2])])
def test_euclidean_kernels_are_rotation_invariant(dim, p, ne):
    """Rotating the domain by 30 degrees leaves every Euclidean distance, det DF and hence the
    spectra of the exp and gauss operators unchanged; the separable kernel measures the L1
    distance, which a rotation changes, so its spectrum must move.  A kernel that used the L1 or
    maximum norm in d >= 2 for exp or gauss fails the first check."""
    lo, hi = [0.0] * dim, [1.0, 0.6, 0.8][:dim]
    F = rotated_box_map(dim, *hi)
    for kind, L, must_match in (("exp", 0.5, True), ("gauss", 0.4, True), ("exp_sep", 0.5, False)):
        wb = np.linalg.eigvalsh(ibq.Problem(dim, p, ne, kernel=kind, L=L, lo=lo, hi=hi).dense_operator())
        wr = np.linalg.eigvalsh(ibq.Problem(dim, p, ne, kernel=kind, L=L, geom=F).dense_operator())
        dev = np.abs(wb - wr).max() / wb.max()
        if must_match:
            assert dev < 1e-13, (kind, dev)
        else:
            assert dev > 1e-4, (kind, dev)


# ---------------------------------------------------------------------------------------------
# NURBS geometry map (Sec. 2.4) used for the quarter-annulus instances
# ---------------------------------------------------------------------------------------------

def test_nurbs_basis_derivative_bernstein_closed_form():
    """On one element (knots 0^{p+1} 1^{p+1}) the B-splines are the Bernstein polynomials and
    d/dx b_{i,p} = p (b_{i-1,p-1} - b_{i,p-1}); checked against that closed form and against
    the zero sum of derivatives (partition of unity)."""
    from math import comb
    from oracle import nurbs
    x = np.linspace(0.0, 1.0, 41)
    for p in (1, 2, 3, 4):
        t = np.array([0.0] * (p + 1) + [1.0] * (p + 1))
        dB = nurbs.basis_derivative_matrix(t, p, x)

        def b(i, q):
            if i < 0 or i > q:
                return np.zeros_like(x)
            return comb(q, i) * x ** i * (1 - x) ** (q - i)
        ref = np.stack([p * (b(i - 1, p - 1) - b(i, p - 1)) for i in range(p + 1)], axis=1)
        assert np.abs(dB - ref).max() < 1e-12
        assert np.abs(dB.sum(axis=1)).max() < 1e-12


def test_nurbs_basis_derivative_finite_differences_multi_element():
    from oracle import nurbs
    t = bspline.open_uniform_knots(3, 5)
    x = np.linspace(0.013, 0.987, 57)
    h = 1e-6
    fd = (bspline.basis_matrix(t, 3, x + h) - bspline.basis_matrix(t, 3, x - h)) / (2 * h)
    assert np.abs(nurbs.basis_derivative_matrix(t, 3, x) - fd).max() < 1e-6


def test_quarter_annulus_exact_geometry_and_volume():
    """The rational quadratic quarter circle is exact: |(x, y)| = 1 + xh_1 and z = xh_3 to
    rounding, the angle runs monotonically from 0 to pi/2; DF agrees with central differences
    and the integral of det DF is the volume 3 pi / 4 (area 3 pi / 4 in 2D)."""
    from oracle import nurbs
    rng = np.random.default_rng(7)
    F = nurbs.quarter_annulus()
    xh = rng.random((200, 3))
    X = F(xh)
    assert np.abs(np.hypot(X[:, 0], X[:, 1]) - (1.0 + xh[:, 0])).max() < 1e-14
    assert np.abs(X[:, 2] - xh[:, 2]).max() < 1e-14
    s = np.linspace(0.0, 1.0, 101)
    ang = np.arctan2(*F(np.stack([0.5 + 0 * s, s, 0 * s], axis=1))[:, 1::-1].T)
    assert abs(ang[0]) < 1e-14 and abs(ang[-1] - np.pi / 2) < 1e-14 and np.all(np.diff(ang) > 0)
    h = 1e-6
    J = F.jacobian(xh)
    Jfd = np.stack([(F(xh + h * np.eye(3)[j]) - F(xh - h * np.eye(3)[j])) / (2 * h) for j in range(3)], axis=2)
    assert np.abs(J - Jfd).max() < 1e-8
    x, w = bspline.gauss_legendre(24)
    g = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    ww = np.einsum("i,j,k->ijk", w, w, w).ravel()
    assert abs((F.detDF(g) * ww).sum() - 0.75 * np.pi) < 1e-12
    F2 = nurbs.quarter_annulus(dim=2)
    g2 = np.stack(np.meshgrid(x, x, indexing="ij"), -1).reshape(-1, 2)
    assert abs((F2.detDF(g2) * np.outer(w, w).ravel()).sum() - 0.75 * np.pi) < 1e-12


def test_nurbs_identity_equals_box_map():
    """A NURBS map whose control net is the degree-1 tensor grid of a box with unit weights is
    the affine box map: same points, same det DF, same IBQ operator."""
    from oracle import nurbs
    lo, hi = np.array([0.0, -1.0]), np.array([2.0, 0.5])
    t = np.array([0.0, 0.0, 1.0, 1.0])
    ctrl = np.zeros((2, 2, 2))
    for j in range(2):
        for i in range(2):
            ctrl[j, i] = [lo[0] + (hi[0] - lo[0]) * i, lo[1] + (hi[1] - lo[1]) * j]
    F = nurbs.NURBSMap([1, 1], [t, t], ctrl, np.ones((2, 2)))
    Pb = ibq.Problem(2, 2, [5, 4], kernel="gauss", L=0.4, lo=lo, hi=hi)
    Pn = ibq.Problem(2, 2, [5, 4], kernel="gauss", L=0.4, geom=F)
    Xb, Jb = Pb.points_and_J()
    Xn, Jn = Pn.points_and_J()
    assert np.abs(Xb - Xn).max() < 1e-14 and np.abs(Jb - Jn).max() < 1e-14
    assert np.abs(Pb.dense_operator() - Pn.dense_operator()).max() < 1e-14


def test_ibq_on_quarter_annulus_converges_to_galerkin():
    """On the curved 2D quarter annulus (J varies from point to point) the IBQ eigenvalues
    approach the brute-force Galerkin eigenvalues of the same space as the mesh is refined."""
    from oracle import nurbs
    F = nurbs.quarter_annulus(dim=2)
    errs = []
    for ne in (6, 12):
        P = ibq.Problem(2, 2, ne, kernel="gauss", L=0.7, geom=F)
        A, Z = galerkin.galerkin_matrices(P, 6)
        lg = sla.eigh(A, Z, eigvals_only=True)[::-1][:6]
        li = np.linalg.eigvalsh(P.dense_operator())[::-1][:6]
        errs.append(np.abs(li - lg).max() / lg[0])
    assert errs[1] < errs[0] / 4
    assert errs[1] < 1e-3


def test_batched_instance_generator_is_seeded():
    from paper_2011_13861_gb300 import inputs as _inputs
    a = _inputs.batched_instances(8)
    b = _inputs.batched_instances(8)
    assert a == b
    for i, c in enumerate(_inputs.batched_instances(64)):
        assert all(8 <= x <= 40 for x in c["ne"]) and c["p"] in (2, 3) and 0.1 <= c["L"] <= 2.0
        assert c["kernel"] == ("exp" if i % 2 == 0 else "gauss")


# ---------------------------------------------------------------------------------------------
# learned warm start: MLP, projector loss, Adam, prolongation between nested spline spaces
# ---------------------------------------------------------------------------------------------

def test_bf16_rounding_matches_torch():
    import torch
    from oracle import mlp
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-8, 8, 1000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -1.0 - 2 ** -8, 0.0, 65504.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)
    assert mlp.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0          # tie to even
    assert mlp.bf16(np.array([1.0 + 3 * 2 ** -9]))[0] == 1.0 + 2 ** -7


def _tiny_net(rng, sizes):
    Ws = [rng.standard_normal((a, b)) / np.sqrt(a) for a, b in zip(sizes[:-1], sizes[1:])]
    bs = [0.1 * rng.standard_normal(b) for b in sizes[1:]]
    return Ws, bs


def test_projector_loss_closed_form_and_invariance():
    from oracle import mlp
    rng = np.random.default_rng(4)
    n, k, B = 9, 3, 4
    out = rng.standard_normal((B, k * n))
    Vs = np.stack([np.linalg.qr(rng.standard_normal((n, k)))[0] for _ in range(B)])
    loss, _ = mlp.projector_loss(out, Vs, k)
    dense = np.mean([np.sum((out[s].reshape(k, n).T @ out[s].reshape(k, n) - Vs[s] @ Vs[s].T) ** 2)
                     for s in range(B)]) / k
    assert abs(loss - dense) < 1e-12 * dense
    R = np.linalg.qr(rng.standard_normal((k, k)))[0] * np.array([1.0, -1.0, 1.0])
    rot = np.stack([(out[s].reshape(k, n).T @ R).T.reshape(-1) for s in range(B)])
    assert abs(mlp.projector_loss(rot, Vs, k)[0] - loss) < 1e-12 * loss
    exact = np.stack([(Vs[s] @ R).T.reshape(-1) for s in range(B)])
    assert abs(mlp.projector_loss(exact, Vs, k)[0]) < 1e-14   # cancellation of k - 2k + k


def test_mlp_forward_and_backward_match_torch_nn():
    """The float64 network (roundings off) against torch.nn: Linear layers with Tanh between
    them and none after the last, same weights (torch stores W^T), float64; the gradients of the
    projector loss from mlp.backward against torch autograd of the same loss.  A tanh on the
    output layer, a bias applied before the activation's input is complete, or transposed
    weights fail here."""
    import torch
    from oracle import mlp
    rng = np.random.default_rng(11)
    n, k, B = 7, 3, 5
    sizes = [4, 16, 16, 16, k * n]
    Ws, bs = _tiny_net(rng, sizes)
    x = rng.standard_normal((B, 4))
    Vs = np.stack([np.linalg.qr(rng.standard_normal((n, k)))[0] for _ in range(B)])
    layers = []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        lin = torch.nn.Linear(W.shape[0], W.shape[1], dtype=torch.float64)
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W.T.copy()))
            lin.bias.copy_(torch.from_numpy(b.copy()))
        layers.append(lin)
        if l < len(Ws) - 1:
            layers.append(torch.nn.Tanh())
    net = torch.nn.Sequential(*layers)
    out_t = net(torch.from_numpy(x))
    out, cache = mlp.forward(Ws, bs, x, rounding=False)
    assert np.abs(out - out_t.detach().numpy()).max() < 1e-14 * max(1.0, np.abs(out).max())
    # projector loss written with torch ops from its definition ||Y Y^T - V V^T||_F^2 / k
    Y = out_t.reshape(B, k, n).transpose(1, 2)
    Vt = torch.from_numpy(Vs)
    loss_t = ((Y @ Y.transpose(1, 2) - Vt @ Vt.transpose(1, 2)) ** 2).sum(dim=(1, 2)).mean() / k
    loss_t.backward()
    loss, g = mlp.projector_loss(out, Vs, k)
    assert abs(loss - loss_t.item()) < 1e-13 * abs(loss)
    dWs, dbs = mlp.backward(Ws, bs, cache, g, rounding=False)
    lins = [m for m in net if isinstance(m, torch.nn.Linear)]
    for l, lin in enumerate(lins):
        assert np.abs(dWs[l] - lin.weight.grad.numpy().T).max() < 1e-13 * np.abs(dWs[l]).max()
        assert np.abs(dbs[l] - lin.bias.grad.numpy()).max() < 1e-13 * np.abs(dbs[l]).max()


def test_mlp_gradient_finite_differences():
    """Backward propagation and the loss gradient against central differences of the float64
    network (roundings off), for every weight and bias of a small 4-layer tanh network."""
    from oracle import mlp
    rng = np.random.default_rng(5)
    n, k, B = 5, 2, 3
    Ws, bs = _tiny_net(rng, [4, 6, 6, 6, k * n])
    x = rng.standard_normal((B, 4))
    Vs = np.stack([np.linalg.qr(rng.standard_normal((n, k)))[0] for _ in range(B)])

    def f(Ws_, bs_):
        out, _ = mlp.forward(Ws_, bs_, x, rounding=False)
        return mlp.projector_loss(out, Vs, k)[0]
    out, cache = mlp.forward(Ws, bs, x, rounding=False)
    _, g = mlp.projector_loss(out, Vs, k)
    dWs, dbs = mlp.backward(Ws, bs, cache, g, rounding=False)
    h = 1e-6
    for l in range(len(Ws)):
        for idx in [(0, 0), (Ws[l].shape[0] - 1, Ws[l].shape[1] - 1), (1, 2)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fd = (f(Wp, bs) - f(Wm, bs)) / (2 * h)
            assert abs(fd - dWs[l][idx]) < 1e-6 * max(1.0, abs(fd)), (l, idx)
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][1] += h
        bm[l][1] -= h
        fd = (f(Ws, bp) - f(Ws, bm)) / (2 * h)
        assert abs(fd - dbs[l][1]) < 1e-6 * max(1.0, abs(fd))


def test_adam_matches_torch():
    import torch
    from oracle import mlp
    rng = np.random.default_rng(6)
    p0 = rng.standard_normal(20)
    grads = [rng.standard_normal(20) for _ in range(3)]
    p = p0.copy()
    m = np.zeros(20)
    v = np.zeros(20)
    for t, g in enumerate(grads, start=1):
        mlp.adam_step(p, g, m, v, t, 1e-2)
    tp = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for g in grads:
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
    assert np.abs(tp.detach().numpy() - p).max() < 1e-12


def test_prolongation_is_exact_and_norm_preserving():
    """Coarse and prolonged fine splines are the same function at random points, and in the
    standard form (Sec. 4.1) the map has orthonormal columns (L2 norms are preserved)."""
    from oracle import prolong
    rng = np.random.default_rng(7)
    for p, nc, nf in [(2, 4, 12), (3, 5, 10), (3, 8, 24)]:
        P = prolong.prolongation_1d(p, nc, nf)
        x = rng.random(200)
        tc = bspline.open_uniform_knots(p, nc)
        tf = bspline.open_uniform_knots(p, nf)
        c = rng.standard_normal(P.shape[1])
        assert np.abs(bspline.basis_matrix(tc, p, x) @ c - bspline.basis_matrix(tf, p, x) @ (P @ c)).max() < 1e-13
        Q = prolong.standard_form_map_1d(p, nc, nf)
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-12


# ---------------------------------------------------------------------------------------
# Multipatch domains (Sec. 3.6): C^0 trial spaces and C^{-1} interpolation spaces at patch
# interfaces (Sec. 6.2, Example 1-1; Sec. 6.3)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("pt", [1, 2, 3])
def test_c_minus1_interpolation_reproduces_a_jump(pt):
    """Interpolation at the one-sided Greville abscissae of a C^{-1} space reproduces every
    piecewise polynomial of degree <= pt with a jump at the interface; the C^{pt-1} space of the
    same mesh cannot."""
    rng = np.random.default_rng(pt)
    s = 1.0 / 3.0
    cl, cr = rng.standard_normal(pt + 1), rng.standard_normal(pt + 1)

    def g(x, side=None):
        left = (x < s) if side is None else ((x < s) | ((x == s) & (np.asarray(side) < 0)))
        return np.where(left, np.polyval(cl, x), np.polyval(cr, x))

    xe = rng.uniform(0, 1, 200)
    xe = xe[np.abs(xe - s) > 1e-9]
    t = bspline.knots_with_interfaces(pt, 6, [s], pt + 1)
    xi, sd = bspline.greville(t, pt), bspline.greville_sides(t, pt)
    assert np.sum(xi == s) == 2 and list(sd[xi == s]) == [-1, 0]
    c = np.linalg.solve(bspline.collocation_matrix(t, pt), g(xi, sd))
    assert np.abs(bspline.basis_matrix(t, pt, xe) @ c - g(xe)).max() < 1e-12
    t0 = bspline.open_uniform_knots(pt, 6)
    c0 = np.linalg.solve(bspline.collocation_matrix(t0, pt), g(bspline.greville(t0, pt)))
    assert np.abs(bspline.basis_matrix(t0, pt, xe) @ c0 - g(xe)).max() > 1e-3


def test_left_limit_evaluation():
    """Left limits at a C^{-1} knot are the values of the left piece; partition of unity holds
    on both sides."""
    t = bspline.knots_with_interfaces(2, 4, [0.5], 3)
    B_r = bspline.basis_matrix(t, 2, [0.5])
    B_l = bspline.basis_matrix(t, 2, [0.5], [-1])
    assert abs(B_r.sum() - 1) < 1e-15 and abs(B_l.sum() - 1) < 1e-15
    n = bspline.dimension(t, 2)
    left_funcs = [i for i in range(n) if t[i + 3] <= 0.5]
    assert B_l[0, left_funcs].sum() == 1.0 and B_r[0, left_funcs].sum() == 0.0
    # the left limit equals the limit of values just left of the knot
    B_near = bspline.basis_matrix(t, 2, [0.5 - 1e-12])
    assert np.abs(B_near - B_l).max() < 1e-10


@pytest.mark.parametrize("dim,p,ne,m", [(1, 2, [6], 2), (2, [2, 2], [6, 2], 2), (2, [3, 1], [3, 2], 1)])
def test_ibq_exact_on_two_patch_affine_domain(dim, p, ne, m):
    """Two affine patches joined with C^0 continuity: the pull-back of the polynomial kernel is
    piecewise polynomial and J = sqrt(det DF) is piecewise constant, jumping at the interface.
    With the C^{-1} interpolation space the IBQ matrix equals the brute-force Galerkin matrix;
    with the C^{pt-1} space of the same mesh it does not."""
    s = 1.0 / 3.0
    F = nurbs.two_patch_bar(a=0.6, split=s, dim=dim)
    itf = [[s]] + [[]] * (dim - 1)
    P = ibq.Problem(dim, p, ne, kernel="poly", L=m, geom=F, interfaces=itf)
    pmax = max(d.p for d in P.dirs)
    A, _ = galerkin.galerkin_matrices(P, q=pmax + m + 2)
    assert np.abs(P.dense()["At"] - A).max() / np.abs(A).max() < 1e-12
    P0 = ibq.Problem(dim, p, ne, kernel="poly", L=m, geom=F)
    A0, _ = galerkin.galerkin_matrices(P0, q=pmax + m + 2)
    assert np.abs(P0.dense()["At"] - A0).max() / np.abs(A0).max() > 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_two_patch_annulus_interface_and_area(dim):
    """The half annulus of two quarter-circle patches of parametric lengths s and 1 - s: F is
    continuous across the interface, det DF has the one-sided closed forms
    (r_out - r_in) sqrt(2) r / s (left) and (r_out - r_in) sqrt(2) r / (1 - s) (right), and the
    volume is pi (r_out^2 - r_in^2) / 2 (times the height)."""
    s, r_in, r_out, h = 1.0 / 3.0, 1.0, 2.0, 1.5
    F = nurbs.two_patch_annulus(r_in, r_out, h, dim, split=s)
    x1 = np.array([0.0, 0.3, 1.0])
    xh = np.zeros((3, dim))
    xh[:, 0] = x1
    xh[:, 1] = s
    if dim == 3:
        xh[:, 2] = 0.4
    left = np.zeros((3, dim), dtype=int)
    left[:, 1] = -1
    assert np.abs(F(xh, left) - F(xh)).max() < 1e-14
    r = r_in + x1 * (r_out - r_in)
    fac = (r_out - r_in) * np.sqrt(2.0) * r * (h if dim == 3 else 1.0)
    assert np.abs(F.detDF(xh, left) - fac / s).max() < 1e-12 * fac.max() / s
    assert np.abs(F.detDF(xh) - fac / (1 - s)).max() < 1e-12 * fac.max() / s
    # volume by Gauss quadrature on each patch (det DF is rational in the angle: 24 points)
    g1, w1 = bspline.gauss_legendre(6, 0.0, 1.0)
    ga, wa = np.concatenate([bspline.gauss_legendre(24, 0.0, s)[0], bspline.gauss_legendre(24, s, 1.0)[0]]), \
        np.concatenate([bspline.gauss_legendre(24, 0.0, s)[1], bspline.gauss_legendre(24, s, 1.0)[1]])
    grids = [g1, ga] + ([g1] if dim == 3 else [])
    wts = [w1, wa] + ([w1] if dim == 3 else [])
    mesh = np.meshgrid(*grids, indexing="ij")
    pts = np.stack([m_.ravel() for m_ in mesh], axis=1)
    ww = np.ones(len(pts))
    for k in range(dim):
        ww = ww * np.meshgrid(*wts, indexing="ij")[k].ravel()
    vol = 0.5 * np.pi * (r_out ** 2 - r_in ** 2) * (h if dim == 3 else 1.0)
    assert abs((F.detDF(pts) * ww).sum() - vol) < 1e-12 * vol


# ---------------------------------------------------------------------------------------------
# stored full-size spectra (written by tests/golden/make_cube_spectra.py from the oracle alone)
# ---------------------------------------------------------------------------------------------

def test_stored_exp_cube_spectrum_invariants():
    """The 24 stored eigenvalues of the 39,304-point exponential cube: the configuration is the
    bench workload's; they are positive and descending, their sum stays below sigma^2 |D| = 1
    (Sec. 3.3: the eigenvalues sum to the total variance), the cube's symmetry group shows as
    the 1-3-3-1-2-1-3-3-3-3 cluster pattern (a 3-fold cluster whose members agree to 1e-13), and
    ARPACK's residuals are at rounding level."""
    from paper_2011_13861_gb300 import inputs
    with open(os.path.join(GOLDEN, "cube_p2_32_exp_L0.5_top24.json")) as f:
        g = json.load(f)
    w = inputs.WORKLOADS["cube-p2-32^3-exp-L0.5"]
    assert {k: g["config"][k] for k in ("dim", "p", "ne", "kernel", "sigma", "L")} == \
        {k: w[k] for k in ("dim", "p", "ne", "kernel", "sigma", "L")}
    ev = np.array(g["eigenvalues"])
    assert np.all(ev > 0) and np.all(np.diff(ev) <= 1e-15 * ev[0]) and ev.sum() < 1.0
    sizes, i = [], 0
    while i < len(ev):
        j = i
        while j + 1 < len(ev) and abs(ev[j + 1] - ev[i]) <= 1e-12 * ev[0]:
            j += 1
        sizes.append(j - i + 1)
        i = j + 1
    assert sizes[:10] == [1, 3, 3, 1, 2, 1, 3, 3, 3, 3], sizes
    assert max(g["relative_residuals"]) < 1e-13


def test_stored_gauss_cube_kronecker_spectrum():
    """The stored 1D eigenpairs of the separable Gaussian cube reproduce the dense 1D oracle and
    its 3D spectrum; on a reduced 3D mesh the same construction matches the full dense oracle."""
    from paper_2011_13861_gb300 import inputs
    with open(os.path.join(GOLDEN, "cube_p3_48_gauss_L0.3_kron.json")) as f:
        g = json.load(f)
    w = inputs.WORKLOADS["cube-p3-48^3-gauss-L0.3"]
    assert (g["config"]["p"], g["config"]["ne"], g["config"]["L"]) == (w["p"], w["ne"], w["L"])
    A1 = ibq.Problem(1, w["p"], w["ne"], kernel="gauss", L=w["L"]).dense_operator()
    U = np.array(g["u_1d"]).T
    mu = np.array(g["mu_1d"])
    assert np.abs(A1 @ U - U * mu).max() < 1e-14 and np.abs(U.T @ U - np.eye(len(mu))).max() < 1e-13
    for lam, (a, b, c) in zip(g["eigenvalues"], g["triples"]):
        assert abs(lam - mu[a] * mu[b] * mu[c]) <= 1e-15 * lam
    assert np.all(np.diff(g["eigenvalues"]) <= 1e-15)
