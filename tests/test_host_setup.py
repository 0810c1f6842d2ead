"""The library's host set-up against the oracle, on the CPU: one direction's factors
(kl_direction_factors: knots, Greville abscissae, Gauss quadrature, Cholesky factor,
collocation, folded factor C_k) and the mapped Greville grid with J (kl_mapped_points: box and
NURBS maps, one-sided evaluation at patch interfaces).  kl_create uploads exactly these arrays,
built by the same host code, so this pins the set-up without a GPU; the GPU tests then check
the operator built from them."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ibq, nurbs, prolong
from paper_2011_13861_gb300 import _binding, build, inputs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _binding.load()


def oracle_C(d):
    # C_k = B~^{-T} M L^{-T}, by triangular and LU solves on the oracle's matrices
    X1 = sla.solve_triangular(d.L, d.M.T, lower=True).T          # M L^{-T}
    return sla.lu_solve(d.Bt_lu, X1, trans=1)                     # B~^{-T} X1


CASES = [
    (1, 1, 0, 0, ()), (2, 7, 0, 0, ()), (3, 5, 0, 0, ()), (4, 9, 0, 0, ()),
    (2, 6, 3, 4, ()), (3, 4, 2, 8, ()), (2, 12, 0, 0, (0.25,)), (3, 6, 2, 6, (1.0 / 3.0, 2.0 / 3.0)),
    (1, 6, 2, 3, (1.0 / 3.0,)),
]


@pytest.mark.parametrize("p,ne,pt,net,itf", CASES)
def test_direction_factors_match_the_oracle(lib, p, ne, pt, net, itf):
    got = _binding.direction_factors(p, ne, pt, net, itf)
    d = ibq.Direction(p, ne, pt or None, net or None, interfaces=itf)
    assert (got["n"], got["nt"]) == (d.n, d.nt)
    np.testing.assert_allclose(got["greville"], d.xi, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(got["side"], np.asarray(d.side, dtype=np.int32))
    np.testing.assert_allclose(got["L"], d.L, rtol=0, atol=1e-13 * np.abs(d.L).max())
    C = oracle_C(d)
    np.testing.assert_allclose(got["C"], C, rtol=0, atol=1e-12 * np.abs(C).max())


def test_cholesky_factor_reproduces_the_gramian(lib):
    got = _binding.direction_factors(3, 8)
    d = ibq.Direction(3, 8)
    L = got["L"]
    assert np.allclose(np.triu(L, 1), 0.0)
    np.testing.assert_allclose(L @ L.T, d.Z, rtol=0, atol=1e-14)


@pytest.mark.parametrize("args,needle", [
    ((0, 4), "degrees and element counts"),
    ((2, 0), "degrees and element counts"),
    ((2, 5000), "4096"),
    ((2, 6, 0, 0, (0.3,)), "interior breakpoint"),
    ((2, 6, 0, 0, (1.0,)), "interior breakpoint"),
])
def test_direction_factors_reject_bad_arguments(lib, args, needle):
    with pytest.raises(_binding.KLError) as e:
        _binding.direction_factors(*args)
    assert e.value.status == 1 and needle in str(e.value)


def oracle_points(dim, p, ne, pt=None, net=None, lo=None, hi=None, geom=None, interfaces=None):
    prob = ibq.Problem(dim, p, ne, pt=pt, net=net, lo=lo, hi=hi, geom=geom, interfaces=interfaces)
    X, J = prob.points_and_J()
    out = np.zeros((X.shape[0], 3))
    out[:, :X.shape[1]] = X
    return out, J


@pytest.mark.parametrize("dim,p,ne,pt,net,lo,hi", [
    (1, 2, 9, None, None, [-1.0], [2.0]),
    (2, [2, 3], [5, 4], None, None, [0.0, -0.5], [1.0, 0.25]),
    (3, 2, [3, 4, 2], [3, 2, 2], [2, 4, 3], [0.0, 0.0, 0.0], [1.0, 2.0, 0.5]),
])
def test_mapped_points_box(lib, dim, p, ne, pt, net, lo, hi):
    X, J = _binding.mapped_points(dim, p, ne, pt, net, lo, hi)
    Xo, Jo = oracle_points(dim, p, ne, pt, net, lo, hi)
    np.testing.assert_allclose(X, Xo, rtol=0, atol=1e-15)
    np.testing.assert_allclose(J, Jo, rtol=1e-15, atol=0)


def as_oracle_map(net):
    return nurbs.NURBSMap(net["deg"], net["knots"], net["ctrl"], net["weights"])


@pytest.mark.parametrize("dim", [2, 3])
def test_mapped_points_quarter_annulus(lib, dim):
    net = inputs.quarter_annulus_net(1.0, 2.0, 1.0, dim)
    p, ne = [2, 3, 2][:dim], [6, 4, 3][:dim]
    X, J = _binding.mapped_points(dim, p, ne, nurbs=net)
    Xo, Jo = oracle_points(dim, p, ne, geom=nurbs.quarter_annulus(1.0, 2.0, 1.0, dim))
    np.testing.assert_allclose(X, Xo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(J, Jo, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dim", [2, 3])
def test_mapped_points_two_patch_annulus_one_sided(lib, dim):
    # the map has a C0 knot at 1/3 in direction 2; the space has a patch interface there, so
    # the two collocated abscissae take det DF from their own side (it jumps by 2 there)
    net = inputs.two_patch_annulus_net(1.0, 2.0, 1.0, dim, 1.0 / 3.0)
    p, ne = [2] * dim, [3, 6, 2][:dim]
    itf = [(), (1.0 / 3.0,), ()][:dim]
    X, J = _binding.mapped_points(dim, p, ne, nurbs=net, interfaces=itf)
    Xo, Jo = oracle_points(dim, p, ne, geom=as_oracle_map(net), interfaces=itf)
    np.testing.assert_allclose(X, Xo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(J, Jo, rtol=1e-13, atol=0)
    jumps = np.isclose(J[:-1] / J[1:], np.sqrt(2.0)) | np.isclose(J[1:] / J[:-1], np.sqrt(2.0))
    assert jumps.any()


def test_mapped_points_reject_bad_geometry(lib):
    with pytest.raises(_binding.KLError):
        _binding.mapped_points(2, 2, 4, lo=[0.0, 1.0], hi=[1.0, 1.0])
    net = inputs.quarter_annulus_net(1.0, 2.0, 1.0, 2)
    net = dict(net, weights=-np.asarray(net["weights"]))
    with pytest.raises(_binding.KLError) as e:
        _binding.mapped_points(2, 2, 4, nurbs=net)
    assert "weights must be positive" in str(e.value)


@pytest.mark.parametrize("p,ne_c,ne_f", [(1, 2, 6), (2, 4, 8), (3, 16, 48), (3, 5, 5), (4, 3, 9)])
def test_prolongation_factor_matches_the_oracle(lib, p, ne_c, ne_f):
    Q = _binding.prolongation_factor(p, ne_c, ne_f)
    Qo = prolong.standard_form_map_1d(p, ne_c, ne_f)
    assert Q.shape == Qo.shape
    np.testing.assert_allclose(Q, Qo, rtol=0, atol=1e-12 * np.abs(Qo).max())
    # nested spaces: Q has orthonormal columns (a standard-form vector keeps its norm)
    np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), rtol=0, atol=1e-12)


def test_prolongation_factor_rejects_non_nested_meshes(lib):
    with pytest.raises(_binding.KLError) as e:
        _binding.prolongation_factor(2, 4, 6)
    assert "refine" in str(e.value)
