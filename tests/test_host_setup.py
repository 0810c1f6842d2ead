"""The library's host set-up of one direction (kl_direction_factors: knots, Greville abscissae,
Gauss quadrature, Cholesky factor, collocation, folded factor C_k) against the oracle's
matrices, on the CPU.  kl_create uploads exactly these arrays, so this pins stage a0 without
a GPU; the GPU tests then check the operator built from them."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ibq
from paper_2011_13861_gb300 import _binding, build


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
