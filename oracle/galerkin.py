"""Brute-force standard Galerkin matrices by tensor Gauss quadrature (TEST INFRASTRUCTURE ONLY).

Sec. 5.1 describes the standard formation: every pair of elements of the
2d-dimensional domain integrated with a tensor Gauss-Legendre rule.  Here that
is written out with no sum factorisation at all: one global list of quadrature
points (q per direction on every element), the d-variate B-spline values at
those points, and

    A_ij = sum_a sum_b w_a w_b Gamma(F(x_a), F(x_b)) B_i(x_a) B_j(x_b) sqrt(detDF(x_a) detDF(x_b))

(eq. GalA_mat) and Z_ij = sum_a w_a B_i(x_a) B_j(x_a) (Sec. 3.5).  Only for tiny meshes.
"""
import numpy as np

from . import bspline
from .kernels import kernel_matrix


def quadrature_1d(t, q):
    br = bspline.breakpoints(t)
    xs, ws = [], []
    for a, b in zip(br[:-1], br[1:]):
        xg, wg = bspline.gauss_legendre(q, a, b)
        xs.append(xg)
        ws.append(wg)
    return np.concatenate(xs), np.concatenate(ws)


def galerkin_matrices(problem, q):
    """Dense (A, Z) of the standard Galerkin method for an oracle Problem, q Gauss points per direction."""
    d = problem.dim
    pts1, wts1, bas1 = [], [], []
    for dd in problem.dirs:
        x, w = quadrature_1d(dd.t, q)
        pts1.append(x)
        wts1.append(w)
        bas1.append(bspline.basis_matrix(dd.t, dd.p, x))
    # tensor quadrature in vec order (direction 1 fastest), basis values by Kronecker products
    grids = np.meshgrid(*list(reversed(pts1)), indexing="ij")
    Xh = np.stack([grids[d - 1 - k].ravel() for k in range(d)], axis=1)
    W = wts1[d - 1]
    Bq = bas1[d - 1]
    for k in range(d - 2, -1, -1):
        W = np.kron(W, wts1[k])
        Bq = np.kron(Bq, bas1[k])
    X = problem.geom(Xh)
    sJ = np.sqrt(problem.geom.detDF(Xh))
    Gam = kernel_matrix(X, X, problem.kernel, problem.sigma, problem.L)
    wJ = W * sJ
    A = Bq.T @ (wJ[:, None] * Gam * wJ[None, :]) @ Bq
    Z = Bq.T @ (W[:, None] * Bq)
    return A, Z
