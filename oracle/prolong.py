"""Exact prolongation between nested spline spaces (TEST INFRASTRUCTURE ONLY).

A coarse space (degree p, ne_c uniform elements) is contained in a fine one of the same
degree whose uniform knots include the coarse knots (ne_f a multiple of ne_c).  Every coarse
B-spline is therefore a fine spline, and its fine coefficients are found by interpolating it
at the fine Greville points with the fine collocation matrix (Sec. 4.2: interpolation at the
Greville abscissae is exact on the space):

    P_k = B~_f^{-1} B_c(x_f),   coefficients c_f = P c_c   (direction k).

In the standard form of Sec. 4.1 (v' = L^T v, Z = L L^T) the map between coarse and fine
standard-form vectors is Q_k = L_f^T P_k L_c^{-T}; in d dimensions the Kronecker product
Q_d (x) ... (x) Q_1 (direction 1 fastest).
"""
import numpy as np

from . import bspline


def prolongation_1d(p, ne_c, ne_f):
    """Fine coefficients of every coarse B-spline: (n_f x n_c)."""
    if ne_f % ne_c:
        raise ValueError("the fine mesh must refine the coarse one")
    tc = bspline.open_uniform_knots(p, ne_c)
    tf = bspline.open_uniform_knots(p, ne_f)
    xf = bspline.greville(tf, p)
    Bf = bspline.collocation_matrix(tf, p, xf)
    Bc = bspline.basis_matrix(tc, p, xf)
    return np.linalg.solve(Bf, Bc)


def standard_form_map_1d(p, ne_c, ne_f):
    """Q = L_f^T P L_c^{-T} between coarse and fine standard-form coefficient vectors."""
    tc = bspline.open_uniform_knots(p, ne_c)
    tf = bspline.open_uniform_knots(p, ne_f)
    Lc = np.linalg.cholesky(bspline.gramian(tc, p))
    Lf = np.linalg.cholesky(bspline.gramian(tf, p))
    P = prolongation_1d(p, ne_c, ne_f)
    return Lf.T @ P @ np.linalg.inv(Lc).T


def kron_dirs(mats):
    """M_d (x) ... (x) M_1 for mats = [M_1, ..., M_d] (vec order, direction 1 fastest)."""
    out = mats[-1]
    for m in reversed(mats[:-1]):
        out = np.kron(out, m)
    return out
