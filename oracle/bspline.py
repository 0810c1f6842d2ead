"""Univariate B-spline machinery for the oracle (TEST INFRASTRUCTURE ONLY).

Follows Sec. 2.3 (B-splines), Sec. 3.5 eq. univariate_mass_matrix with the
Remark after it (exact Gauss-Legendre, p+1 points per element), Sec. 4.2
(collocation at the Greville abscissae, eq. interpolation_matrix) and Sec. 4.3
eq. univariate_mass_matrix2 (mixed mass matrix M_k).

Knot vectors are open and uniform: degree p, ne elements on [0, 1], end knots
of multiplicity p+1, interior knots simple, so the spline space is C^{p-1} and
has n = ne + p functions.  Multipatch domains (Sec. 3.6) add patch interfaces:
interior breakpoints where the trial space is only C^0 (knot multiplicity p) and
the interpolation space is C^{-1} (multiplicity p+1).  A C^{-1} space has two
Greville abscissae at such a knot; the basis is evaluated there from the side of
the function whose support ends or starts at the knot (left / right limit).
"""
import math

import numpy as np
from numpy.polynomial.legendre import leggauss


def open_uniform_knots(p, ne):
    """Open uniform knot vector on [0, 1]: (p+1) zeros, ne-1 interior knots, (p+1) ones."""
    if p < 0 or ne < 1:
        raise ValueError("need p >= 0 and ne >= 1")
    interior = [i / ne for i in range(1, ne)]
    return np.array([0.0] * (p + 1) + interior + [1.0] * (p + 1))


def knots_with_interfaces(p, ne, interfaces=(), mult=None):
    """Open uniform knot vector with each interface value (an interior breakpoint i/ne of the
    uniform mesh) repeated to multiplicity `mult` (p: C^0 there; p + 1: C^{-1})."""
    t = list(open_uniform_knots(p, ne))
    for x in interfaces:
        i = int(round(float(x) * ne))
        if not (0 < i < ne) or abs(float(x) * ne - i) > 1e-12:
            raise ValueError("an interface must be an interior breakpoint of the uniform mesh")
        xv = i / ne
        have = sum(1 for y in t if y == xv)
        t += [xv] * (int(mult) - have)
    return np.array(sorted(t))


def dimension(t, p):
    """Number of B-splines of degree p on knot vector t."""
    return len(t) - p - 1


def greville(t, p):
    """Greville abscissae: the average of the p knots t[i+1] .. t[i+p] (de Boor)."""
    if p < 1:
        raise ValueError("Greville abscissae need p >= 1")
    n = dimension(t, p)
    return np.array([sum(t[i + 1:i + p + 1]) / p for i in range(n)])


def basis_matrix(t, p, x, side=None):
    """Values of all n B-splines of degree p at the points x: B[a, i] = B_{i,p}(x_a).

    Cox-de Boor recursion written out over degrees.  The degree-0 functions are
    indicator functions of [t_i, t_{i+1}); at the right end of the domain the
    last non-empty interval is taken closed so that the basis is a partition of
    unity on the whole closed interval.  Points with side[a] < 0 take the left
    limit instead: the indicators of (t_i, t_{i+1}] (and the first interval closed).
    """
    t = np.asarray(t, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    left = np.zeros(len(x), dtype=bool) if side is None else (np.asarray(side) < 0)
    m = len(t) - 1  # number of knot spans (some empty)
    last = max(i for i in range(m) if t[i] < t[i + 1])
    first = min(i for i in range(m) if t[i] < t[i + 1])
    B = np.zeros((len(x), m))
    for i in range(m):
        if t[i] < t[i + 1]:
            inside = (t[i] <= x) & (x < t[i + 1])
            if i == last:
                inside |= (x == t[i + 1])
            inside_l = (t[i] < x) & (x <= t[i + 1])
            if i == first:
                inside_l |= (x == t[i])
            B[:, i] = np.where(left, inside_l, inside).astype(np.float64)
    for q in range(1, p + 1):
        Bn = np.zeros((len(x), m - q))
        for i in range(m - q):
            left = t[i + q] - t[i]
            right = t[i + q + 1] - t[i + 1]
            term = np.zeros(len(x))
            if left > 0.0:
                term += (x - t[i]) / left * B[:, i]
            if right > 0.0:
                term += (t[i + q + 1] - x) / right * B[:, i + 1]
            Bn[:, i] = term
        B = Bn
    return B


def gauss_legendre(q, a=0.0, b=1.0):
    """q-point Gauss-Legendre rule mapped to [a, b]."""
    xg, wg = leggauss(q)
    return 0.5 * (b - a) * xg + 0.5 * (b + a), 0.5 * (b - a) * wg


def breakpoints(*knot_vectors):
    """Sorted union of the distinct knot values of several knot vectors."""
    return np.unique(np.concatenate([np.asarray(t) for t in knot_vectors]))


def mass_matrix(t_row, p_row, t_col, p_col, q=None):
    """M[i, j] = integral over [0, 1] of B^{row}_i * B^{col}_j.

    Gauss-Legendre on every interval of the union of both knot vectors' breakpoints,
    so each integrand is a polynomial there.  The default rule has enough points to
    be exact for degree p_row + p_col.  With identical spaces and q = p + 1 this is
    the rule of the Remark in Sec. 3.5.
    """
    if q is None:
        q = int(math.ceil((p_row + p_col + 1) / 2.0))
    br = breakpoints(t_row, t_col)
    xs, ws = [], []
    for a, b in zip(br[:-1], br[1:]):
        xg, wg = gauss_legendre(q, a, b)
        xs.append(xg)
        ws.append(wg)
    x = np.concatenate(xs)
    w = np.concatenate(ws)
    Br = basis_matrix(t_row, p_row, x)
    Bc = basis_matrix(t_col, p_col, x)
    return Br.T @ (w[:, None] * Bc)


def gramian(t, p):
    """Univariate mass matrix Z_k (Sec. 3.5 eq. univariate_mass_matrix), p+1 Gauss points per element."""
    return mass_matrix(t, p, t, p, q=p + 1)


def greville_sides(t, p):
    """-1 for a Greville abscissa that sits on an interior knot where its own function's support
    ends (evaluate from the left there), 0 otherwise (the default right-limit evaluation)."""
    x = greville(t, p)
    n = dimension(t, p)
    return np.array([-1 if (t[i + p + 1] == x[i] and t[0] < x[i] < t[-1]) else 0 for i in range(n)])


def collocation_matrix(t, p, x=None, side=None):
    """Collocation matrix B~[i, j] = B~_j(x_i) at the Greville abscissae (Sec. 4.2 eq. interpolation_matrix),
    one-sided at the knots of a C^{-1} space."""
    if x is None:
        x = greville(t, p)
        side = greville_sides(t, p)
    return basis_matrix(t, p, x, side)
