"""Tensor-product NURBS geometry maps for the oracle (TEST INFRASTRUCTURE ONLY).

The paper maps the parametric unit cube onto the physical domain with a NURBS
map F (Sec. 2.4): F(xh) = sum_I R_I(xh) P_I with rational basis
R_I = N_I w_I / sum_J N_J w_J, N_I the tensor-product B-splines.  The IBQ
operator needs F at the Greville points and det DF there (Sec. 4.4.1: J is
sqrt(det DF)).  Everything here is written from that definition:

  * B-spline values by the Cox-de Boor recursion (bspline.basis_matrix);
  * first derivatives by the textbook identity
        d/dx B_{i,p} = p/(t_{i+p} - t_i) B_{i,p-1} - p/(t_{i+p+1} - t_{i+1}) B_{i+1,p-1};
  * DF by the quotient rule on F = P / W with P = sum N w P and W = sum N w.

No sum factorisation and no reuse of library code.
"""
import numpy as np

from . import bspline


def basis_derivative_matrix(t, p, x, side=None):
    """dB[a, i] = d/dx B_{i,p}(x_a) on knot vector t (p >= 1); one-sided (left limit) where
    side[a] < 0."""
    t = np.asarray(t, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = bspline.dimension(t, p)
    Bm = bspline.basis_matrix(t, p - 1, x, side)    # n + 1 functions of degree p - 1
    dB = np.zeros((len(x), n))
    for i in range(n):
        left = t[i + p] - t[i]
        right = t[i + p + 1] - t[i + 1]
        if left > 0.0:
            dB[:, i] += p / left * Bm[:, i]
        if right > 0.0:
            dB[:, i] -= p / right * Bm[:, i + 1]
    return dB


class NURBSMap:
    """F: [0,1]^d -> R^d (d = 2 or 3), tensor-product NURBS.

    deg[k], knots[k] per parametric direction (open knot vectors on [0,1]); ctrl is an array of
    shape (n_d, ..., n_1, d) of control points and weights of shape (n_d, ..., n_1), direction 1
    fastest (the same vec ordering as the spline spaces).
    """

    def __init__(self, deg, knots, ctrl, weights):
        self.deg = [int(p) for p in deg]
        self.knots = [np.asarray(t, dtype=np.float64) for t in knots]
        self.d = len(self.deg)
        self.ctrl = np.asarray(ctrl, dtype=np.float64)
        self.w = np.asarray(weights, dtype=np.float64)
        self.n = [bspline.dimension(t, p) for t, p in zip(self.knots, self.deg)]
        assert self.ctrl.shape == tuple(reversed(self.n)) + (self.d,)
        assert self.w.shape == tuple(reversed(self.n))

    def _eval(self, xh, sides=None):
        xh = np.atleast_2d(np.asarray(xh, dtype=np.float64))
        m = xh.shape[0]
        sd = [None] * self.d if sides is None else [np.asarray(sides)[:, k] for k in range(self.d)]
        B = [bspline.basis_matrix(self.knots[k], self.deg[k], xh[:, k], sd[k]) for k in range(self.d)]
        dB = [basis_derivative_matrix(self.knots[k], self.deg[k], xh[:, k], sd[k]) for k in range(self.d)]
        # flatten the control net in vec order (direction 1 fastest)
        Pw = (self.ctrl * self.w[..., None]).reshape(-1, self.d)     # w_I P_I
        w = self.w.reshape(-1)
        # tensor basis per point, and its derivative along each direction
        def tensor(factors):
            out = factors[self.d - 1]
            for k in range(self.d - 2, -1, -1):
                out = np.einsum("ai,aj->aij", out, factors[k]).reshape(m, -1)
            return out
        N = tensor(B)
        P = N @ Pw
        W = N @ w
        F = P / W[:, None]
        DF = np.zeros((m, self.d, self.d))
        for j in range(self.d):
            fac = [dB[k] if k == j else B[k] for k in range(self.d)]
            Nj = tensor(fac)
            dP = Nj @ Pw
            dW = Nj @ w
            DF[:, :, j] = (dP * W[:, None] - P * dW[:, None]) / (W * W)[:, None]
        return F, DF

    def __call__(self, xh, sides=None):
        return self._eval(xh, sides)[0]

    def jacobian(self, xh, sides=None):
        return self._eval(xh, sides)[1]

    def detDF(self, xh, sides=None):
        """det DF; at a C^0 knot of the map, sides[a, k] < 0 takes the derivative from the left."""
        return np.linalg.det(self.jacobian(xh, sides))


def quarter_annulus(r_in=1.0, r_out=2.0, height=1.0, dim=3):
    """Quarter annulus r in [r_in, r_out], angle in [0, pi/2] (extruded to z in [0, height] for
    dim = 3): degree 2 in every direction, one Bezier element per direction.  The angular
    direction is the exact rational quadratic quarter circle (middle weight sqrt(2)/2);
    radius and height are linear in the parameter (equally spaced control points)."""
    knots = [np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])] * dim
    radii = [r_in, 0.5 * (r_in + r_out), r_out]
    dirs = [(1.0, 0.0), (1.0, 1.0), (0.0, 1.0)]
    wang = [1.0, np.sqrt(0.5), 1.0]
    if dim == 2:
        ctrl = np.zeros((3, 3, 2))
        wts = np.zeros((3, 3))
        for j in range(3):          # angle (direction 2)
            for i in range(3):      # radius (direction 1)
                ctrl[j, i] = [radii[i] * dirs[j][0], radii[i] * dirs[j][1]]
                wts[j, i] = wang[j]
        return NURBSMap([2, 2], knots, ctrl, wts)
    zs = [0.0, 0.5 * height, height]
    ctrl = np.zeros((3, 3, 3, 3))
    wts = np.zeros((3, 3, 3))
    for kz in range(3):
        for j in range(3):
            for i in range(3):
                ctrl[kz, j, i] = [radii[i] * dirs[j][0], radii[i] * dirs[j][1], zs[kz]]
                wts[kz, j, i] = wang[j]
    return NURBSMap([2, 2, 2], knots, ctrl, wts)


def two_patch_annulus(r_in=1.0, r_out=2.0, height=1.0, dim=3, split=1.0 / 3.0):
    """Half annulus r in [r_in, r_out], angle in [0, pi], made of two quarter-annulus patches
    joined with C^0 continuity at the angular parameter `split` (knot of multiplicity 2 in the
    degree-2 angular direction).  Each patch is the exact rational quadratic quarter circle; the
    patches have parametric lengths split and 1 - split, so det DF jumps at the interface unless
    split = 1/2."""
    ka = np.array([0.0, 0.0, 0.0, split, split, 1.0, 1.0, 1.0])
    kl = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    radii = [r_in, 0.5 * (r_in + r_out), r_out]
    dirs = [(1.0, 0.0), (1.0, 1.0), (0.0, 1.0), (-1.0, 1.0), (-1.0, 0.0)]
    wang = [1.0, np.sqrt(0.5), 1.0, np.sqrt(0.5), 1.0]
    if dim == 2:
        ctrl = np.zeros((5, 3, 2))
        wts = np.zeros((5, 3))
        for j in range(5):
            for i in range(3):
                ctrl[j, i] = [radii[i] * dirs[j][0], radii[i] * dirs[j][1]]
                wts[j, i] = wang[j]
        return NURBSMap([2, 2], [kl, ka], ctrl, wts)
    zs = [0.0, 0.5 * height, height]
    ctrl = np.zeros((3, 5, 3, 3))
    wts = np.zeros((3, 5, 3))
    for kz in range(3):
        for j in range(5):
            for i in range(3):
                ctrl[kz, j, i] = [radii[i] * dirs[j][0], radii[i] * dirs[j][1], zs[kz]]
                wts[kz, j, i] = wang[j]
    return NURBSMap([2, 2, 2], [kl, ka, kl], ctrl, wts)


def two_patch_bar(a=0.25, split=0.5, dim=2):
    """Piecewise affine map of [0,1]^dim: direction 1 is degree 1 with a C^0 knot at `split`
    (x_1 = a xi / split on the first patch, a + (1 - a)(xi - split)/(1 - split) on the second),
    the other directions are the identity.  det DF is piecewise constant and jumps at the
    interface unless a = split."""
    k1 = np.array([0.0, 0.0, split, 1.0, 1.0])
    kid = np.array([0.0, 0.0, 1.0, 1.0])
    xs = [0.0, a, 1.0]
    if dim == 1:
        return NURBSMap([1], [k1], np.array(xs)[:, None], np.ones(3))
    if dim == 2:
        ctrl = np.zeros((2, 3, 2))
        for j in range(2):
            for i in range(3):
                ctrl[j, i] = [xs[i], float(j)]
        return NURBSMap([1, 1], [k1, kid], ctrl, np.ones((2, 3)))
    ctrl = np.zeros((2, 2, 3, 3))
    for kz in range(2):
        for j in range(2):
            for i in range(3):
                ctrl[kz, j, i] = [xs[i], float(j), float(kz)]
    return NURBSMap([1, 1, 1], [k1, kid, kid], ctrl, np.ones((2, 2, 3)))
