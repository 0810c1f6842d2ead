"""Interpolation-based-quadrature (IBQ) Galerkin discretisation, written out densely,
and the matrix-free operator of Algorithm 1 (TEST INFRASTRUCTURE ONLY).

Notation follows the paper:
  Z   = Z_d (x) ... (x) Z_1          univariate B-spline mass matrices (Sec. 3.5)
  L   = L_d (x) ... (x) L_1, Z_k = L_k L_k^T                    (Sec. 4.1, eq. cholesky)
  B~  = B~_d (x) ... (x) B~_1        collocation at Greville points (Sec. 4.2)
  M   = M_d (x) ... (x) M_1, M_k[i, j] = int B~_i B_j       (Sec. 4.3)
  J   = diag(sqrt(det DF)) at the mapped Greville points          (Sec. 4.4.1)
  A~  = M^T B~^{-1} J Gamma J B~^{-T} M                            (Sec. 4.3)
  A~' = L^{-1} A~ L^{-T}                                            (Sec. 4.4.1)

Vectors use the paper's vec ordering (Sec. 2.2): index i = i_1 + i_2 n_1 + ...,
i.e. i_1 runs fastest; a tensor is stored as a C-order array [n_d, ..., n_1].
"""
import numpy as np
import scipy.linalg as sla

from . import bspline
from .kernels import kernel_matrix


class Direction:
    """Univariate data of one parametric direction k (trial space p, ne; interpolation space pt, net).

    `interfaces`: patch interfaces of a multipatch domain (Sec. 3.6) in this direction, interior
    breakpoints of both uniform meshes; the trial space is C^0 there and the interpolation space
    C^{-1} (Sec. 6.2, Example 1-1), whose two Greville abscissae at the knot are evaluated from
    the left and from the right."""

    def __init__(self, p, ne, pt=None, net=None, interfaces=()):
        self.p, self.ne = int(p), int(ne)
        self.pt = int(pt if pt else p)
        self.net = int(net if net else ne)
        self.interfaces = tuple(interfaces)
        self.t = bspline.knots_with_interfaces(self.p, self.ne, self.interfaces, self.p)
        self.tt = bspline.knots_with_interfaces(self.pt, self.net, self.interfaces, self.pt + 1)
        self.n = bspline.dimension(self.t, self.p)
        self.nt = bspline.dimension(self.tt, self.pt)
        self.xi = bspline.greville(self.tt, self.pt)              # Greville abscissae of B~
        self.side = bspline.greville_sides(self.tt, self.pt)      # -1: left limit at a C^{-1} knot
        self.Z = bspline.gramian(self.t, self.p)                   # eq. univariate_mass_matrix
        self.L = np.linalg.cholesky(self.Z)                        # eq. cholesky (lower)
        self.M = bspline.mass_matrix(self.tt, self.pt, self.t, self.p)   # eq. univariate_mass_matrix2
        self.Bt = bspline.collocation_matrix(self.tt, self.pt)     # eq. interpolation_matrix
        self.Bt_lu = sla.lu_factor(self.Bt)


class BoxMap:
    """Affine map F(xh) = lo + (hi - lo) * xh of [0,1]^d onto a box; det DF is constant."""

    def __init__(self, lo, hi):
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)

    def __call__(self, xh, sides=None):
        return self.lo + (self.hi - self.lo) * xh

    def detDF(self, xh, sides=None):
        return np.full(xh.shape[0], np.prod(self.hi - self.lo))


class Problem:
    """One discretised KL problem: directions, geometry map and covariance kernel."""

    def __init__(self, dim, p, ne, kernel="exp", sigma=1.0, L=1.0, pt=None, net=None,
                 lo=None, hi=None, geom=None, interfaces=None):
        def per_dir(v):
            return list(v) if np.ndim(v) else [v] * dim
        p, ne = per_dir(p), per_dir(ne)
        pt = per_dir(pt) if pt is not None else [None] * dim
        net = per_dir(net) if net is not None else [None] * dim
        itf = list(interfaces) if interfaces is not None else [()] * dim
        self.dim = dim
        self.dirs = [Direction(p[k], ne[k], pt[k], net[k], itf[k]) for k in range(dim)]
        # geometry map F: the affine box map by default, or any object with F(xh) and detDF(xh)
        # (e.g. a NURBS map, oracle.nurbs.NURBSMap)
        self.geom = geom if geom is not None else BoxMap(lo if lo is not None else [0.0] * dim,
                                                         hi if hi is not None else [1.0] * dim)
        self.kernel, self.sigma, self.L = kernel, float(sigma), float(L)
        self.N = int(np.prod([d.n for d in self.dirs]))
        self.Nt = int(np.prod([d.nt for d in self.dirs]))

    # -- Greville grid -----------------------------------------------------------------
    def parametric_points(self, sides=False):
        """Tensor Greville grid in vec order (k_1 fastest): array Nt x d (and, with sides=True,
        the per-direction evaluation sides of every point)."""
        grids = np.meshgrid(*[d.xi for d in reversed(self.dirs)], indexing="ij")
        # grids[j] varies along axis j of the C-order array [nt_d, ..., nt_1]
        cols = [grids[self.dim - 1 - k].ravel() for k in range(self.dim)]
        xh = np.stack(cols, axis=1)
        if not sides:
            return xh
        sg = np.meshgrid(*[d.side for d in reversed(self.dirs)], indexing="ij")
        return xh, np.stack([sg[self.dim - 1 - k].ravel() for k in range(self.dim)], axis=1)

    def points_and_J(self):
        """Mapped Greville points X = F(xh) and J = sqrt(det DF(xh)) (Sec. 4.4.1); at a patch
        interface det DF is taken from the side the point's interpolation function lives on."""
        xh, sd = self.parametric_points(sides=True)
        return self.geom(xh, sd), np.sqrt(self.geom.detDF(xh, sd))

    # -- Kronecker factors expanded (Sec. 2.2 eq. kron_*) -------------------------------
    def kron(self, attr):
        mats = [getattr(d, attr) for d in reversed(self.dirs)]   # D_d (x) ... (x) D_1
        out = mats[0]
        for m in mats[1:]:
            out = np.kron(out, m)
        return out

    # -- dense IBQ matrices (Sec. 4.2 - 4.4.1) ------------------------------------------
    def dense(self):
        """Return dict with Gamma, G, G~, A~, Z, L and A~' formed densely, step by step."""
        X, J = self.points_and_J()
        Gamma = kernel_matrix(X, X, self.kernel, self.sigma, self.L)      # kernel at Greville pairs
        G = J[:, None] * Gamma * J[None, :]                               # G = J Gamma J
        Bt = self.kron("Bt")
        Gt = np.linalg.solve(Bt, np.linalg.solve(Bt, G).T).T              # G~ = B~^{-1} G B~^{-T}
        M = self.kron("M")
        At = M.T @ Gt @ M                                                 # A~ = M^T G~ M
        Z = self.kron("Z")
        Lf = self.kron("L")
        tmp = sla.solve_triangular(Lf, At, lower=True)                    # L^{-1} A~
        Ap = sla.solve_triangular(Lf, tmp.T, lower=True).T                # (L^{-1} A~) L^{-T}
        return {"Gamma": Gamma, "G": G, "Gt": Gt, "At": At, "Z": Z, "L": Lf, "Ap": Ap, "X": X, "J": J}

    def dense_operator(self):
        """A~' as a dense symmetric matrix (symmetrised against round-off)."""
        Ap = self.dense()["Ap"]
        return 0.5 * (Ap + Ap.T)

    # -- matrix-free application, Algorithm 1 --------------------------------------------
    def _modes(self, v, nvec, sizes):
        return v.reshape((nvec,) + tuple(reversed(sizes)))

    @staticmethod
    def _along(T, axis, fn):
        """Apply fn (acting on the leading axis of a 2D array) along tensor axis."""
        Tm = np.moveaxis(T, axis, 0)
        shape = Tm.shape
        out = fn(Tm.reshape(shape[0], -1))
        return np.moveaxis(out.reshape((out.shape[0],) + shape[1:]), 0, axis)

    def apply(self, v, stage5_rows=2048):
        """y = A~' v for v of shape (N,) or (N, nvec), following the nine stages of Algorithm 1.

        Stage 5 evaluates Gamma on the fly in row blocks of ``stage5_rows`` rows.
        """
        v = np.asarray(v, dtype=np.float64)
        single = v.ndim == 1
        V = v.reshape(self.N, -1)
        nvec = V.shape[1]
        d = self.dim
        n = [dd.n for dd in self.dirs]
        nt = [dd.nt for dd in self.dirs]
        T = V.T.reshape((nvec,) + tuple(reversed(n)))       # [vec, n_d, ..., n_1]
        ax = lambda k: d - k                                 # tensor axis of direction k (0-based)
        # stage 1: V = L^{-T} v   (back substitution with L_k^T in every direction)
        for k, dd in enumerate(self.dirs):
            T = self._along(T, ax(k), lambda A, dd=dd: sla.solve_triangular(dd.L.T, A, lower=False))
        # stage 2: X = M V
        for k, dd in enumerate(self.dirs):
            T = self._along(T, ax(k), lambda A, dd=dd: dd.M @ A)
        # stage 3: Y = B~^{-T} X  (LU factors of B~_k)
        for k, dd in enumerate(self.dirs):
            T = self._along(T, ax(k), lambda A, dd=dd: sla.lu_solve(dd.Bt_lu, A, trans=1))
        X, J = self.points_and_J()
        Y = T.reshape(nvec, self.Nt).T * J[:, None]          # stage 4: Y' = J . Y
        Zp = self.stage5(X, Y, stage5_rows)                  # stage 5: Z' = Gamma Y'
        Zs = Zp * J[:, None]                                 # stage 6: Z = J . Z'
        T = Zs.T.reshape((nvec,) + tuple(reversed(nt)))
        # stage 7: Y = B~^{-1} Z
        for k, dd in enumerate(self.dirs):
            T = self._along(T, ax(k), lambda A, dd=dd: sla.lu_solve(dd.Bt_lu, A, trans=0))
        # stage 8: V = M^T Y
        for k, dd in enumerate(self.dirs):
            T = self._along(T, ax(k), lambda A, dd=dd: dd.M.T @ A)
        # stage 9: v' = L^{-1} V
        for k, dd in enumerate(self.dirs):
            T = self._along(T, ax(k), lambda A, dd=dd: sla.solve_triangular(dd.L, A, lower=True))
        out = T.reshape(nvec, self.N).T
        return out[:, 0] if single else out

    def stage5(self, X, Y, rows=2048, row_index=None):
        """Z'[k] = sum_l Gamma(x_k, x_l) Y[l] with Gamma evaluated on the fly, row block by row block.

        If row_index is given, only those rows are computed (for sampled checks at large sizes).
        """
        Y = np.asarray(Y, dtype=np.float64).reshape(X.shape[0], -1)
        idx = np.arange(X.shape[0]) if row_index is None else np.asarray(row_index)
        out = np.empty((len(idx), Y.shape[1]))
        for s in range(0, len(idx), rows):
            blk = idx[s:s + rows]
            out[s:s + len(blk)] = kernel_matrix(X[blk], X, self.kernel, self.sigma, self.L) @ Y
        return out

    # -- the two halves of Algorithm 1 around stage 5, exposed for stage-wise checks ------
    def forward(self, v):
        """Stages 1-4: u = J . B~^{-T} M L^{-T} v'  (N x nvec -> Nt x nvec)."""
        v = np.asarray(v, dtype=np.float64).reshape(self.N, -1)
        nvec = v.shape[1]
        d = self.dim
        T = v.T.reshape((nvec,) + tuple(reversed([dd.n for dd in self.dirs])))
        for k, dd in enumerate(self.dirs):
            T = self._along(T, d - k, lambda A, dd=dd: sla.solve_triangular(dd.L.T, A, lower=False))
        for k, dd in enumerate(self.dirs):
            T = self._along(T, d - k, lambda A, dd=dd: dd.M @ A)
        for k, dd in enumerate(self.dirs):
            T = self._along(T, d - k, lambda A, dd=dd: sla.lu_solve(dd.Bt_lu, A, trans=1))
        _, J = self.points_and_J()
        return T.reshape(nvec, self.Nt).T * J[:, None]

    def backward(self, z):
        """Stages 6-9: y = L^{-1} M^T B~^{-1} (J . z)  (Nt x nvec -> N x nvec)."""
        z = np.asarray(z, dtype=np.float64).reshape(self.Nt, -1)
        nvec = z.shape[1]
        d = self.dim
        _, J = self.points_and_J()
        T = (z * J[:, None]).T.reshape((nvec,) + tuple(reversed([dd.nt for dd in self.dirs])))
        for k, dd in enumerate(self.dirs):
            T = self._along(T, d - k, lambda A, dd=dd: sla.lu_solve(dd.Bt_lu, A, trans=0))
        for k, dd in enumerate(self.dirs):
            T = self._along(T, d - k, lambda A, dd=dd: dd.M.T @ A)
        for k, dd in enumerate(self.dirs):
            T = self._along(T, d - k, lambda A, dd=dd: sla.solve_triangular(dd.L, A, lower=True))
        return T.reshape(nvec, self.N).T


def generalized_eigs(At, Z, k=None):
    """Largest k eigenvalues (descending) and Z-orthonormal vectors of A~ v = lambda Z v (LAPACK sygvd)."""
    N = At.shape[0]
    k = N if k is None else k
    w, V = sla.eigh(0.5 * (At + At.T), Z, subset_by_index=[N - k, N - 1])
    return w[::-1], V[:, ::-1]


def standard_eigs(Ap, k=None):
    """Largest k eigenvalues (descending) and orthonormal vectors of the symmetric A~'."""
    N = Ap.shape[0]
    k = N if k is None else k
    w, V = sla.eigh(0.5 * (Ap + Ap.T), subset_by_index=[N - k, N - 1])
    return w[::-1], V[:, ::-1]
