"""Covariance kernels for the oracle (TEST INFRASTRUCTURE ONLY).

Sec. 3.1 names the exponential and the squared-exponential (Gaussian) kernel
with variance sigma^2 and a correlation length, but prints no formula.  The
readings used here:

  exp       sigma^2 exp(-||x - x'||_2 / L)
  gauss     sigma^2 exp(-||x - x'||_2^2 / L^2)
  exp_sep   sigma^2 exp(-sum_k |x_k - x'_k| / L)     (separable test kernel)
  poly      sigma^2 prod_k (1 + x_k x'_k)^m, m = int(L) (polynomial test kernel)

The differences x - x' are formed coordinate by coordinate (never through
|x|^2 + |x'|^2 - 2 x.x').
"""
import numpy as np

KINDS = ("exp", "gauss", "exp_sep", "poly")


def kernel_matrix(X1, X2, kind, sigma=1.0, L=1.0):
    """Dense Gamma[a, b] = Gamma(X1[a], X2[b]) for point sets X1 (n1 x d), X2 (n2 x d)."""
    X1 = np.atleast_2d(np.asarray(X1, dtype=np.float64))
    X2 = np.atleast_2d(np.asarray(X2, dtype=np.float64))
    s2 = sigma * sigma
    if kind == "poly":
        m = int(L)
        out = np.ones((X1.shape[0], X2.shape[0]))
        for k in range(X1.shape[1]):
            out *= (1.0 + np.outer(X1[:, k], X2[:, k])) ** m
        return s2 * out
    diff = [X1[:, k][:, None] - X2[:, k][None, :] for k in range(X1.shape[1])]
    if kind == "exp":
        r = np.sqrt(sum(d * d for d in diff))
        return s2 * np.exp(-r / L)
    if kind == "gauss":
        r2 = sum(d * d for d in diff)
        return s2 * np.exp(-r2 / (L * L))
    if kind == "exp_sep":
        r1 = sum(np.abs(d) for d in diff)
        return s2 * np.exp(-r1 / L)
    raise ValueError("unknown kernel kind %r" % (kind,))
