"""Closed-form eigenvalues of the 1D exponential covariance kernel (TEST INFRASTRUCTURE ONLY).

The Remark in Sec. 6.1 validates the 1D reference spectrum against the
analytic solution it cites (Ghanem and Spanos, Ch. 2.3.3).  For the kernel
sigma^2 exp(-|x - x'| / ell) on the interval [-a, a], with c = 1 / ell, the
eigenvalues are

    lambda = sigma^2 * 2 c / (omega^2 + c^2),

where omega runs over the positive roots of

    c - omega tan(omega a) = 0     (even eigenfunctions, cos(omega x))
    omega + c tan(omega a) = 0     (odd eigenfunctions,  sin(omega x)).

Each equation has exactly one root in every branch of tan: the even roots lie
in (j pi, j pi + pi/2) / a and the odd roots in (j pi + pi/2, (j+1) pi) / a,
j = 0, 1, 2, ...  Roots are found by bracketed bisection (scipy brentq).  The
1D eigenvalues of the separable kernel on a box are products of these.
"""
import math

import numpy as np
from scipy.optimize import brentq


def exp_kernel_1d(num, ell=1.0, length=1.0, sigma=1.0):
    """Largest ``num`` eigenvalues (descending) of sigma^2 exp(-|x-x'|/ell) on an interval of given length."""
    a = 0.5 * length
    c = 1.0 / ell
    eps = 1e-13
    vals = []
    for j in range(num):
        lo, hi = j * math.pi / a, (j * math.pi + 0.5 * math.pi) / a
        f_even = lambda w: c - w * math.tan(w * a)
        w_even = brentq(f_even, lo + eps, hi - eps, xtol=1e-15, rtol=1e-15, maxiter=500)
        vals.append(2.0 * c / (w_even * w_even + c * c))
        lo, hi = (j * math.pi + 0.5 * math.pi) / a, ((j + 1) * math.pi) / a
        f_odd = lambda w: w + c * math.tan(w * a)
        w_odd = brentq(f_odd, lo + eps, hi - eps, xtol=1e-15, rtol=1e-15, maxiter=500)
        vals.append(2.0 * c / (w_odd * w_odd + c * c))
    vals = sorted(vals, reverse=True)[:num]
    return sigma * sigma * np.array(vals)


def exp_separable_box(num, ell, lengths, sigma=1.0, per_dir=None):
    """Largest ``num`` eigenvalues of the separable kernel sigma^2 exp(-sum_k |x_k - x'_k| / ell) on a box.

    The operator is the tensor product of 1D operators, so its eigenvalues are all products
    lambda^(1)_{i1} ... lambda^(d)_{id} of 1D eigenvalues (sigma^2 counted once).
    """
    per_dir = per_dir or num
    lists = [exp_kernel_1d(per_dir, ell, Lk, 1.0) for Lk in lengths]
    prods = np.array([1.0])
    for lst in lists:
        prods = np.outer(prods, lst).ravel()
    return sigma * sigma * np.sort(prods)[::-1][:num]
