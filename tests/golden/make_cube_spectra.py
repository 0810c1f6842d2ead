"""Writes the stored full-size spectra under tests/golden/ from the oracle alone.

cube_p2_32_exp_L0.5_top24.json
    The 24 largest eigenvalues of the standard-form IBQ operator A~' (Sec. 4.4.1) on the unit
    cube, degree-2 splines, 32^3 elements (34^3 = 39,304 Greville points), Euclidean
    exponential kernel sigma^2 exp(-|x-x'|/L), sigma = 1, L = 0.5.  The operator is the
    oracle's Algorithm 1 (stages 1-4 `Problem.forward`, stages 6-9 `Problem.backward`) with
    stage 5 done as a product with the dense kernel matrix Gamma (12.4 GB, formed once by
    `oracle.kernels.kernel_matrix` in row blocks), inside ARPACK's implicitly restarted Lanczos
    (`scipy.sparse.linalg.eigsh`, the solver the paper uses, Sec. 4.4.2) at tolerance 1e-13.
    The residual of every stored pair is measured afterwards with the same operator.

cube_p3_48_gauss_L0.3_kron.json
    The separable Gaussian kernel on the unit cube (identity map) makes A~' a Kronecker product
    of three identical 1D operators (Sec. 4.1: every factor of A~' is a Kronecker product when
    Gamma is), so the leading eigenpairs of the 132,651-point cube (degree 3, 48^3 elements,
    L = 0.3) are products of the 1D dense oracle's eigenpairs.  Stored: the 1D eigenvalues and
    eigenvectors (51 x 12, direction-independent) and the index triples (a, b, c) of the 32
    largest products (vector u_c (x) u_b (x) u_a, direction 1 fastest).

Run from the repository root (the first file needs about 20 GB of memory and some minutes):
    python tests/golden/make_cube_spectra.py [exp39k] [gauss133k]
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ibq  # noqa: E402
from oracle.kernels import kernel_matrix  # noqa: E402


def config_hash(cfg):
    return hashlib.sha256(json.dumps(cfg, sort_keys=True).encode()).hexdigest()[:16]


def exp_cube_39k(k=24, tol=1e-13, seed=7):
    from scipy.sparse.linalg import LinearOperator, eigsh
    cfg = {"dim": 3, "p": 2, "ne": 32, "kernel": "exp", "sigma": 1.0, "L": 0.5, "map": "identity"}
    P = ibq.Problem(cfg["dim"], cfg["p"], cfg["ne"], kernel=cfg["kernel"], sigma=cfg["sigma"], L=cfg["L"])
    X, _ = P.points_and_J()
    t0 = time.time()
    Gamma = np.empty((P.Nt, P.Nt))
    rows = 512
    for s in range(0, P.Nt, rows):
        Gamma[s:s + rows] = kernel_matrix(X[s:s + rows], X, P.kernel, P.sigma, P.L)
    t_form = time.time() - t0
    napply = [0]

    def matvec(v):
        napply[0] += 1
        u = P.forward(v.reshape(P.N, -1))           # stages 1-4
        return P.backward(Gamma @ u).reshape(v.shape)   # stage 5 (dense), stages 6-9

    op = LinearOperator((P.N, P.N), matvec=matvec, dtype=np.float64)
    v0 = np.random.default_rng(seed).uniform(-1.0, 1.0, P.N)
    t0 = time.time()
    w, V = eigsh(op, k=k, which="LA", tol=tol, ncv=3 * k, v0=v0)
    t_solve = time.time() - t0
    order = np.argsort(w)[::-1]
    w, V = w[order], V[:, order]
    res = [float(np.linalg.norm(matvec(V[:, i]) - w[i] * V[:, i]) / abs(w[i])) for i in range(k)]
    return {
        "config": cfg, "config_hash": config_hash(cfg), "N": P.N,
        "source": "oracle.ibq.Problem.forward / backward around a dense oracle.kernels.kernel_matrix "
                  "product, scipy.sparse.linalg.eigsh (ARPACK IRLM) at tol %.0e, start vector seed %d"
                  % (tol, seed),
        "eigenvalues": [float(x) for x in w], "relative_residuals": res,
        "operator_applications": napply[0], "seconds_gamma": t_form, "seconds_eigsh": t_solve,
    }


def gauss_cube_133k(k=32, r=12):
    cfg = {"dim": 3, "p": 3, "ne": 48, "kernel": "gauss", "sigma": 1.0, "L": 0.3, "map": "identity"}
    P1 = ibq.Problem(1, cfg["p"], cfg["ne"], kernel="gauss", sigma=1.0, L=cfg["L"])
    mu, U = ibq.standard_eigs(P1.dense_operator())
    # fix each 1D vector's sign (largest-magnitude entry positive) so the file is reproducible
    for j in range(U.shape[1]):
        if U[np.argmax(np.abs(U[:, j])), j] < 0:
            U[:, j] = -U[:, j]
    trip = sorted(((mu[a] * mu[b] * mu[c], a, b, c) for a in range(r) for b in range(r) for c in range(r)),
                  key=lambda t: (-t[0], t[1], t[2], t[3]))[:k]
    return {
        "config": cfg, "config_hash": config_hash(cfg), "N": P1.N ** 3,
        "source": "oracle.ibq.standard_eigs of the 1D oracle.ibq.Problem(1, 3, 48, gauss, L=0.3) "
                  "dense operator; 3D pairs are products (separable kernel, identity map)",
        "mu_1d": [float(x) for x in mu[:r]],
        "u_1d": [[float(x) for x in U[:, j]] for j in range(r)],
        "triples": [[int(a), int(b), int(c)] for _, a, b, c in trip],
        "eigenvalues": [float(t[0]) for t in trip],
    }


def main(argv):
    which = argv[1:] or ["gauss133k", "exp39k"]
    if "gauss133k" in which:
        out = gauss_cube_133k()
        with open(os.path.join(HERE, "cube_p3_48_gauss_L0.3_kron.json"), "w") as f:
            json.dump(out, f, indent=1)
    if "exp39k" in which:
        out = exp_cube_39k()
        with open(os.path.join(HERE, "cube_p2_32_exp_L0.5_top24.json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv)
