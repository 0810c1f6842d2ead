"""Learned warm start for the eigensolver (no counterpart in the paper).

A small network maps the parameters of a quarter-annulus KL problem (correlation length L,
kernel type, inner and outer radius) to k standard-form vectors of a coarse trial space
(degree p, ne_c elements per direction).  It is trained on eigenvectors that the solver itself
computes on coarse meshes, with the loss on orthogonal projectors (invariant under rotations
and sign flips of the predicted vectors).  For a fine problem of the same degree whose
element counts are multiples of ne_c, the prediction is carried exactly to the fine space
(kl_prolong: every coarse spline is a fine spline) and becomes the start block of kl_eigs.
When the warm-started solve does not converge within its restart budget, the problem is
solved again from the seeded random start (the method without the network).

Every numerical step runs in the library's kernels: the network's forward and backward
passes and Adam (kl_mlp_*), the coarse solves, the prolongation and the fine solve; this
module only builds the problems, moves tensors between them and keeps the bookkeeping.
"""
import math
import time

import numpy as np

from . import _binding as B
from .inputs import quarter_annulus_net

N_FEATURES = 4


def features(prm):
    """Network inputs of one parameter set: log L, +1 (exponential) / -1 (Gaussian), 5 (r_in - 1),
    5 (r_out - 2) (all of order one on the ranges used)."""
    return [math.log(prm["L"]), 1.0 if prm["kernel"] == "exp" else -1.0, 5.0 * (prm["r_in"] - 1.0),
            5.0 * (prm["r_out"] - 2.0)]


def problem(prm, p, ne, height=1.0, sigma=1.0):
    """The KL problem of one parameter set on the quarter annulus (degree p, ne elements per
    direction, the NURBS net of quarter_annulus_net)."""
    net = quarter_annulus_net(prm["r_in"], prm["r_out"], height, 3)
    return B.KLProblem(3, p, ne, kernel=prm["kernel"], sigma=sigma, L=prm["L"], nurbs=net)


class WarmStart:
    """Network + coarse space.  k: number of predicted vectors (the start block width);
    width x depth: hidden layers (tanh); seed: initial weights."""

    def __init__(self, p=3, ne_coarse=16, k=32, width=256, depth=4, seed=5):
        self.p, self.ne_c, self.k = int(p), int(ne_coarse), int(k)
        self.n = (self.ne_c + self.p) ** 3          # open uniform knots: ne + p splines per direction
        # targets are the eigenvectors scaled by sqrt(n) (entries of order one, like the outputs of
        # the initial network); the projector loss is then n^2 times that of unit vectors
        self.scale = math.sqrt(self.n)
        self.net = B.MLP(N_FEATURES, width, depth, self.k * self.n, seed)
        self.history = []

    # ---- training data ------------------------------------------------------------------
    def targets(self, params, tol=1e-4, block=16, method=0, precision=B.KL_P_FP32, maxiter=60, batch=64):
        """Solve every coarse problem for its k leading eigenvectors, `batch` problems at a time
        through kl_eigs_batched (one shared stage-5 launch per step; batch=1 solves them one by
        one with kl_eigs).  By default the plain method runs in float32 to residual 1e-4: the
        targets then span the eigenspaces to ~1e-3, far below the network's own error (sines
        of a few 1e-2).  Returns (X, T, stats): X (S, 4) and T (S, k n) float32 CUDA tensors
        (vector j of sample s at T[s, j n:(j+1) n], scaled by sqrt(n))."""
        import torch
        X = torch.tensor([features(q) for q in params], dtype=torch.float32, device="cuda")
        T = torch.empty((len(params), self.k * self.n), dtype=torch.float32, device="cuda")
        applies, unconv = 0, 0
        t0 = time.perf_counter()
        for c0 in range(0, len(params), max(1, batch)):
            chunk = params[c0:c0 + max(1, batch)]
            probs = [problem(q, self.p, self.ne_c) for q in chunk]
            if len(probs) > 1:
                _, vecs, infos, _, _ = B.eigs_batched(probs, self.k, tol=tol, method=method, block=block,
                                                      precision=precision, maxiter=maxiter)
            else:
                _, v, info = probs[0].eigs(self.k, tol=tol, method=method, block=block, precision=precision,
                                           maxiter=maxiter, raise_on_nonconv=False)
                vecs, infos = [v], [info]
            for j, (v, info) in enumerate(zip(vecs, infos)):
                T[c0 + j] = (v * self.scale).to(torch.float32).reshape(-1)
                applies += info["applies"]
                unconv += int(info["converged"] < self.k)
            for pr in probs:
                pr.close()
        torch.cuda.synchronize()
        return X, T, {"solves": len(params), "seconds": time.perf_counter() - t0, "applies": applies,
                      "not_converged": unconv}

    def fit(self, X, T, epochs=200, batch=64, lr=1e-3, seed=6, stages=8):
        """Adam epochs over (X, T) with a stepwise cosine decay of the learning rate (`stages`
        constant pieces); returns the per-epoch mean loss of unit-norm vectors
        (||Y Y^T - V V^T||_F^2 / k)."""
        t0 = time.perf_counter()
        stages = max(1, min(int(stages), int(epochs)))
        hist = []
        done = 0
        for i in range(stages):
            e = (epochs * (i + 1)) // stages - done
            if e <= 0:
                continue
            lr_i = lr * 0.5 * (1.0 + math.cos(math.pi * (i + 0.5) / stages))
            hist += list(self.net.train(X, T, self.k, self.n, e, min(batch, X.shape[0]), lr_i, seed + i))
            done += e
        hist = np.asarray(hist) / float(self.n) ** 2
        self.history += list(hist)
        self.fit_seconds = time.perf_counter() - t0
        return hist

    # ---- prediction ---------------------------------------------------------------------
    def predict(self, prm):
        """(k, n) float64 standard-form vectors of the coarse space."""
        import torch
        x = torch.tensor([features(prm)], dtype=torch.float32, device="cuda")
        return self.net.forward(x).reshape(self.k, self.n).to(torch.float64) / self.scale

    def start_block(self, fine, prm):
        """The prediction carried to the trial space of `fine` (same degree, element counts a
        multiple of the coarse ones): (k, N_fine) float64."""
        coarse = problem(prm, self.p, self.ne_c)
        try:
            return B.prolong(coarse, fine, self.predict(prm))
        finally:
            coarse.close()

    def solve(self, fine, prm, nev, tol=1e-8, maxiter=40, fallback=True, block=None, **eig_kw):
        """The nev leading eigenpairs of `fine` from the warm start.  By default the k predicted
        vectors form the start block (block = k, basis 3 k, tensor-core float32 first phase for
        blocks wider than 16); with block < k they are compressed
        by Rayleigh-Ritz to the `block` leading Ritz vectors (kl_eig_opts.nstart).  When the
        warm solve has not converged after `maxiter` restarts, or the prediction holds NaN or
        Inf, the seeded random start with the same options takes over (fallback=True).  Returns (evals, evecs, info) with
        info['path'] = 'warm' | 'fallback' and info['warm'] = the warm attempt's info."""
        import torch
        kw = dict(method=1, precision=B.KL_P_TC64)
        kw.update(eig_kw)
        block = self.k if block is None else min(int(block), self.k)
        if block == self.k:
            kw.setdefault("ncv", max(3 * block, -(-(nev + 2 * block) // block) * block))
        if block > 16:
            # a tensor-core float32 launch costs the same for up to 32 vectors: for wide start
            # blocks it is the cheaper first phase (the scalar float32 kernel's cost grows with the
            # block width)
            kw.setdefault("low_precision", B.KL_P_TC32)
        t0 = time.perf_counter()
        start = self.start_block(fine, prm).contiguous()
        torch.cuda.synchronize()
        t_start = time.perf_counter() - t0
        try:
            ev, vecs, info = fine.eigs(nev, tol=tol, block=block, start=start, maxiter=maxiter,
                                       raise_on_nonconv=False, **kw)
        except B.KLError as err:
            # a prediction with NaN or Inf (KL_ERR_NUMERIC) is a failed warm start, not a failed solve
            if not fallback or B.STATUS.get(err.status) != "KL_ERR_NUMERIC":
                raise
            info = {"converged": -1, "error": str(err)}
        info["ms_start_block"] = 1e3 * t_start
        if info["converged"] >= nev or not fallback:
            info["path"] = "warm"
            return ev, vecs, info
        ev2, vecs2, info2 = fine.eigs(nev, tol=tol, block=block, **kw)
        info2["path"] = "fallback"
        info2["warm"] = info
        return ev2, vecs2, info2
