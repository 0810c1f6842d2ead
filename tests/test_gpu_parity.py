"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Element-by-element comparisons on seeded synthetic inputs at sizes the oracle finishes in
seconds, spanning several 128/256-point tiles and a ragged tail; the float64 bar is the
matvec relative error 1e-12 (max abs error / max abs value), the float32 bar 2e-5.
"""
import numpy as np
import pytest

from oracle import ibq
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5

CASES = [
    # dim, p, ne, kernel, L, pt, net, lo, hi
    (1, 2, 300, "exp", 0.3, None, None, None, None),
    (2, [2, 3], [23, 17], "gauss", 0.4, None, None, [0.0, -1.0], [2.0, 0.5]),
    (3, 2, [9, 10, 11], "exp", 0.5, None, None, None, None),
    (3, [2, 2, 3], [6, 5, 7], "gauss", 0.3, [3, 2, 3], [8, 7, 9], None, None),
    (2, 2, [20, 20], "exp_sep", 1.0, None, None, None, None),
    (3, 2, [4, 5, 3], "poly", 2, None, None, [0.0, 0.0, 0.0], [1.5, 1.0, 2.0]),
]


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / np.abs(b).max()


def make(kl, case):
    dim, p, ne, kern, L, pt, net, lo, hi = case
    P = ibq.Problem(dim, p, ne, kernel=kern, L=L, pt=pt, net=net, lo=lo, hi=hi, sigma=1.3)
    G = kl.KLProblem(dim, p, ne, kernel=kern, L=L, pt=pt, net=net, lo=lo, hi=hi, sigma=1.3)
    return P, G


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%s" % (c[0], c[3]))
def test_setup_factors_and_points(kl, case):
    P, G = make(kl, case)
    assert (G.N, G.Nt) == (P.N, P.Nt)
    for k, d in enumerate(P.dirs):
        # C_k = B~_k^{-T} M_k L_k^{-T} composed from the oracle's univariate matrices
        ref = np.linalg.solve(d.Bt.T, d.M @ np.linalg.inv(d.L).T)
        assert rel(G.factor(k), ref) < 1e-13
    X, J = G.points()
    Xo, Jo = P.points_and_J()
    assert np.abs(X - Xo).max() < 1e-15 * max(1.0, np.abs(Xo).max())
    assert rel(J, Jo) < 1e-15


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%s" % (c[0], c[3]))
def test_stagewise_parity_fp64(kl, case):
    import torch
    P, G = make(kl, case)
    v = inputs.random_block(P.N, 3, seed=11)
    vd = torch.from_numpy(v.T.copy()).cuda()
    u = G.forward(vd).cpu().numpy().T
    assert rel(u, P.forward(v)) < 1e-13                                    # stages 1-4
    X, _ = P.points_and_J()
    z = G.covmv(torch.from_numpy(u.T.copy()).cuda()).cpu().numpy().T
    assert rel(z, P.stage5(X, u)) < FP64_TOL                               # stage 5
    y = G.backward(torch.from_numpy(z.T.copy()).cuda()).cpu().numpy().T
    assert rel(y, P.backward(z)) < 1e-13                                   # stages 6-9
    yf = G.apply(vd).cpu().numpy().T
    Ap = P.dense_operator()
    assert rel(yf, Ap @ v) < FP64_TOL                                      # all nine stages


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%s" % (c[0], c[3]))
def test_double_float_stage5_meets_fp64_tolerance(kl, case):
    """KL_P_DF64 (double-float arithmetic on the float32 pipe) against the float64 oracle."""
    import torch
    P, G = make(kl, case)
    v = inputs.random_block(P.N, 3, seed=13)
    vd = torch.from_numpy(v.T.copy()).cuda()
    X, _ = P.points_and_J()
    u = P.forward(v)
    z = G.covmv(torch.from_numpy(u.T.copy()).cuda(), precision=kl.KL_P_DF64).cpu().numpy().T
    assert rel(z, P.stage5(X, u)) < FP64_TOL
    y = G.apply(vd, precision=kl.KL_P_DF64).cpu().numpy().T
    assert rel(y, P.dense_operator() @ v) < FP64_TOL


@pytest.mark.parametrize("case", CASES[:4], ids=lambda c: "%dd-%s" % (c[0], c[3]))
def test_apply_fp32(kl, case):
    import torch
    P, G = make(kl, case)
    v = inputs.random_block(P.N, 5, seed=12)
    y = G.apply(torch.from_numpy(v.T.copy()).cuda(), precision=kl.KL_P_FP32).cpu().numpy().T
    assert rel(y, P.dense_operator() @ v) < FP32_TOL
    X, _ = P.points_and_J()
    u = P.forward(v)
    z = G.covmv(torch.from_numpy(u.T.copy()).cuda(), precision=kl.KL_P_FP32).cpu().numpy().T
    assert rel(z, P.stage5(X, u)) < FP32_TOL


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%s" % (c[0], c[3]))
@pytest.mark.parametrize("nvec", [16, 3, 17])
def test_tensor_core_stage5(kl, case, nvec):
    """KL_P_TC32: float32 kernel values split into three bfloat16 terms, tcgen05 MMA with float32
    accumulation in tensor memory; float32-level agreement with the float64 oracle."""
    import torch
    P, G = make(kl, case)
    X, _ = P.points_and_J()
    u = inputs.random_block(P.Nt, nvec, seed=31)
    z = G.covmv(torch.from_numpy(u.T.copy()).cuda(), precision=kl.KL_P_TC32).cpu().numpy().T
    assert rel(z, P.stage5(X, u)) < FP32_TOL
    v = inputs.random_block(P.N, nvec, seed=32)
    y = G.apply(torch.from_numpy(v.T.copy()).cuda(), precision=kl.KL_P_TC32).cpu().numpy().T
    assert rel(y, P.dense_operator() @ v) < FP32_TOL


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dd-%s" % (c[0], c[3]))
@pytest.mark.parametrize("nvec", [32, 3, 33])
def test_tensor_core_fp64_class_stage5(kl, case, nvec):
    """KL_P_TC64: double-float kernel values and float64 u cut into exact bfloat16 slices, slice
    products summed on the tensor cores; float64 tolerance against the float64 oracle."""
    import torch
    P, G = make(kl, case)
    X, _ = P.points_and_J()
    u = inputs.random_block(P.Nt, nvec, seed=41)
    # one vector with a large dynamic range (per-vector power-of-two scaling)
    u[:, 0] *= np.exp(np.linspace(-20.0, 5.0, P.Nt))
    z = G.covmv(torch.from_numpy(u.T.copy()).cuda(), precision=kl.KL_P_TC64).cpu().numpy().T
    zo = P.stage5(X, u)
    for v in range(nvec):
        assert rel(z[:, v], zo[:, v]) < FP64_TOL, v
    v = inputs.random_block(P.N, nvec, seed=42)
    y = G.apply(torch.from_numpy(v.T.copy()).cuda(), precision=kl.KL_P_TC64).cpu().numpy().T
    assert rel(y, P.dense_operator() @ v) < FP64_TOL


def test_tensor_core_fp64_class_zero_and_tiny_vectors(kl):
    """A zero vector gives zero; a vector scaled by 2^-900 gives the scaled product."""
    import torch
    P, G = make(kl, CASES[2])
    X, _ = P.points_and_J()
    u = inputs.random_block(P.Nt, 3, seed=43)
    u[:, 1] = 0.0
    u[:, 2] *= 2.0 ** -900
    z = G.covmv(torch.from_numpy(u.T.copy()).cuda(), precision=kl.KL_P_TC64).cpu().numpy().T
    zo = P.stage5(X, u)
    assert np.all(z[:, 1] == 0.0)
    assert rel(z[:, 0], zo[:, 0]) < FP64_TOL
    assert rel(z[:, 2], zo[:, 2]) < FP64_TOL


@pytest.mark.parametrize("nvec", [1, 2, 7, 16, 17, 33])
def test_block_widths(kl, nvec):
    """Vector groups of the stage-5 kernels (16 in float64, 32 in float32 and on the tensor cores)
    and their tails."""
    import torch
    P, G = make(kl, CASES[2])
    v = inputs.random_block(P.N, nvec, seed=nvec)
    vd = torch.from_numpy(v.T.copy()).cuda()
    ref = P.dense_operator() @ v
    assert rel(G.apply(vd).cpu().numpy().T, ref) < FP64_TOL
    assert rel(G.apply(vd, precision=kl.KL_P_DF64).cpu().numpy().T, ref) < FP64_TOL
    assert rel(G.apply(vd, precision=kl.KL_P_TC64).cpu().numpy().T, ref) < FP64_TOL
    assert rel(G.apply(vd, precision=kl.KL_P_FP32).cpu().numpy().T, ref) < FP32_TOL
    assert rel(G.apply(vd, precision=kl.KL_P_TC32).cpu().numpy().T, ref) < FP32_TOL


def test_deterministic(kl):
    import torch
    _, G = make(kl, CASES[2])
    v = torch.from_numpy(inputs.random_block(G.N, 4, seed=5).T.copy()).cuda()
    a = G.apply(v)
    b = G.apply(v)
    assert torch.equal(a, b)


def test_invalid_arguments(kl):
    import torch
    with pytest.raises(kl.KLError):
        kl.KLProblem(3, 2, 4, kernel="exp", L=-1.0)
    with pytest.raises(kl.KLError):
        kl.KLProblem(4, 2, 4)
    with pytest.raises(kl.KLError):
        kl.KLProblem(2, 0, 4)
    _, G = make(kl, CASES[0])
    with pytest.raises(kl.KLError):
        G.eigs(0)
    # an empty block is a no-op
    e = torch.empty((0, G.N), dtype=torch.float64, device="cuda")
    assert G.apply(e).shape == (0, G.N)


def test_to_bspline(kl):
    """v = L^{-T} v': the B-spline coefficients satisfy v^T Z v = v'^T v' (Sec. 4.1)."""
    import torch
    P, G = make(kl, CASES[1])
    vp = inputs.random_block(P.N, 2, seed=3)
    v = G.to_bspline(torch.from_numpy(vp.T.copy()).cuda()).cpu().numpy().T
    Z = P.kron("Z")
    assert np.abs(v.T @ Z @ v - vp.T @ vp).max() < 1e-12 * np.abs(vp.T @ vp).max()


@pytest.mark.parametrize("dim,p,ne", [(1, 1, 1), (2, 1, [1, 2]), (3, 1, 1), (1, 2, 253)],
                         ids=["2pts", "6pts", "8pts", "255pts"])
def test_tiny_problems_every_precision(kl, dim, p, ne):
    """Degenerate sizes: 2 to 8 points (one partial tile in every kernel, a single row block on
    the tensor cores) and 255 points (one point short of two symmetric tiles), 3 vectors, every
    stage-5 arithmetic against the oracle."""
    import torch
    P = ibq.Problem(dim, p, ne, kernel="exp", L=0.7, sigma=0.9)
    G = kl.KLProblem(dim, p, ne, kernel="exp", L=0.7, sigma=0.9)
    X, _ = P.points_and_J()
    u = inputs.random_block(P.Nt, 3, seed=77)
    ref = P.stage5(X, u)
    ud = torch.from_numpy(u.T.copy()).cuda()
    for prec, tol in ((kl.KL_P_FP64, FP64_TOL), (kl.KL_P_DF64, FP64_TOL), (kl.KL_P_TC64, FP64_TOL),
                      (kl.KL_P_FP32, FP32_TOL), (kl.KL_P_TC32, FP32_TOL)):
        z = G.covmv(ud, precision=prec).cpu().numpy().T
        assert rel(z, ref) < tol, (prec, rel(z, ref))
    v = inputs.random_block(P.N, 2, seed=78)
    y = G.apply(torch.from_numpy(v.T.copy()).cuda()).cpu().numpy().T
    assert rel(y, P.dense_operator() @ v) < FP64_TOL


def test_packed_double_float_pairs_are_bit_identical(kl):
    """The tensor-core float64-class producers evaluate two kernel values per packed float32-pair
    instruction; kl_df2_selftest runs the scalar and the packed double-float code on the same
    random points (spans 1/4 to 64, so the exponential's clamp is reached) for the exponential,
    Gaussian and separable-exponential kernels, their six slices and the slices' double-float
    sum, and counts differing float words: none may differ."""
    assert kl.df2_selftest(1 << 20, seed=7) == 0
    assert kl.df2_selftest(0) == 0
