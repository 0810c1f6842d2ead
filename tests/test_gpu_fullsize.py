"""Full-size checks at the sizes the bench runs: sampled outputs the oracle computes one by one,
and properties that hold at any size (Kronecker spectrum of a separable kernel, residuals
measured with the oracle's own operator)."""
import numpy as np
import pytest

from oracle import ibq
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


@pytest.fixture(scope="module")
def cube_exp(kl):
    w = inputs.WORKLOADS["cube-p2-32^3-exp-L0.5"]
    P = ibq.Problem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    G = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    return P, G


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "df64"])
def test_stage5_sampled_rows_at_39k_points(kl, cube_exp, prec):
    import torch
    P, G = cube_exp
    X, _ = P.points_and_J()
    u = inputs.random_block(P.Nt, 4, seed=21)
    z = G.covmv(torch.from_numpy(u.T.copy()).cuda(), precision=prec).cpu().numpy().T
    rows = np.random.default_rng(5).choice(P.Nt, size=64, replace=False)
    rows = np.concatenate([rows, [0, P.Nt - 1]])
    ref = P.stage5(X, u, row_index=rows)
    assert rel(z[rows], ref) < 1e-12


def test_contractions_at_39k_points(kl, cube_exp):
    import torch
    P, G = cube_exp
    v = inputs.random_block(P.N, 2, seed=22)
    u = G.forward(torch.from_numpy(v.T.copy()).cuda()).cpu().numpy().T
    assert rel(u, P.forward(v)) < 1e-13
    z = inputs.random_block(P.Nt, 2, seed=23)
    y = G.backward(torch.from_numpy(z.T.copy()).cuda()).cpu().numpy().T
    assert rel(y, P.backward(z)) < 1e-13


def test_eigenpairs_at_39k_points_against_oracle_operator(kl, cube_exp):
    """20 leading pairs from the double-float solver; residuals of the first and the 20th pair
    measured with the oracle's matrix-free float64 operator (Algorithm 1 on the CPU), and the
    eigenvalues agree with the float64 GPU solver."""
    import torch
    P, G = cube_exp
    start = torch.from_numpy(inputs.random_block(G.N, 4, seed=1).T.copy()).cuda()
    ev, vec, info = G.eigs(20, 1e-8, method=0, block=4, start=start, precision=2)
    assert max(info["resid"]) <= 1e-8
    V = vec.cpu().numpy().T
    for i in (0, 19):
        r = P.apply(V[:, i], stage5_rows=512) - ev[i] * V[:, i]
        assert np.linalg.norm(r) <= 1.5e-8 * abs(ev[i])
    ev64, _, _ = G.eigs(20, 1e-8, method=0, block=4, start=start, want_vectors=False)
    assert np.abs(ev - ev64).max() / ev64[0] < 1e-10


def test_gaussian_cube_at_133k_points_kronecker_spectrum(kl):
    """Unit cube, p=3, 48^3 elements (132,651 points), Gaussian kernel L=0.3: the kernel is a
    product over coordinates and the map is the identity, so A~' = A~'_3 (x) A~'_2 (x) A~'_1 and the
    spectrum is every product of three 1D eigenvalues (1D operator from the dense oracle)."""
    import torch
    w = inputs.WORKLOADS["cube-p3-48^3-gauss-L0.3"]
    mu = np.linalg.eigvalsh(ibq.Problem(1, w["p"], w["ne"], kernel="gauss", L=w["L"]).dense_operator())[::-1][:20]
    ref = np.sort(np.einsum("i,j,k->ijk", mu, mu, mu).ravel())[::-1][:20]
    G = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    start = torch.from_numpy(inputs.random_block(G.N, 16, seed=1).T.copy()).cuda()
    ev, _, info = G.eigs(20, 1e-8, method=1, block=16, start=start, precision=2, want_vectors=False)
    assert max(info["resid"]) <= 1e-8
    assert np.abs(ev - ref).max() / ref[0] < 1e-10
