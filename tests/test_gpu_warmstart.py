"""The learned warm start through the C ABI: the network's forward pass, loss, gradient and Adam
step against the float64 oracle with the same bfloat16 roundings (oracle/mlp.py), the exact
prolongation against the Kronecker product of the 1D maps (oracle/prolong.py), and what a
trained network gains over the random start on a small quarter-annulus problem."""
import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import prolong as oprol

pytestmark = pytest.mark.gpu


def orthonormal_targets(rng, batch, n, k):
    """(batch, k n) float32 rows holding k orthonormal vectors of length n each."""
    T = np.zeros((batch, k * n))
    for s in range(batch):
        Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
        T[s] = Q.T.reshape(-1)
    return T.astype(np.float32)


def as64(params):
    Ws, bs = params
    return [W.astype(np.float64) for W in Ws], [b.astype(np.float64) for b in bs]


def abs_bound(Ws, x):
    """Per-output sum of |terms| through the network (bf16-rounded magnitudes): the scale against
    which a float32 sum and an occasional one-ulp bfloat16 difference in a layer input are measured."""
    h = np.abs(omlp.bf16(x))
    for l, W in enumerate(Ws):
        h = h @ np.abs(omlp.bf16(W))
        if l < len(Ws) - 1:
            h = np.minimum(h, 1.0)      # |tanh| <= 1
    return h


# n_in, width, depth, k, n, batch: ragged tiles (width 80, batch 37, n_out 600 = 4 M-tiles + 88
# rows), a split contraction over n_out in dH = dZ W^T, three N-tiles for batch 530, inner
# dimensions that are not multiples of 8 (width 20, n_out 21: the float32-FMA GEMM), and a
# first layer on the tensor cores (8 inputs)
SHAPES = [(4, 80, 3, 4, 150, 37), (4, 64, 1, 2, 40, 9), (5, 48, 2, 3, 200, 530), (3, 20, 2, 3, 7, 5),
          (8, 32, 1, 2, 64, 16)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "w%d-d%d-b%d" % (s[1], s[2], s[5]))
def test_forward_matches_oracle(kl, shape):
    import torch
    n_in, width, depth, k, n, batch = shape
    rng = np.random.default_rng(11)
    net = kl.MLP(n_in, width, depth, k * n, seed=3)
    Ws, bs = as64(net.get_params())
    bs = [rng.uniform(-0.3, 0.3, b.shape) for b in bs]
    net.set_params(Ws, bs)
    Ws, bs = as64(net.get_params())
    x = rng.uniform(-1.5, 1.5, (batch, n_in)).astype(np.float32)
    out = net.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref, _ = omlp.forward(Ws, bs, x.astype(np.float64), rounding=True)
    ref_exact, _ = omlp.forward(Ws, bs, x.astype(np.float64), rounding=False)
    scale = abs_bound(Ws, x)
    err = np.abs(out - ref)
    # float32 sums: a few units of 2^-24 of the absolute scale; a rare one-ulp (2^-8) difference in a
    # bfloat16-rounded hidden input is allowed at the 2^-8 level of that scale
    assert np.all(err <= 2.0 ** -8 * scale + 1e-30), err.max()
    assert np.median(err / scale) < 1e-6
    # the roundings matter: the exact float64 network is much farther away than the kernel
    assert np.abs(ref_exact - ref).max() > 20 * np.median(err)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "w%d-d%d-b%d" % (s[1], s[2], s[5]))
def test_loss_and_gradient_match_oracle(kl, shape):
    """Loss and gradients of the tensor-core network against the oracle, which models every
    bfloat16 rounding of the kernels.  The two still differ because the kernels form their float32
    sums in another order than the float64 oracle: where such a sum lies within 2^-24 of a
    bfloat16 rounding boundary, the rounded factor comes out one bfloat16 unit (2^-8 of itself)
    apart.  The backward pass rounds the layer input h and the propagated gradient d of every
    layer, and a flip in d at one layer reaches every earlier layer, so a weight-gradient entry of
    the first of four layers can carry up to about four such flips per summand: 4 x 2^-8 = 1.6e-2
    of the sum of its summands' magnitudes, which for these random inputs stays within about the
    largest gradient entry.  Hence the bar 2e-2 x max|ref| on the largest error.  Flips are rare
    (most sums are far from a boundary), so the median error sits at the float32 level: the second
    bar, 1e-3 x max|ref|, is loose for it on purpose and catches a systematic error such as a
    missing rounding or a transposed product."""
    import torch
    n_in, width, depth, k, n, batch = shape
    rng = np.random.default_rng(12)
    net = kl.MLP(n_in, width, depth, k * n, seed=4)
    Ws, bs = as64(net.get_params())
    Ws[-1] = Ws[-1] / np.sqrt(n)
    bs = [rng.uniform(-0.2, 0.2, b.shape) for b in bs]
    net.set_params(Ws, bs)
    Ws, bs = as64(net.get_params())
    x = rng.uniform(-1.0, 1.0, (batch, n_in)).astype(np.float32)
    T = orthonormal_targets(rng, batch, n, k)
    loss, (dWs, dbs) = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(T).cuda(), k, n)
    out, cache = omlp.forward(Ws, bs, x.astype(np.float64), rounding=True)
    Vs = np.stack([T[s].astype(np.float64).reshape(k, n).T for s in range(batch)])
    ref_loss, gout = omlp.projector_loss(out, Vs, k)
    rdW, rdb = omlp.backward(Ws, bs, cache, gout, rounding=True)
    assert abs(float(loss.mean()) - ref_loss) <= 1e-4 * abs(ref_loss)
    for l in range(len(Ws)):
        for g, r in ((dWs[l], rdW[l]), (dbs[l], rdb[l])):
            e = np.abs(g.astype(np.float64) - r)
            assert e.max() <= 2e-2 * np.abs(r).max(), (l, e.max(), np.abs(r).max())
            assert np.median(e) <= 1e-3 * np.abs(r).max(), (l, np.median(e))


def test_adam_step_matches_oracle(kl):
    import torch
    n_in, width, depth, k, n, batch = 4, 40, 2, 3, 30, 24
    rng = np.random.default_rng(13)
    net = kl.MLP(n_in, width, depth, k * n, seed=8)
    Ws0, bs0 = as64(net.get_params())
    x = torch.from_numpy(rng.uniform(-1, 1, (batch, n_in)).astype(np.float32)).cuda()
    T = torch.from_numpy(orthonormal_targets(rng, batch, n, k)).cuda()
    _, (gW, gb) = net.loss_grad(x, T, k, n)
    lr = 1e-3
    net.train(x, T, k, n, epochs=1, batch=batch, lr=lr, seed=1)       # one step over the whole set
    Ws1, bs1 = as64(net.get_params())
    for P0, G, P1 in list(zip(Ws0, gW, Ws1)) + list(zip(bs0, gb, bs1)):
        g = G.astype(np.float64).ravel()
        ref = omlp.adam_step(P0.ravel().copy(), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
        big = np.abs(g) > 1e-3 * np.abs(g).max()
        d = np.abs(P1.ravel() - ref)
        assert np.all(d[big] <= 2e-3 * lr + 1e-6 * np.abs(ref[big])), d[big].max()
        assert np.all(d <= 2 * lr + 1e-6)


def test_training_lowers_loss(kl):
    """Targets that depend smoothly on the input (rotations of a fixed frame): Adam epochs lower
    the projector loss by a large factor."""
    import torch
    rng = np.random.default_rng(14)
    k, n, S = 3, 60, 128
    Q0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    X = rng.uniform(-1, 1, (S, 2))
    T = np.zeros((S, k * n), np.float32)
    for s in range(S):
        c, sn = np.cos(X[s, 0]), np.sin(X[s, 0])
        V = Q0[:, :k].copy()
        V[:, 0] = c * Q0[:, 0] + sn * Q0[:, k]
        V[:, 1] = np.cos(X[s, 1]) * Q0[:, 1] + np.sin(X[s, 1]) * Q0[:, k + 1]
        T[s] = V.T.reshape(-1)
    net = kl.MLP(2, 64, 2, k * n, seed=1)
    Ws, bs = net.get_params()
    Ws[-1] = Ws[-1] / np.sqrt(n)
    net.set_params(Ws, bs)
    hist = net.train(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(T).cuda(), k, n,
                     epochs=150, batch=32, lr=3e-3, seed=2)
    assert hist[-1] < 0.05 * hist[0], (hist[0], hist[-1])


PROLONG_CASES = [
    # dim, p, ne_coarse, ne_fine
    (1, 2, [3], [9]),
    (2, 3, [2, 3], [4, 6]),
    (3, 2, [2, 3, 2], [4, 3, 6]),
    (3, 3, [2, 2, 3], [6, 4, 3]),
]


@pytest.mark.parametrize("case", PROLONG_CASES, ids=lambda c: "%dd-p%d" % (c[0], c[1]))
def test_prolong_matches_oracle(kl, case):
    import torch
    dim, p, nc, nf = case
    C = kl.KLProblem(dim, p, nc, kernel="exp", L=0.5)
    F = kl.KLProblem(dim, p, nf, kernel="exp", L=0.5)
    rng = np.random.default_rng(15)
    v = rng.standard_normal((5, C.N))
    y = kl.prolong(C, F, torch.from_numpy(v).cuda()).cpu().numpy()
    Q = oprol.kron_dirs([oprol.standard_form_map_1d(p, nc[i], nf[i]) for i in range(dim)])
    ref = v @ Q.T
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    # one vector alone, and the identity when the meshes agree
    y1 = kl.prolong(C, F, torch.from_numpy(v[2]).cuda()).cpu().numpy()
    assert np.abs(y1 - ref[2]).max() <= 1e-12 * np.abs(ref).max()
    yi = kl.prolong(C, C, torch.from_numpy(v).cuda()).cpu().numpy()
    assert np.abs(yi - v).max() <= 1e-12 * np.abs(v).max()


def test_prolong_rejects_non_nested(kl):
    import torch
    C = kl.KLProblem(2, 2, [3, 3])
    F = kl.KLProblem(2, 2, [4, 6])
    G = kl.KLProblem(2, 3, [6, 6])
    v = torch.zeros((1, C.N), dtype=torch.float64, device="cuda")
    for bad in (F, G):
        with pytest.raises(kl.KLError):
            kl.prolong(C, bad, v)


# ---- the gain of a trained network ----------------------------------------------------------

SMALL = dict(p=2, ne_coarse=4, k=8, width=128, depth=3)
FINE_NE = 12
NEV = 6
# correlation lengths the 4-element coarse mesh resolves (at L ~ 0.1 its leading eigenvectors are
# mesh artefacts and not even the exact coarse eigenvectors approximate the fine ones)
L_RANGE = (0.4, 2.0)


@pytest.fixture(scope="module")
def trained(kl):
    from paper_2011_13861_gb300 import inputs, warmstart
    ws = warmstart.WarmStart(seed=5, **SMALL)
    X, T, stats = ws.targets(inputs.warmstart_params(96, seed=5, L_range=L_RANGE), block=8)
    assert stats["not_converged"] == 0
    hist = ws.fit(X, T, epochs=400, batch=32, lr=1e-3, seed=6)
    assert hist[-1] < 0.1 * hist[0], (hist[0], hist[-1])
    return ws


def test_warm_start_gains_over_random_start(kl, trained):
    """Unseen parameter sets: the prolonged prediction is close to the fine eigenspace and the
    warm-started solve needs fewer operator applications than the same solver from the random
    start, with the same eigenvalues."""
    from paper_2011_13861_gb300 import inputs, warmstart
    ws = trained
    gains = []
    for prm in inputs.warmstart_params(3, seed=6, L_range=L_RANGE):
        fine = warmstart.problem(prm, SMALL["p"], FINE_NE)
        # the same solver and options (block k, basis 3 k), seeded random start
        ev_r, vec_r, info_r = fine.eigs(NEV, tol=1e-8, method=1, block=SMALL["k"], ncv=3 * SMALL["k"],
                                        precision=kl.KL_P_TC64)
        ev_w, vec_w, info_w = ws.solve(fine, prm, NEV, tol=1e-8)
        assert info_w["path"] == "warm"
        assert np.abs(ev_w - ev_r).max() <= 1e-6 * ev_r[0]
        start = ws.start_block(fine, prm)
        # the NEV leading eigenvectors lie close to the predicted span
        Qs, _ = np.linalg.qr(start.cpu().numpy().T)
        proj = Qs.T @ vec_r.cpu().numpy().T
        sines = np.sqrt(np.clip(1 - np.linalg.svd(proj, compute_uv=False) ** 2, 0, None))
        assert sines.max() < 0.5, sines
        gains.append(info_r["applies"] / info_w["applies"])
    # a Krylov method gains from a start block only the iterations that take a random block down
    # to the start's accuracy (sines 0.05 - 0.3 here, against tan ~ sqrt(N) for a random block)
    assert min(gains) > 0.95 and np.mean(gains) > 1.05, gains


def test_fallback_when_the_warm_solve_stalls(kl):
    """An untrained network, a short correlation length (slowly decaying spectrum) and a budget of
    one restart of the float64 iteration: the warm attempt does not converge and the random-start
    solve takes over and converges."""
    from paper_2011_13861_gb300 import warmstart
    ws = warmstart.WarmStart(seed=9, **SMALL)
    prm = {"kernel": "gauss", "L": 0.1, "r_in": 1.0, "r_out": 2.0}
    fine = warmstart.problem(prm, SMALL["p"], FINE_NE)
    ev, vec, info = ws.solve(fine, prm, NEV, tol=1e-10, maxiter=1, ncv=24, block=SMALL["k"], method=0,
                             precision=kl.KL_P_FP64)
    assert info["warm"]["applies"] > 0
    assert info["path"] == "fallback"
    assert info["warm"]["converged"] < NEV
    assert info["converged"] >= NEV
    ev_r, _, _ = fine.eigs(NEV, tol=1e-10, method=1, block=SMALL["k"], precision=kl.KL_P_TC64)
    assert np.abs(ev - ev_r).max() <= 1e-8 * ev_r[0]


def test_wide_start_is_compressed_by_rayleigh_ritz(kl):
    """A start subspace wider than the block (kl_eig_opts.nstart): exact leading eigenvectors
    padded with random columns are compressed to the block leading Ritz vectors, and the solve
    returns the same eigenpairs as from a random start."""
    import torch
    from paper_2011_13861_gb300 import inputs as inp
    G = kl.KLProblem(3, 2, 6, kernel="exp", L=0.7)
    ev0, vec0, _ = G.eigs(6, tol=1e-10, method=0, block=4)
    pad = torch.from_numpy(inp.random_block(G.N, 6, seed=4).T.copy()).cuda()
    start = torch.cat([vec0, pad], dim=0).contiguous()            # 12 columns, block 4
    ev1, _, info1 = G.eigs(6, tol=1e-10, method=0, block=4, start=start)
    assert np.abs(ev1 - ev0).max() <= 1e-10 * ev0[0]
    assert info1["converged"] >= 6 and max(info1["resid"]) <= 1e-10
    # a start block of exact eigenvectors spans an invariant subspace: the solver must still find
    # the remaining wanted pairs (fresh directions when the expansion is rank deficient)
    ev2, _, info2 = G.eigs(6, tol=1e-10, method=0, block=4, start=vec0[:4].contiguous())
    assert np.abs(ev2 - ev0).max() <= 1e-10 * ev0[0]
    with pytest.raises(ValueError):
        G.eigs(6, method=0, block=8, start=vec0[:4].contiguous())


@pytest.mark.parametrize("prec", ["fp32", "tc32"])
def test_float32_class_plain_solve(kl, prec):
    """The plain method in float32-class arithmetic (the warm start's training solves): converged
    to residual 1e-5, eigenvalues within float32 accuracy of the float64 solve, and eigenvectors
    spanning the same subspace to ~1e-4."""
    # a box with unequal sides: no symmetry-degenerate eigenvalues
    G = kl.KLProblem(3, 2, [6, 5, 4], kernel="gauss", L=0.6, lo=[0.0, 0.0, 0.0], hi=[1.0, 0.83, 0.61])
    p = kl.KL_P_FP32 if prec == "fp32" else kl.KL_P_TC32
    ev0, V0, _ = G.eigs(8, tol=1e-10, method=0, block=4)
    ev1, V1, info = G.eigs(8, tol=1e-5, method=0, block=4, precision=p, raise_on_nonconv=False)
    assert info["converged"] >= 8 and max(info["resid"]) <= 1e-5, (info["converged"], info["resid"])
    assert np.abs(ev1 - ev0).max() <= 1e-5 * ev0[0], np.abs(ev1 - ev0).max() / ev0[0]
    s = np.linalg.svd(V0[:6].cpu().numpy() @ V1[:6].cpu().numpy().T, compute_uv=False)
    assert np.sqrt(max(0.0, 1.0 - s.min() ** 2)) < 1e-3, s


def test_fallback_when_the_prediction_is_not_finite(kl):
    """A network whose output is NaN (a poisoned bias) makes the warm start fail with
    KL_ERR_NUMERIC inside the solver; the random-start solve takes over."""
    from paper_2011_13861_gb300 import warmstart
    ws = warmstart.WarmStart(seed=9, **SMALL)
    Ws, bs = ws.net.get_params()
    bs[-1][3] = np.nan
    ws.net.set_params(Ws, bs)
    prm = {"kernel": "exp", "L": 0.8, "r_in": 1.0, "r_out": 2.0}
    fine = warmstart.problem(prm, SMALL["p"], FINE_NE)
    ev, _, info = ws.solve(fine, prm, NEV, tol=1e-8)
    assert info["path"] == "fallback" and "NUMERIC" in info["warm"]["error"]
    assert info["converged"] >= NEV
