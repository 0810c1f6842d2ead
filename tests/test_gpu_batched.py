"""Many independent instances in one batched stage-5 launch (kl_apply_batched) and solved
together (kl_eigs_batched), against the oracle and against the single-instance path."""
import numpy as np
import pytest

from oracle import ibq, nurbs
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu


def small_instances():
    # uneven sizes, both geometries, every kernel kind the batched kernels switch on
    return [
        dict(dim=3, p=2, ne=[5, 4, 6], kernel="exp", L=0.4, annulus=True),
        dict(dim=3, p=3, ne=[3, 5, 4], kernel="gauss", L=0.8, annulus=True),
        dict(dim=2, p=2, ne=[11, 7], kernel="exp", L=0.3, annulus=False),
        dict(dim=3, p=2, ne=[6, 6, 5], kernel="gauss", L=1.7, annulus=False),
        dict(dim=2, p=2, ne=[9, 10], kernel="exp_sep", L=0.6, annulus=True),
        dict(dim=3, p=2, ne=[3, 2, 3], kernel="poly", L=2, annulus=False),
    ]


def make(kl, c):
    if c["annulus"]:
        net = inputs.quarter_annulus_net(dim=c["dim"])
        F = nurbs.NURBSMap(net["deg"], net["knots"], net["ctrl"], net["weights"])
        P = ibq.Problem(c["dim"], c["p"], c["ne"], kernel=c["kernel"], L=c["L"], sigma=1.2, geom=F)
        G = kl.KLProblem(c["dim"], c["p"], c["ne"], kernel=c["kernel"], L=c["L"], sigma=1.2, nurbs=net)
    else:
        P = ibq.Problem(c["dim"], c["p"], c["ne"], kernel=c["kernel"], L=c["L"], sigma=1.2)
        G = kl.KLProblem(c["dim"], c["p"], c["ne"], kernel=c["kernel"], L=c["L"], sigma=1.2)
    return P, G


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


@pytest.mark.parametrize("prec,tol", [(2, 1e-12), (1, 2e-5)], ids=["df64", "fp32"])
def test_apply_batched_against_oracle(kl, prec, tol):
    import torch
    cases = small_instances()
    PG = [make(kl, c) for c in cases]
    nvs = [3, 1, 4, 2, 5, 3]
    vs = [inputs.random_block(P.N, nv, seed=50 + i) for i, ((P, G), nv) in enumerate(zip(PG, nvs))]
    vd = [torch.from_numpy(v.T.copy()).cuda() for v in vs]
    ys = kl.apply_batched([G for _, G in PG], vd, precision=prec)
    for (P, G), v, y, x in zip(PG, vs, ys, vd):
        assert rel(y.cpu().numpy().T, P.dense_operator() @ v) < tol
        # the single-instance path agrees (different kernels, same arithmetic class)
        assert rel(y.cpu().numpy().T, G.apply(x, precision=prec).cpu().numpy().T) < tol
    # deterministic: a second batched call is bit-identical
    ys2 = kl.apply_batched([G for _, G in PG], vd, precision=prec)
    assert all(torch.equal(a, b) for a, b in zip(ys, ys2))
    # a batch of 12 (timed split sizes, then the captured graph) in a different order, twice
    order = [5, 0, 3, 1, 4, 2, 0, 3, 2, 5, 1, 4]
    PG2 = [make(kl, cases[i]) for i in order]
    vd2 = [torch.from_numpy(inputs.random_block(P.N, 2, seed=70 + j).T.copy()).cuda() for j, (P, _) in enumerate(PG2)]
    for _ in range(2):
        ys3 = kl.apply_batched([G for _, G in PG2], vd2, precision=prec)
        for (P, G), x, y in zip(PG2, vd2, ys3):
            assert rel(y.cpu().numpy().T, P.dense_operator() @ x.cpu().numpy().T) < tol


@pytest.mark.parametrize("method", [0, 1])
def test_eigs_batched_against_oracle(kl, method):
    cases = small_instances()[:5]
    PG = [make(kl, c) for c in cases]
    k = 8
    ev, vecs, infos, sts, binfo = kl.eigs_batched([G for _, G in PG], k, 1e-8, method=method, block=4,
                                                  precision=kl.KL_P_DF64)
    assert all(s == 0 for s in sts)
    assert binfo["rounds"] > 0 and binfo["cols_per_split"] in (1024, 2048, 4096, 8192)
    for i, (P, G) in enumerate(PG):
        lam = np.linalg.eigvalsh(P.dense_operator())[::-1][:k]
        assert np.abs(ev[i] - lam).max() / lam[0] < 1e-10, i
        assert max(infos[i]["resid"]) <= 1e-8
        V = vecs[i].cpu().numpy().T
        assert np.abs(V.T @ V - np.eye(k)).max() < 1e-12
        # residuals with the oracle operator
        R = P.dense_operator() @ V - V * ev[i]
        assert (np.linalg.norm(R, axis=0) / np.abs(ev[i])).max() < 2e-8


