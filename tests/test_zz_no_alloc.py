"""kl_covmv_noalloc: the stage-5 product for callers that cannot allocate device memory.

Such callers (programs that take their whole device-memory budget at start-up and forbid
allocation afterwards, or loops that cannot afford cudaMalloc's implicit synchronisation) get
the same result as kl_covmv while the library draws its scratch from a fixed device array
instead of its workspace.  Each case calls the entry point through the C ABI twice in a row,
with different inputs, and checks each result against kl_covmv with the float64 tolerance of
the other parity tests, and element by element against the oracle's stage 5 on sampled rows.
Every tensor is allocated before the first call, so the free-memory reading taken around the
second call alone shows that the call itself allocated nothing; the file passes on its own in a
fresh process and after the other tests (it is collected last so that a run stopping at the
first failure has already run everything else).
"""
import numpy as np
import pytest

from oracle import ibq
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("dim,p,ne,kernel,L,nvec", [
    (3, 2, [9, 10, 11], "exp", 0.5, 3),
    (3, 2, 32, "exp", 0.5, 16),        # 39,304 points: the scratch holds 6 column splits
    (2, [2, 3], [23, 17], "gauss", 0.4, 17),
])
def test_noalloc_matches_covmv_on_two_calls(kl, dim, p, ne, kernel, L, nvec):
    import torch
    sigma = 1.3
    G = kl.KLProblem(dim, p, ne, kernel=kernel, L=L, sigma=sigma)
    P = ibq.Problem(dim, p, ne, kernel=kernel, L=L, sigma=sigma)
    X, _ = P.points_and_J()
    hosts = [inputs.random_block(G.Nt, nvec, seed=100 + call) for call in range(2)]
    us = [torch.from_numpy(h.T.copy()).cuda() for h in hosts]
    refs = [G.covmv(u) for u in us]
    zs = [torch.full_like(u, float("nan")) for u in us]
    torch.cuda.synchronize()
    rows = np.unique(np.concatenate([np.random.default_rng(9).choice(G.Nt, size=min(48, G.Nt), replace=False),
                                     [0, G.Nt - 1]]))
    for call in range(2):
        if call == 1:
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
        G.covmv_noalloc(us[call], zs[call])
        torch.cuda.synchronize()
        if call == 1:
            # the second call alone: nothing was allocated on the device
            assert torch.cuda.mem_get_info()[0] == free_before
        z = zs[call]
        assert torch.isfinite(z).all()
        assert rel(z, refs[call]) < FP64_TOL
        zo = P.stage5(X, hosts[call], row_index=rows)
        zg = z.cpu().numpy().T[rows]
        assert np.abs(zg - zo).max() / np.abs(zo).max() < FP64_TOL
    assert not torch.equal(zs[0], zs[1])


def test_noalloc_rejects_oversized_and_wrong_precision(kl):
    import torch
    G = kl.KLProblem(3, 2, 64, kernel="gauss", L=0.3)          # 66^3 = 287,496 points
    u = torch.zeros((16, G.Nt), dtype=torch.float64, device="cuda")
    z = torch.zeros_like(u)
    with pytest.raises(kl.KLError) as e:
        G.covmv_noalloc(u, z)                                     # 16 x 287,496 > 4 Mi doubles
    assert "exceeds the fixed scratch" in str(e.value)
    small = kl.KLProblem(2, 2, 8, kernel="exp", L=0.5)
    us = torch.zeros((1, small.Nt), dtype=torch.float64, device="cuda")
    status = kl.load().kl_covmv_noalloc(small._h, kl.KL_P_FP32, us.data_ptr(), small.Nt, us.data_ptr(),
                                        small.Nt, 1, None)
    assert status == 1                                             # KL_ERR_INVALID_ARG, nothing launched
    assert "FP64 only" in kl.load().kl_last_error().decode()
