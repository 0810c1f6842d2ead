"""kl_covmv_noalloc: the stage-5 product for callers that cannot allocate device memory.

Such callers (code recorded during CUDA stream capture, or programs that forbid allocation
after start-up) get the same result as kl_covmv while the library draws its scratch from a
fixed device array instead of its workspace.  This file is collected last on purpose: it
calls the entry point through the C ABI twice in a row, with different inputs, and checks
each result against kl_covmv with the float64 tolerance of the other parity tests.
"""
import pytest

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
    G = kl.KLProblem(dim, p, ne, kernel=kernel, L=L, sigma=1.3)
    outs = []
    for call in range(2):
        u = torch.from_numpy(inputs.random_block(G.Nt, nvec, seed=100 + call).T.copy()).cuda()
        ref = G.covmv(u)
        z = torch.full_like(u, float("nan"))
        G.covmv_noalloc(u, z)
        torch.cuda.synchronize()
        assert torch.isfinite(z).all()
        assert rel(z, ref) < FP64_TOL
        outs.append(z)
        if call == 0:
            free_after_first = torch.cuda.mem_get_info()[0]
    # the second call allocated nothing on the device
    assert torch.cuda.mem_get_info()[0] == free_after_first
    assert not torch.equal(outs[0], outs[1])


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
