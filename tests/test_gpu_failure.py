"""Failure detection without a GPU fault: a bounded wait that nothing completes reports
KL_ERR_TIMEOUT and leaves the context usable; non-finite data ends a solve with KL_ERR_NUMERIC;
a solve that runs out of restarts reports KL_ERR_NOT_CONVERGED (and the warm start falls back,
tests/test_gpu_warmstart.py)."""
import numpy as np
import pytest

from oracle import ibq
from paper_2011_13861_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(kl):
    import torch
    st, msg = kl.wait_selftest(0.05)
    assert kl.STATUS[st] == "KL_ERR_TIMEOUT", msg
    st2, _ = kl.wait_selftest(5.0)            # out of range: rejected on the host
    assert kl.STATUS[st2] == "KL_ERR_INVALID_ARG"
    # the context still works: a float64 application against the oracle
    P = ibq.Problem(2, 2, [4, 5], kernel="exp", L=0.5)
    G = kl.KLProblem(2, 2, [4, 5], kernel="exp", L=0.5)
    v = inputs.random_block(P.N, 2, seed=3)
    y = G.apply(torch.from_numpy(v.T.copy()).cuda()).cpu().numpy().T
    ref = P.dense_operator() @ v
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_non_finite_start_is_reported(kl):
    import torch
    G = kl.KLProblem(2, 2, [5, 5], kernel="exp", L=0.5)
    start = torch.from_numpy(inputs.random_block(G.N, 4, seed=4).T.copy()).cuda()
    start[1, 7] = float("nan")
    with pytest.raises(kl.KLError) as e:
        G.eigs(4, 1e-8, method=0, block=4, start=start)
    assert "NUMERIC" in str(e.value)
    ev, _, info = G.eigs(4, 1e-8, method=0, block=4)     # the handle is still usable
    assert info["converged"] >= 4


def test_restart_budget_reports_not_converged(kl):
    G = kl.KLProblem(2, 2, [8, 8], kernel="gauss", L=0.1)
    ev, _, info = G.eigs(6, 1e-12, method=0, block=2, ncv=12, maxiter=1, raise_on_nonconv=False)
    assert kl.STATUS[info["status"]] == "KL_ERR_NOT_CONVERGED" and info["converged"] < 6
