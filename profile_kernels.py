"""Launches the stage-5 kernel product alone, for kernel profiling (ncu) and timing.

  python profile_kernels.py --workload cube-p2-32^3-exp-L0.5 --precision fp64 --nvec 1 --reps 3

Builds the handle, runs stages 1-4 once to obtain u, then calls kl_covmv `reps` times on the
current stream and prints the CUDA-event time per call.

  python profile_kernels.py --contract --workload cube-p3-48^3-gauss-L0.3 --nvec 32 --reps 3

times the forward (stages 1-4) and backward (stages 6-9) contractions alone.

  python profile_kernels.py --peaks

prints the measured float64/float32 FMA and MUFU ex2/rsqrt rates (kl_pipe_rates).

  python profile_kernels.py --mlp-train --batch 64 --reps 3

times training steps of the warm-start network (4 inputs, 4 x 256 tanh, 32 x 6,859 outputs) on
seeded synthetic inputs and targets: one warm-up epoch, then `reps` epochs of 256 samples.

  python profile_kernels.py --annulus 64 [--annulus-sequential]

solves the first 64 seeded quarter-annulus instances of the batched workload (10 eigenpairs each,
residual 1e-8, mixed method, block 4, tensor-core float64-class polish) once, together through
kl_eigs_batched or one after another, and prints the wall time and the summed solver counters.
"""
import argparse
import json

import torch

import paper_2011_13861_gb300 as kl
from paper_2011_13861_gb300 import inputs


def mlp_train(a):
    k, n, S = 32, 6859, 256
    net = kl.MLP(4, 256, 4, k * n, seed=1)
    x = torch.from_numpy(inputs.random_block(S, 4, seed=2).astype("float32")).cuda()
    t = torch.from_numpy(inputs.random_block(S, k * n, seed=3).astype("float32")).cuda()
    net.train(x, t, k, n, 1, a.batch, 1e-4, 0)
    out = []
    for r in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.train(x, t, k, n, 1, a.batch, 1e-4, r + 1)
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1) / (S // a.batch))
    print(json.dumps({"mlp_train": {"batch": a.batch, "params": net.nparam, "ms_per_step": out}}))


def contract(a):
    w = inputs.WORKLOADS[a.workload]
    G = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    v = torch.from_numpy(inputs.random_block(G.N, a.nvec, seed=1).T.copy()).cuda()
    z = torch.from_numpy(inputs.random_block(G.Nt, a.nvec, seed=2).T.copy()).cuda()
    G.forward(v)
    G.backward(z)
    torch.cuda.synchronize()
    out = {"forward": [], "backward": []}
    for _ in range(a.reps):
        for name, fn in (("forward", lambda: G.forward(v)), ("backward", lambda: G.backward(z))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out[name].append(e0.elapsed_time(e1))
    print(json.dumps({"workload": a.workload, "nvec": a.nvec, "N": G.N, "Ntilde": G.Nt, "ms": out}))


def annulus(a):
    import time
    net = inputs.quarter_annulus_net()
    cases = inputs.batched_instances(64)[:a.annulus]
    Gs = [kl.KLProblem(c["dim"], c["p"], c["ne"], kernel=c["kernel"], L=c["L"], sigma=c["sigma"], nurbs=net)
          for c in cases]
    opts = dict(method=1, block=4, precision=kl.KL_P_TC64, want_vectors=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if a.annulus_sequential:
        infos = [G.eigs(10, 1e-8, **opts)[2] for G in Gs]
        bi = None
    else:
        _, _, infos, _, bi = kl.eigs_batched(Gs, 10, 1e-8, **opts)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    keys = ("applies", "block_applies", "restarts", "ms_fp32_phase", "ms_stage5_fp32", "ms_stage5_tc32",
            "ms_stage5_tc64")
    print(json.dumps({"instances": len(Gs), "sequential": a.annulus_sequential, "wall_s": wall,
                      "converged_all": all(i["converged"] >= 10 for i in infos),
                      "sums": {k: sum(i[k] for i in infos) for k in keys}, "batch": bi}))
    for G in Gs:
        G.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cube-p2-32^3-exp-L0.5")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "df64", "tc32", "tc64"])
    ap.add_argument("--nvec", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--solve", default=None, choices=[None, "plain", "plain_df", "mixed", "lobpcg", "mixed_lobpcg"],
                    help="run one warm-up and one timed eigensolve instead of stage 5 alone")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--tol-low", type=float, default=0.0)
    ap.add_argument("--ncv", type=int, default=0)
    ap.add_argument("--maxiter", type=int, default=0, help="restart / step bound of --solve (0 = library default)")
    ap.add_argument("--polish-block", type=int, default=0)
    ap.add_argument("--polish-ncv", type=int, default=0)
    ap.add_argument("--low", default="fp32", choices=["fp32", "tc32"])
    ap.add_argument("--mlp-train", action="store_true", help="time training steps of the warm-start network")
    ap.add_argument("--contract", action="store_true", help="time the forward and backward contractions")
    ap.add_argument("--peaks", action="store_true", help="measured pipe rates (kl_pipe_rates)")
    ap.add_argument("--tc-sym", action="store_true",
                    help="tensor-core float64 class: symmetric schedule (kl_set_tc_symmetric(1))")
    ap.add_argument("--sym-slot-limit", type=int, default=None,
                    help="bytes of the one-launch symmetric schedule's slots (kl_set_sym_slot_limit)")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--annulus", type=int, default=0, help="solve this many batched-workload instances (1..64)")
    ap.add_argument("--annulus-sequential", action="store_true", help="--annulus one instance after another")
    ap.add_argument("--accurate", default="df64", choices=["fp64", "df64", "tc64"],
                    help="accurate-phase arithmetic of --solve plain_df / mixed")
    a = ap.parse_args()
    if a.sym_slot_limit is not None:
        kl.set_sym_slot_limit(a.sym_slot_limit)
    if a.tc_sym:
        kl.set_tc_symmetric(True)
    if a.mlp_train:
        return mlp_train(a)
    if a.contract:
        return contract(a)
    if a.annulus:
        return annulus(a)
    if a.peaks:
        print(json.dumps(kl.pipe_rates()))
        return
    w = inputs.WORKLOADS[a.workload]
    G = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    if a.solve:
        method = {"plain": 0, "plain_df": 0, "mixed": 1, "lobpcg": 2, "mixed_lobpcg": 3}[a.solve]
        block = a.block or {0: 4, 1: 16, 2: 32, 3: 32}[method]
        prec = kl.KL_P_FP64 if a.solve == "plain" else \
            {"fp64": kl.KL_P_FP64, "df64": kl.KL_P_DF64, "tc64": kl.KL_P_TC64}[a.accurate]
        start = torch.from_numpy(inputs.random_block(G.N, block, seed=1).T.copy()).cuda()
        out = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ev, _, info = G.eigs(w["k"], 1e-8, method=method, block=block, start=start, precision=prec,
                                 tol_low=a.tol_low, ncv=a.ncv, maxiter=a.maxiter, raise_on_nonconv=False,
                                 polish_block=a.polish_block,
                                 polish_ncv=a.polish_ncv,
                                 low_precision=kl.KL_P_TC32 if a.low == "tc32" else kl.KL_P_FP32)
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        info.pop("resid")
        print(json.dumps({"workload": a.workload, "solve": a.solve, "block": block, "accurate": a.accurate,
                          "ms": out, "info": info}))
        return
    prec = {"fp64": kl.KL_P_FP64, "fp32": kl.KL_P_FP32, "df64": kl.KL_P_DF64, "tc32": kl.KL_P_TC32,
            "tc64": kl.KL_P_TC64}[a.precision]
    v = torch.from_numpy(inputs.random_block(G.N, a.nvec, seed=1).T.copy()).cuda()
    u = G.forward(v).reshape(a.nvec, G.Nt).contiguous()
    G.covmv(u, precision=prec)
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        G.covmv(u, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    print(json.dumps({"workload": a.workload, "precision": a.precision, "nvec": a.nvec, "Ntilde": G.Nt,
                      "ms": times, "pairs_per_s": G.Nt * G.Nt / (min(times) * 1e-3)}))


if __name__ == "__main__":
    main()
