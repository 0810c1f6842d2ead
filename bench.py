"""Benchmark: time to the 20 leading Karhunen-Loeve eigenpairs at relative residual 1e-8 and the
kernel-evaluation rate, plain float64 block Lanczos vs the mixed-precision form, on the unit-cube
workload (degree-2 splines, 32^3 elements, 34^3 = 39,304 Greville points, exponential kernel
exp(-|x-x'|/L), sigma = 1, L = 0.5).

One step = one complete eigensolve through the C ABI (kl_eigs): every operator application runs
all nine stages of Algorithm 1 on the GPU.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

--impl reference times the CPU oracle (plain NumPy float64 stage-5 product on the host cores) on
a bounded sample of the same workload, in the same unit.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 20 eigenpairs @res 1e-8 and kernel evals/s, chosen form vs plain FP64"
UNIT = "kernel evals/s"
DEFAULT_WORKLOAD = "cube-p2-32^3-exp-L0.5"
TOL = 1e-8
FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64 vector rate (nominal)
# algorithmic float64 flops of one kernel evaluation (paper's convention: one flop per add,
# subtract, multiply; FMA = 2): distance 3 sub + 3 mul + 2 add, pre-scaled coordinates carry 1/L
# (a 9th flop per evaluation, the scaling by 1/L, is folded into set-up); sqrt by one Heron correction
# (mul, fma, mul, fma = 6); exp by Tang's method (fma, sub, fma, 4 fma + mul, fma = 16);
# plus 2 flops per vector for the product.  The kernel is symmetric, so the method needs only half
# of the evaluations (one per unordered pair): algorithmic flops per ordered pair = eval/2 + 2b.
FLOPS_PER_EVAL = {"exp": 8 + 6 + 16, "gauss": 8 + 16, "exp_sep": 3 + 2 + 16, "poly": 12}
# DRAM bytes per launch of covmv64_sym_kernel<EXP, 4> at 39,304 points (ncu capture, see
# profiles/stage5_fp64_sym_cube-p2-32^3-exp.md): 5.4 MB read + 136.3 MB written (partial slots)
SYM64_NV4_TRAFFIC_BYTES = 5.377536e6 + 136.273408e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--plain-block", type=int, default=4)
    ap.add_argument("--mixed-block", type=int, default=4)
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-instance quarter-annulus batch")
    ap.add_argument("--no-large-cube", action="store_true",
                    help="skip the 132,651-point Gaussian cube (mixed precision with blocks of 16)")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the learned warm start")
    ap.add_argument("--warm-train-solves", type=int, default=2000,
                    help="coarse (16^3, p=3) training solves of the warm-start network (2000 = the full set)")
    ap.add_argument("--warm-epochs", type=int, default=100)
    ap.add_argument("--warm-eval", type=int, default=2, help="unseen parameter sets solved at 48^3")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for nm, val in zip(names, f[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(w, rows, seed=0):
    """Kernel evaluations per second of the oracle's float64 stage-5 product on `rows` rows."""
    import numpy as np

    from oracle import ibq
    from paper_2011_13861_gb300 import inputs
    P = ibq.Problem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    X, _ = P.points_and_J()
    u = inputs.random_block(P.Nt, 1, seed=seed)
    idx = np.linspace(0, P.Nt - 1, rows).astype(np.int64)
    t0 = time.perf_counter()
    P.stage5(X, u, rows=256, row_index=idx)
    dt = time.perf_counter() - t0
    return rows * P.Nt / dt, dt, P.Nt


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2011_13861_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    rows = 20000
    for _ in range(args.warmup):
        oracle_rate(w, rows // 4)
    rates, secs = [], []
    for _ in range(args.steps):
        r, dt, Nt = oracle_rate(w, rows)
        rates.append(r)
        secs.append(dt)
    value = statistics.mean(rates)
    sample = "%d of %d rows of the float64 stage-5 product (oracle.ibq.Problem.stage5), %d columns each" % (
        rows, Nt, Nt)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "Ntilde": Nt, "L2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def flush_l2(buf):
    buf.add_(1.0)


def measure_batched(kl, inputs):
    """64 seeded instances on the quarter annulus (quadratic NURBS map, radius 1..2, height 1),
    elements per direction 8..40, degree 2-3, exponential / Gaussian kernels, L log-uniform in
    [0.1, 2], 10 eigenpairs each: solved together (kl_eigs_batched: one batched stage-5 launch
    per step for every instance in its float32 phase, then the tensor-core polish per
    instance) against the same solves one after another."""
    import numpy as np
    import torch
    net = inputs.quarter_annulus_net()
    cases = inputs.batched_instances(64)
    t0 = time.perf_counter()
    Gs = [kl.KLProblem(c["dim"], c["p"], c["ne"], kernel=c["kernel"], L=c["L"], sigma=c["sigma"], nurbs=net)
          for c in cases]
    t_create = time.perf_counter() - t0
    opts = dict(method=1, block=4, precision=kl.KL_P_TC64, want_vectors=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev_b, _, infos, sts, bi = kl.eigs_batched(Gs, 10, TOL, **opts)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    ev_s = [G.eigs(10, TOL, **opts)[0] for G in Gs]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    Nt = np.array([G.Nt for G in Gs], dtype=float)
    out = {"workload": "64 quarter-annulus instances (seed 2011), k=10 each", "create_s": t_create,
           "batched_s": t_batch, "sequential_s": t_seq, "batched_vs_sequential": t_seq / t_batch,
           "converged": int(sum(1 for x in sts if x == 0)), "max_resid": max(max(i["resid"]) for i in infos),
           "max_rel_eig_diff_batched_vs_sequential": float(max(np.abs(ev_b[i] - ev_s[i]).max() / abs(ev_s[i][0])
                                                              for i in range(len(Gs)))),
           "batched_stage5_ms": bi["ms_stage5"], "batched_launches": bi["rounds"], "requests": bi["requests"],
           "cols_per_split": bi["cols_per_split"], "points_min_max": [int(Nt.min()), int(Nt.max())],
           "sum_pairs_per_application": float((Nt ** 2).sum()),
           "timing": "wall clock with a device synchronisation on both sides, one run each"}
    for G in Gs:
        G.close()
    return out


def measure_warm_start(kl, inputs, train_solves, epochs, n_eval):
    """Learned warm start on the quarter annulus: a 4 x 256 bfloat16 network trained on the
    32 leading eigenvectors of `train_solves` coarse problems (p=3, 16^3 elements; kernel, L and
    radii drawn with seed 5), then used, prolonged exactly to 48^3 elements, as the start block
    of the mixed solver (20 eigenpairs, residual 1e-8) for unseen parameter sets (seed 6); against
    the same solver from the random start (block 32, basis 96 and the tensor-core float32 first
    phase as the warm start; and block 16 with the scalar float32 first phase, the best random-start
    configuration) and, for the first parameter set, random-start float64 block Lanczos (block 4).
    Also timed: the 32 predicted vectors compressed by Rayleigh-Ritz to a block-16 start."""
    import numpy as np
    import torch
    from paper_2011_13861_gb300 import warmstart
    ws = warmstart.WarmStart(p=3, ne_coarse=16, k=32, width=256, depth=4, seed=5)
    X, T, st = ws.targets(inputs.warmstart_params(train_solves, seed=5))
    hist = ws.fit(X, T, epochs=epochs, batch=64, lr=1e-3, seed=6)
    torch.cuda.synchronize()
    out = {"workload": "quarter annulus r_in~U(0.8,1.2) r_out~U(1.8,2.2) h=1, exp/gauss, L~logU(0.1,2); "
                       "coarse p=3 16^3 (6,859 dof), fine p=3 48^3 (132,651 dof), k=20 of a 32-vector start",
           "train_solves": st["solves"], "train_targets_s": st["seconds"], "train_not_converged": st["not_converged"],
           "epochs": epochs, "fit_s": ws.fit_seconds, "loss_first_last": [float(hist[0]), float(hist[-1])],
           "network": "4 x 256 tanh, bfloat16 weights and layer inputs, float32 sums, %d parameters" % ws.net.nparam,
           "eval": []}
    del X, T
    k = 20

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r

    for i, prm in enumerate(inputs.warmstart_params(n_eval, seed=6)):
        fine = warmstart.problem(prm, 3, 48)
        mixed = dict(method=1, precision=kl.KL_P_TC64)
        # workspaces of every width and precision allocated before any timed solve
        for nv, pr in ((32, kl.KL_P_TC32), (32, kl.KL_P_FP32), (16, kl.KL_P_FP32), (32, kl.KL_P_TC64)):
            fine.apply(torch.zeros((nv, fine.N), dtype=torch.float64, device="cuda"), precision=pr)
        tw, (ev_w, vec_w, iw) = timed(lambda: ws.solve(fine, prm, k, tol=TOL))
        t32, (ev_r, _, i32) = timed(lambda: fine.eigs(k, TOL, block=32, ncv=96, low_precision=kl.KL_P_TC32,
                                                      want_vectors=False, **mixed))
        t16, (_, _, i16) = timed(lambda: fine.eigs(k, TOL, block=16, want_vectors=False, **mixed))
        tc, (_, _, ic) = timed(lambda: ws.solve(fine, prm, k, tol=TOL, block=16))
        # subspace of the prediction against the converged eigenvectors (diagnostic)
        start = ws.start_block(fine, prm)
        Qs, _ = torch.linalg.qr(start.T)
        cosv = torch.linalg.svdvals(Qs.T @ vec_w.T).cpu().numpy()
        row = {"kernel": prm["kernel"], "L": prm["L"], "r_in": prm["r_in"], "r_out": prm["r_out"],
               "path": iw["path"], "warm_s": tw, "warm_applies": iw["applies"], "warm_restarts": iw["restarts"],
               "warm_start_block_ms": iw.get("ms_start_block", iw.get("warm", {}).get("ms_start_block")),
               "random32_s": t32, "random32_applies": i32["applies"], "random16_s": t16,
               "random16_applies": i16["applies"], "gain_vs_random32": t32 / tw, "gain_vs_random16": t16 / tw,
               "warm_compressed16_s": tc, "warm_compressed16_applies": ic["applies"],
               "max_resid_warm": max(iw["resid"][:k]),
               "max_rel_eig_diff_warm_vs_random": float(np.max(np.abs(ev_w - ev_r) / np.abs(ev_r))),
               "prediction_max_sine_top20": float(np.sqrt(max(0.0, 1.0 - cosv.min() ** 2)))}
        if i == 0:
            tp, (ev_p, _, ip) = timed(lambda: fine.eigs(k, TOL, method=0, block=4, want_vectors=False))
            row.update({"fp64_lanczos_s": tp, "fp64_lanczos_applies": ip["applies"], "gain_vs_fp64_lanczos": tp / tw,
                        "max_rel_eig_diff_warm_vs_fp64": float(np.max(np.abs(ev_w - ev_p) / np.abs(ev_p)))})
        out["eval"].append(row)
        fine.close()
    out["timing"] = "wall clock with a device synchronisation on both sides, one run each (warm includes " \
                    "the network forward pass and the prolongation)"
    return out


def measure_large_cube(kl, inputs, flush, stream):
    """Unit cube, p=3, 48^3 elements (132,651 points), Gaussian kernel L=0.3, 20 eigenpairs:
    the mixed form with blocks of 16 (float32 phase, tensor-core float64-class polish) against
    one plain float64 block-4 solve of the same problem on the same GPU."""
    import numpy as np
    import torch
    w = inputs.WORKLOADS["cube-p3-48^3-gauss-L0.3"]
    k = w["k"]
    G = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    N, Nt = G.N, G.Nt
    s16 = torch.from_numpy(inputs.random_block(N, 16, seed=1).T.copy()).cuda()
    s4 = torch.from_numpy(inputs.random_block(N, 4, seed=1).T.copy()).cuda()

    def timed_once(fn):
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    def mixed():
        return G.eigs(k, TOL, method=1, block=16, start=s16, precision=kl.KL_P_TC64)

    mixed()
    ms_m = []
    for _ in range(2):
        t, (ev_m, vec_m, info_m) = timed_once(mixed)
        ms_m.append(t)
    ms_p, (ev_p, _, info_p) = timed_once(lambda: G.eigs(k, TOL, method=0, block=4, start=s4, want_vectors=False))
    ych = G.apply(vec_m)
    lam = torch.from_numpy(np.asarray(ev_m)).cuda().reshape(-1, 1)
    resid = ((ych - lam * vec_m).norm(dim=1) / lam.abs().reshape(-1)).max().item()
    ms_mixed = statistics.mean(ms_m)
    out = {"workload": "cube-p3-48^3-gauss-L0.3", "N": N, "Ntilde": Nt, "k": k,
           "chosen_form": "float32 stage-5 block Lanczos (block 16) + block-32 tensor-core float64-class polish "
                          "(20 wanted + 12 guard vectors)",
           "chosen_ms": ms_mixed, "plain_fp64_ms": ms_p, "speedup": ms_p / ms_mixed,
           "chosen_applies": info_m["applies"], "plain_applies": info_p["applies"],
           "chosen_stage5_ms": {"fp32": info_m["ms_stage5_fp32"], "tc64": info_m["ms_stage5_tc64"]},
           "plain_stage5_fp64_ms_per_call": info_p["ms_stage5_fp64"] / max(info_p["stage5_calls_fp64"], 1),
           "max_rel_eig_diff_vs_plain": float(np.max(np.abs(np.asarray(ev_m) - np.asarray(ev_p)) /
                                                     np.abs(np.asarray(ev_p)))),
           "max_resid_chosen": max(info_m["resid"]), "max_resid_chosen_fp64_operator": resid,
           "max_resid_plain": max(info_p["resid"]),
           "plain_evals_per_s": info_p["applies"] * float(Nt) * Nt / (ms_p * 1e-3),
           "timing": "CUDA events; chosen form mean of 2 after 1 warm-up, plain float64 once; L2 flushed"}
    G.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2011_13861_gb300 as kl
    from paper_2011_13861_gb300 import inputs

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    w = inputs.WORKLOADS[args.workload]
    k = w["k"]
    G = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    N, Nt = G.N, G.Nt
    # each rank solves its own instance (independent problems: weak scaling, no collective)
    seed = 1 + rank
    start_p = torch.from_numpy(inputs.random_block(N, args.plain_block, seed=seed).T.copy()).cuda()
    start_m = torch.from_numpy(inputs.random_block(N, args.mixed_block, seed=seed).T.copy()).cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def solve_plain():
        return G.eigs(k, TOL, method=0, block=args.plain_block, start=start_p)

    def solve_mixed():
        # float32 stage 5 until the estimates reach tol_low, then a polish block of max(k, 32)
        # whose stage 5 runs on the tensor cores with exact slicing (float64-class); residuals
        # from the polish operator's products, re-checked below with the float64 operator
        return G.eigs(k, TOL, method=1, block=args.mixed_block, start=start_m, precision=kl.KL_P_TC64)

    def solve_plain_df():
        return G.eigs(k, TOL, method=0, block=args.plain_block, start=start_p, precision=kl.KL_P_DF64)

    for _ in range(args.warmup):
        solve_plain()
        solve_mixed()
        solve_plain_df()
    torch.cuda.synchronize()

    def timed(fn, clocks=None):
        times, infos = [], []
        if clocks:
            clocks.start()
        launches0 = kl.kernel_launches()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush_l2(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ev, vec, info = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append((ev, info))
        if world > 1:
            dist.barrier()
        launches = kl.kernel_launches() - launches0
        clk = clocks.stop() if clocks else None
        return times, infos, launches, clk

    clocks = ClockSampler(local)
    t_plain, i_plain, launches_plain, clk = timed(solve_plain, clocks)
    t_mixed, i_mixed, launches_mixed, _ = timed(solve_mixed)
    t_pdf, i_pdf, _, _ = timed(solve_plain_df)

    ms_plain = statistics.mean(t_plain)
    ms_mixed = statistics.mean(t_mixed)
    ms_pdf = statistics.mean(t_pdf)
    if world > 1:
        ms_plain, ms_mixed, ms_pdf = max_over_ranks([ms_plain, ms_mixed, ms_pdf], device="cuda")
    # untimed: float64-operator residuals of the chosen form's eigenvectors
    ev_chk, vec_chk, _ = solve_mixed()
    ych = G.apply(vec_chk)
    lam = torch.from_numpy(np.asarray(ev_chk)).cuda().reshape(-1, 1)
    fp64_resid = ((ych - lam * vec_chk).norm(dim=1) / lam.abs().reshape(-1)).max().item()
    info_p = i_plain[-1][1]
    info_m = i_mixed[-1][1]
    ev_p, ev_m = i_plain[-1][0], i_mixed[-1][0]
    applies_p = info_p["applies"]
    value = world * applies_p * float(Nt) * Nt / (ms_plain * 1e-3)

    # roofline of the dominant kernel (float64 stage 5) from the events recorded around it
    fl = FLOPS_PER_EVAL[w["kernel"]]
    calls = info_p["stage5_calls_fp64"]
    ms5 = info_p["ms_stage5_fp64"] / max(calls, 1)
    vecs_per_call = applies_p / max(calls, 1)
    flops_per_pair = 0.5 * fl + 2 * vecs_per_call
    flops_per_launch = float(Nt) * Nt * flops_per_pair
    achieved = flops_per_launch / (ms5 * 1e-3) / 1e12
    stage5_share = info_p["ms_stage5_fp64"] / ms_plain

    # end to end through the public API with host buffers: create + H2D start block + solve + D2H vectors
    def e2e_once():
        t0 = time.perf_counter()
        G2 = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
        host = torch.from_numpy(inputs.random_block(N, args.plain_block, seed=seed).T.copy()).pin_memory()
        dev = host.to("cuda", non_blocking=True)
        ev, vec, info = G2.eigs(k, TOL, method=0, block=args.plain_block, start=dev)
        out = torch.empty((k, N), dtype=torch.float64).pin_memory()
        out.copy_(vec, non_blocking=True)
        torch.cuda.synchronize()
        G2.close()
        return time.perf_counter() - t0, info
    e2e_t, e2e_info = e2e_once()
    e2e_value = world * e2e_info["applies"] * float(Nt) * Nt / e2e_t

    large_cube = None
    if world == 1 and not args.no_large_cube:
        large_cube = measure_large_cube(kl, inputs, flush, stream)
    batched = None
    if world == 1 and not args.no_batched:
        batched = measure_batched(kl, inputs)
    warm = None
    if world == 1 and not args.no_warm_start:
        warm = measure_warm_start(kl, inputs, args.warm_train_solves, args.warm_epochs, args.warm_eval)

    cpu = None
    if rank == 0 and world == 1:
        rows = 15000
        r, dt, _ = oracle_rate(w, rows)
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d of %d rows of the float64 stage-5 product (NumPy, single thread), %.1f s" % (
                   rows, Nt, dt)}

    peaks = read_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_plain, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "dim": w["dim"], "degree": w["p"], "elements": w["ne"],
                   "kernel": w["kernel"], "L": w["L"], "sigma": w["sigma"], "N": N, "Ntilde": Nt, "k": k,
                   "tol": TOL, "plain": "float64 thick-restart block Lanczos, block %d" % args.plain_block,
                   "L2": "flushed between steps (256 MB write)"},
        "time_to_solution_s": {"plain_fp64": ms_plain / 1e3, "chosen_mixed": ms_mixed / 1e3,
                               "plain_df64": ms_pdf / 1e3, "speedup": ms_plain / ms_mixed},
        "plain_df64": {"method": "double-float stage 5 (float64-accurate) block Lanczos, block %d" % args.plain_block,
                       "ms": ms_pdf, "applies": i_pdf[-1][1]["applies"],
                       "max_resid": max(i_pdf[-1][1]["resid"]),
                       "max_rel_eig_diff_vs_plain": float(np.max(np.abs(i_pdf[-1][0] - ev_p) / np.abs(ev_p))),
                       "stage5_df64_ms_per_call": i_pdf[-1][1]["ms_stage5_df64"] /
                       max(i_pdf[-1][1]["stage5_calls_df64"], 1)},
        "plain_fp64": {"applies": applies_p, "block_applies": info_p["block_applies"],
                       "restarts": info_p["restarts"], "max_resid": max(info_p["resid"]),
                       "evals_per_s": value, "eigenvalues": [float(x) for x in ev_p]},
        "chosen_form": {"method": "float32 stage-5 block Lanczos (block %d, symmetric tiles) + block-%d polish "
                                  "with the tensor-core float64-class stage 5 (exact bfloat16 slicing)"
                                  % (args.mixed_block, min(max(k, 32), 48)),
                        "ms": ms_mixed, "applies": info_m["applies"], "applies_tc64": info_m["applies_tc64"],
                        "max_resid": max(info_m["resid"]), "max_resid_fp64_operator": fp64_resid,
                        "stage5_tc64_ms_per_call": info_m["ms_stage5_tc64"] / max(info_m["stage5_calls_tc64"], 1),
                        "max_rel_eig_diff_vs_plain": float(np.max(np.abs(ev_m - ev_p) / np.abs(ev_p))),
                        "evals_per_s": world * info_m["applies"] * float(Nt) * Nt / (ms_mixed * 1e-3),
                        "ms_fp32_phase": info_m["ms_fp32_phase"],
                        "stage5_fp32_ms_per_call": info_m["ms_stage5_fp32"] / max(info_m["stage5_calls_fp32"], 1),
                        "stage5_fp64_ms_per_call": info_m["ms_stage5_fp64"] / max(info_m["stage5_calls_fp64"], 1)},
        "roofline": {"bound": "alu", "kernel": "covmv64_sym_kernel (float64 stage 5, symmetric tiles, exponential)",
                     "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_NOMINAL_TFLOPS,
                     "traffic": SYM64_NV4_TRAFFIC_BYTES if (w["kernel"] == "exp" and Nt == 39304
                                                            and args.plain_block == 4) else None,
                     "peak_source": "nominal GB300 FP64 vector rate (recipe table; MEASURED_PEAKS.json has no "
                                    "FP64 figure); own DFMA microbenchmark: 1.00 TFLOP/s",
                     "flops_per_pair": flops_per_pair, "ms_per_launch": ms5, "launches": calls,
                     "stage5_share_of_step": stage5_share},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": N * args.plain_block * 8,
                "d2h_bytes_per_step": k * N * 8 + k * 8, "seconds": e2e_t},
        "gpu_launches": launches_plain,
        "clocks": clk,
        "peaks_file": {k2: peaks.get(k2) for k2 in ("hbm_gbs", "bf16_tflops", "sm_max_mhz")},
    }
    if large_cube:
        line["cube_p3_48_gauss_mixed_blocks16"] = large_cube
    if batched:
        line["batched_annulus_instances_64"] = batched
    if warm:
        line["learned_warm_start"] = warm
    if cpu:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
