"""Benchmark: time to the 20 leading Karhunen-Loeve eigenpairs at relative residual 1e-8, chosen
(mixed-precision) form against plain float64, on the largest single-GPU workload: the unit cube,
degree-3 splines, 48^3 elements (51^3 = 132,651 Greville points), Gaussian kernel
exp(-|x-x'|^2/L^2), sigma = 1, L = 0.3.

One step = one complete eigensolve of the chosen form through the C ABI (kl_eigs): block Lanczos
with a float32 stage 5 (block 16) until the residual estimates reach 1e-6, then a block-32
polish whose stage 5 runs on the tensor cores in float64-class arithmetic (exact bfloat16
slicing); every operator application runs all nine stages of Algorithm 1 on the GPU.  The line
also carries the plain float64 solve of the same problem, the accuracy of every mode against
the oracle's Kronecker spectrum, the kernel-evaluation rates and the roofline fraction of each
stage-5 kernel.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

--impl reference times the CPU oracle (Algorithm 1 in NumPy, stage 5 spread over the host
cores) on a bounded sample of the same workload and reports its time to solution in the same
unit (extrapolated from the sample; the sample is stated in the line).
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
UNIT = "s"
DEFAULT_WORKLOAD = "cube-p3-48^3-gauss-L0.3"
SECONDARY_WORKLOAD = "cube-p2-32^3-exp-L0.5"
TOL = 1e-8
GOLDEN = os.path.join(ROOT, "tests", "golden")
# stored oracle spectra (written by tests/golden/make_cube_spectra.py, which calls only the oracle)
STORED = {"cube-p3-48^3-gauss-L0.3": "cube_p3_48_gauss_L0.3_kron.json",
          "cube-p2-32^3-exp-L0.5": "cube_p2_32_exp_L0.5_top24.json"}
# reduced meshes of the same problems, on which the oracle's ARPACK solve runs to the end
REDUCED = {"cube-p3-48^3-gauss-L0.3": "cube-p3-16^3-gauss-L0.3",
           "cube-p2-32^3-exp-L0.5": "cube-p2-16^3-exp-L0.5"}


# DRAM bytes (read + write) per launch from one ncu capture of the same kernel on the same
# workload and vector count (profiles/stage5_dram_cube-p3-48^3-gauss.md); None where the kernel
# changed after the capture
TRAFFIC = {("tc64", "cube-p3-48^3-gauss-L0.3", 32): 61230592.0 + 29322240.0,
           ("tc32", "cube-p3-48^3-gauss-L0.3", 32): 29455616.0 + 3426816.0,
           ("fp32", "cube-p3-48^3-gauss-L0.3", 16): 10383616.0 + 58083584.0}


def flops_per_eval(kind):
    """Algorithmic flops of one kernel evaluation: 3 subtractions, 3 multiplications, 2 additions
    and the scaling by 1/L (9), plus one exponential and, for the exponential kernel, one square
    root, each counted as one operation."""
    return 9 + 1 + (1 if kind == "exp" else 0)


def stage5_flops(kind, Nt, nvec, symmetric):
    """Algorithmic flops of one stage-5 launch over nvec vectors: Ntilde^2 ordered pairs, each with
    2 nvec flops of product; the kernel values once per ordered pair, or once per unordered pair
    when the kernel evaluates each value for both (k, l) and (l, k)."""
    evals = float(Nt) * Nt * (0.5 if symmetric else 1.0)
    return evals * flops_per_eval(kind) + float(Nt) * Nt * 2.0 * nvec, evals


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--block", type=int, default=16, help="block size of the chosen form's float32 phase")
    ap.add_argument("--plain-block", type=int, default=4)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain float64 solve of the workload")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 39,304-point exponential cube (chosen form and plain float64)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-instance quarter-annulus batch")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the learned warm start")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle's cpu_baseline leg")
    ap.add_argument("--cpu-seconds", type=float, default=5.0,
                    help="host seconds per oracle sample (rate samples of the cpu_baseline leg)")
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


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


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


# ---------------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline leg and the reference arm only)
# ---------------------------------------------------------------------------------------------
_OW = None


def _oracle_worker_init(w, seed):
    """Pool worker: one oracle problem, its mapped points and a seeded vector, BLAS on one thread."""
    global _OW
    from oracle import ibq
    from paper_2011_13861_gb300 import inputs
    P = ibq.Problem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    X, _ = P.points_and_J()
    _OW = (P, X, inputs.random_block(P.Nt, 1, seed=seed))


def _block_rows(Nt):
    """Row-block height for the oracle's stage 5 that keeps its temporaries (rows x Ntilde) near
    1 Mi entries, so that they stay in the host caches."""
    return max(8, min(256, (1 << 20) // max(Nt, 1)))


def _oracle_rows(idx):
    P, X, u = _OW
    P.stage5(X, u, rows=_block_rows(P.Nt), row_index=idx)
    return len(idx)


def _oracle_stage5_rows(args):
    P, X, _ = _OW
    u, idx = args
    return P.stage5(X, u, rows=_block_rows(P.Nt), row_index=idx)


class OracleHost:
    """The oracle as it stands, timed on the host cores: its stage 5 (Algorithm 1, line 5) split
    by rows over `cores` spawned worker processes (one BLAS thread each), the other stages in this
    process.  Spawned workers never touch the GPU."""

    def __init__(self, w, cores, seed=0):
        import multiprocessing as mp
        self.w, self.cores = w, cores
        old = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in old:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init, initargs=(w, seed))
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        from oracle import ibq
        self.P = ibq.Problem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
        self.pool.map(_oracle_rows, [[0]] * cores)      # workers started and initialised

    def close(self):
        self.pool.close()
        self.pool.join()

    def rate(self, seconds):
        """Kernel evaluations per second of the oracle's stage 5 on an evenly spread row sample
        sized to take about `seconds` (grown from a short probe)."""
        import numpy as np
        Nt = self.P.Nt
        rows = max(self.cores, 64)
        while True:
            idx = np.linspace(0, Nt - 1, rows).astype(np.int64)
            chunks = np.array_split(idx, self.cores * 4)
            t0 = time.perf_counter()
            self.pool.map(_oracle_rows, chunks)
            dt = time.perf_counter() - t0
            if dt >= 0.5 * seconds or rows >= Nt:
                return rows * float(Nt) / dt, rows, dt
            rows = min(Nt, int(rows * max(2.0, 0.7 * seconds / max(dt, 1e-3))))

    def arpack(self, k, tol, seed=1):
        """The oracle's matrix-free operator (stages 1-4 and 6-9 here, stage 5 on the pool)
        inside ARPACK's implicitly restarted Lanczos (scipy eigsh, the paper's solver): time to
        the k largest eigenpairs and the number of operator applications."""
        import numpy as np
        from scipy.sparse.linalg import LinearOperator, eigsh
        P = self.P
        X, _ = P.points_and_J()
        chunks = np.array_split(np.arange(P.Nt), self.cores * 2)
        n = [0]

        def matvec(v):
            n[0] += 1
            u = P.forward(v.reshape(P.N, -1))
            z = np.concatenate(self.pool.map(_oracle_stage5_rows, [(u, c) for c in chunks]))
            return P.backward(z).reshape(v.shape)

        op = LinearOperator((P.N, P.N), matvec=matvec, dtype=np.float64)
        v0 = np.random.default_rng(seed).uniform(-1.0, 1.0, P.N)
        t0 = time.perf_counter()
        w, _ = eigsh(op, k=k, which="LA", tol=tol, v0=v0)
        return time.perf_counter() - t0, n[0], np.sort(w)[::-1]


def oracle_time_to_solution(w, cores, seconds, reduced=None):
    """The oracle's time to the workload's k eigenpairs on `cores` host cores.  Small workloads
    run ARPACK to the end; for large ones ARPACK runs on the reduced mesh of the same problem
    (its application count stands for the full mesh's) and the full-mesh time is that count times
    Ntilde^2 over the oracle's evaluation rate measured on a row sample of the full mesh."""
    from paper_2011_13861_gb300 import inputs
    out = {"cores": cores}
    if reduced is None:
        oh = OracleHost(w, cores)
        try:
            t, napp, _ = oh.arpack(w["k"], TOL)
            r, rows, dt = oh.rate(seconds)
        finally:
            oh.close()
        out.update(seconds=t, applications=napp, rate=r, extrapolated=False,
                   sample="ARPACK (scipy eigsh, k=%d, tol 1e-8) with the oracle's operator to the end, %d "
                          "applications, %.2f s" % (w["k"], napp, t))
        return out
    wr = inputs.WORKLOADS[reduced]
    oh = OracleHost(wr, cores)
    try:
        tr, napp, _ = oh.arpack(w["k"], TOL)
    finally:
        oh.close()
    oh = OracleHost(w, cores)
    try:
        r, rows, dt = oh.rate(seconds)
    finally:
        oh.close()
    Nt = oh.P.Nt
    out.update(seconds=napp * float(Nt) * Nt / r, applications=napp, rate=r, extrapolated=True,
               reduced_seconds=tr, sample_rows=rows, sample_seconds=dt,
               sample="extrapolated: ARPACK (scipy eigsh, k=%d, tol 1e-8) with the oracle's operator on "
                      "the reduced mesh %s took %d applications (%.1f s); the oracle's stage 5 ran %d of "
                      "%d rows of the full mesh in %.1f s (%.3g evals/s); time = applications x "
                      "Ntilde^2 / rate" % (w["k"], reduced, napp, tr, rows, Nt, dt, r))
    return out


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2011_13861_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    reduced = REDUCED.get(args.workload)
    cores = host_cores()
    napp, tred = None, None
    if reduced is not None:
        oh = OracleHost(inputs.WORKLOADS[reduced], cores)
        try:
            tred, napp, _ = oh.arpack(w["k"], TOL)
        finally:
            oh.close()
    oh = OracleHost(w, cores)
    Nt = oh.P.Nt
    secs, rows_used = [], 0
    try:
        if reduced is None:
            for _ in range(args.warmup):
                oh.arpack(w["k"], TOL)
            for _ in range(args.steps):
                t, napp, _ = oh.arpack(w["k"], TOL)
                secs.append(t)
            sample = "ARPACK (scipy eigsh, k=%d, tol 1e-8) with the oracle's operator to the end (%d applications)" % (
                w["k"], napp)
        else:
            for _ in range(args.warmup):
                oh.rate(0.3 * args.cpu_seconds)
            for _ in range(args.steps):
                r, rows_used, _ = oh.rate(args.cpu_seconds)
                secs.append(napp * float(Nt) * Nt / r)
            sample = ("extrapolated per step: %d ARPACK applications (counted on the reduced mesh %s, %.1f s) x "
                      "Ntilde^2 / the oracle's stage-5 rate on %d sampled rows of the full mesh"
                      % (napp, reduced, tred, rows_used))
    finally:
        oh.close()
    value = statistics.mean(secs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * value,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "Ntilde": Nt, "k": w["k"], "tol": TOL,
                                            "L2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline_leg(w, workload, seconds):
    """The oracle on this machine's host cores: time to solution with every core (the value, same unit
    as the line) and the single-core evaluation rate (the paper's setting: one core)."""
    cores = host_cores()
    allc = oracle_time_to_solution(w, cores, seconds, REDUCED.get(workload))
    one = OracleHost(w, 1)
    try:
        r1, rows1, dt1 = one.rate(seconds)
    finally:
        one.close()
    return {"value": allc["seconds"], "unit": UNIT, "cores": cores, "kind": "oracle", "sample": allc["sample"],
            "evals_per_s_all_cores": allc["rate"], "evals_per_s_one_core": r1,
            "one_core_sample": "%d rows of the oracle's stage 5 on one core in %.1f s" % (rows1, dt1),
            "applications": allc["applications"], "extrapolated": allc["extrapolated"],
            "time_to_solution_one_core_s": allc["applications"] * float(w_nt(w)) ** 2 / r1}


def w_nt(w):
    import numpy as np
    ne = w["ne"] if np.ndim(w["ne"]) else [w["ne"]] * w["dim"]
    return int(np.prod([n + w["p"] for n in ne]))


# ---------------------------------------------------------------------------------------------
# accuracy against the stored oracle spectra
# ---------------------------------------------------------------------------------------------
def mode_accuracy(workload, ev, vecs, k):
    """Per-mode relative eigenvalue error against the stored oracle spectrum and, where the file
    holds eigenvectors (the separable Gaussian cube: Kronecker products of 1D oracle pairs), the
    largest principal-angle sine between each computed eigenvector cluster and the oracle's
    eigenspace of that eigenvalue."""
    import numpy as np
    name = STORED.get(workload)
    if name is None:
        return None
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    ref = np.array(g["eigenvalues"])
    ev = np.asarray(ev)[:k]
    out = {"reference": g["source"], "rel_eig_err": [float(x) for x in np.abs(ev - ref[:k]) / np.abs(ref[:k])]}
    out["max_rel_eig_err"] = max(out["rel_eig_err"])
    if "u_1d" not in g or vecs is None:
        out["subspace_sine"] = None
        return out
    U = np.array(g["u_1d"]).T
    trip = g["triples"]
    V = vecs.cpu().numpy().T if hasattr(vecs, "cpu") else np.asarray(vecs)
    sines = [None] * k
    rtol = 1e-9 * ref[0]
    i = 0
    while i < k:
        j = i
        while j + 1 < k and abs(ref[j + 1] - ref[i]) <= rtol:
            j += 1
        members = [t for lam, t in zip(ref, trip) if abs(lam - ref[i]) <= rtol]
        Q = np.stack([np.kron(U[:, c], np.kron(U[:, b], U[:, a])) for a, b, c in members], axis=1)
        Q, _ = np.linalg.qr(Q)
        Vc = V[:, i:j + 1]
        s = float(np.linalg.norm(Vc - Q @ (Q.T @ Vc), 2))
        for m in range(i, j + 1):
            sines[m] = s
        i = j + 1
    out["subspace_sine"] = sines
    out["max_subspace_sine"] = max(sines)
    return out


def flush_l2(buf):
    buf.add_(1.0)


# ---------------------------------------------------------------------------------------------
# secondary legs
# ---------------------------------------------------------------------------------------------
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
    # the first batched call also allocates every handle's solver workspace, times the column
    # split candidates and captures the launch graphs: timed separately, then the steady state
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kl.eigs_batched(Gs, 10, TOL, **opts)
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
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
           "batched_first_call_s": t_first,
           "batched_s": t_batch, "sequential_s": t_seq, "batched_vs_sequential": t_seq / t_batch,
           "converged": int(sum(1 for x in sts if x == 0)), "max_resid": max(max(i["resid"]) for i in infos),
           "max_rel_eig_diff_batched_vs_sequential": float(max(np.abs(ev_b[i] - ev_s[i]).max() / abs(ev_s[i][0])
                                                              for i in range(len(Gs)))),
           "batched_stage5_ms": bi["ms_stage5"], "batched_launches": bi["rounds"], "requests": bi["requests"],
           "cols_per_split": bi["cols_per_split"], "points_min_max": [int(Nt.min()), int(Nt.max())],
           "sum_pairs_per_application": float((Nt ** 2).sum()),
           "timing": "wall clock with a device synchronisation on both sides, one run each, after one "
                     "untimed batched call (workspaces, column-split choice, graph capture: batched_first_call_s)"}
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
    configuration) and, for the first parameter set, random-start float64 block Lanczos (block 4)."""
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
        start = ws.start_block(fine, prm)
        Qs, _ = torch.linalg.qr(start.T)
        cosv = torch.linalg.svdvals(Qs.T @ vec_w.T).cpu().numpy()
        row = {"kernel": prm["kernel"], "L": prm["L"], "r_in": prm["r_in"], "r_out": prm["r_out"],
               "path": iw["path"], "warm_s": tw, "warm_applies": iw["applies"], "warm_restarts": iw["restarts"],
               "random32_s": t32, "random32_applies": i32["applies"], "random16_s": t16,
               "random16_applies": i16["applies"], "gain_vs_random32": t32 / tw, "gain_vs_random16": t16 / tw,
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


def roofline_entry(name, bound, kind, Nt, nvec, symmetric, ms, launches, peak_flops, peak_label, traffic=None):
    flops, evals = stage5_flops(kind, Nt, nvec, symmetric)
    achieved = flops / (ms * 1e-3) / 1e12
    peak = peak_flops / 1e12
    return {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_label,
            "flops_per_launch": flops, "executed_evals_per_launch": evals,
            "logical_evals_per_launch": float(Nt) * Nt, "vectors_per_launch": nvec,
            "ms_per_launch": ms, "launches": launches}


def timed_events(fn, flush, stream, clocks=None, steps=1, barrier=None):
    import torch
    times, outs = [], []
    if clocks:
        clocks.start()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    for _ in range(steps):
        flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        outs.append(out)
    if barrier:
        barrier()
    clk = clocks.stop() if clocks else None
    return times, outs, clk


def measure_secondary(kl, inputs, flush, stream, plain_block, mixed_block, steps, dfma_flops):
    """The 39,304-point exponential cube (p=2, 32^3, L=0.5): chosen form against plain float64,
    eigenvalues per mode against the stored oracle spectrum (dense Gamma inside ARPACK)."""
    import numpy as np
    import torch
    w = inputs.WORKLOADS[SECONDARY_WORKLOAD]
    k = w["k"]
    G = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    sp = torch.from_numpy(inputs.random_block(G.N, plain_block, seed=1).T.copy()).cuda()
    sm = torch.from_numpy(inputs.random_block(G.N, mixed_block, seed=1).T.copy()).cuda()
    plain = lambda: G.eigs(k, TOL, method=0, block=plain_block, start=sp, want_vectors=False)  # noqa: E731
    chosen = lambda: G.eigs(k, TOL, method=1, block=mixed_block, start=sm, precision=kl.KL_P_TC64,  # noqa: E731
                            want_vectors=False)
    for _ in range(2):
        plain()
        chosen()
    tp, op, _ = timed_events(plain, flush, stream, steps=steps)
    tc, oc, _ = timed_events(chosen, flush, stream, steps=steps)
    ev_p, _, ip = op[-1]
    ev_c, _, ic = oc[-1]
    Nt = G.Nt
    ms_p, ms_c = statistics.mean(tp), statistics.mean(tc)
    calls = max(ip["stage5_calls_fp64"], 1)
    out = {"workload": SECONDARY_WORKLOAD, "N": G.N, "Ntilde": Nt, "k": k,
           "plain_fp64_s": ms_p / 1e3, "chosen_s": ms_c / 1e3, "speedup": ms_p / ms_c,
           "plain": "float64 thick-restart block Lanczos, block %d" % plain_block,
           "chosen": "float32 stage-5 block Lanczos (block %d) + block-32 polish: one tensor-core "
                     "float64-class stage 5, float32 correction blocks" % mixed_block,
           "plain_applies": ip["applies"], "chosen_applies": ic["applies"],
           "plain_evals_per_s": ip["applies"] * float(Nt) * Nt / (ms_p * 1e-3),
           "chosen_evals_per_s": ic["applies"] * float(Nt) * Nt / (ms_c * 1e-3),
           "max_resid_plain": max(ip["resid"]), "max_resid_chosen": max(ic["resid"]),
           "accuracy_plain": mode_accuracy(SECONDARY_WORKLOAD, ev_p, None, k),
           "accuracy_chosen": mode_accuracy(SECONDARY_WORKLOAD, ev_c, None, k),
           "plain_stage5_fp64_ms_per_call": ip["ms_stage5_fp64"] / calls,
           "chosen_stage5_ms": {"fp32": ic["ms_stage5_fp32"], "tc64": ic["ms_stage5_tc64"],
                                "tc32": ic["ms_stage5_tc32"]},
           "timing": "CUDA events, mean of %d after 2 warm-ups each, L2 flushed" % steps}
    out["roofline_plain_fp64"] = roofline_entry(
        "covmv64_sym_kernel (float64 stage 5, symmetric tiles)", "alu", w["kernel"], Nt,
        ip["applies"] / calls, True, ip["ms_stage5_fp64"] / calls, calls, dfma_flops,
        "measured float64 FMA rate x 2 (kl_pipe_rates, this run)")
    G.close()
    return out


# ---------------------------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------------------------
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
    barrier = dist.barrier if world > 1 else None
    pipes = kl.pipe_rates()
    dfma_flops, ffma_flops = 2.0 * pipes["dfma_per_s"], 2.0 * pipes["ffma_per_s"]

    w = inputs.WORKLOADS[args.workload]
    k = w["k"]
    G = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
    N, Nt = G.N, G.Nt
    seed = 1 + rank      # each rank solves its own instance: independent problems, no collective
    start_c = torch.from_numpy(inputs.random_block(N, args.block, seed=seed).T.copy()).cuda()
    start_p = torch.from_numpy(inputs.random_block(N, args.plain_block, seed=seed).T.copy()).cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def solve_chosen():
        # float32 stage 5 until the estimates reach 1e-6, then a polish block of max(k, 32) whose
        # first application runs on the tensor cores with exact slicing (float64-class) and whose
        # correction blocks take the float32 stage 5
        return G.eigs(k, TOL, method=1, block=args.block, start=start_c, precision=kl.KL_P_TC64)

    for _ in range(args.warmup):
        solve_chosen()
    torch.cuda.synchronize()
    launches0 = kl.kernel_launches()
    clocks = ClockSampler(local)
    t_c, outs, clk = timed_events(solve_chosen, flush, stream, clocks, args.steps, barrier)
    launches = (kl.kernel_launches() - launches0) / args.steps
    ms_c = statistics.mean(t_c)
    if world > 1:
        ms_c = max_over_ranks([ms_c], device="cuda")[0]
    ev_c, vec_c, info_c = outs[-1]
    # untimed: residuals of the chosen form's eigenvectors under the float64 operator, and the
    # accuracy of every mode against the oracle's spectrum
    ych = G.apply(vec_c)
    lam = torch.from_numpy(np.asarray(ev_c)).cuda().reshape(-1, 1)
    fp64_resid = ((ych - lam * vec_c).norm(dim=1) / lam.abs().reshape(-1)).cpu().numpy()
    acc_c = mode_accuracy(args.workload, ev_c, vec_c, k)
    del ych

    plain = None
    if not args.no_plain:
        tp, op, _ = timed_events(lambda: G.eigs(k, TOL, method=0, block=args.plain_block, start=start_p),
                                 flush, stream, steps=1)
        ev_p, vec_p, info_p = op[-1]
        calls = max(info_p["stage5_calls_fp64"], 1)
        plain = {"method": "float64 thick-restart block Lanczos, block %d, every application float64" % args.plain_block,
                 "seconds": tp[0] / 1e3, "applies": info_p["applies"], "restarts": info_p["restarts"],
                 "max_resid": max(info_p["resid"]),
                 "evals_per_s": info_p["applies"] * float(Nt) * Nt / (tp[0] * 1e-3),
                 "accuracy": mode_accuracy(args.workload, ev_p, vec_p, k),
                 "max_rel_eig_diff_chosen_vs_plain": float(np.max(np.abs(ev_c - ev_p) / np.abs(ev_p))),
                 "roofline": roofline_entry("covmv64_sym_kernel (float64 stage 5, symmetric tiles)", "alu",
                                            w["kernel"], Nt, info_p["applies"] / calls, True,
                                            info_p["ms_stage5_fp64"] / calls, calls, dfma_flops,
                                            "measured float64 FMA rate x 2 (kl_pipe_rates, this run)"),
                 "timing": "CUDA events, one run, L2 flushed"}
        del vec_p

    # roofline of each stage-5 kernel of the chosen form, from the events the library records
    # around every stage-5 launch on the launching stream during the timed solves
    rl = {}
    nc32 = info_c["stage5_calls_fp32"]
    if nc32:
        # float32 calls: the float32 phase's blocks and the polish's correction blocks; the kernel
        # runs groups of at most 16 vectors (a 32-vector call is two launches of the 16-wide kernel)
        v32 = (info_c["applies"] - info_c["applies_fp64"] - info_c["applies_df64"] - info_c["applies_tc64"]
               - info_c["applies_tc32"])
        g32 = max(nc32, -(-v32 // 16))
        rl["fp32"] = roofline_entry("covmv32_kernel (float32 stage 5, packed pair FMAs, %g-vector groups)" % (v32 / g32),
                                    "alu", w["kernel"], Nt, v32 / g32, v32 / g32 <= 8, info_c["ms_stage5_fp32"] / g32,
                                    g32, ffma_flops, "measured float32 FMA rate x 2 (kl_pipe_rates, this run)",
                                    TRAFFIC.get(("fp32", args.workload, int(round(v32 / g32)))))
    nc64 = info_c["stage5_calls_tc64"]
    if nc64:
        nv64 = info_c["applies_tc64"] / nc64
        rl["tc64"] = roofline_entry(
            "covmv_tcx_kernel<64> (tensor-core float64-class stage 5, exact bf16 slices)", "alu", w["kernel"], Nt,
            nv64, False, info_c["ms_stage5_tc64"] / nc64, nc64, ffma_flops,
            "measured float32 FMA rate x 2 (kl_pipe_rates, this run): the kernel's double-float "
            "kernel values and slicing run on the float32 pipe, its bound",
            TRAFFIC.get(("tc64", args.workload, int(round(nv64)))))
    nt32 = info_c["stage5_calls_tc32"]
    if nt32:
        nvt = info_c["applies_tc32"] / nt32
        rl["tc32"] = roofline_entry(
            "covmv_tcx_kernel<32> (tensor-core float32 class, the polish's correction blocks)", "alu", w["kernel"],
            Nt, nvt, False, info_c["ms_stage5_tc32"] / nt32, nt32, ffma_flops,
            "measured float32 FMA rate x 2 (kl_pipe_rates, this run): kernel values and slicing on the float32 pipe",
            TRAFFIC.get(("tc32", args.workload, int(round(nvt)))))
    share = {key: (info_c["ms_stage5_" + key] / ms_c) for key in ("fp32", "tc64", "tc32")}
    dom = max(rl, key=lambda key: share[key]) if rl else None
    roofline = dict(rl[dom]) if dom else None
    if roofline is not None:
        roofline["share_of_step"] = share[dom]

    # end to end through the public API with host buffers: create + H2D start block + solve + D2H
    def e2e_once():
        t0 = time.perf_counter()
        G2 = kl.KLProblem(w["dim"], w["p"], w["ne"], kernel=w["kernel"], sigma=w["sigma"], L=w["L"])
        host = torch.from_numpy(inputs.random_block(N, args.block, seed=seed).T.copy()).pin_memory()
        dev = host.to("cuda", non_blocking=True)
        ev, vec, info = G2.eigs(k, TOL, method=1, block=args.block, start=dev, precision=kl.KL_P_TC64)
        out = torch.empty((k, N), dtype=torch.float64).pin_memory()
        out.copy_(vec, non_blocking=True)
        torch.cuda.synchronize()
        G2.close()
        return time.perf_counter() - t0
    e2e_t = e2e_once()
    if world > 1:
        e2e_t = max_over_ranks([e2e_t], device="cuda")[0]

    secondary = batched = warm = None
    if world == 1 and not args.no_secondary:
        secondary = measure_secondary(kl, inputs, flush, stream, 4, 16, 3, dfma_flops)
    if world == 1 and not args.no_batched:
        batched = measure_batched(kl, inputs)
    if world == 1 and not args.no_warm_start:
        warm = measure_warm_start(kl, inputs, args.warm_train_solves, args.warm_epochs, args.warm_eval)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_leg(w, args.workload, args.cpu_seconds)

    peaks = read_peaks()
    line = {
        "metric": METRIC, "value": ms_c / 1e3, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_c, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 + f64-class (bf16 tcgen05 slices); f64 polish solver, df64 float32-phase basis products",
        "data": "synthetic",
        "config": {"workload": args.workload, "dim": w["dim"], "degree": w["p"], "elements": w["ne"],
                   "kernel": w["kernel"], "L": w["L"], "sigma": w["sigma"], "N": N, "Ntilde": Nt, "k": k,
                   "tol": TOL, "chosen_form": "block Lanczos, float32 stage 5 (block %d) to 1e-6, then a "
                                              "block-32 polish: one tensor-core float64-class stage 5 on "
                                              "the float32 Ritz block, float32 correction blocks"
                                              % args.block,
                   "L2": "flushed between steps (256 MB write)"},
        "chosen": {"seconds": ms_c / 1e3, "step_ms": t_c, "applies": info_c["applies"],
                   "applies_tc64": info_c["applies_tc64"], "restarts": info_c["restarts"],
                   "max_resid": max(info_c["resid"]), "max_resid_fp64_operator": float(fp64_resid.max()),
                   "resid_fp64_operator": [float(x) for x in fp64_resid],
                   "evals_per_s": info_c["applies"] * float(Nt) * Nt / (ms_c * 1e-3),
                   "ms_fp32_phase": info_c["ms_fp32_phase"],
                   "stage5_ms": {"fp32": info_c["ms_stage5_fp32"], "tc64": info_c["ms_stage5_tc64"],
                                 "tc32": info_c["ms_stage5_tc32"]},
                   "accuracy": acc_c},
        "plain_fp64": plain,
        "speedup_vs_plain_fp64": (plain["seconds"] / (ms_c / 1e3)) if plain else None,
        "eigenvalues": [float(x) for x in ev_c],
        "roofline": roofline,
        "rooflines": rl,
        "pipe_rates": pipes,
        "e2e": {"value": e2e_t, "unit": UNIT, "h2d_bytes_per_step": N * args.block * 8,
                "d2h_bytes_per_step": k * N * 8 + k * 8,
                "what": "kl_create + pinned host start block copied in + kl_eigs + eigenvectors copied out"},
        "gpu_launches": int(round(launches)),
        "clocks": clk,
        "peaks_file": {k2: peaks.get(k2) for k2 in ("hbm_gbs", "bf16_tflops", "sm_max_mhz")},
    }
    if secondary:
        line["cube_p2_32_exp_secondary"] = secondary
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
