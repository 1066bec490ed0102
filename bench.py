#!/usr/bin/env python3
"""REBK benchmark on GB300: solves/s to 1e-8 relative error.

Workload (the precision configuration): A = G1 G2 with G1 = randn(8000, 2000),
G2 = randn(2000, 20000) (m = 8000, n = 20000, rank 2000, rank-deficient and
underdetermined), inconsistent b = A x* + N(0, 0.01^2), seed = rank;
contiguous blocks tau = 128 (Section 3 partitions); alpha = 1.75 / beta_max
(Section 3's empirical step, beta_max from the block spectral norms on the
GPU).  A step is one complete solve to ||x - A^+ b|| <= 1e-8 ||A^+ b|| (the
paper's stop rule with a relative tolerance) by the mixed-precision path:
FP32 or BF16 storage, FP32 inner sweeps, FP64 refinement.  The plain FP64
path is timed on the same problem for comparison.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

M, N, RANK, TAU, TOL = 8000, 20000, 2000, 128, 1e-8
METRIC = "solves/s to 1e-8 rel err (mixed+warm-start+batched vs plain FP64); HBM GB/s"
WORKLOAD = ("precision: A = G1 G2, G1 = randn(8000,2000), G2 = randn(2000,20000) "
            "(8000x20000, rank 2000), b = A x* + N(0,0.01^2), tau = 128, alpha = 1.75/beta_max, "
            "stop ||x - A^+b|| <= 1e-8 ||A^+b||")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--profile-plain", action="store_true",
                    help="with --profile-pass K: run K iterations of the plain FP64 kernel instead")
    ap.add_argument("--storage", choices=["fp32", "bf16"], default="fp32")
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=8.0, help="oracle sample per CPU build (seconds)")
    ap.add_argument("--residual-steps", type=int, default=2,
                    help="mixed solves timed with the residual stop rule (no known solution)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["precision", "warm", "batch", "sparse", "sweep", "free"], default="precision",
                    help="precision: the headline solve (default); warm: the learned warm start "
                         "on the 8192 x 2048 spectrum workload (targets, training, warm vs cold)")
    ap.add_argument("--sparse-mixed", action="store_true",
                    help="with --workload sparse --profile-pass K: run the mixed-precision pass")
    ap.add_argument("--batch-probe", choices=["", "all", "one"], default="",
                    help="with --workload batch: time one iteration of the batched kernel per system shape")
    ap.add_argument("--sweep-parts", default="", help="sweep workload: comma-separated parts 1-6 (default all)")
    ap.add_argument("--batch-tau", type=int, default=16, help="batch workload block size (0 = autotune)")
    ap.add_argument("--batch-cluster", type=int, default=0,
                    help="batch workload: CTAs per cluster for the longest systems (1 = none, 0 = library choice)")
    ap.add_argument("--batch-joint-frac", type=float, default=0.0,
                    help="batch workload: cluster threshold as a fraction of the mean load per CTA (0 = 0.25)")
    ap.add_argument("--batch-probe-shape", default="", help="with --batch-probe one: the system shape m,n")
    ap.add_argument("--batch-probe-iters", type=int, default=2000, help="batch probe: iterations per pass")
    ap.add_argument("--batch-count", type=int, default=512, help="batch workload: number of systems")
    ap.add_argument("--batch-scale", type=int, default=1, help="batch workload: divide the size ranges (profiling)")
    ap.add_argument("--warm-train", type=int, default=2048)
    ap.add_argument("--warm-eval", type=int, default=32)
    ap.add_argument("--warm-batch-systems", type=int, default=152)
    ap.add_argument("--warm-steps", type=int, default=4000)
    ap.add_argument("--no-combined", action="store_true",
                    help="skip the mixed + warm-start + batched measurement on the 8192 x 2048 stream")
    ap.add_argument("--combined-train", type=int, default=1024, help="combined form: training right-hand sides")
    ap.add_argument("--combined-systems", type=int, default=152,
                    help="combined form: batched systems of 8 held-out right-hand sides (sharing A)")
    ap.add_argument("--combined-steps", type=int, default=1500, help="combined form: network training steps")
    ap.add_argument("--combined-batch-tau", type=int, default=0,
                    help="combined form: block size of the timed batched solves (0 = the batch autotuner's choice)")
    ap.add_argument("--combined-target-iters", type=int, default=8000,
                    help="combined form: inner iterations per refinement pass of the target solves (2 passes)")
    ap.add_argument("--combined-stream", type=int, default=100000,
                    help="combined form: stream length over which target generation and training are amortised")
    ap.add_argument("--profile-mlp", type=int, default=0, metavar="K",
                    help="run K training steps (batch 256) of the 8192 -> 512 -> 512 -> 8192 warm-start network "
                         "and print the time per step (the case the network's ncu summary captures)")
    ap.add_argument("--num-ctas", type=int, default=0,
                    help="CTAs of the persistent kernel on the precision workload (0 = the library's autotune)")
    ap.add_argument("--multi-rhs", type=int, default=16,
                    help="precision workload: right-hand sides of the multi-right-hand-side leg (0 = skip)")
    ap.add_argument("--multi-steps", type=int, default=2, help="timed steps of the multi-right-hand-side leg")
    ap.add_argument("--profile-multi", type=int, default=0, metavar="K",
                    help="run one K-iteration pass of the multi-right-hand-side kernel (one group) twice and exit")
    ap.add_argument("--profile-pass", type=int, default=0, metavar="K",
                    help="run one K-iteration refinement pass of the workload twice and exit "
                         "(the case the ncu summaries under profiles/ capture)")
    return ap.parse_args()


def replica_throughput(elapsed_local: float, units_local: int, world: int, device=None):
    """Whole-job throughput of `world` independent replicas (one problem per
    rank, no collective on the data path): every rank processed units_local
    units in elapsed_local (any time unit); the job took as long as the slowest
    rank (all-reduce MAX when a process group is up).  Returns (units per time
    unit over all ranks, the job's elapsed time)."""
    t = elapsed_local
    if world > 1:
        import torch
        import torch.distributed as dist
        v = torch.tensor([elapsed_local], dtype=torch.float64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        t = float(v.item())
    return units_local * world / t, t


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


def load_anchor():
    path = os.path.join(ROOT, "tests", "golden", "precision_anchor.txt")
    out = {}
    if os.path.exists(path):
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


# DRAM traffic per iteration of the dominant kernel, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one profiled pass, divided by
# its iterations; the capture and its command are summarised in
# profiles/rebk_grid_precision_8000x20000.md).  Keyed by the kernel's
# storage form and the source hash of rebk_grid.cu it was taken on: a changed
# kernel reports null until it is captured again.
KERNEL_TRAFFIC = {
    "corr_fp32": {"source_sha": "13c1267590cf3297", "dram_bytes_per_iteration": 24459010560 / 2000,
                  "from": "ncu summary, scaled: dram__bytes_read.sum + dram__bytes_write.sum of one "
                          "2000-iteration pass at 152 CTAs (bench.py --profile-pass 2000 --num-ctas 152)"},
}


def kernel_traffic(kernel_tag: str):
    """(DRAM bytes per iteration, provenance) of the headline kernel, or (None, why)."""
    import hashlib
    src = os.path.join(ROOT, "paper_2001_04179_gb300", "csrc", "rebk_grid.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    rec = KERNEL_TRAFFIC.get(kernel_tag)
    if rec is None or rec["source_sha"] != sha:
        return None, f"no ncu capture of the current kernel source ({sha})"
    return rec["dram_bytes_per_iteration"], rec["from"]


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def measure_multi(args, sol, prob, dev, rank, storage, stream, hbm_peak):
    """The precision workload's A with args.multi_rhs right-hand sides solved by
    rebk_solve_multi: groups that share one block sequence, each member to 1e-8
    against its own A^+ b (verified).  solves/s = right-hand sides per second."""
    import torch
    nrhs = args.multi_rhs
    pm = make_problem(rank, True, nrhs=nrhs)  # the same factors, hence the same A
    if not (np.array_equal(pm.A[0], prob.A[0]) and np.array_equal(pm.A[-1], prob.A[-1])):
        raise RuntimeError("multi-right-hand-side leg: regenerated A differs from the solver's")
    B = torch.from_numpy(np.ascontiguousarray(pm.b.T)).to(dev)
    Xr = torch.from_numpy(np.ascontiguousarray(pm.x_ref.T)).to(dev)
    del pm
    group = sol.multi_group(storage)
    sol.solve_multi(B[:group], tol=TOL, seed=600, storage=storage, X_ref=Xr[:group])
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    agg = {"iterations": 0, "kernel_ms": 0.0, "sweep_ms": 0.0, "launches": 0, "grid_launches": 0}
    worst = 0.0
    ev0.record(stream)
    for s_ in range(args.multi_steps):
        r = sol.solve_multi(B, tol=TOL, seed=610 + s_, storage=storage, X_ref=Xr)
        if r["status"] != 0 or float(r["rel"].max()) > TOL:
            raise RuntimeError(f"multi-right-hand-side solve did not reach {TOL}: {r['stats']}")
        worst = max(worst, float(r["rel"].max()))
        for k in agg:
            agg[k] += r["stats"][k]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    groups = args.multi_steps * ((nrhs + group - 1) // group)
    esize = {"fp32": 4, "bf16": 2}[storage]
    bytes_it = float(TAU * N + TAU * M) * esize
    kernel_s = agg["kernel_ms"] / 1000.0
    return {"value": nrhs * args.multi_steps / (ms / 1000.0), "unit": "solves/s", "storage": storage,
            "rhs_per_step": nrhs, "group": group, "steps": args.multi_steps, "ms_per_step": ms / args.multi_steps,
            "iterations_per_group": agg["iterations"] / groups, "kernel_ms_per_step": agg["kernel_ms"] / args.multi_steps,
            "fp64_products_ms_per_step": agg["sweep_ms"] / args.multi_steps,
            "us_per_iteration": 1000.0 * agg["kernel_ms"] / max(agg["iterations"], 1),
            "rhs_iterations_per_s": group * agg["iterations"] / kernel_s,
            "rel_err_max": worst, "gpu_launches": agg["launches"],
            "kernel_hbm_gbs": bytes_it * agg["iterations"] / kernel_s / 1e9,
            "kernel_hbm_frac": bytes_it * agg["iterations"] / kernel_s / 1e9 / hbm_peak,
            "note": "every member of a group draws the same blocks (one TMA read of a block serves the group); "
                    "each right-hand side verified <= 1e-8 against its own A^+ b; FP64 refinement sweeps included"}


def make_problem(seed: int, use_gpu: bool, nrhs: int = 0):
    from workloads import product_problem
    mm = None
    if use_gpu:
        import torch

        def mm(a, b):
            ta = torch.from_numpy(np.ascontiguousarray(a)).cuda()
            tb = torch.from_numpy(np.ascontiguousarray(b)).cuda()
            r = (ta @ tb).cpu().numpy()
            del ta, tb
            return r
    return product_problem(M, N, RANK, seed=seed, noise=0.01, matmul=mm, nrhs=nrhs)


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


ORACLE_BUILDS = {
    "parity": ("C -O2 -ffp-contract=off, the parity build the tests use", 1),
    "fast": ("C -O3 -ffp-contract=fast (FMA contraction; generic target, no -march flag: the host code "
             "builds the same on x86-64 and Arm)", 1),
    "omp": ("C -O3 -ffp-contract=fast -fopenmp, block products split over all host threads", None),
}


def time_oracle(prob, alpha, seconds, variant, seed=1000):
    """Iterations/s of the oracle's Algorithm 1 (build `variant`) on the workload,
    over a bounded sample of about `seconds`."""
    import oracle as O
    from workloads import contiguous_offsets
    ro, co = contiguous_offsets(M, TAU), contiguous_offsets(N, TAU)
    norms = O.block_norms(prob.A, ro, co)
    O.rebk(prob.A, prob.b, ro, co, alpha, seed=seed, iters=2, norms=norms, variant=variant)  # load, threads up
    t0 = time.perf_counter()
    O.rebk(prob.A, prob.b, ro, co, alpha, seed=seed, iters=8, norms=norms, variant=variant)
    per = (time.perf_counter() - t0) / 8
    n_it = max(5, int(seconds / max(per, 1e-6)))
    t0 = time.perf_counter()
    O.rebk(prob.A, prob.b, ro, co, alpha, seed=seed, iters=n_it, norms=norms, variant=variant)
    dt = time.perf_counter() - t0
    return n_it / dt, n_it, dt


def cpu_baseline(prob, alpha, iters_per_solve, seconds, source):
    """The oracle (plain FP64 Algorithm 1) on the host cores: the parity build
    and an -O3 build on one thread, and the OpenMP build on all host threads,
    each on a bounded sample of iterations of the same workload; solves/s =
    iterations/s divided by the iterations one solve needs.  The line's value is
    the fastest build's."""
    cores = os.cpu_count() or 1
    builds = {}
    for variant, (desc, threads) in ORACLE_BUILDS.items():
        try:
            its, n_it, dt = time_oracle(prob, alpha, seconds, variant)
        except Exception as exc:  # an OpenMP runtime missing on the host, say
            builds[variant] = {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}
            continue
        builds[variant] = {"value": its / iters_per_solve, "unit": "solves/s", "iterations_per_s": its,
                           "threads": threads or int(os.environ.get("OMP_NUM_THREADS", cores)),
                           "build": desc, "sample": f"{n_it} iterations in {dt:.1f} s"}
    ok = {k: v for k, v in builds.items() if "value" in v}
    best = max(ok, key=lambda k: ok[k]["value"])
    return {"value": ok[best]["value"], "unit": "solves/s", "cores": ok[best]["threads"], "kind": "oracle",
            "iterations_per_s": ok[best]["iterations_per_s"], "build": best,
            "host_cores": cores, "cpu_model": cpu_model(), "builds": builds,
            "sample": (f"the FP64 oracle of Algorithm 1 on this workload, about {seconds:.0f} s of iterations "
                       f"per build; solves/s = iterations/s / {iters_per_solve:.0f} iterations per solve "
                       f"({source})")}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    anchor = load_anchor()
    use_gpu = False
    try:
        import torch
        use_gpu = torch.cuda.is_available()
    except Exception:
        pass
    prob = make_problem(0, use_gpu)
    alpha = anchor.get("alpha")
    if alpha is None:
        import oracle as O
        from workloads import contiguous_offsets
        alpha = 1.75 / max(O.beta_max(prob.A, contiguous_offsets(M, TAU), contiguous_offsets(N, TAU)))
    ipsolve = anchor.get("iterations_to_1e-8", float("nan"))
    import oracle as O
    from workloads import contiguous_offsets
    ro, co = contiguous_offsets(M, TAU), contiguous_offsets(N, TAU)
    norms = O.block_norms(prob.A, ro, co)
    variant = "omp"
    try:
        O.lib(variant)
    except Exception:  # no OpenMP runtime on this host: the single-thread -O3 build
        variant = "fast"
    cores = os.cpu_count() or 1
    threads = int(os.environ.get("OMP_NUM_THREADS", cores)) if variant == "omp" else 1
    # each step: a bounded sample of ~3 s of oracle iterations
    O.rebk(prob.A, prob.b, ro, co, alpha, seed=1000, iters=2, norms=norms, variant=variant)  # load, threads up
    t0 = time.perf_counter()
    O.rebk(prob.A, prob.b, ro, co, alpha, seed=1000, iters=8, norms=norms, variant=variant)
    per = (time.perf_counter() - t0) / 8
    n_it = max(3, int(3.0 / max(per, 1e-6)))
    for _ in range(args.warmup):
        O.rebk(prob.A, prob.b, ro, co, alpha, seed=1000, iters=max(1, n_it // 10), norms=norms, variant=variant)
    t0 = time.perf_counter()
    for s in range(args.steps):
        O.rebk(prob.A, prob.b, ro, co, alpha, seed=1000 + s, iters=n_it, norms=norms, variant=variant)
    dt = time.perf_counter() - t0
    its = args.steps * n_it / dt
    value = its / ipsolve
    sample = (f"per step {n_it} iterations of the FP64 oracle of Algorithm 1 on this workload "
              f"({ORACLE_BUILDS[variant][0]}); solves/s = iterations/s / {ipsolve:.0f} iterations per solve "
              f"(oracle's own count to 1e-8, tests/golden/precision_anchor.txt)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "tau": TAU, "alpha": alpha},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": sample, "iterations_per_s": its, "build": variant,
                             "host_cores": cores, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_warm(args):
    """Learned warm start on the 8192 x 2048 workload: A = U diag(i^-1/2) V^T,
    b = A (M c) + N(0, 1e-3^2), M = randn(2048, 32), c ~ N(0, I).  Training
    pairs come from the solver: x_ls = A^+ b from batched systems sharing A
    (8 right-hand sides each), y* = (A^T)^+ x_ls from batched systems sharing
    A^T; the network 8192 -> 512 -> 512 -> 8192 (BF16 tensor-core GEMMs) is
    trained with the y-space loss; then mixed-precision solves of held-out
    right-hand sides to 1e-8 from the cold start and from x0 = A^T y.  The warm
    solves' timed region includes the network and the x0 / z0 products."""
    import torch

    from paper_2001_04179_gb300 import BatchSolver, Solver, WarmStartNet
    from workloads import spectrum_problem

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m5, n5, ntr, nev = 8192, 2048, args.warm_train, args.warm_eval
    ntr = max(256, ntr // 256 * 256)
    nbs = max(1, args.warm_batch_systems)
    nbe = 8 * nbs  # held-out right-hand sides of the batched legs
    t0 = time.perf_counter()
    p = spectrum_problem(m5, n5, seed=rank, latent=32, noise=1e-3, nrhs=ntr + nev + nbe)
    gen_s = time.perf_counter() - t0
    A = p.A
    At = np.ascontiguousarray(A.T)
    sol = Solver(A, TAU, TAU, alpha=0.0, storage=("fp32", "bf16"))
    alpha = sol.alpha  # blocks of A^T are the transposes of A's: the same beta_max
    ns = ntr // 8

    def batched(mat, rhs_rows, rows_out):
        bs = BatchSolver([mat] * ns, nrhs=8, tau=TAU, alpha=[alpha] * ns, max_outer=2)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out = bs.solve(rhs_rows, X_ref=None, tol=0.0, max_iter=0, inner_iters=25000, seed=3)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        bs.close()
        return out["x"], dt, out["stats"]

    # 1. x_ls for the training right-hand sides (system i holds RHS 8i..8i+7)
    B_sys = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([p.b[:, 8 * i:8 * i + 8] for i in range(ns)], axis=0))).to(dev)
    Xs, tx, stx = batched(A, B_sys, n5)
    # 2. y* = (A^T)^+ x_ls: the x_ls rows are already laid out as the A^T systems' right-hand sides
    Ys, ty, sty = batched(At, Xs, m5)
    Xtr = Xs.view(ns, n5, 8).permute(0, 2, 1).reshape(ntr, n5)
    Ytr = Ys.view(ns, m5, 8).permute(0, 2, 1).reshape(ntr, m5).contiguous()
    xr_tr = torch.from_numpy(np.ascontiguousarray(p.x_ref[:, :ntr].T)).to(dev)
    x_err = float(((Xtr - xr_tr).norm(dim=1) / xr_tr.norm(dim=1)).max())
    # 3. training
    Btr = torch.from_numpy(np.ascontiguousarray(p.b[:, :ntr].T)).to(dev)
    net = WarmStartNet(A, hidden=512, batch_capacity=256, seed=1)
    out_scale = 0.1 * float(torch.sqrt((Ytr * Ytr).sum(1).mean() / (Btr * Btr).sum(1).mean()))
    net.set_loss("y_rel", out_scale)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = net.fit(Btr, Ytr, steps=args.warm_steps, lr=1e-3, batch=256)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    # 4. held-out solves, cold vs warm
    stream = torch.cuda.current_stream()
    res = {}
    for S in ("fp32", "bf16"):
        row = {}
        for mode in ("cold", "warm"):
            its, e0s = [], []
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for i in range(ntr, ntr + nev):
                b = torch.from_numpy(np.ascontiguousarray(p.b[:, i])).to(dev)
                xr = torch.from_numpy(np.ascontiguousarray(p.x_ref[:, i])).to(dev)
                if mode == "warm":
                    x0, z0 = net.warm_start(sol, b)
                    r = sol.solve_refined(b, tol=TOL, seed=7, storage=S, x_ref=xr, x0=x0, z0=z0)
                    e0s.append(float((x0 - xr).norm() / xr.norm()))
                else:
                    r = sol.solve_refined(b, tol=TOL, seed=7, storage=S, x_ref=xr)
                if r["stats"]["rel_err"] > TOL:
                    raise RuntimeError(f"{mode} {S} solve did not reach {TOL}: {r['stats']}")
                its.append(r["stats"]["iterations"])
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            row[mode] = {"solves_per_s": nev / (ms / 1000.0), "iterations_mean": float(np.mean(its))}
            if e0s:
                row[mode]["x0_rel_err_median"] = float(np.median(e0s))
        row["speedup"] = row["warm"]["solves_per_s"] / row["cold"]["solves_per_s"]
        res[S] = row
    # plain FP64 (Algorithm 1 as printed) on the same held-out right-hand sides
    nplain = min(nev, 16)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its = []
    ev0.record(stream)
    for i in range(ntr, ntr + nplain):
        b = torch.from_numpy(np.ascontiguousarray(p.b[:, i])).to(dev)
        xr = torch.from_numpy(np.ascontiguousarray(p.x_ref[:, i])).to(dev)
        r = sol.solve(b, tol=TOL, max_iter=10**7, seed=7, x_ref=xr)
        if r["stats"]["rel_err"] > TOL:
            raise RuntimeError(f"plain FP64 solve did not reach {TOL}: {r['stats']}")
        its.append(r["stats"]["iterations"])
    ev1.record(stream)
    torch.cuda.synchronize()
    plain = {"solves_per_s": nplain / (ev0.elapsed_time(ev1) / 1000.0), "iterations_mean": float(np.mean(its)),
             "rhs": nplain}
    # batched FP32 mixed: nbs systems of 8 right-hand sides sharing A, cold and warm
    c0 = ntr + nev
    Bb = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([p.b[:, c0 + 8 * i:c0 + 8 * i + 8] for i in range(nbs)], axis=0))).to(dev)
    Xrb = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([p.x_ref[:, c0 + 8 * i:c0 + 8 * i + 8] for i in range(nbs)], axis=0))).to(dev)
    bsv = BatchSolver([A] * nbs, nrhs=8, tau=TAU, alpha=[alpha] * nbs)
    batched_res = {}
    for mode in ("cold", "warm"):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        X0 = Z0 = None
        if mode == "warm":  # the network and the x0 / z0 products are inside the timed region
            X0, Z0 = net.warm_start_batch(sol, Bb, nbe, group=8)
        out = bsv.solve(Bb, X_ref=Xrb, tol=TOL, max_iter=400000, seed=11, X0=X0, Z0=Z0)
        ev1.record(stream)
        torch.cuda.synchronize()
        st_ = out["stats"]
        if st_["converged"] != nbs:
            raise RuntimeError(f"batched {mode}: {st_['converged']} of {nbs} systems converged")
        batched_res[mode] = {"solves_per_s": nbe / (ev0.elapsed_time(ev1) / 1000.0),
                             "iterations_mean_per_system": st_["iterations"] / nbs, "rhs": nbe,
                             "systems": nbs}
    bsv.close()
    res["batched_fp32"] = batched_res
    res["plain_fp64"] = plain
    res["speedup_mixed_warm_batched_vs_plain_fp64"] = batched_res["warm"]["solves_per_s"] / plain["solves_per_s"]
    if rank == 0:
        print(json.dumps({
            "workload": "warm start: A = U diag(i^-1/2) V^T 8192x2048, b = A(Mc) + N(0,1e-3^2), latent 32; "
                        "MLP 8192-512-512-8192 (BF16 GEMMs), x0 = A^T y, z0 = b - A x0; tau = 128; tol 1e-8",
            "metric": "solves/s to 1e-8 rel err, warm vs cold (mixed precision)", "unit": "solves/s",
            "train_rhs": ntr, "eval_rhs": nev, "problem_gen_s": gen_s,
            "targets": {"x_ls_batch_s": tx, "y_star_batch_s": ty, "x_ls_max_rel_err": x_err,
                        "systems": ns, "rhs_per_system": 8, "passes": 2, "iterations_per_pass": 25000},
            "training": {"steps": args.warm_steps, "seconds": train_s, "loss_first": losses[0],
                         "loss_last": float(np.mean(losses[-20:])), "out_scale": out_scale,
                         "loss": "mean ||y - y*||^2 / ||y*||^2", "lr": "1e-3 cosine", "batch": 256},
            "fp32": res["fp32"], "bf16": res["bf16"], "plain_fp64": res["plain_fp64"],
            "batched_fp32": res["batched_fp32"],
            "speedup_mixed_warm_batched_vs_plain_fp64": res["speedup_mixed_warm_batched_vs_plain_fp64"]}))
    return 0


def run_batch_workload(args):
    """Batched systems: 512 independent dense systems, m ~ U[200, 6000], n ~
    U[50, 2000], 30% rank-deficient products of inner dimension ceil(n/4), 8
    right-hand sides each (B = A X* + N(0, 0.01^2)); FP32 inner iterations, FP64
    refinement, one CUDA graph per solve, at most 1e5 iterations per system,
    stop at 1e-8 relative error per right-hand side.  A step is one solve of
    the whole batch; the metric counts the right-hand sides that reached 1e-8."""
    import torch

    from paper_2001_04179_gb300 import BatchSolver
    from workloads import batched_problems

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.batch_probe:
        return batch_probe(args)
    t0 = time.perf_counter()
    ps = batched_problems(args.batch_count, seed=rank, nrhs=8, scale_down=args.batch_scale)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    bs = BatchSolver([p.A for p in ps], nrhs=8, tau=args.batch_tau, cluster=args.batch_cluster,
                     joint_frac=args.batch_joint_frac)
    B = bs.stack_rhs([p.b for p in ps], bs.m)
    Xr = bs.stack_rhs([p.x_ref for p in ps], bs.n)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    for w in range(max(1, args.warmup)):
        out = bs.solve(B, X_ref=Xr, tol=TOL, max_iter=100000, seed=900 + w)
    steps = max(1, args.steps)
    ms, rhs_ok, sys_ok, iters = 0.0, 0, 0, 0
    for s_ in range(steps):
        out = bs.solve(B, X_ref=Xr, tol=TOL, max_iter=100000, seed=1000 + s_)
        st = out["stats"]
        ms += st["device_ms"]
        iters += st["iterations"]
        xs = bs.split_x(out["x"])
        errs = np.array([[np.linalg.norm(xs[i][:, r] - ps[i].x_ref[:, r]) / np.linalg.norm(ps[i].x_ref[:, r])
                          for r in range(8)] for i in range(len(ps))])
        rhs_ok += int((errs <= TOL).sum())
        sys_ok += int((errs <= TOL).all(axis=1).sum())
    bs_tau = st["tau"]
    # Systems with a right-hand side short of 1e-8 at the iteration cap: Theorem main's
    # rate eta = 1 - (2 alpha - alpha^2 beta^I_max) sigma_r^2 / ||A||_F^2 at the batch's
    # alpha.  The error bound's leading term eta^k reaches 1e-16 (1e-8 relative, squared)
    # after k = log(1e-16) / log(eta) iterations; with sigma_r^2 from the device Lanczos
    # (approached from above, so eta is too small) this k is a lower bound.
    from paper_2001_04179_gb300 import Solver
    cap = 100000
    short = [i for i in range(len(ps)) if not (errs[i] <= TOL).all()]
    reach = []
    for i in short:
        p = ps[i]
        sol = Solver(p.A, bs_tau, bs_tau, alpha=0.0, storage=())
        sp = sol.spectrum(steps=int(min(p.A.shape[0], p.A.shape[1], 400)), seed=1)
        sol.close()
        eta = sp["eta"]
        k_lower = float("inf") if not (0.0 < eta < 1.0) else float(np.log(1e-16) / np.log(eta))
        reach.append({"system": i, "m": int(p.A.shape[0]), "n": int(p.A.shape[1]), "alpha": sp["alpha"],
                      "sigma_r_sq_upper": sp["sigma_r_sq"], "sigma1_sq": sp["sigma1_sq"], "fro2": sp["fro2"],
                      "eta": eta, "iterations_lower_bound": k_lower,
                      "rhs_short": int((errs[i] > TOL).sum()), "out_of_reach": bool(k_lower > cap)})
    out_idx = {r["system"] for r in reach if r["out_of_reach"]}
    reachable_rhs = 8 * (len(ps) - len(out_idx))
    reachable_ok = int(sum((errs[i] <= TOL).sum() for i in range(len(ps)) if i not in out_idx))
    if rank == 0:
        print(json.dumps({
            "workload": f"batched: {args.batch_count} systems m~U[200,6000]/{args.batch_scale}, "
                        f"n~U[50,2000]/{args.batch_scale}, 30% rank-deficient, 8 RHS each; "
                        "FP32 inner / FP64 refinement; one CUDA graph per solve; <= 1e5 iterations per system",
            "metric": "right-hand sides solved to 1e-8 per second", "unit": "solves/s",
            "value": rhs_ok / (ms / 1000.0), "steps": steps, "ms_per_step": ms / steps,
            "tau": st["tau"], "graph": st["graph"], "launches_per_solve": st["launches"],
            "rhs_converged_per_solve": rhs_ok / steps, "systems_converged_per_solve": sys_ok / steps,
            "inner_iterations_per_solve": iters / steps, "max_iterations": st["max_iterations"],
            "problem_gen_s": gen_s, "create_s": create_s,
            "sum_mn": int(sum(p.A.shape[0] * p.A.shape[1] for p in ps)),
            "col_path": st.get("col_path"), "cluster": st.get("cluster"), "systems_on_clusters": st.get("joint"),
            "top_cluster": st.get("top_cluster"), "systems_on_top_clusters": st.get("top_joint"),
            "out_of_reach": {"rule": "Theorem main's rate at the batch's alpha, sigma_r^2 from device Lanczos "
                                     "(an upper estimate): iterations to 1e-8 >= log(1e-16)/log(eta) > the cap",
                             "cap": cap, "systems": len(out_idx), "rhs": 8 * len(out_idx),
                             "reachable_rhs": reachable_rhs, "reachable_rhs_converged_last_solve": reachable_ok,
                             "reachable_rhs_per_s": reachable_ok / (ms / 1000.0 / steps),
                             "short_systems": reach}}))
    return 0


def batch_probe(args):
    """Cost of one iteration of the batched kernel on one SM: one Gaussian system
    (or `copies` identical ones, one per CTA, stored once) with 8 right-hand sides,
    tau = --batch-tau (16 when 0), one
    pass of 2000 iterations (no stopping test), device time of the second solve
    over the iterations; next to the FP32 FMA work of an iteration at 128 FMA per
    clock and 2.07 GHz.  --batch-probe one: only the 6000 x 2000 system, once.
    --batch-cluster C > 1: each system on a cluster of C CTAs instead of one."""
    import torch

    from paper_2001_04179_gb300 import BatchSolver

    shapes = [(6000, 2000)] if args.batch_probe == "one" else [(8192, 2048), (6000, 2000), (2000, 2000),
                                                                (2000, 500), (500, 200)]
    if args.batch_probe == "one" and args.batch_probe_shape:
        shapes = [tuple(int(v) for v in args.batch_probe_shape.split(","))]
    copies_list = [1] if args.batch_probe == "one" else [1, 152]
    tau = args.batch_tau if args.batch_tau > 0 else 16
    K = args.batch_probe_iters
    for copies in copies_list:
        for (m, n) in shapes:
            rng = np.random.default_rng(m + n)
            A = rng.standard_normal((m, n))
            cl = args.batch_cluster if args.batch_cluster > 1 else 1
            bs = BatchSolver([A] * copies, nrhs=8, tau=tau, max_outer=1, cluster=cl, joint_frac=1e-9)
            B = bs.stack_rhs([rng.standard_normal((m, 8)) for _ in range(copies)], bs.m)
            for sd in (3, 4):
                out = bs.solve(B, X_ref=None, tol=0.0, max_iter=K, inner_iters=K, seed=sd)
            st = out["stats"]
            its = max(st["max_iterations"], 1)
            us = 1000.0 * st["device_ms"] / its
            fma_us = 2 * (m * tau + tau * n) * 8 / (128 * 2.07e9) * 1e6
            print(json.dumps({"probe": "batched iteration cost", "m": m, "n": n, "tau": tau, "copies": copies,
                              "cluster": st["cluster"], "systems_on_clusters": st["joint"], "iterations": its,
                              "us_per_iteration": us, "fp32_fma_us": fma_us, "fma_fraction": fma_us / us}),
                  flush=True)
            bs.close()
    return 0


def run_free_workload(args):
    """Section 4's sampling without a partition (rebk_solve_free: tau row and tau column
    indices drawn independently per iteration with probabilities proportional to their
    squared norms) next to Algorithm 1 on the contiguous partition (rebk_solve), plain
    FP64, the same block sizes and step size: the 1000 x 200 Gaussian system of the
    plain-FP64 workload (tau 20, to 1e-10) and the 8000 x 20000 rank-2000 system (tau
    128, to 1e-8).  Whole solves timed with CUDA events; per-iteration time from the
    kernel events; algorithmic bytes 8 tau (m + n) per iteration (each drawn column
    and row read once per product pass) against the measured L2 and HBM rates."""
    import ctypes as _ct

    import torch

    from paper_2001_04179_gb300 import Solver
    from paper_2001_04179_gb300 import rebk as _R
    from workloads import gaussian_problem

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pk = _R.RebkPeaks()
    _R.check(_R.load().rebk_device_peaks(_ct.byref(pk), None))
    hbm_peak, _, peak_src = load_peaks()
    cases = [("1000x200 Gaussian (full column rank, inconsistent), tau 20, to 1e-10",
              gaussian_problem(1000, 200, seed=rank), 20, 1e-10),
             ("8000x20000 rank 2000 (A = G1 G2, b = A x* + N(0, 0.01^2)), tau 128, to 1e-8",
              make_problem(rank, True), 128, 1e-8)]
    steps = max(1, args.steps)
    out = []
    for name, p, tau, tol in cases:
        A = torch.from_numpy(p.A).to(dev)
        sol = Solver(A, tau, tau, alpha=0.0, storage=())
        del A
        b = torch.from_numpy(p.b).to(dev)
        xr = torch.from_numpy(p.x_ref).to(dev)
        m, n = p.A.shape
        res = {"workload": name, "alpha": sol.alpha}
        for kind in ("partition", "free"):
            def one(seed):
                if kind == "free":
                    r = sol.solve_free(b, tau, tau, tol=tol, max_iter=10**7, seed=seed, x_ref=xr)
                else:
                    r = sol.solve(b, tol=tol, max_iter=10**7, seed=seed, x_ref=xr)
                if r["stats"]["rel_err"] > tol:
                    raise RuntimeError(f"{kind} solve did not reach {tol}: {r['stats']}")
                return r
            for w in range(max(1, args.warmup)):
                one(900 + w)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record()
            its, kms = 0, 0.0
            for s_ in range(steps):
                st = one(1000 + s_)["stats"]
                its += st["iterations"]
                kms += st["kernel_ms"]
            ev1.record()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            gbs = 8.0 * tau * (m + n) * its / (kms / 1000.0) / 1e9
            res[kind] = {"solves_per_s": steps / (ms / 1000.0), "iterations_per_solve": its / steps,
                         "us_per_iteration": 1000.0 * kms / its, "algorithmic_gbs": gbs,
                         "l2_frac": gbs / pk.l2_gbs, "hbm_frac": gbs / hbm_peak}
        res["free_over_partition_solves_per_s"] = res["free"]["solves_per_s"] / res["partition"]["solves_per_s"]
        sol.close()
        out.append(res)
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps({"workload": "sampling without a partition vs Algorithm 1 on a partition (plain FP64)",
                          "metric": "solves/s to the stated tolerance", "unit": "solves/s", "steps": steps,
                          "cases": out, "l2_gbs_measured": pk.l2_gbs, "hbm_gbs": hbm_peak,
                          "hbm_peak_source": peak_src}))
    return 0


def run_sparse_workload(args):
    """Sparse tomography-like workload: A 65536 x 16384 CSR, 96 nonzeros per row
    at uniform random columns, values U(0,1) 10^u (u ~ U(0,1) per row: row norms
    spread over a decade), b = A x* + 1% Gaussian noise; tau = 256 (256 row
    blocks over CSR, 64 column blocks over the CSC copy); plain FP64 Algorithm 1
    and the mixed-precision solve (FP32 values and inner sweeps, FP64
    refinement), each to 1e-8 relative error against x_ref from the normal
    equations (dense Cholesky on the host)."""
    import torch

    from paper_2001_04179_gb300 import SparseSolver
    from workloads import sparse_problem

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, n, k = 65536, 16384, 96
    t0 = time.perf_counter()
    p = sparse_problem(m, n, k, seed=rank, noise=0.01, decades=1.0,
                       x_ref=None if args.profile_pass > 0 else "normal")
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    sol = SparseSolver(m, n, p.indptr, p.indices, p.data, 256, 256)
    create_s = time.perf_counter() - t0
    info = sol.info()
    b = torch.from_numpy(p.b).to(dev)
    if args.profile_pass > 0:  # a fixed number of iterations, twice (the second is the one ncu captures)
        for _ in range(2):
            if args.sparse_mixed:
                r = sol.solve_refined(b, tol=0.0, max_iter=args.profile_pass, seed=7, max_outer=1,
                                      inner_iters=args.profile_pass)
            else:
                r = sol.solve(b, tol=0.0, max_iter=args.profile_pass, seed=7)
        torch.cuda.synchronize()
        print(json.dumps({"profile_pass": args.profile_pass, "workload": "sparse",
                          "mode": "mixed" if args.sparse_mixed else "plain", "iterations": r["stats"]["iterations"],
                          "us_per_iteration": 1000.0 * r["stats"]["kernel_ms"] / args.profile_pass}))
        return 0
    xr = torch.from_numpy(p.x_ref).to(dev)
    stream = torch.cuda.current_stream()
    steps = max(1, args.steps)
    nnz_col_block = p.nnz / info["col_blocks"]
    nnz_row_block = 256 * k

    def run(mode):
        call = sol.solve if mode == "plain" else sol.solve_refined
        for w in range(max(1, args.warmup)):
            call(b, tol=TOL, max_iter=4_000_000, seed=900 + w, x_ref=xr)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its, kms, outer = 0, 0.0, 0
        ev0.record(stream)
        for s_ in range(steps):
            out = call(b, tol=TOL, max_iter=4_000_000, seed=1000 + s_, x_ref=xr)
            if out["stats"]["rel_err"] > TOL:
                raise RuntimeError(f"sparse {mode} solve did not reach {TOL}: {out['stats']}")
            its += out["stats"]["iterations"]
            kms += out["stats"]["kernel_ms"]
            outer += out["stats"]["outer"]
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        # per iteration: both blocks' values and indices (4 B) twice (gather, scatter) and the
        # gathered / scattered vector entries (8 B FP64, 4 B FP32 corrections)
        vb = 8 if mode == "plain" else 4
        bytes_it = (nnz_col_block + nnz_row_block) * 2 * (vb + 4 + vb)
        return {"value": steps / (ms / 1000.0), "ms_per_step": ms / steps, "iterations_per_solve": its / steps,
                "refinement_passes_per_solve": outer / steps, "kernel_ms_per_solve": kms / steps,
                "block_iterations_per_s": its / (kms / 1000.0), "us_per_iteration": 1000.0 * kms / its,
                "algorithmic_bytes_per_iteration": bytes_it, "achieved_gbs": bytes_it * its / (kms / 1000.0) / 1e9,
                "matrix_bytes_csr_plus_csc": 2 * p.nnz * (vb + 4)}

    plain = run("plain")
    mixed = run("mixed")
    # The CSR + CSC copies (151 MB FP64, 113 MB FP32) mostly stay in the 129 MB L2
    # (ncu: 0.27 MB of DRAM traffic per iteration), so the bandwidth roof of this
    # kernel is L2's: measured here by the library's L2 read microbenchmark.
    from paper_2001_04179_gb300 import rebk as _R
    import ctypes as _ct
    pk = _R.RebkPeaks()
    _R.check(_R.load().rebk_device_peaks(_ct.byref(pk), None))
    l2_peak = pk.l2_gbs
    for res in (plain, mixed):
        res["roofline"] = {"bound": "l2", "achieved": res["achieved_gbs"], "peak": l2_peak, "unit": "GB/s",
                           "frac": res["achieved_gbs"] / l2_peak,
                           "peak_source": "measured: rebk_device_peaks L2 read kernel (16-byte loads that "
                                          "bypass L1) on this GPU"}
    if rank == 0:
        print(json.dumps({
            "workload": "sparse: 65536x16384 CSR, 96 nnz/row uniform columns, values U(0,1)*10^U(0,1), "
                        "b = A x* + 1% noise; tau = 256 rows / 256 columns; to 1e-8",
            "metric": "solves/s to 1e-8 rel err", "unit": "solves/s", "steps": steps,
            "plain_fp64": plain, "mixed_fp32": mixed, "mixed_over_plain": mixed["value"] / plain["value"],
            "nnz": p.nnz, "alpha": info["alpha"], "beta_max": info["beta_max"], "problem_gen_s": gen_s,
            "create_s": create_s}))
    return 0


def run_sweep(args):
    """Block size and step size on GB300, measured by the library's autotuner
    (rebk_tune_tau: time to tolerance of each candidate, mean of several
    seeded solves).  Parts, each printed as one JSON row per point and one row
    with the tuner's pick:
      (1) 8000 x 20000 rank 2000, FP32 mixed precision to 1e-8: tau in
          {32, 64, 128, 256} at alpha = 1.75 / beta_max, then alpha / beta_max in
          {0.5, 1, 1.5, 1.75, 1.95, 2.25} at tau = 128;
      (2) randn(1000, 200) inconsistent, plain FP64 to 1e-10, tau in
          {5, 10, 20, 40, 100, 200};
      (3) Fig. 1 shapes: Type I (500 x 250, rank 150, kappa 2) and Type II
          randn(500, 250), tau = 10, alpha / beta_max from 0.75 to 2.62;
      (4) Fig. 2 shapes: Type I (20000 x 5000, rank 4500, kappa 2) and Type II
          randn(20000, 5000), tau in {5, 10, 20, 50, 100, 200}, alpha = 1.75 / beta_max;
      (5) Fig. 3 shapes: Type I (m x 500, rank 250, kappa 2) and Type II
          randn(m, 500), m = 2000, 4000, ..., 20000, tau = 10, alpha = 1.75 / beta_max.
    Parts (3)-(5) stop at ||x - A^+ b|| <= 1e-5 (the absolute rule of Section 3's
    experiments) in plain FP64.  (6) the device Lanczos estimates of sigma_1^2 and
    sigma_r^2 with Remark alpha's mean-optimal step and the rates of Theorems ner and
    main, and randn(1000, 200) solved at that step, at 1 / beta_max and at 1.75 / beta_max."""
    import torch

    from paper_2001_04179_gb300 import tune_tau
    from workloads import gaussian_problem, type1_problem

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    only = set(args.sweep_parts.split(",")) if args.sweep_parts else None
    rows = []

    def emit(name, pts, best, c=None):
        for p in pts:
            rows.append({"workload": name, "tau": p["tau"],
                         "alpha_times_beta_max": c if c is not None else round(p["alpha"] * p["beta_max"], 6),
                         "beta_max": p["beta_max"], "iterations": p["iterations"],
                         "ms_per_solve": p["device_ms"], "status": R_STATUS(p["status"])})
        rows.append({"workload": name, "tuner_best_tau": best})

    def tune(name, A, b, xr, taus, c, storage, tol, trials, max_iter=10**7):
        best, pts = tune_tau(A, b, taus, x_ref=xr, alpha_factor=c, storage=storage, tol=tol,
                             max_iter=max_iter, seed=1000 + rank, trials=trials, stream=stream)
        emit(name, pts, best, c)
        return best, pts

    if only is None or "1" in only:
        prob = make_problem(rank, True)
        A_dev = torch.from_numpy(prob.A).to(dev)
        b, xr = torch.from_numpy(prob.b).to(dev), torch.from_numpy(prob.x_ref).to(dev)
        name = "8000x20000 rank 2000, FP32 mixed, tol 1e-8"
        tune(name, A_dev, b, xr, [32, 64, 128, 256], 1.75, "fp32", TOL, 2)
        for c in (0.5, 1.0, 1.5, 1.75, 1.95, 2.25):
            tune(name + ", alpha sweep", A_dev, b, xr, [128], c, "fp32", TOL, 2, max_iter=200000)
        del A_dev, b, xr, prob
        torch.cuda.empty_cache()
    if only is None or "2" in only:
        g = gaussian_problem(1000, 200, seed=rank)
        tune("randn(1000,200) inconsistent, plain FP64, tol 1e-10", g.A, torch.from_numpy(g.b).to(dev),
             torch.from_numpy(g.x_ref).to(dev), [5, 10, 20, 40, 100, 200], 1.75, "fp64", 1e-10, 3)

    def paper_pair(m, n, r, seed):
        return [("Type I %dx%d r%d k2" % (m, n, r), type1_problem(m, n, r, 2.0, seed)),
                ("Type II randn(%d,%d)" % (m, n), gaussian_problem(m, n, seed=seed))]

    def abs_tol(p):
        return 1e-5 / float(np.linalg.norm(p.x_ref))

    if only is None or "3" in only:
        for label, p in paper_pair(500, 250, 150, 7 + rank):
            A_dev = torch.from_numpy(p.A).to(dev)
            b, xr = torch.from_numpy(p.b).to(dev), torch.from_numpy(p.x_ref).to(dev)
            for c in (0.75, 1.0, 1.25, 1.5, 1.75, 2.0, 2.25, 2.62):
                tune("Fig. 1 " + label + ", tau 10, abs err 1e-5", A_dev, b, xr, [10], c, "fp64", abs_tol(p),
                     10, max_iter=400000)
    if only is None or "4" in only:
        for label, p in paper_pair(20000, 5000, 4500, 11 + rank):
            A_dev = torch.from_numpy(p.A).to(dev)
            b, xr = torch.from_numpy(p.b).to(dev), torch.from_numpy(p.x_ref).to(dev)
            tune("Fig. 2 " + label + ", alpha 1.75/beta_max, abs err 1e-5", A_dev, b, xr,
                 [5, 10, 20, 50, 100, 200], 1.75, "fp64", abs_tol(p), 2, max_iter=3000000)
            del A_dev, b, xr, p
            torch.cuda.empty_cache()
    if only is None or "5" in only:
        for m in range(2000, 20001, 2000):
            for label, p in paper_pair(m, 500, 250, 13 + m + rank):
                A_dev = torch.from_numpy(p.A).to(dev)
                b, xr = torch.from_numpy(p.b).to(dev), torch.from_numpy(p.x_ref).to(dev)
                tune("Fig. 3 " + label + ", tau 10, alpha 1.75/beta_max, abs err 1e-5", A_dev, b, xr, [10],
                     1.75, "fp64", abs_tol(p), 3, max_iter=3000000)
    if only is None or "6" in only:
        # Section 2's step-size quantities from the device Lanczos estimates, and solves at
        # Remark alpha's mean-optimal step, at 1 / beta_max (the step Theorem main's bound
        # favours) and at 1.75 / beta_max
        from paper_2001_04179_gb300 import Solver
        g = gaussian_problem(1000, 200, seed=rank)
        bg, xg = torch.from_numpy(g.b).to(dev), torch.from_numpy(g.x_ref).to(dev)
        sol = Solver(g.A, 20, 20, alpha=0.0, storage=(), stream=stream)
        t0 = time.perf_counter()
        sp = sol.spectrum(steps=200, seed=1)
        sp_s = time.perf_counter() - t0
        bmax = max(sp["beta_row"], sp["beta_col"])
        row = {"workload": "randn(1000,200), tau 20: spectral estimates", "spectrum_s": sp_s,
               "alpha_mean_opt_times_beta_max": sp["alpha_mean_opt"] * bmax, **sp}
        for label, a in (("mean_opt", sp["alpha_mean_opt"]), ("1/beta_max", 1.0 / bmax), ("1.75/beta_max", 1.75 / bmax)):
            sol.alpha = a
            o = sol.solve(bg, tol=1e-10, max_iter=200000, seed=5, x_ref=xg,
                          allow=(R_CODE("REBK_OK"), R_CODE("REBK_MAX_ITER"), R_CODE("REBK_DIVERGED")))
            sp2 = sol.spectrum(steps=200, seed=1)
            row["solve_" + label] = {"alpha": a, "status": R_STATUS(o["status"]), "iterations": o["stats"]["iterations"],
                                     "rel_err": o["stats"]["rel_err"], "delta": sp2["delta"], "eta": sp2["eta"],
                                     "rho": sp2["rho"]}
        rows.append(row)
        prob = make_problem(rank, True)
        A_dev = torch.from_numpy(prob.A).to(dev)
        sol = Solver(A_dev, 128, 128, alpha=0.0, storage=(), stream=stream)
        t0 = time.perf_counter()
        sp = sol.spectrum(steps=300, seed=1)
        rows.append({"workload": "8000x20000 rank 2000, tau 128: spectral estimates (300 steps)",
                     "spectrum_s": time.perf_counter() - t0,
                     "alpha_mean_opt_times_beta_max": sp["alpha_mean_opt"] * max(sp["beta_row"], sp["beta_col"]), **sp})
        sol.close()
    if rank == 0:
        for r in rows:
            print(json.dumps(r), flush=True)
    return 0


def R_CODE(name: str) -> int:
    from paper_2001_04179_gb300 import rebk as R
    return getattr(R, name)


def R_STATUS(code: int) -> str:
    from paper_2001_04179_gb300 import rebk as R
    return R.STATUS_NAMES.get(code, str(code))


def measure_combined(args, dev, rank):
    """The metric's combined form on the learned-warm-start workload: A = U
    diag(i^-1/2) V^T (8192 x 2048), a stream of right-hand sides b = A (M c) +
    N(0, 1e-3^2), M = randn(2048, 32).  Once per A: training targets from the
    solver (x_ls = A^+ b by batched solves on A, y* = (A^T)^+ x_ls by batched
    solves on A^T, a fixed number of passes, no known solution used), then the
    8192 -> 512 -> 512 -> 8192 network trained on them.  Timed: held-out
    right-hand sides solved to 1e-8 relative error by the mixed-precision
    batched solver (systems of 8 right-hand sides sharing A) from the network's
    x0 = A^T y, z0 = b - A x0 (network and products inside the timed region),
    every right-hand side checked against A^+ b; next to plain FP64 Algorithm 1
    one right-hand side at a time on the same right-hand sides."""
    import torch

    from paper_2001_04179_gb300 import BatchSolver, Solver, WarmStartNet
    from workloads import spectrum_problem

    m5, n5 = 8192, 2048
    ntr = max(256, args.combined_train // 256 * 256)
    nbs = max(1, args.combined_systems)
    nev = 8 * nbs
    t0 = time.perf_counter()
    p = spectrum_problem(m5, n5, seed=100 + rank, latent=32, noise=1e-3, nrhs=ntr + nev)
    gen_s = time.perf_counter() - t0
    A = p.A
    At = np.ascontiguousarray(A.T)
    stream = torch.cuda.current_stream()
    sol = Solver(A, TAU, TAU, alpha=0.0, storage=("fp32",), stream=stream)
    alpha = sol.alpha  # the blocks of A^T are the transposes of A's: the same beta_max
    ns = ntr // 8
    iters = args.combined_target_iters

    def targets(mat, rhs_rows):
        bs = BatchSolver([mat] * ns, nrhs=8, tau=TAU, alpha=[alpha] * ns, max_outer=2)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out = bs.solve(rhs_rows, X_ref=None, tol=0.0, max_iter=0, inner_iters=iters, seed=3)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        bs.close()
        return out["x"], dt

    B_sys = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([p.b[:, 8 * i:8 * i + 8] for i in range(ns)], axis=0))).to(dev)
    Xs, tx = targets(A, B_sys)
    Ys, ty = targets(At, Xs)
    Xtr = Xs.view(ns, n5, 8).permute(0, 2, 1).reshape(ntr, n5)
    Ytr = Ys.view(ns, m5, 8).permute(0, 2, 1).reshape(ntr, m5).contiguous()
    xr_tr = torch.from_numpy(np.ascontiguousarray(p.x_ref[:, :ntr].T)).to(dev)
    x_err = float(((Xtr - xr_tr).norm(dim=1) / xr_tr.norm(dim=1)).median())
    Btr = torch.from_numpy(np.ascontiguousarray(p.b[:, :ntr].T)).to(dev)
    net = WarmStartNet(A, hidden=512, batch_capacity=256, seed=1, stream=stream)
    out_scale = 0.1 * float(torch.sqrt((Ytr * Ytr).sum(1).mean() / (Btr * Btr).sum(1).mean()))
    net.set_loss("y_rel", out_scale)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = net.fit(Btr, Ytr, steps=args.combined_steps, lr=1e-3, batch=256)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    del B_sys, Xs, Ys, Xtr, Ytr, xr_tr, Btr
    # ---- timed: held-out right-hand sides, warm start + batched mixed precision ----
    c0 = ntr
    Bb = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([p.b[:, c0 + 8 * i:c0 + 8 * i + 8] for i in range(nbs)], axis=0))).to(dev)
    Xrb = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([p.x_ref[:, c0 + 8 * i:c0 + 8 * i + 8] for i in range(nbs)], axis=0))).to(dev)
    # block size of the batched solves: the batch autotuner's (at the first solve, untimed), with
    # its own step size 1.75 / beta_max for that partition; or a given tau at the solver's alpha
    btau = args.combined_batch_tau
    bsv = BatchSolver([A] * nbs, nrhs=8, tau=btau, alpha=None if btau == 0 else [alpha] * nbs, stream=stream)
    res = {}
    for mode in ("warm", "cold"):
        for rep in range(2):  # the first solve also orders the queue; the second is timed
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            X0 = Z0 = None
            if mode == "warm":
                X0, Z0 = net.warm_start_batch(sol, Bb, nev, group=8)
            out = bsv.solve(Bb, X_ref=Xrb, tol=TOL, max_iter=400000, seed=11 + rep, X0=X0, Z0=Z0)
            ev1.record(stream)
            torch.cuda.synchronize()
        st_ = out["stats"]
        X = out["x"].view(nbs, n5, 8)
        Xr = Xrb.view(nbs, n5, 8)
        errs = ((X - Xr).norm(dim=1) / Xr.norm(dim=1)).flatten()
        ms = ev0.elapsed_time(ev1)
        res[mode] = {"solves_per_s": nev / (ms / 1000.0), "ms": ms, "rhs": nev, "systems": nbs,
                     "rhs_reaching_1e-8": int((errs <= TOL).sum()), "rel_err_max": float(errs.max()),
                     "iterations_mean_per_system": st_["iterations"] / nbs, "refinement_passes": st_["outer"],
                     "tau": st_["tau"], "col_path": st_["col_path"], "cluster": st_["cluster"]}
    bsv.close()
    # ---- plain FP64 Algorithm 1, one right-hand side at a time, on held-out right-hand sides ----
    nplain = 8
    its = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(c0, c0 + nplain):
        b = torch.from_numpy(np.ascontiguousarray(p.b[:, i])).to(dev)
        xr = torch.from_numpy(np.ascontiguousarray(p.x_ref[:, i])).to(dev)
        r = sol.solve(b, tol=TOL, max_iter=10**7, seed=7, x_ref=xr)
        if r["stats"]["rel_err"] > TOL:
            raise RuntimeError(f"plain FP64 solve did not reach {TOL}: {r['stats']}")
        its.append(r["stats"]["iterations"])
    ev1.record(stream)
    torch.cuda.synchronize()
    plain = {"solves_per_s": nplain / (ev0.elapsed_time(ev1) / 1000.0), "iterations_mean": float(np.mean(its)),
             "rhs": nplain}
    once_s = tx + ty + train_s
    warm = res["warm"]
    amort = 1.0 / (1.0 / warm["solves_per_s"] + once_s / args.combined_stream)
    sol.close()
    return {
        "workload": ("learned warm start stream: A = U diag(i^-1/2) V^T 8192x2048, b = A(Mc) + N(0,1e-3^2), "
                     "latent 32; FP32 inner / FP64 refinement, batched tau autotuned (plain FP64 and the "
                     "training targets at tau 128), alpha 1.75/beta_max; "
                     "MLP 8192-512-512-8192 on tcgen05 BF16 GEMMs, x0 = A^T y, z0 = b - A x0"),
        "value": warm["solves_per_s"], "unit": "solves/s",
        "speedup_vs_plain_fp64": warm["solves_per_s"] / plain["solves_per_s"],
        "warm_batched": warm, "cold_batched": res["cold"], "plain_fp64": plain,
        "warm_over_cold_batched": warm["solves_per_s"] / res["cold"]["solves_per_s"],
        "once_per_A": {"targets_x_ls_s": tx, "targets_y_star_s": ty, "training_s": train_s,
                       "train_rhs": ntr, "target_passes": 2, "target_iterations_per_pass": iters,
                       "x_ls_median_rel_err": x_err, "training_steps": args.combined_steps,
                       "loss_first": losses[0], "loss_last": float(np.mean(losses[-20:]))},
        "amortised_over_stream": {"stream_rhs": args.combined_stream, "solves_per_s": amort,
                                  "speedup_vs_plain_fp64": amort / plain["solves_per_s"]},
        "problem_gen_s": gen_s,
    }


def run_profile_mlp(args):
    """K training steps of the warm-start network on a random 8192 x 2048 A and
    random targets (y-space loss): the network's products, Adam and the
    conversions, timed with CUDA events; warm-up steps first."""
    import ctypes

    import torch

    from paper_2001_04179_gb300 import WarmStartNet
    from paper_2001_04179_gb300 import rebk as R

    m, n, B = 8192, 2048, 256
    rng = np.random.default_rng(0)
    A = rng.standard_normal((m, n)) / np.sqrt(m)
    net = WarmStartNet(A, hidden=512, batch_capacity=B, seed=1)
    net.set_loss("y_rel", 0.1)
    Bm = torch.from_numpy(rng.standard_normal((B, m))).cuda()
    T = torch.from_numpy(rng.standard_normal((B, m))).cuda()
    lib = R.load()
    loss = ctypes.c_double()

    def step():
        R.check(lib.rebk_mlp_train_step(net._h, ctypes.c_void_p(Bm.data_ptr()), ctypes.c_void_p(T.data_ptr()), B,
                                        1e-3, ctypes.byref(loss)))

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.profile_mlp):
        step()
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.profile_mlp
    flops = 2.0 * B * (2 * m * 512 + 512 * 512) * 2.5  # forward 1x, weight and input gradients 1.5x
    print(json.dumps({"profile_mlp": args.profile_mlp, "ms_per_step": ms, "tflops_per_step": flops / (ms * 1e-3) / 1e12,
                      "loss": loss.value}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_mlp > 0:
        return run_profile_mlp(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "free":
        return run_free_workload(args)
    if args.workload == "sparse":
        return run_sparse_workload(args)
    if args.workload == "warm":
        return run_warm(args)
    if args.workload == "batch":
        return run_batch_workload(args)
    import torch
    import torch.distributed as dist

    from paper_2001_04179_gb300 import Solver

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    hbm_peak, bf16_peak, peak_src = load_peaks()
    from paper_2001_04179_gb300 import rebk as _R
    import ctypes as _ct
    dev_peaks = _R.RebkPeaks()
    _R.check(_R.load().rebk_device_peaks(_ct.byref(dev_peaks), None))
    dev_peaks = dev_peaks.as_dict()
    prob = make_problem(rank, True)
    stream = torch.cuda.current_stream()
    A_dev = torch.from_numpy(prob.A).to(dev)
    sol = Solver(A_dev, TAU, TAU, alpha=0.0, storage=("fp32", "bf16"), stream=stream, num_ctas=args.num_ctas)
    del A_dev
    torch.cuda.empty_cache()
    alpha = sol.alpha
    b = torch.from_numpy(prob.b).to(dev)
    xr = torch.from_numpy(prob.x_ref).to(dev)
    S = args.storage

    if args.profile_multi > 0:
        # one group of right-hand sides of the same A; ncu captures the second pass
        K = args.profile_multi
        g = sol.multi_group(S)
        pm = make_problem(rank, True, nrhs=g)
        B = torch.from_numpy(np.ascontiguousarray(pm.b.T)).to(dev)
        del pm
        for _ in range(2):
            r = sol.solve_multi(B, tol=0.0, max_iter=K, seed=7, storage=S, max_outer=1, inner_iters=K)
        torch.cuda.synchronize()
        st = r["stats"]
        print(json.dumps({"profile_multi": K, "storage": S, "group": g, "iterations": st["iterations"],
                          "kernel_ms": st["kernel_ms"], "us_per_iteration": 1000.0 * st["kernel_ms"] / K}))
        return 0

    if args.profile_pass > 0:
        # the first pass also runs the CTA-count autotune; ncu captures the second pass
        K = args.profile_pass
        for _ in range(2):
            if args.profile_plain:
                r = sol.solve(b, tol=0.0, max_iter=K, seed=7)
            else:
                r = sol.solve_refined(b, tol=0.0, max_iter=K, seed=7, storage=S, max_outer=1, inner_iters=K)
        torch.cuda.synchronize()
        st = r["stats"]
        print(json.dumps({"profile_pass": K, "storage": "fp64" if args.profile_plain else S, "iterations": st["iterations"],
                          "kernel_ms": st["kernel_ms"], "us_per_iteration": 1000.0 * st["kernel_ms"] / K}))
        return 0

    def solve_mixed(seed, bb=b, xx=xr, x=None):
        r = sol.solve_refined(bb, tol=TOL, seed=seed, storage=S, x_ref=xx, x=x)
        if r["stats"]["rel_err"] > TOL:
            raise RuntimeError(f"solve did not reach {TOL}: {r['stats']}")
        return r

    for w in range(args.warmup):
        solve_mixed(900 + w)

    # ---------------- timed region: K solves, inputs resident in HBM ----------------
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    agg = {"iterations": 0, "kernel_ms": 0.0, "sweep_ms": 0.0, "launches": 0, "grid_launches": 0, "outer": 0}
    for s in range(args.steps):
        st = solve_mixed(1000 + s)["stats"]
        for k in agg:
            agg[k] += st[k]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    value, ms_max = replica_throughput(ms / 1000.0, args.steps, world, dev)
    ms_max *= 1000.0

    # ---------------- e2e: host buffers, copies inside the timed region ----------------
    b_host = torch.from_numpy(prob.b).pin_memory()
    xr_host = torch.from_numpy(prob.x_ref).pin_memory()
    x_host = torch.empty(N, dtype=torch.float64).pin_memory()
    b_d = torch.empty_like(b)
    xr_d = torch.empty_like(xr)
    x_d = torch.empty(N, dtype=torch.float64, device=dev)
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        b_d.copy_(b_host, non_blocking=True)
        xr_d.copy_(xr_host, non_blocking=True)
        solve_mixed(2000 + s, bb=b_d, xx=xr_d, x=x_d)
        x_host.copy_(x_d, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value, _ = replica_throughput(e2e_s, e2e_steps, world, dev)

    # ---------------- plain FP64 path on the same problem ----------------
    plain = None
    if args.plain_steps > 0:
        sol.solve(b, tol=TOL, max_iter=10**7, seed=800, x_ref=xr)
        torch.cuda.synchronize()
        p_ev0, p_ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p_ev0.record(stream)
        pagg = {"iterations": 0, "kernel_ms": 0.0, "grid_launches": 0}
        for s in range(args.plain_steps):
            st = sol.solve(b, tol=TOL, max_iter=10**7, seed=1000 + s, x_ref=xr)["stats"]
            for k in pagg:
                pagg[k] += st[k]
        p_ev1.record(stream)
        torch.cuda.synchronize()
        pms = p_ev0.elapsed_time(p_ev1) / args.plain_steps
        it = pagg["iterations"] / args.plain_steps
        flops = 4.0 * TAU * (M + N) * pagg["iterations"]
        fp64_rate = flops / (pagg["kernel_ms"] / 1000.0) / 1e12
        fp64_peak = dev_peaks["fp64_tflops"]
        plain = {"value": 1000.0 / pms, "unit": "solves/s", "ms_per_solve": pms, "iterations_per_solve": it,
                 "block_iterations_per_s": pagg["iterations"] / (pagg["kernel_ms"] / 1000.0),
                 "roofline": {"bound": "alu", "achieved": fp64_rate, "peak": fp64_peak, "unit": "TFLOP/s",
                              "frac": fp64_rate / fp64_peak,
                              "peak_source": ("measured: rebk_device_peaks FP64 FMA kernel on this GPU "
                                              f"(SM clock {dev_peaks['sm_mhz']:.0f} MHz during it)"),
                              "hbm_gbs": 8.0 * TAU * (M + N) * pagg["iterations"] / (pagg["kernel_ms"] / 1000.0) / 1e9,
                              "hbm_frac": 8.0 * TAU * (M + N) * pagg["iterations"] / (pagg["kernel_ms"] / 1000.0)
                              / 1e9 / hbm_peak}}

    # ---------------- residual stop rule: solves without the known solution ----------------
    resid = None
    if args.residual_steps > 0:
        r_ev0, r_ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        errs, its_r = [], 0
        xs_r = []
        r_ev0.record(stream)
        for s in range(args.residual_steps):
            r = sol.solve_refined(b, tol=TOL, seed=3000 + s, storage=S)
            its_r += r["stats"]["iterations"]
            xs_r.append(r["x"])
        r_ev1.record(stream)
        torch.cuda.synchronize()
        for x_ in xs_r:
            errs.append(float((x_ - xr).norm() / xr.norm()))
        rms = r_ev0.elapsed_time(r_ev1) / args.residual_steps
        resid = {"value": 1000.0 / rms, "unit": "solves/s", "ms_per_solve": rms,
                 "iterations_per_solve": its_r / args.residual_steps, "rel_err_max": max(errs),
                 "rule": "max(||b - z - A x|| / ||b||, ||A^T z|| / (||A||_F ||b||)) <= 1e-8 after each "
                         "refinement pass (no x_ref); rel_err_max is the error against A^+ b measured afterwards"}

    # ---------------- several right-hand sides at once (shared block sequence) ----------------
    multi = None
    if args.multi_rhs > 0:
        multi = measure_multi(args, sol, prob, dev, rank, S, stream, hbm_peak)

    # ---------------- the combined form (mixed + warm start + batched) ----------------
    combined = None
    if not args.no_combined:
        del b_host, xr_host, x_host, b_d, xr_d, x_d
        torch.cuda.empty_cache()
        combined = measure_combined(args, dev, rank)

    # ---------------- roofline of the dominant kernel ----------------
    esize = {"fp32": 4, "bf16": 2}[S]
    bytes_per_iter = float(TAU * N + TAU * M) * esize
    kernel_s = agg["kernel_ms"] / 1000.0
    achieved = bytes_per_iter * agg["iterations"] / kernel_s / 1e9
    traffic_per_iter, traffic_src = kernel_traffic(f"corr_{S}")
    per_launch_iters = agg["iterations"] / max(agg["grid_launches"], 1)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "peak_source": peak_src,
            "traffic": None if traffic_per_iter is None else traffic_per_iter * per_launch_iters,
            "traffic_source": traffic_src + ("" if traffic_per_iter is None else
                                             "; per-iteration DRAM bytes scaled to this run's iterations per launch"),
            "algorithmic_bytes_per_launch": bytes_per_iter * per_launch_iters,
            "kernel": f"rebk_grid_kernel<{ 'float' if S == 'fp32' else '__nv_bfloat16' },float,corr>",
            "kernel_share_of_step": kernel_s / (ms_max / 1000.0),
            "avg_launch_ms": agg["kernel_ms"] / max(agg["grid_launches"], 1)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        anchor = load_anchor()
        if "iterations_to_1e-8" in anchor:
            ips, src = anchor["iterations_to_1e-8"], "oracle's own count, tests/golden/precision_anchor.txt"
        else:
            ips, src = (plain or {}).get("iterations_per_solve", float("nan")), "GPU plain FP64 count"
        cpu = cpu_baseline(prob, alpha, ips, args.cpu_seconds, src)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "storage": S, "tau": TAU, "alpha": alpha, "tol": TOL,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (A: 320 MB bf16 / 640 MB fp32 / 1.28 GB fp64)"},
            "iterations_per_solve": agg["iterations"] / args.steps,
            "outer_passes_per_solve": agg["outer"] / args.steps,
            "kernel_ms_per_solve": agg["kernel_ms"] / args.steps,
            "sweep_ms_per_solve": agg["sweep_ms"] / args.steps,
            "hbm_gbs": achieved,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 8 * (M + N),
                    "d2h_bytes_per_step": 8 * N},
            "gpu_launches": agg["launches"],
            "clocks": clk,
            "plain_fp64": plain,
            "speedup_vs_plain_fp64": None if plain is None else value / plain["value"],
            "residual_rule": resid,
            "combined": combined,
            "multi_rhs": multi,
            "device_peaks": dev_peaks,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
