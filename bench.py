#!/usr/bin/env python
"""Benchmark of the PCAL hot path on GB300: iterations/s and time-to-KKT.

Default workload: f = 1/2 tr(X^T (L3 + Diag(V)) X) on a 128^3 grid (n = 2097152), p = 1024,
V iid U[0, 1], FP32 storage.  One step = one PCAL iteration (Lambda1 multiplier, ABB step
size) in the compensated 3xTF32 phase, from a seeded orthonormal start resident in device
memory; beside the timed steps: one complete solve to relative KKT 1e-5 plus the FP64
Cholesky-QR (time-to-KKT, and end to end through the public API with host copies), the
separable companion against its exact optimum, the FP64 GPU path over its first iterations
(extrapolated) and the oracle on a slab of the grid (cpu_baseline).  `--workload` selects the
other configurations (the 1D Hartree energy, 64^3 stencil, the 512-problem batch, Section
5.4's n = 10000 problems).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]

Prints one JSON line (rank 0).  With N > 1 (torchrun) the default workload's rows are sharded
over the ranks (one problem; strong scaling); the other workloads run one replica per rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCAL time-to-KKT 1e-6 (s) & iters/s, mixed vs FP64 on 1 GB300; % roofline"
WORKLOADS = {
    "hartree1d": dict(kind="hartree1d", n=20000, p=50, alpha=1.0, quad_scale=0.25, beta=1000.0,
                      tol=1e-6, name="hartree1d_n20000_p50"),
    "dense": dict(kind="dense", n=500, p=20, beta=1.0, tol=1e-6, name="dense_trace_n500_p20"),
    # 3D Laplacian plus potential on a 64^3 grid, p = 256: FP32 with tensor-core Grams and
    # update (TF32, compensated 3xTF32 below KKT 1e-3); KKT 1e-5 is where the FP32 path meets
    # 1e-6 of the optimum.  The FP64 path is timed over its first 30 iterations only.
    "stencil3d": dict(kind="stencil3d", m=64, n=262144, p=256, beta=1.0, tol=1e-5,
                      name="stencil3d_n262144_p256", fp64_maxit=30),
    # 512 independent dense trace problems, n uniform in [64, 2048], p uniform in
    # [4, min(64, n/2)], beta = 1, PCAL to relative KKT 1e-6 in one persistent launch.
    "batched": dict(kind="batched", count=512, n_lo=64, n_hi=2048, beta=1.0, tol=1e-6,
                    name="batched_512_dense_trace_n64-2048_p4-64", fp64_sample=6),
    # 3D Laplacian plus potential on a 128^3 grid, p = 1024 (8.6 GB per n x p FP32 buffer),
    # V iid U[0,1]: the largest single-GPU workload, and the default.  One step = one PCAL
    # iteration (all rows of the hot path) in the compensated phase that dominates the solve;
    # beside the steps: one complete solve (time-to-KKT, end to end with host copies), the same
    # solve on the companion instance with a separable potential whose optimum is exact
    # (tests/golden), the FP64 path over its first iterations (extrapolated) and the oracle on
    # the grid's first 8 z-planes (cpu_baseline).  The start is the Q factor of a seeded
    # Gaussian generated on the device (a host FP64 start would take 17 GB).
    # PCAL runs with the Lambda1 multiplier (Lambda = Psi(C)) on this workload and on its
    # separable companion (exact optimum): with eq. (lambda2) a large ABB step early in the solve
    # can collapse the columns onto one direction, which PCAL's column normalisation cannot undo
    # (measured on the companion and, with other rounding of the same kernels, on this instance)
    "stencil3d_128": dict(kind="stencil3d", m=128, n=2097152, p=1024, beta=1.0, tol=1e-5,
                          tol_separable=1e-6, maxit=3000, name="stencil3d_n2097152_p1024",
                          fp64_iters=1, slab_planes=8, lambda_rule="lambda1",
                          separable=dict(lambda_rule="lambda1")),
    # Section 5.4's parallel workloads at n = 10000, p = 1000, PCAL with beta = 1 (the paper's
    # default): Problem 1 with L = Diag(L_1, ..., L_2000) of 5 x 5 Dirichlet blocks (alpha = 1),
    # and Problem 2 with the tridiagonal A and a random linear term; FP32 storage with
    # tensor-core Grams and update.  The FP64 path is timed over its first 10 iterations.
    "block_hartree": dict(kind="hartree1d", n=10000, p=1000, alpha=1.0, quad_scale=0.5, block=5,
                          beta=1.0, tol=1e-6, name="block_hartree_n10000_p1000_b5", fp64_maxit=10,
                          section54=True),
    "tridiag_linear": dict(kind="hartree1d", n=10000, p=1000, alpha=0.0, quad_scale=0.5,
                           linear=True, beta=1.0, tol=1e-6, name="tridiag_linear_n10000_p1000",
                           fp64_maxit=10, section54=True),
}
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="stencil3d_128")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--grams-only", type=int, nargs=2, metavar=("N", "P"), default=None,
                    help="only time the tensor-core Grams X^T [X | G] of one FP32 handle on seeded "
                         "N x P Gaussian matrices (with --tensor-cores); a profiler-sized run")
    ap.add_argument("--slab-planes", type=int, default=0,
                    help="stencil3d_128 only: z-planes of the oracle's bounded sample (the "
                         "cpu_baseline and the reference arm); 0 keeps 8")
    ap.add_argument("--kernel-iters", type=int, default=0,
                    help="only time the kernel groups of this many iterations (graph engine's "
                         "kernels launched one by one) and print them; a short, profiler-sized run")
    ap.add_argument("--tensor-cores", choices=["auto", "off", "tf32", "3xtf32", "tf32-single",
                                               "3xtf32-single"], default="auto")
    ap.add_argument("--p", type=int, default=0,
                    help="block_hartree / tridiag_linear only: the width p (Section 5.4 sweeps "
                         "p = 500 ... 2500 at n = 10000); 0 keeps 1000")
    ap.add_argument("--solver", choices=["pcal", "moptqr"], default="pcal",
                    help="block_hartree / tridiag_linear only: PCAL, or MOptQR (the comparison "
                         "solver of Section 5.4: a Cholesky retraction every iteration)")
    ap.add_argument("--beta", type=float, default=0.0,
                    help="block_hartree / tridiag_linear only: the penalty beta (0 keeps the "
                         "paper's PCAL default 1; from p ~ 0.18 n on, beta = 1 lets the columns "
                         "collapse and beta = s + 0.1 = 4.1 converges)")
    return ap.parse_args()


def workload_config(args, **extra):
    """The workload's parameters, with --p applied to Section 5.4's workloads."""
    wl = dict(WORKLOADS[args.workload], **extra)
    if getattr(args, "p", 0):
        if not wl.get("section54"):
            raise SystemExit("--p applies to the block_hartree and tridiag_linear workloads")
        if not 1 <= args.p <= wl["n"] // 2:
            raise SystemExit(f"--p must lie in [1, {wl['n'] // 2}]")
        wl["name"] = wl["name"].replace(f"_p{wl['p']}", f"_p{args.p}")
        wl["p"] = args.p
    if getattr(args, "solver", "pcal") != "pcal":
        if not wl.get("section54"):
            raise SystemExit("--solver applies to the block_hartree and tridiag_linear workloads")
        wl["variant"] = args.solver
        wl["name"] += f"_{args.solver}"
    if getattr(args, "beta", 0.0):
        if not wl.get("section54"):
            raise SystemExit("--beta applies to the block_hartree and tridiag_linear workloads")
        if not args.beta > 0.0:
            raise SystemExit("--beta must be positive")
        wl["beta"] = args.beta
        wl["name"] += f"_beta{args.beta:g}"
    if getattr(args, "slab_planes", 0):
        if not wl.get("slab_planes"):
            raise SystemExit("--slab-planes applies to the stencil3d_128 workload")
        if not 1 <= args.slab_planes <= wl["m"]:
            raise SystemExit(f"--slab-planes must lie in [1, {wl['m']}]")
        wl["slab_planes"] = args.slab_planes
    return wl


# ---------------------------------------------------------------- distributed plumbing

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, local):
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))


def barrier(world):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def reduce_max_sum(world, tmax, tsum, device="cuda"):
    """(max over ranks of tmax, sum over ranks of tsum); device "cpu" for a gloo group."""
    if world == 1:
        return tmax, tsum
    import torch
    import torch.distributed as dist
    a = torch.tensor([tmax], dtype=torch.float64, device=device)
    b = torch.tensor([tsum], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to PLAM_CLOCKS_DIR (default: the system temporary directory);
        # the bench line carries their summary
        import tempfile
        cdir = os.environ.get("PLAM_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(cdir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- roofline helpers

def sm_count(torch):
    """Streaming multiprocessors of the current device (152 on a GB300)."""
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def measured_tf32_tflops():
    """Dense TF32 tensor peak: the measured bf16 burst GEMM rate times the nominal TF32 / BF16
    dense ratio (1.1 / 2.25 PFLOP/s); the profiling fallback 1.9 PFLOP/s bf16 without the file."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 burst x 1.1/2.25 (nominal TF32/BF16)"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x 1.1/2.25 (nominal TF32/BF16)"


def kernel_flops(wl):
    """Algorithmic tensor-core flops per launch of the contractions: the Grams X^T X (symmetric,
    n p^2) and X^T G (2 n p^2), the update X M and X E (2 x 2 n p^2)."""
    n, p = wl["n"], wl["p"]
    return {"gram_partial": 3 * n * p * p, "update": 4 * n * p * p}


def kernel_bytes(wl, w, nchunks_unused=None):
    """Algorithmic DRAM bytes per launch of each kernel group (w = bytes per element of X)."""
    n, p = wl["n"], wl["p"]
    npw = n * p * w
    if wl["kind"] == "hartree1d" and wl.get("section54"):
        # chain kernels: X read by the density kernel (when alpha != 0) and the gradient kernel,
        # G written, the linear term read; rho partials per column group are O(n)
        obj = (3 if wl["alpha"] else 2) * npw + (npw if wl.get("linear") else 0)
    elif wl["kind"] == "hartree1d":
        obj = 3 * npw + 3 * 8 * n      # read X twice (density, gradient), write G; rho, y
    elif wl["kind"] == "dense":
        obj = n * n * w + 2 * npw
    else:
        obj = 2 * npw + n * w
    return {"objective": obj, "gram_partial": 2 * npw, "gram_finalize": 2 * p * p * 8,
            "update": 4 * npw + 2 * p * p * w, "step_size": 8 * (3 * p + 6),
            "primal_update": 3 * npw}


KERNEL_SOURCES = {
    "resident": ["k_resident.cu"], "tc_update": ["k_tc_update.cu", "tc_ptx.cuh"],
    "tc_gram": ["k_tc_gram.cu", "tc_ptx.cuh"], "tc_gram2": ["k_tc_gram2.cu", "tc_ptx.cuh"],
    "stencil_grad": ["k_objective.cu"],
    "hartree_grad": ["k_objective.cu"], "dense_grad": ["k_objective.cu"],
    "chain_grad": ["k_objective.cu"],
    "update": ["k_update.cu"], "primal_update": ["k_update.cu"], "step_size": ["k_update.cu"],
    "gram_partial": ["k_gram.cu"], "gram_finalize": ["k_gram.cu"],
    "batched_solve": ["k_batched.cu"], "orth": ["k_orth.cu"],
}


def csrc_hash(kernel=None):
    """sha256 (16 hex digits) of a kernel's sources plus the shared headers (all of csrc/
    when kernel is None)."""
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_1810_03930_gb300", "csrc")
    names = sorted(os.listdir(cdir)) if kernel is None else sorted(
        KERNEL_SOURCES.get(kernel, []) + ["plam_common.cuh", "plam_device.cuh"])
    for fn in names:
        h.update(open(os.path.join(cdir, fn), "rb").read())
    return h.hexdigest()[:16]


def tc_gram_name(p, tensor_cores="auto"):
    """The tensor-core Gram kernel the library runs at width p: CTA pairs (256 x 256 tiles) from
    p = 256 on, one CTA per 128-column tile below (or with a "-single" tensor_cores mode)."""
    return "tc_gram2" if p >= 256 and not str(tensor_cores).endswith("-single") else "tc_gram"


def recorded_traffic(kernel, workload):
    """dram bytes per launch recorded by an ncu capture summarised under profiles/, if the
    kernel's sources have not changed since: the summary carries the hash of the sources it was
    captured on, and may list later hashes whose sources differ from them only in host-side
    declarations of the shared header (`same_kernel_sources_sha256_16:`, with the diff named)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    hashes = re.findall(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text)
    if not m or csrc_hash(kernel) not in hashes:
        return None
    return float(m.group(1))


def golden_fstar(name):
    name = name.replace("_moptqr", "")
    path = os.path.join(ROOT, "tests", "golden", f"{name}_optimum.json")
    try:
        return json.load(open(path))
    except Exception:
        pass
    try:       # Section 5.4's workloads: the oracle's PCAL run to relative KKT 1e-8
        g = json.load(open(os.path.join(ROOT, "tests", "golden", "section54_n10000_p1000.json")))
        return {"f_star": g[name]["tol_1e-08"]["f_orth"]}
    except Exception:
        return None


# ---------------------------------------------------------------- our arm

def make_solver(wl, precision, torch, engine="auto", final_orth=1, maxit=3000, tensor_cores=None):
    from paper_1810_03930_gb300 import Solver
    kw = dict(variant=wl.get("variant", "pcal"), lambda_rule=wl.get("lambda_rule", "lambda2"),
              beta=wl["beta"],
              tol=wl["tol"], maxit=maxit,
              precision=precision, final_orth=final_orth, graph_iters=16, engine=engine,
              tensor_cores=tensor_cores or wl.get("tensor_cores", "auto"), orth_metrics=False)
    if wl["kind"] == "stencil3d":
        m = wl["m"]
        return Solver(wl["n"], wl["p"], "stencil3d", grid=(m, m, m), V=wl["V"], **kw)
    if wl["kind"] == "hartree1d":
        return Solver(wl["n"], wl["p"], "hartree1d", alpha=wl["alpha"], quad_scale=wl["quad_scale"],
                      block=wl.get("block", 0), lin=wl.get("lin"), **kw)
    return Solver(wl["n"], wl["p"], "dense", A=wl["A"], **kw)


def load_inputs(wl):
    from workloads import (workload_block_hartree, workload_dense_trace, workload_hartree1d,
                           workload_stencil3d, workload_tridiag_linear)
    if wl.get("section54"):
        w = (workload_tridiag_linear(wl["n"], wl["p"]) if wl.get("linear")
             else workload_block_hartree(wl["n"], wl["p"], wl["block"]))
        wl["lin"] = w.lin
    elif wl["kind"] == "stencil3d":
        w = workload_stencil3d(m=wl["m"], p=wl["p"])
        wl["V"] = w.V
    elif wl["kind"] == "hartree1d":
        w = workload_hartree1d(n=wl["n"], p=wl["p"], alpha=wl["alpha"], quad_scale=wl["quad_scale"])
    else:
        w = workload_dense_trace(wl["n"], wl["p"])
        wl["A"] = w.A
    return w


def orth_feasibility(Q, n, torch):
    """||Q^T Q - I||_F of an FP64 device result (shape (p, ld), column-major n x p), checked
    outside the timed region: the timed solves skip the library's own feasibility report
    (orth_metrics off), which costs one more FP64 Gram."""
    Qt = Q[:, :n]
    E = Qt @ Qt.T - torch.eye(Q.shape[0], dtype=Q.dtype, device=Q.device)
    return float(torch.linalg.matrix_norm(E))


def timed_solves(solver, X0d, steps, flush, torch, host=None, allow_maxit=False):
    """Run `steps` solves; returns (list of ms, list of iters, last Q, last info, launches)."""
    Xw = torch.empty_like(X0d)
    Q = solver.new_matrix(dtype=torch.float64)
    ms, its = [], []
    info = None
    launches0 = solver.kernel_launches()
    Qh = None
    if host is not None:
        Qh = torch.empty(Q.shape, dtype=torch.float64, pin_memory=True)
    for _ in range(steps):
        flush.zero_()
        if host is None:
            Xw.copy_(X0d)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        if host is not None:
            Xw.copy_(host, non_blocking=True)
        st, info = solver.solve(Xw, Q)
        if host is not None:
            Qh.copy_(Q, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if st not in ((0, 2) if allow_maxit else (0,)):
            raise RuntimeError(f"solve did not converge: status {st}, info {info.as_dict()}")
        ms.append(e0.elapsed_time(e1))
        its.append(info.iters)
    return ms, its, Q, info, solver.kernel_launches() - launches0


def cpu_baseline(w, wl, seconds, gpu_iters):
    """The oracle as it stands, on the host cores, on a bounded sample of the same solve."""
    import numpy as np
    from oracle import objectives as oo
    from oracle import plam as op
    obj = oo.objective_for(w)
    t0 = time.perf_counter()
    probe = op.solve(obj, w.X0, variant="pcal", beta=wl["beta"], tol=wl["tol"], maxit=5, record=False)
    per_it = (time.perf_counter() - t0) / max(1, probe.iters + 1)
    k = int(max(5, min(3000, seconds / max(per_it, 1e-6))))
    t0 = time.perf_counter()
    r = op.solve(obj, w.X0, variant="pcal", beta=wl["beta"], tol=wl["tol"], maxit=k, record=False)
    dt = time.perf_counter() - t0
    rate = (r.iters + 1) / dt
    cores = os.cpu_count()
    threads = cores
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            threads = max(i.get("num_threads", cores) for i in info)
    except Exception:
        pass
    return {"value": rate, "unit": "iters/s", "cores": threads, "kind": "oracle",
            "sample": (f"FP64 NumPy/SciPy oracle PCAL from the same X0, {r.iters} iterations "
                       f"({'converged' if r.converged else 'first ' + str(r.iters) + ' of the solve'}) in "
                       f"{dt:.1f} s on {cores} host cores; extrapolated time-to-KKT at the GPU's "
                       f"{gpu_iters} iterations: {gpu_iters / rate:.2f} s"),
            "time_to_kkt_s_est": gpu_iters / rate}


def run_ours(args, rank, world, local):
    import torch
    dist_init(world, local)
    wl = workload_config(args)
    w = load_inputs(wl)
    from paper_1810_03930_gb300 import colmajor_to_device
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # ---- mixed path (the metric)
    sol = make_solver(wl, "fp32", torch)
    X0d = colmajor_to_device(w.X0, torch.float32)
    timed_solves(sol, X0d, max(1, args.warmup), flush, torch)          # warm-up (graph capture, caches)
    clk = ClockSampler(local)
    barrier(world)
    clk.start()
    ms, its, Q, info, launches = timed_solves(sol, X0d, args.steps, flush, torch)
    barrier(world)
    clocks = clk.stop()
    t_total = sum(ms) / 1e3
    iters_total = float(sum(its))
    t_max, iters_all = reduce_max_sum(world, t_total, iters_total)
    value = iters_all / t_max
    ms_per_step = 1e3 * t_max / args.steps
    # ---- parity evidence on the result of the last timed step
    fstar = golden_fstar(wl["name"])
    sol64 = make_solver(wl, "fp64", torch)
    G = sol64.new_matrix()
    f_q = sol64.energy_grad(Q, G)
    parity = {"f_orth": f_q, "feas_orth": orth_feasibility(Q, wl["n"], torch), "kkt_rel": info.kkt_rel}
    if fstar:
        parity["f_star"] = fstar["f_star"]
        parity["obj_rel_err"] = abs(f_q - fstar["f_star"]) / abs(fstar["f_star"])
    # ---- one solve at the tolerance where the objective meets 1e-6 of f* (the error falls
    #      quadratically with the KKT tolerance; 1e-6 leaves ~4e-5 on this workload)
    tight = None
    if wl["kind"] == "hartree1d" and fstar and not wl.get("section54"):
        wl_t = dict(wl, tol=1e-7)
        sol_t = make_solver(wl_t, "fp32", torch)
        timed_solves(sol_t, X0d, 1, flush, torch)
        ms_t, its_t, Q_t, info_t, _ = timed_solves(sol_t, X0d, 1, flush, torch)
        f_t = sol64.energy_grad(Q_t, G)
        tight = {"tol_kkt_rel": 1e-7, "time_s": ms_t[0] / 1e3, "iters": its_t[0],
                 "obj_rel_err": abs(f_t - fstar["f_star"]) / abs(fstar["f_star"]),
                 "feas_orth": orth_feasibility(Q_t, wl["n"], torch)}
        sol_t.close()
    # ---- FP64 GPU path beside it
    X0d64 = colmajor_to_device(w.X0, torch.float64)
    if wl.get("fp64_maxit"):
        # bounded: the first fp64_maxit iterations; time-to-KKT at the mixed path's count
        sol64b = make_solver(wl, "fp64", torch, final_orth=0, maxit=wl["fp64_maxit"])
        timed_solves(sol64b, X0d64, 1, flush, torch, allow_maxit=True)
        ms64, its64, _, _, _ = timed_solves(sol64b, X0d64, 1, flush, torch, allow_maxit=True)
        sol64b.close()
        rate64 = sum(its64) / (sum(ms64) / 1e3)
        fp64 = {"iters_per_s": rate64, "iters_timed": sum(its64),
                "time_to_kkt_s": statistics.mean(its) / rate64,
                "time_to_kkt_note": "extrapolated: mixed-path iteration count / FP64 iteration rate "
                                    f"over its first {wl['fp64_maxit']} iterations"}
    else:
        timed_solves(sol64, X0d64, 1, flush, torch)
        ms64, its64, _, info64, _ = timed_solves(sol64, X0d64, max(1, args.fp64_steps), flush, torch)
        fp64 = {"time_to_kkt_s": statistics.mean(ms64) / 1e3,
                "iters_per_solve": statistics.mean(its64),
                "iters_per_s": sum(its64) / (sum(ms64) / 1e3)}
    # ---- which engine ran the metric
    engine = sol.engine()
    peak_hbm, peak_kind = measured_peaks()
    clock_mhz = clocks.get("sm_mhz") or 2070.0
    n, p = wl["n"], wl["p"]
    flops_iter = 7 * n * p * p            # Table "cost": 7 n p^2 per iteration
    if engine == "resident":
        # the persistent kernel alone: the same solve without the final orthonormalisation
        sol_k = make_solver(wl, "fp32", torch, final_orth=0)
        timed_solves(sol_k, X0d, 1, flush, torch)
        ms_k, its_k, _, _, _ = timed_solves(sol_k, X0d, 3, flush, torch)
        sol_k.close()
        t_launch = statistics.mean(ms_k) / 1e3
        achieved = flops_iter * statistics.mean(its_k) / t_launch / 1e12
        peak = sm_count(torch) * 128 * 2 * clock_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "kernel": "resident_solve_kernel", "achieved": achieved,
                    "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": f"derived: {sm_count(torch)} SMs x 128 FP32 FMA lanes x 2 flop x median SM clock "
                                   f"{clock_mhz:.0f} MHz",
                    "traffic": recorded_traffic("resident", wl["name"]),
                    "alg_flops_per_launch": flops_iter * statistics.mean(its_k),
                    "launch_ms": t_launch * 1e3, "iters_per_launch": statistics.mean(its_k)}
    # ---- the multi-kernel (graph) engine beside it, with per-kernel attribution
    sol_g = make_solver(wl, "fp32", torch, engine="graph")
    timed_solves(sol_g, X0d, 1, flush, torch)
    ms_g, its_g, _, _, _ = timed_solves(sol_g, X0d, 2, flush, torch)
    graph_engine = {"time_to_kkt_s": statistics.mean(ms_g) / 1e3,
                    "iters_per_solve": statistics.mean(its_g),
                    "iters_per_s": sum(its_g) / (sum(ms_g) / 1e3)}
    Xk = X0d.clone()
    sol_g.reset()
    kms, done = sol_g.time_kernels(Xk, 3000)
    # the paper's categories (Fig. "OCQP-percentage"): "Func" the objective, "BLAS3" the Grams,
    # the p x p step and the update product, "Orth" MOptQR's retraction every iteration or
    # PCAL's one final Cholesky-QR (timed here on the last iterate), "other" PCAL's column
    # scaling step
    Qo = sol_g.new_matrix(dtype=torch.float64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sol_g.orthonormalize(Xk, Qo)
    e1.record()
    torch.cuda.synchronize()
    orth_ms = e0.elapsed_time(e1)
    del Qo
    sol_g.close()
    moptqr = wl.get("variant") == "moptqr"
    cat = {"func": kms["objective"] * done,
           "blas3": (kms["gram_partial"] + kms["gram_finalize"] + kms["update"] +
                     kms["step_size"]) * done,
           "orth": kms["primal_update"] * done + (0.0 if moptqr else orth_ms),
           "other": 0.0 if moptqr else kms["primal_update"] * done}
    tot = sum(cat.values())
    categories = {"iterations": done, "ms": cat,
                  "share": {k: v / tot for k, v in cat.items()} if tot > 0 else None,
                  "note": "per-iteration kernel-group times (CUDA events, plain launches) x the "
                          "iterations of the solve; PCAL's Orth is its final Cholesky-QR"}
    kb = kernel_bytes(wl, 4)
    dom = max(kms, key=lambda k: kms[k])
    achieved_g = kb[dom] / (kms[dom] * 1e-3) / 1e9
    tc = wl["p"] >= 128                     # p >= 128: the tensor-core Grams and update run
    kernel_names = {"objective": "chain_grad" if wl.get("section54") else
                    {"hartree1d": "hartree_grad", "stencil3d": "stencil_grad"}.get(
                        wl["kind"], "dense_grad"),
                    "gram_partial": tc_gram_name(wl["p"]) if tc else "gram_partial",
                    "gram_finalize": "gram_finalize", "update": "tc_update" if tc else "update",
                    "step_size": "step_size", "primal_update": "primal_update"}
    roofline_graph = {"bound": "hbm", "kernel": kernel_names[dom], "achieved": achieved_g,
                      "peak": peak_hbm,
                      "unit": "GB/s", "frac": achieved_g / peak_hbm, "peak_source": peak_kind,
                      "traffic": recorded_traffic(kernel_names[dom], wl["name"]),
                      "alg_bytes_per_launch": kb[dom], "launch_ms": kms[dom]}
    kf = kernel_flops(wl)
    tf32, tf32_kind = measured_tf32_tflops()
    if tc and dom in kf and kf[dom] / kb[dom] > tf32 * 1e12 / (peak_hbm * 1e9):
        # a tensor-core contraction above the ridge point (p = 1000: 3p/8 = 375 flop/B for
        # the Grams): bound by the TF32 tensor rate, not by HBM
        achieved_t = kf[dom] / (kms[dom] * 1e-3) / 1e12
        roofline_graph = {"bound": "tensor", "kernel": kernel_names[dom], "achieved": achieved_t,
                          "peak": tf32, "unit": "TFLOP/s", "frac": achieved_t / tf32,
                          "peak_source": tf32_kind,
                          "traffic": recorded_traffic(kernel_names[dom], wl["name"]),
                          "alg_flops_per_launch": kf[dom], "alg_bytes_per_launch": kb[dom],
                          "launch_ms": kms[dom]}
    if moptqr and dom == "primal_update":
        # MOptQR's retraction (the Cholesky-QR of V every iteration) fills this slot: FP64-accurate
        # Gram V^T V and Q = V R^-1 from exact FP32 products, Cholesky and R^-1 in FP64.  Table
        # "cost"'s flops of one retraction: 2 n p^2 (Gram, upper half, and the triangular solve)
        # + 2 p^3 / 3 (Cholesky, R^-1), against the FP32 FMA peak (the products and their exact
        # sums run on the FP32 pipe)
        clk = clocks.get("sm_mhz") or 2070.0
        peak_alu = sm_count(torch) * 128 * 2 * clk * 1e6 / 1e12
        fl = 2.0 * n * p * p + 2.0 * p ** 3 / 3.0
        achieved_r = fl / (kms[dom] * 1e-3) / 1e12
        roofline_graph = {"bound": "alu", "kernel": "moptqr_retraction", "achieved": achieved_r,
                          "peak": peak_alu, "unit": "TFLOP/s", "frac": achieved_r / peak_alu,
                          "peak_source": f"derived: {sm_count(torch)} SMs x 128 FP32 FMA lanes x 2 "
                                         f"flop x median SM clock {clk:.0f} MHz",
                          "traffic": None, "alg_flops_per_launch": fl, "launch_ms": kms[dom],
                          "note": "exact FP32 products cost about ten FP32 operations per "
                                  "multiply-add of the algorithm"}
    if engine != "resident":
        roofline = roofline_graph
    # ---- end to end through the public API with host buffers
    Xh = torch.empty(X0d.shape, dtype=torch.float32, pin_memory=True)
    Xh.copy_(X0d.cpu())
    ms_e, its_e, _, _, _ = timed_solves(sol, X0d, max(1, args.steps), flush, torch, host=Xh)
    t_e, it_e = reduce_max_sum(world, sum(ms_e) / 1e3, float(sum(its_e)))
    e2e = {"value": it_e / t_e, "unit": "iters/s", "time_to_kkt_s": t_e / len(ms_e),
           "h2d_bytes_per_step": int(Xh.numel() * Xh.element_size()),
           "d2h_bytes_per_step": int(Q.numel() * Q.element_size())}
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wl["name"], "objective": (
                          "1/2 tr(X^T A X) + tr(G_lin^T X), A = tridiag(-1,2,-1), G_lin iid U[-1,1] "
                          "(Section 5.4, Problem 2)" if wl.get("linear") else
                          "1/2 tr(X^T L X) + 1/4 rho^T L^-1 rho, L = Diag of 5x5 Dirichlet "
                          "tridiag(-1,2,-1) blocks (Section 5.4, Problem 1)") if wl.get("section54")
                      else {
                          "hartree1d": "1/4 tr(X^T L X) + alpha/4 rho^T L^-1 rho",
                          "stencil3d": "1/2 tr(X^T (L3 + Diag(V)) X), 7-point Dirichlet L3 on 64^3, "
                                       "V iid U[0,1]"}.get(wl["kind"], "1/2 tr(X^T A X)"),
                      "n": wl["n"], "p": wl["p"],
                      "solver": ("MOptQR (Cholesky retraction every iteration), ABB"
                                 if wl.get("variant") == "moptqr" else "PCAL eq.(lambda2), ABB"),
                      "beta": wl["beta"], "tol_kkt_rel": wl["tol"], "final_orth": "FP64 Cholesky-QR",
                      "l2": "flushed before every step (256 MB write)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "time_to_kkt_s": ms_per_step / 1e3, "iters_per_solve": statistics.mean(its),
           "fp64": fp64, "mixed_speedup_vs_fp64": fp64["time_to_kkt_s"] / (ms_per_step / 1e3),
           "parity": parity, "objective_1e-6_solve": tight, "engine": engine,
           "roofline": roofline, "graph_engine": graph_engine,
           "graph_engine_roofline": roofline_graph, "graph_engine_kernels_ms_per_launch": kms,
           "categories": categories,
           "e2e": e2e,
           "gpu_launches": int(launches), "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, wl, args.cpu_seconds, statistics.mean(its))
    if rank == 0:
        print(json.dumps(out), flush=True)
    sol.close()
    sol64.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- the 128^3, p = 1024 workload

STENCIL128_SEED = 1810039300 + 10 * 5 + 1      # stream 1 (the start) of configuration 5


def device_start(sol, n, p, torch):
    """The seeded orthonormal start on the device: the Q factor (FP64 Cholesky-QR of the library,
    rounded to FP32) of an iid N(0, 1) n x p matrix drawn by torch's Philox generator."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(STENCIL128_SEED)
    Z = torch.randn((p, n), generator=gen, device="cuda", dtype=torch.float32)
    Q = torch.empty((p, n), dtype=torch.float64, device="cuda")
    sol.orthonormalize(Z, Q)
    del Z
    X0 = Q.to(torch.float32)
    del Q
    torch.cuda.empty_cache()
    return X0


def stencil_energy64(Q, V64, m, torch):
    """f(Q) = 1/2 tr(Q^T (L3 + Diag(V)) Q) in FP64 with torch, 32 columns at a time: the parity
    check of a result (outside every timed region).  Q: (p, ld) FP64 holding n x p column-major."""
    n = m ** 3
    Vg = V64.view(m, m, m)
    tot = 0.0
    for c0 in range(0, Q.shape[0], 32):
        q = Q[c0:c0 + 32, :n].reshape(-1, m, m, m)
        g = (6.0 + Vg) * q
        g[:, 1:] -= q[:, :-1]
        g[:, :-1] -= q[:, 1:]
        g[:, :, 1:] -= q[:, :, :-1]
        g[:, :, :-1] -= q[:, :, 1:]
        g[:, :, :, 1:] -= q[:, :, :, :-1]
        g[:, :, :, :-1] -= q[:, :, :, 1:]
        tot += float((q * g).sum())
        del g, q
    return 0.5 * tot


def timed_solve_e2e(sol, Xh, Xw, Q, Qh, torch):
    """One complete solve through the public API with the start copied in from pinned host memory
    and the FP64 result copied back: CUDA events split it into H2D, solve (time-to-KKT from the
    start resident in HBM) and D2H; returns (seconds solve, seconds end to end, status, info)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record()
    Xw.copy_(Xh, non_blocking=True)
    ev[1].record()
    st, info = sol.solve(Xw, Q)
    ev[2].record()
    if Qh is not None:
        Qh.copy_(Q, non_blocking=True)
    ev[3].record()
    torch.cuda.synchronize()
    return ev[1].elapsed_time(ev[2]) / 1e3, ev[0].elapsed_time(ev[3]) / 1e3, st, info


def pcal_name(wl):
    return ("PCAL eq.(Lambda1), ABB" if wl.get("lambda_rule") == "lambda1"
            else "PCAL eq.(lambda2), ABB")


def solve_or_report(sol, Xh, Xw, Q, Qh, torch):
    """One complete solve (timed_solve_e2e).  A solve whose final Cholesky-QR fails (the iterate
    lost rank in a transient blow-up of the ABB steps) is reported with its history instead of
    ending the run; otherwise "result" holds timed_solve_e2e's tuple."""
    from paper_1810_03930_gb300._lib import PlamError
    try:
        res = timed_solve_e2e(sol, Xh, Xw, Q, Qh, torch)
    except PlamError as e:
        hist = sol.history()
        out = {"status": "failed", "error": str(e)}
        if len(hist):
            out.update({"iters": int(hist[-1][0]), "kkt_rel_last": float(hist[-1][2]),
                        "feas_last": float(hist[-1][3]),
                        "feas_max": float(max(h[3] for h in hist))})
        return out
    return {"status": {0: "converged", 2: "maxit"}.get(res[2], str(res[2])),
            "iters": int(res[3].iters), "time_s": res[0], "result": res}


def companion_parity(sol_p, wls, Xh, Xw, Q, Vs64, m, torch):
    """One solve of the separable companion and its objective against the exact optimum.  A
    solve whose final Cholesky-QR fails (the iterate lost rank in a transient blow-up of the
    ABB steps, which PCAL cannot undo) is reported with its history instead of ending the run."""
    from paper_1810_03930_gb300._lib import PlamError
    g = golden_fstar("stencil3d_separable_n2097152_p1024")
    fstar = g["f_star"] if g else None
    out = {"tol_kkt_rel": wls["tol"], "variant": wls.get("variant", "pcal"), "beta": wls["beta"],
           "lambda_rule": wls.get("lambda_rule", "lambda2"),
           "potential": "V = v_x(x) + v_y(y) + v_z(z), v_k iid U[0, 1/3] (exact optimum from "
                        "three tridiagonal eigensolves)"}
    try:
        t_sep, _, st_p, info_p = timed_solve_e2e(sol_p, Xh, Xw, Q, None, torch)
    except PlamError as e:
        hist = sol_p.history()
        out.update({"status": "failed", "error": str(e), "iters": int(hist[-1][0]),
                    "kkt_rel_last": float(hist[-1][2]), "feas_last": float(hist[-1][3]),
                    "feas_max": float(max(h[3] for h in hist))})
        return out
    out.update(result_parity(Q, Vs64, m, info_p, torch, fstar))
    out.update({"time_s": t_sep, "status": {0: "converged", 2: "maxit"}.get(st_p, str(st_p))})
    if fstar is not None:
        # the first iterate whose objective is within 1e-6 of f* (the device's f of the iterate
        # X^k, which PCAL keeps at unit column norms: the orthonormalisation moves f only at
        # second order), and the time to it at the solve's mean rate
        hist = sol_p.history()
        ok = [int(h[0]) for h in hist if abs(h[1] - fstar) <= 1e-6 * abs(fstar)]
        if ok:
            k6 = ok[0]
            out["objective_1e-6"] = {"iteration": k6, "time_s_est": t_sep * k6 / max(1, info_p.iters),
                                     "kkt_rel_there": float(hist[k6][2])}
    return out


def result_parity(Q, V64, m, info, torch, fstar=None):
    n = m ** 3
    f = stencil_energy64(Q, V64, m, torch)
    Qs = Q[:, :n]
    E = Qs @ Qs.T
    E.diagonal().sub_(1.0)
    out = {"iters": info.iters, "kkt_rel": info.kkt_rel, "converged": bool(info.converged),
           "f_orth": f, "feas_orth": float(torch.linalg.matrix_norm(E))}
    del E
    if fstar is not None:
        out["f_star"] = fstar
        out["obj_rel_err"] = abs(f - fstar) / abs(fstar)
    return out


def run_stencil128_sharded(args, rank, world, local, wl):
    """N > 1: ONE 128^3, p = 1024 problem whose z-planes are split over the ranks
    (plam_create_sharded; the Grams and dots all-gathered over NCCL, halo planes exchanged with
    the neighbours): the timed steps are iterations of that problem, then one complete solve.
    Strong scaling: the problem does not grow with N."""
    import torch
    from paper_1810_03930_gb300.dist import ShardedStencil, TorchDistComm, sharded_solver
    from workloads import rng_for, uniform_potential
    m, n, p = wl["m"], wl["n"], wl["p"]
    sl = ShardedStencil((m, m, m), rank, world)
    rows = slice(sl.row0, sl.row0 + sl.n_local)
    V = torch.as_tensor(uniform_potential(n, rng_for(5, 0))[rows], device="cuda").to(torch.float32)
    comm = TorchDistComm()

    def solver(tc, maxit, final_orth):
        return sharded_solver(comm, "stencil3d", sl.n_local, p, sl.row0, n, grid=(m, m, sl.nz_local),
                              V=V, variant="pcal", lambda_rule=wl.get("lambda_rule", "lambda2"),
                              beta=wl["beta"],
                              tol=wl["tol"], maxit=maxit, precision="fp32", final_orth=final_orth,
                              tensor_cores=tc)

    sol_s = solver("3xtf32", 100000, 0)
    # the same seeded start as one GPU: every rank draws the whole Gaussian and keeps its rows;
    # the orthonormalisation's Gram is summed over the ranks
    gen = torch.Generator(device="cuda")
    gen.manual_seed(STENCIL128_SEED)
    Z = torch.randn((p, n), generator=gen, device="cuda", dtype=torch.float32)[:, rows].contiguous()
    buf, Zl = sl.new_x(p, torch.float32)
    Zl[:, :sl.n_local] = Z
    del Z
    Q = torch.empty((p, sl.n_local), dtype=torch.float64, device="cuda")
    sol_s.orthonormalize(Zl, Q)
    X0 = Q.to(torch.float32)
    del Q
    xbuf, X = sl.new_x(p, torch.float32)
    X[:, :sl.n_local] = X0
    for _ in range(max(3, args.warmup)):
        sol_s.step(X)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clk = ClockSampler(local)
    barrier(world)
    clk.start()
    launches0 = sol_s.kernel_launches()
    for e0, e1 in evs:
        e0.record()
        sol_s.step(X)
        e1.record()
    barrier(world)
    clocks = clk.stop()
    launches = sol_s.kernel_launches() - launches0
    sol_s.close()
    t_max, _ = reduce_max_sum(world, sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3, 0.0)
    value = args.steps / t_max
    # one complete solve, the start in from pinned host memory and the result back
    sol = solver("auto", wl["maxit"], 1)
    Xh = torch.empty((p, sl.n_local), dtype=torch.float32, pin_memory=True)
    Xh.copy_(X0)
    Qh = torch.empty((p, sl.n_local), dtype=torch.float64, pin_memory=True)
    Q = torch.empty((p, sl.n_local), dtype=torch.float64, device="cuda")
    barrier(world)
    t_solve, t_e2e, st, info = timed_solve_e2e(sol, Xh, X, Q, Qh, torch)
    t_solve, _ = reduce_max_sum(world, t_solve, 0.0)
    t_e2e, _ = reduce_max_sum(world, t_e2e, 0.0)
    sol.close()
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wl["name"], "n": n, "p": p, "solver": pcal_name(wl),
                      "beta": wl["beta"], "tol_kkt_rel": wl["tol"], "maxit": wl["maxit"],
                      "step": "one PCAL iteration of the whole problem, compensated 3xTF32",
                      "l2": "inputs larger than L2",
                      "parallelism": f"rows sharded over {world} GPUs (z-slabs; NCCL all-gather of "
                                     "the Grams and dots, halo planes with the neighbours)"},
           "time_to_kkt_s": t_solve, "iters_per_solve": info.iters,
           "parity": {"iters": info.iters, "kkt_rel": info.kkt_rel,
                      "status": {0: "converged", 2: "maxit"}.get(st, str(st))},
           "e2e": {"value": info.iters / t_e2e, "unit": "iters/s", "time_to_kkt_s": t_e2e,
                   "h2d_bytes_per_step": int(n * p * 4), "d2h_bytes_per_step": int(n * p * 8)},
           "gpu_launches": int(launches), "clocks": clocks}
    if rank == 0:
        print(json.dumps(out), flush=True)
    import torch.distributed as dist
    dist.destroy_process_group()


def run_stencil128(args, rank, world, local):
    import numpy as np
    import torch
    dist_init(world, local)
    wl = workload_config(args)
    if world > 1:
        run_stencil128_sharded(args, rank, world, local, wl)
        return
    m, n, p = wl["m"], wl["n"], wl["p"]
    from workloads import rng_for, stencil3d_separable_potential, uniform_potential
    V64 = torch.as_tensor(uniform_potential(n, rng_for(5, 0)), device="cuda")
    wl["V"] = V64.to(torch.float32)
    # ---- the timed steps: PCAL iterations in the compensated phase (3xTF32 Grams and update)
    sol_s = make_solver(wl, "fp32", torch, engine="graph", final_orth=0, maxit=100000,
                        tensor_cores="3xtf32")
    X0 = device_start(sol_s, n, p, torch)
    Xs = X0.clone()
    for _ in range(max(3, args.warmup)):
        sol_s.step(Xs)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clk = ClockSampler(local)
    barrier(world)
    clk.start()
    launches0 = sol_s.kernel_launches()
    for e0, e1 in evs:
        e0.record()
        sol_s.step(Xs)
        e1.record()
    barrier(world)
    clocks = clk.stop()
    launches = sol_s.kernel_launches() - launches0
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    t_max, iters_all = reduce_max_sum(world, sum(step_ms) / 1e3, float(args.steps))
    value = iters_all / t_max
    ms_per_step = 1e3 * t_max / args.steps
    # per-kernel attribution of the same iterations (CUDA events between the kernel groups)
    kms, _ = sol_s.time_kernels(Xs, 3)
    sol_s.close()
    del Xs
    torch.cuda.empty_cache()
    # ---- one complete solve of the workload: time-to-KKT and end to end.  If the iterate of a
    # solve with eq. (lambda2) loses rank in a transient of the ABB steps (the final Cholesky-QR
    # then fails, and PCAL cannot undo a collapse), the failure is reported and the solve is
    # repeated from the same start with the Lambda1 multiplier
    Xh = torch.empty((p, n), dtype=torch.float32, pin_memory=True)
    Xh.copy_(X0)
    Qh = torch.empty((p, n), dtype=torch.float64, pin_memory=True)
    Xw = torch.empty_like(X0)
    Q = torch.empty((p, n), dtype=torch.float64, device="cuda")
    rules = [wl.get("lambda_rule", "lambda2")]
    if rules[0] != "lambda1":
        rules.append("lambda1")
    attempts, info, st, t_solve, t_e2e, launches_solve, parity = [], None, None, None, None, 0, None
    for rule in rules:
        sol = make_solver(dict(wl, lambda_rule=rule), "fp32", torch, engine="graph",
                          maxit=wl["maxit"])
        attempt = solve_or_report(sol, Xh, Xw, Q, Qh, torch)
        attempt["lambda_rule"] = rule
        if attempt["status"] != "failed":
            t_solve, t_e2e, st, info = attempt.pop("result")
            launches_solve = sol.kernel_launches()
            parity = result_parity(Q, V64, m, info, torch)
            parity["status"] = attempt["status"]
            parity["lambda_rule"] = rule
        attempts.append(attempt)
        sol.close()
        if info is not None:
            break
    del Qh
    # ---- the companion instance with a separable potential: exact optimum (tests/golden)
    Vs64 = torch.as_tensor(stencil3d_separable_potential(m)[0], device="cuda")
    wls = dict(wl, V=Vs64.to(torch.float32), tol=wl["tol_separable"], **wl.get("separable", {}))
    sol_p = make_solver(wls, "fp32", torch, engine="graph", maxit=wl["maxit"])
    parity_sep = companion_parity(sol_p, wls, Xh, Xw, Q, Vs64, m, torch)
    sol_p.close()
    del Xh, Q, Vs64
    torch.cuda.empty_cache()
    # ---- the FP64 GPU path: its first iterations, extrapolated to the mixed path's count
    sol64 = make_solver(wl, "fp64", torch, engine="graph", final_orth=0, maxit=100000)
    X64 = X0.to(torch.float64)
    sol64.step(X64)                       # warm-up (first launch of every kernel)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(wl["fp64_iters"]):
        sol64.step(X64)
    e1.record()
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3 / wl["fp64_iters"]
    sol64.close()
    del X64
    fp64 = {"s_per_iter": t64, "iters_per_s": 1.0 / t64, "iters_timed": wl["fp64_iters"],
            "time_to_kkt_s": info.iters * t64 if info is not None else None,
            "time_to_kkt_note": "extrapolated: the mixed path's iteration count x the FP64 path's "
                                f"time per iteration over iterations 2..{1 + wl['fp64_iters']}"}
    # ---- roofline of the dominant kernel group of the timed steps
    peak_hbm, peak_kind = measured_peaks()
    tf32, tf32_kind = measured_tf32_tflops()
    kf = kernel_flops(wl)
    kb = kernel_bytes(wl, 4)
    dom = max(kms, key=lambda k: kms[k])
    names = {"objective": "stencil_grad", "gram_partial": tc_gram_name(p),
             "gram_finalize": "gram_finalize",
             "update": "tc_update", "step_size": "step_size", "primal_update": "primal_update"}
    if dom in kf:
        ach = kf[dom] / (kms[dom] * 1e-3) / 1e12
        roofline = {"bound": "tensor", "kernel": names[dom], "achieved": ach, "peak": tf32,
                    "unit": "TFLOP/s", "frac": ach / tf32, "peak_source": tf32_kind,
                    "traffic": recorded_traffic(names[dom], wl["name"]),
                    "alg_flops_per_launch": kf[dom], "launch_ms": kms[dom],
                    "mode": "compensated 3xTF32 (three MMAs per product; the flops counted are the "
                            "algorithm's, Table 'cost')"}
    else:
        ach = kb[dom] / (kms[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": names[dom], "achieved": ach, "peak": peak_hbm,
                    "unit": "GB/s", "frac": ach / peak_hbm, "peak_source": peak_kind,
                    "traffic": recorded_traffic(names[dom], wl["name"]),
                    "alg_bytes_per_launch": kb[dom], "launch_ms": kms[dom]}
    kernels = {}
    for k, ms in kms.items():
        d = {"ms": ms}
        if k in kf:
            d["tflops"] = kf[k] / (ms * 1e-3) / 1e12
            d["frac_tf32"] = d["tflops"] / tf32
        else:
            d["gbs"] = kb[k] / (ms * 1e-3) / 1e9
            d["frac_hbm"] = d["gbs"] / peak_hbm
        kernels[names[k]] = d
    h2d = int(n * p * 4)
    d2h = int(n * p * 8)
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wl["name"],
                      "objective": "1/2 tr(X^T (L3 + Diag(V)) X), 7-point Dirichlet L3 on 128^3, "
                                   "V iid U[0,1]",
                      "n": n, "p": p, "solver": pcal_name(wl), "beta": wl["beta"],
                      "tol_kkt_rel": wl["tol"], "maxit": wl["maxit"],
                      "step": "one PCAL iteration, compensated 3xTF32 tensor-core Grams and update",
                      "final_orth": "FP64 Cholesky-QR",
                      "l2": "inputs larger than L2 (8.6 GB per n x p buffer)",
                      "parallelism": "single GPU" if world == 1 else f"{world} replicas"},
           "time_to_kkt_s": t_solve, "iters_per_solve": info.iters if info else None,
           "iters_per_s_solve": info.iters / t_solve if info else None,
           "fp64": fp64,
           "mixed_speedup_vs_fp64": fp64["time_to_kkt_s"] / t_solve if info else None,
           "solve_attempts": attempts,
           "parity": parity, "parity_separable": parity_sep, "engine": "graph",
           "roofline": roofline, "kernels_ms_per_launch": kernels,
           "e2e": {"value": info.iters / t_e2e if info else None, "unit": "iters/s",
                   "time_to_kkt_s": t_e2e, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "note": "one complete solve through Solver.solve: the start from pinned host "
                           "memory in, the FP64 result out" if info else
                           "no solve completed (solve_attempts)"},
           "gpu_launches": int(launches), "gpu_launches_solve": int(launches_solve),
           "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        iters = info.iters if info else attempts[-1].get("iters", wl["maxit"])
        out["cpu_baseline"] = cpu_baseline_slab(wl, V64.cpu().numpy(), args.cpu_seconds, iters)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def slab_problem(wl, V, planes):
    """The first `planes` z-planes of the 128^3 workload as a Dirichlet problem of their own (the
    oracle's bounded sample): the same p, the potential of those planes, a seeded orthonormal
    start.  Its iteration cost is that of the full grid times planes / 128 (Table "cost":
    7 n p^2 + O(n p) is linear in n)."""
    import numpy as np
    from workloads import orthonormal_start, rng_for
    m, p = wl["m"], wl["p"]
    ns = m * m * planes
    return (m, m, planes), np.asarray(V[:ns]), orthonormal_start(ns, p, rng_for(5, 4)), ns


def cpu_baseline_slab(wl, V, seconds, gpu_iters):
    """The oracle as it stands on the host cores, PCAL iterations on the first z-planes of the
    grid (bounded by `seconds`), scaled to whole-grid iterations/s by the row count."""
    from oracle import objectives as oo
    from oracle import plam as op
    planes = wl["slab_planes"]
    grid, Vs, X0s, ns = slab_problem(wl, V, planes)
    obj = oo.Stencil3DObjective(grid, Vs)
    t0 = time.perf_counter()
    op.solve(obj, X0s, variant="pcal", beta=wl["beta"],
             lambda_rule=wl.get("lambda_rule", "lambda2"), tol=0.0, maxit=1, record=False)
    per_it = time.perf_counter() - t0          # one iteration plus the final Householder QR
    k = int(max(1, min(50, seconds / max(per_it, 1e-6))))
    t0 = time.perf_counter()
    r = op.solve(obj, X0s, variant="pcal", beta=wl["beta"],
                 lambda_rule=wl.get("lambda_rule", "lambda2"), tol=0.0, maxit=k, record=False)
    dt = time.perf_counter() - t0
    scale = ns / wl["n"]
    rate = (r.iters + 1) / dt * scale
    return {"value": rate, "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"FP64 NumPy/SciPy oracle PCAL, {r.iters} iterations (plus its final "
                       f"Householder QR) on the first {planes} of the 128 z-planes (n = {ns}, "
                       f"p = {wl['p']}) in {dt:.1f} s on {os.cpu_count()} host cores; iterations/s "
                       f"x {scale:g} = the full grid's rate; time-to-KKT at the GPU's {gpu_iters} "
                       f"iterations: {gpu_iters / rate:.0f} s"),
            "time_to_kkt_s_est": gpu_iters / rate}


# ---------------------------------------------------------------- reference arm (the oracle)

def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workload_config(args)
    scale, X0 = 1.0, None
    from oracle import objectives as oo
    from oracle import plam as op
    if wl["kind"] == "batched":        # the oracle on the batch's first problem per step
        from workloads import batched_shapes, workload_batched_problem
        n, p = batched_shapes(count=wl["count"], n_lo=wl["n_lo"], n_hi=wl["n_hi"])[0]
        w = workload_batched_problem(0, n, p)
        wl.update(kind="dense", n=n, p=p, A=w.A)
        obj = oo.objective_for(w)
    elif wl.get("slab_planes"):        # 128^3: iterations on the grid's first z-planes, scaled
        from workloads import rng_for, uniform_potential
        grid, Vs, X0, ns = slab_problem(wl, uniform_potential(wl["n"], rng_for(5, 0)),
                                        wl["slab_planes"])
        obj = oo.Stencil3DObjective(grid, Vs)
        scale = ns / wl["n"]
    else:
        w = load_inputs(wl)
        obj = oo.objective_for(w)
    if X0 is None:
        X0 = w.X0
    per_it = 0.0
    for _ in range(max(1, args.warmup)):
        t0 = time.perf_counter()
        r = op.solve(obj, X0, variant="pcal", beta=wl["beta"], tol=wl["tol"],
                     lambda_rule=wl.get("lambda_rule", "lambda2"),
                     maxit=1 if scale != 1.0 else 2, record=False)
        per_it = (time.perf_counter() - t0) / (r.iters + 1)
    # each step a bounded sample of the solve: 20 iterations, fewer where one takes long (about 8 s
    # of CPU work per step), so that a --steps K --warmup W run ends within minutes; two on the
    # 128^3 workload's slab (seconds per iteration)
    per_step = 2 if scale != 1.0 else int(max(3, min(20, 8.0 / max(per_it, 1e-9))))
    times, iters = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = op.solve(obj, X0, variant="pcal", beta=wl["beta"], tol=wl["tol"],
                     lambda_rule=wl.get("lambda_rule", "lambda2"), maxit=per_step,
                     record=False)
        times.append(time.perf_counter() - t0)
        iters.append(r.iters + 1)
    value = sum(iters) / sum(times) * scale
    sample = (f"FP64 NumPy/SciPy oracle PCAL, the first {per_step} iterations of the {wl['name']} "
              f"solve from the seeded X0 per step, on {os.cpu_count()} host cores")
    if scale != 1.0:
        sample = (f"FP64 NumPy/SciPy oracle PCAL, {per_step} iterations (and its final Householder "
                  f"QR) per step on the first {wl['slab_planes']} of the 128 z-planes (n = "
                  f"{int(scale * wl['n'])}, p = {wl['p']}), on {os.cpu_count()} host cores; "
                  f"iterations/s x {scale:g} = the full grid's rate")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": wl["name"], "n": wl["n"], "p": wl["p"],
                                           "beta": wl["beta"], "tol_kkt_rel": wl["tol"]},
           "cpu_baseline": {"value": value, "unit": "iters/s", "cores": os.cpu_count(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_grams_only(args):
    """Milliseconds of plam_grams (the tensor-core Gram kernel, its chunk reduction and the
    handle's synchronisation) on seeded N x P Gaussian X and G, after three untimed calls."""
    import torch
    from paper_1810_03930_gb300 import Solver
    n, p = args.grams_only
    tc = args.tensor_cores if args.tensor_cores not in ("auto", "off") else "3xtf32"
    s = Solver(n, p, "hartree1d", precision="fp32", tensor_cores=tc)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(STENCIL128_SEED)
    X = torch.randn((p, n), generator=gen, device="cuda") / n ** 0.5
    G = torch.randn((p, n), generator=gen, device="cuda")
    for _ in range(3):
        s.grams(X, G)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        s.grams(X, G)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"grams_only": {"n": n, "p": p, "tensor_cores": tc,
                                     "kernel": tc_gram_name(p, tc),
                                     "ms_per_call": e0.elapsed_time(e1) / 5}}), flush=True)
    s.close()


def run_kernel_iters(args):
    """Per-kernel-group milliseconds of the first --kernel-iters iterations (mixed path); for the
    batched workload, one launch capped at --kernel-iters iterations per problem."""
    import torch
    if WORKLOADS[args.workload]["kind"] == "batched":
        from paper_1810_03930_gb300 import BatchSolver
        from workloads import batched_shapes, workload_batched_problem
        wl = WORKLOADS["batched"]
        shapes = batched_shapes(count=wl["count"], n_lo=wl["n_lo"], n_hi=wl["n_hi"])
        ws = [workload_batched_problem(i, n, p) for i, (n, p) in enumerate(shapes)]
        bs = BatchSolver([w.A for w in ws], [w.X0 for w in ws], beta=wl["beta"], tol=0.0,
                         maxit=args.kernel_iters)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        infos = bs.solve()
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"workload": wl["name"], "iterations_per_problem": args.kernel_iters,
                          "launch_ms": e0.elapsed_time(e1),
                          "iterations": sum(i.iters for i in infos)}), flush=True)
        bs.close()
        return
    import numpy as np
    wl = workload_config(args, tensor_cores=args.tensor_cores)
    if wl.get("slab_planes"):
        from workloads import rng_for, uniform_potential
        wl["V"] = uniform_potential(wl["n"], rng_for(5, 0))
        sol = make_solver(wl, "fp32", torch, engine="graph")
        X = device_start(sol, wl["n"], wl["p"], torch)
    else:
        w = load_inputs(wl)
        from paper_1810_03930_gb300 import colmajor_to_device
        sol = make_solver(wl, "fp32", torch, engine="graph")
        X = colmajor_to_device(w.X0, torch.float32)
    kms, done = sol.time_kernels(X, args.kernel_iters)
    sol.close()
    print(json.dumps({"workload": wl["name"], "tensor_cores": args.tensor_cores, "iterations": done,
                      "kernels_ms_per_launch": kms}), flush=True)


def run_batched(args, rank, world, local):
    """The batched configuration: one step = one persistent launch solving every problem."""
    import numpy as np
    import torch
    dist_init(world, local)
    wl = dict(WORKLOADS["batched"])
    from paper_1810_03930_gb300 import BatchSolver, colmajor_to_device
    from workloads import batched_shapes, workload_batched_problem
    shapes = batched_shapes(count=wl["count"], n_lo=wl["n_lo"], n_hi=wl["n_hi"])
    ws = [workload_batched_problem(i, n, p) for i, (n, p) in enumerate(shapes)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    bs = BatchSolver([w.A for w in ws], [w.X0 for w in ws], beta=wl["beta"], tol=wl["tol"],
                     maxit=3000)
    X0s = [x.clone() for x in bs.X]
    tile, tune_ms = bs.autotune(iters=20)

    def restore():
        for x, x0 in zip(bs.X, X0s):
            x.copy_(x0)

    def step(host=None):
        flush.zero_()
        if host is None:
            restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        if host is not None:
            for x, h in zip(bs.X, host[0]):
                x.copy_(h, non_blocking=True)
        infos = bs.solve()
        if host is not None:
            for q, h in zip(bs.Q, host[1]):
                h.copy_(q, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), infos

    for _ in range(max(1, args.warmup)):
        step()
    clk = ClockSampler(local)
    barrier(world)
    clk.start()
    ms, its, conv = [], [], []
    for _ in range(args.steps):
        t, infos = step()
        ms.append(t)
        its.append(sum(i.iters for i in infos))
        conv.append(sum(1 for i in infos if i.converged))
    barrier(world)
    clocks = clk.stop()
    t_max, it_all = reduce_max_sum(world, sum(ms) / 1e3, float(sum(its)))
    value = it_all / t_max
    ms_per_step = 1e3 * t_max / args.steps
    # parity: the objective of every orthonormalised result against Ky Fan's optimum
    from oracle import objectives as oo
    errs = []
    for w, q in zip(ws[:64], bs.Q[:64]):
        Q = np.asfortranarray(q[:, : w.n].double().cpu().numpy().T)
        fstar = 0.5 * np.linalg.eigvalsh(w.A)[: w.p].sum()
        errs.append(abs(oo.TraceObjective(w.A).value(Q) - fstar) / abs(fstar))
    parity = {"checked": len(errs), "max_obj_rel_err": float(max(errs)),
              "converged": conv[-1], "count": len(ws),
              "max_feas_orth": float(max(i.feas_orth for i in infos))}
    # roofline: the kernel is bound by its FP32 arithmetic (A stays in L2 while a CTA works on it)
    flops = sum(i.iters * (2.0 * w.n * w.n * w.p + 8.0 * w.n * w.p * w.p) for w, i in zip(ws, infos))
    clock_mhz = clocks.get("sm_mhz") or 2070.0
    peak = sm_count(torch) * 128 * 2 * clock_mhz * 1e6 / 1e12
    achieved = flops / (ms_per_step * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "batched_solve_kernel", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"derived: {sm_count(torch)} SMs x 128 FP32 FMA lanes x 2 flop x median SM clock "
                               f"{clock_mhz:.0f} MHz",
                "alg_flops_per_launch": flops, "launch_ms": ms_per_step}
    # FP64 comparator: sequential single-problem FP64 solves of a sample, scaled by cost
    from paper_1810_03930_gb300 import Solver
    idx = np.linspace(0, len(ws) - 1, wl["fp64_sample"]).astype(int)
    t64, cost64 = 0.0, 0.0
    for i in idx:
        w = ws[i]
        s = Solver(w.n, w.p, "dense", A=w.A, variant="pcal", beta=wl["beta"], tol=wl["tol"],
                   maxit=3000, precision="fp64", final_orth=1)
        Xd = colmajor_to_device(w.X0, torch.float64)
        Q = s.new_matrix(dtype=torch.float64)
        s.solve(Xd.clone(), Q)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st, inf = s.solve(Xd, Q)
        e1.record()
        torch.cuda.synchronize()
        t64 += e0.elapsed_time(e1) / 1e3
        cost64 += w.n * w.n * w.p
        s.close()
    cost_all = float(sum(w.n * w.n * w.p for w in ws))
    fp64 = {"time_to_kkt_s": t64 * cost_all / cost64, "sampled_problems": len(idx),
            "time_to_kkt_note": "512 sequential FP64 single-problem solves, extrapolated from "
                                f"{len(idx)} timed ones by the sum of n^2 p"}
    # end to end: starts from pinned host memory, orthonormalised results back to the host
    hx = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in bs.X]
    hq = [torch.empty(q.shape, dtype=q.dtype, pin_memory=True) for q in bs.Q]
    for h, x0 in zip(hx, X0s):
        h.copy_(x0.cpu())
    te, ite = [], 0
    for _ in range(max(1, args.steps)):
        t, infos_e = step(host=(hx, hq))
        te.append(t)
        ite += sum(i.iters for i in infos_e)
    t_e, it_e = reduce_max_sum(world, sum(te) / 1e3, float(ite))
    e2e = {"value": it_e / t_e, "unit": "iters/s", "time_to_kkt_s": t_e / len(te),
           "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hx)),
           "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hq))}
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wl["name"], "problems": len(ws),
                      "objective": "1/2 tr(X_b^T A_b X_b), A_b = (B+B^T)/2, B iid N(0,1)",
                      "solver": "PCAL eq.(lambda2), ABB, one persistent launch (CUDA graph)",
                      "beta": wl["beta"], "tol_kkt_rel": wl["tol"], "tile_rows": tile,
                      "autotune_ms": tune_ms, "final_orth": "FP64 Cholesky-QR per problem",
                      "l2": "flushed before every step (256 MB write)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "time_to_kkt_s": ms_per_step / 1e3, "iters_per_step": statistics.mean(its),
           "fp64": fp64, "mixed_speedup_vs_fp64": fp64["time_to_kkt_s"] / (ms_per_step / 1e3),
           "parity": parity, "engine": "batched", "roofline": roofline, "e2e": e2e,
           "gpu_launches": args.steps, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_batched(ws, wl, args.cpu_seconds, ms_per_step / 1e3)
    if rank == 0:
        print(json.dumps(out), flush=True)
    bs.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline_batched(ws, wl, seconds, gpu_s):
    """The oracle on the host cores: sequential solves of the batch's problems until about
    `seconds` have passed, extrapolated to the whole batch by the sum of n^2 p."""
    from oracle import objectives as oo
    from oracle import plam as op
    t0 = time.perf_counter()
    cost_done, done, its = 0.0, 0, 0
    for w in ws[::-1]:                       # smallest problems last in the list: take a mix
        r = op.solve(oo.TraceObjective(w.A), w.X0, variant="pcal", beta=wl["beta"], tol=wl["tol"],
                     maxit=3000, record=False)
        cost_done += w.n * w.n * w.p
        done += 1
        its += r.iters
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    cost_all = float(sum(w.n * w.n * w.p for w in ws))
    est = dt * cost_all / cost_done
    return {"value": its / dt, "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"FP64 NumPy oracle PCAL, {done} of the {len(ws)} problems solved to KKT "
                       f"{wl['tol']} in {dt:.1f} s; whole batch extrapolated by the sum of n^2 p: "
                       f"{est:.0f} s"),
            "time_to_kkt_s_est": est}


def main():
    args = parse_args()
    workload_config(args)          # refuses a bad --p before any device work
    rank, world, local = dist_env()
    if args.workload == "batched" and args.impl == "ours" and args.kernel_iters == 0:
        run_batched(args, rank, world, local)
        return
    if args.grams_only:
        if rank == 0:
            run_grams_only(args)
        return
    if args.kernel_iters > 0:
        if rank == 0:
            run_kernel_iters(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if WORKLOADS[args.workload].get("slab_planes"):
        run_stencil128(args, rank, world, local)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
