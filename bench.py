"""Benchmark: f(A)b solves/s of sketched FOM + sketched GMRES on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl skf|reference]

Default workload (cd3d_n100): 3D convection-diffusion, 7-point centred
differences on a 100^3 grid (N = 1e6, 6.94e6 nonzeros), FP64 values, seeded
N(0,1) right-hand side normalised, f(z) = log(1+z)/z, m = 200, k = 2,
sparse-sign sketch s = 800, zeta = 8.

One step = one pass of the whole path over one right-hand side through the
public API: skf_sfom_sgmres, both approximants of f(A) b from one truncated
Arnoldi process with fused sketches (the basis both methods use, as in the
reference arm's pair), one whitening QR, both adaptive-quadrature tails and
one pass over V_m for both recombinations (--separate: skf_sfom and
skf_sgmres, two Arnoldi processes).  value = solves/s over all GPUs (2
solves per step per GPU).  Under torchrun each rank runs an
independent replica (the path has no data-path exchange; scaling "weak").
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_PEAK_FALLBACK = 6800.0
# DRAM bytes (read + write) per Arnoldi step, summed over the spmv and update
# kernels of one ncu capture of those kernels as they stand; keyed by workload,
# basis dtype and sketch, and removed whenever those kernels change.
FP32_STEP_TRAFFIC = 1511.9e6   # DRAM bytes per FP32 step at N = 16.8M (ncu, the current kernels)
# ncu dram bytes per Arnoldi step, for step kernels unchanged since their capture;
# k_arnoldi_persist is one launch for all m steps: per-step bytes are the
# difference of two captures (m = 40 and m = 12) over 28 steps; the FP32 entry
# is the two step kernels of one step (spmv 1125.4 MB + update 386.4 MB)
NCU_TRAFFIC_PER_STEP = {("cd3d_n100", "f64", "sparse_sign", True): 91.4e6,
                        ("cd3d_n100", "f64", "sparse_sign", False): None,
                        ("cd3d_n256_fp32", "f32", "sparse_sign", False): FP32_STEP_TRAFFIC}


BASIS_BYTES = {"f64": 8, "f32": 4, "bf16": 2}
DTYPE_NAME = {"f64": "f64", "f32": "f32", "bf16": "bf16-storage/f32"}
METRIC = {"f64": "f(A)b solves/s (sFOM + sGMRES, FP64)",
          "f32": "f(A)b solves/s (sFOM + sGMRES, FP32 basis and arithmetic, FP64 tail)",
          "bf16": "f(A)b solves/s (sFOM + sGMRES, BF16 basis, FP32 arithmetic, FP64 tail)"}


SKETCH_KIND = {"sparse_sign": lambda skf: skf.SPARSE_SIGN, "srht": lambda skf: skf.SRHT,
               "srdct": lambda skf: skf.SRDCT}


def basis_torch(name: str):
    import torch
    return {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[name]


def reference_error_fp64(skf, A, S, b_dev, f, wl, x_fom, x_gm, dev):
    """Relative 2-norm error of the reduced-precision results against the FP64
    GPU path on the same operator (values widened exactly), sketch and rule."""
    import numpy as np
    import torch
    op64 = skf.upload_csr(A.rowptr, A.colind, A.values.astype(np.float64), device=dev)
    p64 = skf.make_params(wl.m, wl.k, tol=1e-10)
    r_f = skf.sfom(op64.csr, S, b_dev, f, p64)
    r_g = skf.sgmres(op64.csr, S, b_dev, f, p64)
    torch.cuda.synchronize()
    e_f = float(torch.linalg.norm(x_fom - r_f) / torch.linalg.norm(r_f))
    e_g = float(torch.linalg.norm(x_gm - r_g) / torch.linalg.norm(r_g))
    del op64, r_f, r_g
    torch.cuda.empty_cache()
    return {"rel_err_vs_fp64_gpu": {"sfom": e_f, "sgmres": e_g}, "target": 1e-6,
            "meets_target": bool(max(e_f, e_g) <= 1e-6)}


# ---- replicas: one independent solve stream per GPU, no data-path collective.
# The timed region is bracketed by barriers; the job's time is the slowest
# rank's, and its throughput counts every rank's solves.
def replica_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_max(v: float, world: int, device) -> float:
    """Max of a per-rank value over the ranks (device: where the process
    group's tensors live: cuda under NCCL, cpu under gloo)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, solves_per_rank: int, t_max_ms: float) -> float:
    """Whole-job solves/s: every rank's solves over the slowest rank's time."""
    return world * solves_per_rank / (t_max_ms / 1e3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


def workload_spec(name: str):
    from workloads import WORKLOADS
    return WORKLOADS[name]


def build_inputs(name: str):
    """Seeded synthetic operator and right-hand side (numpy, host)."""
    from workloads.configs import quad_scale
    wl = workload_spec(name)
    A = wl.operator()
    b = wl.rhs(A.n)
    return wl, A, b


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
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
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def cpu_baseline_sample(name: str, budget_s: float = 20.0, sketch: str = "sparse_sign"):
    """The oracle, as it stands, on a bounded sample of the workload: the
    first j_s Arnoldi steps at full N (scaled to m linearly) and both tails
    (sFOM by quadrature, sGMRES) on the j_s-column sample, scaled by (m/j_s)^2
    for their O(s m^2) dense work."""
    import numpy as np
    from oracle import sketched as osk
    from oracle.arnoldi import arnoldi_trunc
    from oracle.sketch import Sketch
    from workloads import csr_to_scipy
    from workloads.configs import quad_scale
    wl, A, b = build_inputs(name)
    As = csr_to_scipy(A.astype(np.float64))
    S = Sketch(sketch, A.n, wl.s, wl.zeta, 13)
    c = quad_scale(wl.func, wl.lam_lo or 0.0, float(abs(As).sum(1).max()))
    t0 = time.perf_counter()
    ar = arnoldi_trunc(As, b, 2, wl.k, S)
    per_step_probe = (time.perf_counter() - t0) / 2
    js = int(max(4, min(wl.m, (0.6 * budget_s) // max(per_step_probe, 1e-6))))
    t0 = time.perf_counter()
    ar = arnoldi_trunc(As, b, js, wl.k, S)
    t_arn = time.perf_counter() - t0
    W = osk.whiten(ar["SV"], ar["SAV"], S @ b)
    t0 = time.perf_counter()
    ell = wl.extra.get("ell")
    osk.sgmres_quadrature(W, wl.func, c, ell=ell, tol=1e-10)
    osk.sfom_quadrature(W, wl.func, c, ell=ell, tol=1e-10)
    t_tail = time.perf_counter() - t0
    per_pair = t_arn * (wl.m / js) * 2 + t_tail * (wl.m / js) ** 2
    cores = len(os.sched_getaffinity(0))
    return {"value": 2.0 / per_pair, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{js} of {wl.m} Arnoldi steps at full N (x{wl.m / js:.1f}, twice: one basis per method) + "
                      f"sFOM/sGMRES tails on the {js}-column sample (x{(wl.m / js) ** 2:.0f}); "
                      f"BLAS threads {os.environ.get('OMP_NUM_THREADS', 'default')}, SciPy CSR matvec single-threaded",
            "seconds": round(t_arn + t_tail, 2)}


def oracle_pair(name: str, sketch: str = "sparse_sign", m: int | None = None):
    """One sFOM + sGMRES pair of the workload by the oracle as it stands, on the
    full operator: one truncated Arnoldi process (the basis both methods
    use), both tails (adaptive quadrature, tol 1e-10) and both
    recombinations; m < wl.m gives a bounded prefix (the warm-up)."""
    import numpy as np
    from oracle import sketched as osk
    from oracle.arnoldi import arnoldi_trunc
    from oracle.sketch import Sketch
    from workloads import csr_to_scipy
    from workloads.configs import quad_scale
    wl, A, b = build_inputs(name)
    As = csr_to_scipy(A.astype(np.float64))
    S = Sketch(sketch, A.n, wl.s, wl.zeta, 13)
    c = quad_scale(wl.func, wl.lam_lo or 0.0, float(abs(As).sum(1).max()))
    mm = m or wl.m
    ell = wl.extra.get("ell")
    t0 = time.perf_counter()
    ar = arnoldi_trunc(As, b, mm, wl.k, S)
    W = osk.whiten(ar["SV"], ar["SAV"], S @ b)
    yg, _ = osk.sgmres_quadrature(W, wl.func, c, ell=ell, tol=1e-10)
    yf, _ = osk.sfom_quadrature(W, wl.func, c, ell=ell, tol=1e-10)
    xg, xf = ar["V"] @ yg, ar["V"] @ yf
    return time.perf_counter() - t0, wl, A


def run_reference(args, rank: int):
    """The oracle as it stands on the host cores, rank 0 only.  Each timed
    step is one whole pair of the workload (nothing extrapolated): one
    Arnoldi process shared by the two methods, both tails, both
    recombinations.  Warm-up steps run a short prefix (untimed)."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_pair(args.workload, args.sketch, m=4)
    times = []
    for _ in range(args.steps):
        dt, wl, A = oracle_pair(args.workload, args.sketch)
        times.append(dt)
    total = sum(times)
    value = 2.0 * args.steps / total
    cores = len(os.sched_getaffinity(0))
    sample = (f"whole sFOM + sGMRES pairs on the full workload (N = {A.n}, m = {wl.m}): one truncated Arnoldi "
              f"process shared by both methods, both tails, both recombinations; BLAS threads "
              f"{os.environ.get('OMP_NUM_THREADS', 'default')}, SciPy CSR matvec single-threaded")
    line = {"metric": "f(A)b solves/s (sFOM + sGMRES, FP64)", "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "N": int(A.n), "nnz": int(A.nnz), "m": wl.m, "k": wl.k,
                       "s": wl.s, "zeta": wl.zeta, "sketch": args.sketch, "f": wl.func},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "timed_s": round(total, 1)}
    print(json.dumps(line), flush=True)


def run_block(args, wl, A, op, dev, rank):
    """skf_solve_block in its lockstep SpMM form (nrhs right-hand sides, one
    operator and sketch) against nrhs skf_solve calls on the same inputs:
    CUDA events, median of the steps, L2 flushed; the results must be
    bit-identical."""
    import numpy as np
    import torch
    import paper_2208_11447_gb300 as skf
    from workloads.configs import quad_scale
    m = args.m or wl.m
    bdt = basis_torch(args.basis)
    S = skf.Sketch(SKETCH_KIND[args.sketch](skf), A.n, wl.s, wl.zeta, 13)
    f = skf.make_func(wl.func, quad_scale(wl.func, wl.lam_lo or 0.0, op.csr.norm_inf()))
    p = skf.make_params(m, wl.k, basis_dtype=bdt, tol=1e-10)
    B = torch.as_tensor(np.stack([wl.rhs(A.n) * (1.0 + 0.1 * q) + 1e-3 * q for q in range(args.nrhs)]),
                        device=dev).contiguous()
    Xb, Xs = torch.empty_like(B), torch.empty_like(B)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def block():
        with skf.block_mode(1):   # the lockstep SpMM form
            skf.solve_block(skf.SGMRES, op.csr, S, B, f, p, X=Xb)

    def singles():
        # the Arnoldi form of the lockstep columns (two-kernel), for a like comparison
        with skf.arnoldi_mode(skf.ARNOLDI_TWO_KERNEL):
            for q in range(args.nrhs):
                skf.solve(skf.SGMRES, op.csr, S, B[q], f, p, x=Xs[q])

    res = {"mode": "block", "workload": args.workload, "basis": args.basis, "m": m, "nrhs": args.nrhs}
    for name, fn in (("block", block), ("singles", singles)):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            ev0.record()
            fn()
            ev1.record()
            ev1.synchronize()
            ts.append(ev0.elapsed_time(ev1))
        res[name + "_ms"] = round(statistics.median(ts), 3)
    res["speedup"] = round(res["singles_ms"] / res["block_ms"], 3)
    res["bitwise_equal"] = bool(torch.equal(Xb, Xs))
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_arnoldi_only(args, wl, A, b, op, dev, rank, world):
    """Time skf_arnoldi_trunc alone (m steps of the two step kernels)."""
    import torch
    import paper_2208_11447_gb300 as skf
    m = args.m or wl.m
    bdt = basis_torch(args.basis)
    S = skf.Sketch(SKETCH_KIND[args.sketch](skf), A.n, wl.s, wl.zeta, 13)
    b_dev = torch.as_tensor(b, device=dev)
    for _ in range(args.warmup):
        skf.arnoldi_trunc(op.csr, S, b_dev, m, wl.k, basis_dtype=bdt)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(args.steps):
        ev0.record()
        skf.arnoldi_trunc(op.csr, S, b_dev, m, wl.k, basis_dtype=bdt)
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    if rank == 0:
        us = statistics.median(times) * 1e3 / m
        print(json.dumps({"mode": "arnoldi", "workload": args.workload, "basis": args.basis, "m": m,
                          "us_per_step": round(us, 2)}), flush=True)



# ----------------------------------------------------------------- batched workload
BATCH_TOL = 1e-6          # error gate of a batched FP32-basis solve against the FP64 one
BATCH_FUNC = "invsqrt"


def batch_inputs(n_rhs: int):
    """Host inputs of the batched workload: the seeded layout, its operators
    (FP32-rounded values), quadrature scales and right-hand sides."""
    from workloads.batch import batch_layout, quad_scale_invsqrt
    layout = batch_layout(n_rhs=n_rhs)
    ops = []
    for M in layout.mats:
        A = M.operator()
        ops.append((A, quad_scale_invsqrt(A, M.lam_lo())))
    rhs = [r.rhs(layout.mats[r.mat].N) for r in layout.rhs]
    return layout, ops, rhs


def cpu_batch_sample(layout, ops, rhs, budget_s: float = 20.0):
    """The oracle, as it stands, on a bounded sample of the batched workload:
    a few Arnoldi steps of one right-hand side on each operator (per-step
    time per operator), and the sGMRES tail on a j_t-column basis of the
    smallest operator (its cost depends on m and s = 4m only); scaled to the
    batch as sum_r (m_r t_step(A_r) + (m_r / j_t)^3 t_tail)."""
    import numpy as np
    from oracle import sketched as osk
    from oracle.arnoldi import arnoldi_trunc
    from oracle.sketch import Sketch
    from workloads import csr_to_scipy
    per_op = max(0.5, 0.5 * budget_s / len(ops))
    t_step = []
    spent = 0.0
    for i, (A, c) in enumerate(ops):
        r = next(j for j, q in enumerate(layout.rhs) if q.mat == i)
        q = layout.rhs[r]
        As = csr_to_scipy(A.astype(np.float64))
        S = Sketch("sparse_sign", A.n, q.s, 8, q.sketch_seed)
        t0 = time.perf_counter()
        arnoldi_trunc(As, rhs[r], 2, 2, S)
        probe = (time.perf_counter() - t0) / 2
        js = int(max(2, min(q.m, per_op // max(probe, 1e-6))))
        t0 = time.perf_counter()
        arnoldi_trunc(As, rhs[r], js, 2, S)
        dt = time.perf_counter() - t0
        spent += dt
        t_step.append(dt / js)
    i0 = min(range(len(ops)), key=lambda i: ops[i][0].n)
    A, c = ops[i0]
    r = next(j for j, q in enumerate(layout.rhs) if q.mat == i0)
    jt = 48
    As = csr_to_scipy(A.astype(np.float64))
    S = Sketch("sparse_sign", A.n, 4 * jt, 8, layout.rhs[r].sketch_seed)
    ar = arnoldi_trunc(As, rhs[r], jt, 2, S)
    W = osk.whiten(ar["SV"], ar["SAV"], S @ rhs[r])
    t0 = time.perf_counter()
    osk.sgmres_quadrature(W, BATCH_FUNC, c, tol=1e-10)
    t_tail = time.perf_counter() - t0
    spent += t_tail
    total = sum(q.m * t_step[q.mat] + (q.m / jt) ** 3 * t_tail for q in layout.rhs)
    return {"value": len(layout.rhs) / total, "unit": "solves/s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle",
            "sample": f"per operator a few Arnoldi steps of one right-hand side at full N (per-step time x m_r "
                      f"for each of its right-hand sides) + one sGMRES tail on a {jt}-column basis, s = {4 * jt} "
                      f"(x (m_r/{jt})^3); SciPy CSR matvec single-threaded",
            "seconds": round(spent, 2)}


def run_reference_batch(args, rank: int):
    if rank != 0:
        return
    layout, ops, rhs = batch_inputs(args.batch_rhs)
    for _ in range(args.warmup):
        cpu_batch_sample(layout, ops, rhs, budget_s=1.0)
    budget = min(args.ref_budget, 150.0 / max(1, args.steps))
    vals = [cpu_batch_sample(layout, ops, rhs, budget_s=budget) for _ in range(args.steps)]
    value = statistics.mean(v["value"] for v in vals)
    cb = vals[-1]
    print(json.dumps({
        "metric": "f(A)b solves/s at rel err <= 1e-6 (batched sGMRES)", "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": len(layout.rhs) * 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "batch_cd_8x64", **layout.summary()},
        "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def batch_arms(dev, steps: int, warmup: int, lanes_arg, world: int = 1, n_rhs: int = 64, with_e2e: bool = False,
               clocks=None):
    """The batched workload's arms, all through the public API on the same
    operators, sketches, right-hand sides and rules:
      * FP64 basis, one problem at a time (skf_sgmres per problem);
      * FP64 basis as one batch (skf_solve_batched captured into one CUDA
        graph, replayed once per step): bit-identical to the one-at-a-time
        results (error 0 <= 1e-6);
      * FP32 basis as one batch: its error against the FP64 results per
        problem, and how well the solve's own flag (nodes needing the FP64
        factor) predicts a miss of 1e-6.
    Returns the timings (ms, summed over steps) and per-problem errors."""
    import numpy as np
    import torch
    import paper_2208_11447_gb300 as skf

    layout, ops, rhs = batch_inputs(n_rhs)
    nprob = len(layout.rhs)
    op32, op64 = [], []
    for A, c in ops:
        op32.append(skf.upload_csr(A.rowptr, A.colind, A.values, device=dev))
        op64.append(skf.upload_csr(A.rowptr, A.colind, A.values.astype(np.float64), device=dev))
    sketches, funcs, b_dev = [], [], []
    for q, b in zip(layout.rhs, rhs):
        sketches.append(skf.Sketch(skf.SPARSE_SIGN, layout.mats[q.mat].N, q.s, 8, q.sketch_seed))
        funcs.append(skf.make_func(BATCH_FUNC, ops[q.mat][1]))
        b_dev.append(torch.as_tensor(b, device=dev))
    p32 = [skf.make_params(q.m, 2, basis_dtype=torch.float32, tol=1e-10) for q in layout.rhs]
    p64 = [skf.make_params(q.m, 2, basis_dtype=torch.float64, tol=1e-10) for q in layout.rhs]
    info_sz = ctypes.sizeof(skf.Info)
    x64 = [torch.empty_like(b) for b in b_dev]
    x64b = [torch.empty_like(b) for b in b_dev]
    x32 = [torch.empty_like(b) for b in b_dev]
    inf64 = torch.zeros((nprob, info_sz), dtype=torch.uint8, device=dev)
    inf64b = torch.zeros_like(inf64)
    inf32 = torch.zeros_like(inf64)
    probs64 = [(skf.SGMRES, op64[q.mat].csr, sketches[r], b_dev[r], funcs[r], p64[r], x64b[r], inf64b[r])
               for r, q in enumerate(layout.rhs)]
    probs32 = [(skf.SGMRES, op32[q.mat].csr, sketches[r], b_dev[r], funcs[r], p32[r], x32[r], inf32[r])
               for r, q in enumerate(layout.rhs)]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def fp64_one_at_a_time():
        for r, q in enumerate(layout.rhs):
            skf.sgmres(op64[q.mat].csr, sketches[r], b_dev[r], funcs[r], p64[r], x=x64[r], info=inf64[r])

    def timed(fn, k):
        tot = 0.0
        for _ in range(k):
            flush.zero_()
            ev0.record(stream)
            fn()
            ev1.record(stream)
            ev1.synchronize()
            tot += ev0.elapsed_time(ev1)
        return tot

    def statuses(buf):
        return sorted({skf.read_info(buf[r])["status_name"] for r in range(nprob)})

    out = {"layout": layout, "ops": ops, "rhs": rhs, "nprob": nprob}
    # plain FP64 path, one problem at a time
    for _ in range(warmup):
        fp64_one_at_a_time()
    torch.cuda.synchronize()
    replica_barrier(world)
    out["t64"] = replica_max(timed(fp64_one_at_a_time, steps), world, dev)
    out["status64"] = statuses(inf64)
    # FP64 batch as one CUDA graph
    lane_times = None
    if lanes_arg == "auto":
        graph64, lane_times = skf.BatchGraph.autotune(probs64)
        lanes = graph64.lanes
        del graph64
    else:
        lanes = int(lanes_arg)
    l0 = skf.kernel_launch_count()
    graph64 = skf.BatchGraph(probs64, lanes=lanes)          # one eager run + capture
    out["launches_per_batch"] = (skf.kernel_launch_count() - l0) // 2
    for _ in range(warmup):
        graph64.replay()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    replica_barrier(world)
    torch.cuda.synchronize()
    out["t64b"] = replica_max(timed(graph64.replay, steps), world, dev)
    replica_barrier(world)
    if clocks is not None:
        out["clk"] = clocks.stop()
    out["equal64"] = all(bool(torch.equal(a, b)) for a, b in zip(x64b, x64))
    out["errs64b"] = [float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(x64b, x64)]
    out["status64b"] = statuses(inf64b)
    out["lanes"], out["lane_times"] = lanes, lane_times
    if with_e2e:
        # right-hand sides from pinned host memory, results back
        b_host = [torch.as_tensor(b).pin_memory() for b in rhs]
        x_host = [torch.empty(b.numel(), dtype=torch.float64).pin_memory() for b in b_dev]
        e2e_ms = 0.0
        replica_barrier(world)
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for bd, bh in zip(b_dev, b_host):
                bd.copy_(bh, non_blocking=True)
            graph64.replay()
            for xh, xd in zip(x_host, x64b):
                xh.copy_(xd, non_blocking=True)
            torch.cuda.synchronize()
            e2e_ms += (time.perf_counter() - t0) * 1e3
        out["e2e_ms"] = replica_max(e2e_ms, world, dev)
    del graph64
    # FP32-basis batch as one CUDA graph
    graph32 = skf.BatchGraph(probs32, lanes=lanes)
    for _ in range(warmup):
        graph32.replay()
    torch.cuda.synchronize()
    replica_barrier(world)
    out["t32"] = replica_max(timed(graph32.replay, steps), world, dev)
    del graph32
    out["errs32"] = [float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(x32, x64)]
    out["flags32"] = [skf.read_info(inf32[r])["nodes_fp64"] > 0 for r in range(nprob)]
    out["status32"] = statuses(inf32)
    # mixed precision: the library's plan (one pilot Arnoldi process per
    # operator) picks an FP32 basis where cond(R) 2^-24 <= 1e-6, FP64 elsewhere
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cond, use32 = skf.plan_basis_precision(probs32, BATCH_TOL)
    out["plan_ms"] = (time.perf_counter() - t0) * 1e3
    xmx = [torch.empty_like(b) for b in b_dev]
    infmx = torch.zeros_like(inf64)
    probsmx = [(skf.SGMRES, (op32 if use32[r] else op64)[q.mat].csr, sketches[r], b_dev[r], funcs[r],
                (p32 if use32[r] else p64)[r], xmx[r], infmx[r]) for r, q in enumerate(layout.rhs)]
    graphmx = skf.BatchGraph(probsmx, lanes=lanes)
    for _ in range(warmup):
        graphmx.replay()
    torch.cuda.synchronize()
    replica_barrier(world)
    out["tmx"] = replica_max(timed(graphmx.replay, steps), world, dev)
    del graphmx
    out["errsmx"] = [float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) for a, b in zip(xmx, x64)]
    out["usemx"] = use32
    out["condmx"] = cond
    out["statusmx"] = statuses(infmx)
    return out


def batch_summary(o, steps: int, world: int = 1):
    """The three arms as JSON-ready numbers (solves/s, errors against the FP64
    one-at-a-time results, counts within the 1e-6 gate)."""
    nprob, tol = o["nprob"], BATCH_TOL
    v64b = replica_value(world, nprob * steps, o["t64b"])
    v64 = replica_value(world, nprob * steps, o["t64"])
    v32 = replica_value(world, nprob * steps, o["t32"])
    vmx = replica_value(world, nprob * steps, o["tmx"])
    errs, flags = o["errs32"], o["flags32"]
    return {
        "fp64_one_at_a_time": {"value": round(v64, 3), "unit": "solves/s",
                               "ms_per_batch": round(o["t64"] / steps, 3), "status": o["status64"]},
        "fp64_batched": {"value": round(v64b, 3), "unit": "solves/s", "ms_per_batch": round(o["t64b"] / steps, 3),
                         "speedup_vs_fp64_one_at_a_time": round(v64b / v64, 3),
                         "max_rel_err": max(o["errs64b"]), "bitwise_equal": o["equal64"],
                         "within_1e-6": sum(1 for e in o["errs64b"] if e <= tol), "of": nprob,
                         "status": o["status64b"], "lanes": o["lanes"]},
        "fp32_batched": {"value": round(v32, 3), "unit": "solves/s", "ms_per_batch": round(o["t32"] / steps, 3),
                         "speedup_vs_fp64_one_at_a_time": round(v32 / v64, 3),
                         "max_rel_err": max(errs), "median_rel_err": statistics.median(errs),
                         "within_1e-6": sum(1 for e in errs if e <= tol), "of": nprob, "status": o["status32"],
                         "flag_nodes_fp64": {
                             "flagged_err_gt_tol": sum(1 for f, e in zip(flags, errs) if f and e > tol),
                             "flagged_err_le_tol": sum(1 for f, e in zip(flags, errs) if f and e <= tol),
                             "unflagged_err_gt_tol": sum(1 for f, e in zip(flags, errs) if not f and e > tol),
                             "unflagged_err_le_tol": sum(1 for f, e in zip(flags, errs) if not f and e <= tol)}},
        "mixed_batched": {"value": round(vmx, 3), "unit": "solves/s", "ms_per_batch": round(o["tmx"] / steps, 3),
                          "speedup_vs_fp64_one_at_a_time": round(vmx / v64, 3),
                          "speedup_vs_fp64_batched": round(vmx / v64b, 3),
                          "fp32_problems": sum(1 for u in o["usemx"] if u), "of": nprob,
                          "max_rel_err": max(o["errsmx"]), "within_1e-6": sum(1 for e in o["errsmx"] if e <= tol),
                          "max_rel_err_fp32_problems": max([e for e, u in zip(o["errsmx"], o["usemx"]) if u],
                                                           default=0.0),
                          "status": o["statusmx"], "plan_ms": round(o["plan_ms"], 1),
                          "policy": "skf_plan_basis_precision: FP32 basis where cond(R) 2^-24 <= 1e-6 (cond(R) "
                                    "of the whitening of a pilot basis, one pilot Arnoldi process per operator), "
                                    "FP64 elsewhere; planned once outside the timed region"},
        "errors_vs": "FP64 one-at-a-time GPU path, same problems; gate 1e-6",
    }


def run_batch(args, rank, world, local, dev):
    """Batched workload (bench.py --mode batch): the FP64 batch is the
    headline (the fastest arm that meets 1e-6 on every problem)."""
    clocks = ClockSampler(local)
    o = batch_arms(dev, args.steps, args.warmup, args.lanes, world, args.batch_rhs, with_e2e=True, clocks=clocks)
    layout, ops, rhs, nprob = o["layout"], o["ops"], o["rhs"], o["nprob"]
    summ = batch_summary(o, args.steps, world)
    value = replica_value(world, nprob * args.steps, o["t64b"])
    e2e_value = replica_value(world, nprob * args.steps, o["e2e_ms"])
    # whole-batch effective bandwidth over the algorithmic Arnoldi bytes (FP64)
    alg = 0
    for q in layout.rhs:
        A = ops[q.mat][0]
        alg += q.m * (A.nnz * 12 + 4 * (A.n + 1) + 3 * A.n * 8)
    hbm_peak, hbm_src = measured_peaks()
    gbs = alg / (o["t64b"] / args.steps * 1e-3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_batch_sample(layout, ops, rhs, budget_s=args.ref_budget)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    clk = o["clk"]
    if rank == 0:
        nbytes_b = int(sum(b.nbytes for b in rhs))
        print(json.dumps({
            "metric": "f(A)b solves/s at rel err <= 1e-6 (batched sGMRES)",
            "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(o["t64b"] / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch_cd_8x64", **layout.summary(), "k": 2, "s": "4 m_r", "zeta": 8,
                       "f": BATCH_FUNC, "method": "sgmres", "quad_tol": 1e-10, "basis": "f64", "values": "f32-rounded",
                       "lanes": o["lanes"], "lane_autotune_ms": o["lane_times"], "graph": "one CUDA graph per batch",
                       "parallelism": f"replicas x{world}", "l2": "flushed between steps"},
            "accuracy": {"vs": "FP64 one-at-a-time GPU path, same problems",
                         "max_rel_err": summ["fp64_batched"]["max_rel_err"],
                         "bitwise_equal": o["equal64"], "within_1e-6": summ["fp64_batched"]["within_1e-6"],
                         "of": nprob, "status": o["status64b"]},
            "fp64_one_at_a_time": summ["fp64_one_at_a_time"],
            "speedup_vs_fp64_one_at_a_time": summ["fp64_batched"]["speedup_vs_fp64_one_at_a_time"],
            "fp32_batched": summ["fp32_batched"],
            "mixed_batched": summ["mixed_batched"],
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(gbs / hbm_peak, 4), "traffic": None, "peak_source": hbm_src,
                         "kernel": "whole FP64 batch: algorithmic Arnoldi bytes (sum_r m_r (B_A + 3 N 8)) over the "
                                   "batch time, tails included"},
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 3), "unit": "solves/s", "h2d_bytes_per_step": nbytes_b,
                    "d2h_bytes_per_step": nbytes_b},
            "gpu_launches": int(o["launches_per_batch"] * args.steps),
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
        }), flush=True)


def precision_extras(dev, reps: int = 3):
    """The reduced-precision workload (3D n = 256, N = 16.8M, m = 120,
    z^-1/2): per basis type (FP32, BF16) the truncated-Arnoldi step time
    (CUDA events around skf_arnoldi_trunc, median of reps, L2 flushed), its
    fraction of the measured HBM copy rate for the algorithmic bytes, and the
    relative error of both solves against the FP64 GPU path on the same
    operator (values widened exactly), sketch and rule."""
    import numpy as np
    import torch
    import paper_2208_11447_gb300 as skf
    from workloads.configs import quad_scale
    wl, A, b = build_inputs("cd3d_n256_fp32")
    A32 = A.astype(np.float32)
    op32 = skf.upload_csr(A32.rowptr, A32.colind, A32.values, device=dev)
    S = skf.Sketch(skf.SPARSE_SIGN, A.n, wl.s, wl.zeta, 13)
    c = quad_scale(wl.func, wl.lam_lo or 0.0, op32.csr.norm_inf())
    f = skf.make_func(wl.func, c)
    b_dev = torch.as_tensor(b, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hbm_peak, hbm_src = measured_peaks()
    res = {"workload": "cd3d_n256 (N = 16,777,216, nnz = 117,047,296, m = 120, k = 2, s = 480, zeta = 8, z^-1/2)"}
    xs = {}
    for name, bdt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        ts = []
        for r in range(reps + 1):
            flush.zero_()
            ev0.record(stream)
            skf.arnoldi_trunc(op32.csr, S, b_dev, wl.m, wl.k, basis_dtype=bdt)
            ev1.record(stream)
            ev1.synchronize()
            if r > 0:
                ts.append(ev0.elapsed_time(ev1))
        us = statistics.median(ts) * 1e3 / wl.m
        alg = A.nnz * 8 + 4 * (A.n + 1) + (wl.k + 1) * A.n * BASIS_BYTES[name]
        p = skf.make_params(wl.m, wl.k, basis_dtype=bdt, tol=1e-10)
        xs[name] = (skf.sfom(op32.csr, S, b_dev, f, p), skf.sgmres(op32.csr, S, b_dev, f, p))
        res[name] = {"us_per_step": round(us, 2), "alg_bytes_per_step": int(alg),
                     "hbm_frac": round(alg / (us * 1e-6) / 1e9 / hbm_peak, 4), "of": hbm_src,
                     # ncu DRAM bytes of the two step kernels per step (one capture of the
                     # current kernels); FP32 basis only
                     "traffic": FP32_STEP_TRAFFIC if name == "f32" else None}
    torch.cuda.synchronize()
    del op32
    op64 = skf.upload_csr(A.rowptr, A.colind, A.values.astype(np.float64), device=dev)
    p64 = skf.make_params(wl.m, wl.k, tol=1e-10)
    r_f = skf.sfom(op64.csr, S, b_dev, f, p64)
    r_g = skf.sgmres(op64.csr, S, b_dev, f, p64)
    torch.cuda.synchronize()
    for name in ("f32", "bf16"):
        xf, xg = xs[name]
        res[name]["rel_err_vs_fp64_gpu"] = {
            "sfom": float(torch.linalg.vector_norm(xf - r_f) / torch.linalg.vector_norm(r_f)),
            "sgmres": float(torch.linalg.vector_norm(xg - r_g) / torch.linalg.vector_norm(r_g))}
    del op64, xs, r_f, r_g
    torch.cuda.empty_cache()
    return res


def sketch_extras(dev, op, A, b_dev, wl, m: int = 12, reps: int = 3):
    """Truncated-Arnoldi step of the default operator (FP64 basis, the
    two-kernel form) with each sketch kind: sparse-sign, SRHT and the
    paper's SRDCT (N = 1e6 = 2^6 5^6: the FFT form of the DCT-II).  CUDA
    events around skf_arnoldi_trunc over m steps, median of reps, L2
    flushed; sparse-sign in the two-kernel form for a like comparison."""
    import torch
    import paper_2208_11447_gb300 as skf
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    with skf.arnoldi_mode(skf.ARNOLDI_TWO_KERNEL):
        for kind in ("sparse_sign", "srht", "srdct"):
            S = skf.Sketch(SKETCH_KIND[kind](skf), A.n, wl.s, wl.zeta if kind == "sparse_sign" else 0, 13)
            ts = []
            for r in range(reps + 1):
                flush.zero_()
                ev0.record(stream)
                skf.arnoldi_trunc(op.csr, S, b_dev, m, wl.k)
                ev1.record(stream)
                ev1.synchronize()
                if r > 0:
                    ts.append(ev0.elapsed_time(ev1))
            out[kind] = {"us_per_step": round(statistics.median(ts) * 1e3 / m, 2)}
            del S
    out["workload"] = f"cd3d_n100 (N = 1e6), FP64 basis, k = {wl.k}, s = {wl.s}, m = {m}, two-kernel Arnoldi form"
    return out


def graph_extras(dev, reps: int = 2):
    """The quadrature-batched graph workloads (N = 4e6 directed power-law
    graph, FP32 values and basis, m = 150, k = 3, s = 600, 128 fixed
    Gauss-Jacobi nodes of z^-1/2): rows carrying in-degrees (graph_n4m) and
    rows carrying the power-law out-degrees (graph_n4m_t, row split).  Per
    workload the FP32 truncated-Arnoldi step (CUDA events around
    skf_arnoldi_trunc, median of reps, L2 flushed), its fraction of the
    measured HBM copy rate for the algorithmic bytes, and the relative error
    of the FP32 sGMRES solve against the FP64 GPU path on the same operator
    (values widened exactly), sketch and rule.  The slice layout is chosen
    first by skf_csr_autotune (its per-candidate step times are reported)."""
    import numpy as np
    import torch
    import paper_2208_11447_gb300 as skf
    from workloads.configs import quad_scale
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hbm_peak, hbm_src = measured_peaks()
    res = {}
    for name in ("graph_n4m", "graph_n4m_t"):
        wl, A, b = build_inputs(name)
        L = np.diff(A.rowptr)
        A32 = A.astype(np.float32)
        op32 = skf.upload_csr(A32.rowptr, A32.colind, A32.values, device=dev)
        S = skf.Sketch(skf.SPARSE_SIGN, A.n, wl.s, wl.zeta, 13)
        c = quad_scale(wl.func, wl.lam_lo or 0.0, op32.csr.norm_inf())
        t_nodes, w_nodes = skf.quadrature_rule(skf.make_func(wl.func, c), int(wl.extra["ell"]))
        f = skf.make_func(wl.func, c, nodes=t_nodes, weights=w_nodes)
        b_dev = torch.as_tensor(b, device=dev)
        tune = skf.csr_autotune(op32.csr, S, wl.k, basis_dtype=torch.float32, m_probe=6)   # the slice layout
        ts = []
        for r in range(reps + 1):
            flush.zero_()
            ev0.record(stream)
            skf.arnoldi_trunc(op32.csr, S, b_dev, wl.m, wl.k, basis_dtype=torch.float32)
            ev1.record(stream)
            ev1.synchronize()
            if r > 0:
                ts.append(ev0.elapsed_time(ev1))
        us = statistics.median(ts) * 1e3 / wl.m
        alg = A.nnz * 8 + 4 * (A.n + 1) + (wl.k + 1) * A.n * 4
        i32 = skf.new_info(dev)
        x32 = skf.sgmres(op32.csr, S, b_dev, f, skf.make_params(wl.m, wl.k, basis_dtype=torch.float32, tol=1e-10),
                         info=i32)
        torch.cuda.synchronize()
        del op32
        op64 = skf.upload_csr(A.rowptr, A.colind, A.values.astype(np.float64), device=dev)
        i64 = skf.new_info(dev)
        x64 = skf.sgmres(op64.csr, S, b_dev, f, skf.make_params(wl.m, wl.k, tol=1e-10), info=i64)
        torch.cuda.synchronize()
        cond64 = skf.read_info(i64)["cond_est"]
        err = float(torch.linalg.vector_norm(x32 - x64) / torch.linalg.vector_norm(x64))
        res[name] = {"rows": "power-law out-degrees (row split)" if name.endswith("_t") else "in-degrees",
                     "N": int(A.n), "nnz": int(A.nnz), "max_row": int(L.max()), "rows_over_32": int((L > 32).sum()),
                     "layout": tune["choice"], "layout_us_per_step": [round(x, 1) for x in tune["times_us"]],
                     "us_per_step": round(us, 2), "alg_bytes_per_step": int(alg),
                     "hbm_frac": round(alg / (us * 1e-6) / 1e9 / hbm_peak, 4), "of": hbm_src,
                     "rel_err_vs_fp64_gpu": err, "cond_R_fp64": cond64,
                     "tolerance": {"rule": "max(1e-6, 2^-24 cond(R)) (FP32 basis against FP64, cond(R) of the "
                                           "FP64 whitening)", "value": max(1e-6, 2.0 ** -24 * cond64),
                                   "met": err <= max(1e-6, 2.0 ** -24 * cond64)}}
        del op64, x32, x64, S
        torch.cuda.empty_cache()
    res["workload"] = "graph N = 4e6, FP32 values and basis, m = 150, k = 3, s = 600, 128 nodes, sGMRES z^-1/2"
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="cd3d_n100")
    ap.add_argument("--impl", default="skf", choices=["skf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--arnoldi-reps", type=int, default=5)
    ap.add_argument("--arnoldi-form", default="auto", choices=["auto", "persistent", "two_kernel"],
                    help="form of the FP64 Arnoldi process (skf_set_arnoldi_mode)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra keys of the default line (reduced-precision workload, batch arms)")
    ap.add_argument("--nrhs", type=int, default=4, help="right-hand sides of the block (block mode)")
    ap.add_argument("--mode", default="solve", choices=["solve", "arnoldi", "batch", "block"],
                    help="arnoldi: time only skf_arnoldi_trunc (the dominant kernels), e.g. under ncu; "
                         "batch: the batched workload (8 operators, 64 right-hand sides) as one CUDA graph")
    ap.add_argument("--lanes", default="auto",
                    help="concurrent streams of the batched solve (batch mode): a count, or auto (timed choice of 4/8/16)")
    ap.add_argument("--separate", action="store_true",
                    help="time each pair as two independent solves (skf_sfom + skf_sgmres, two Arnoldi processes) "
                         "instead of skf_sfom_sgmres")
    ap.add_argument("--two-pass", action="store_true",
                    help="two-pass truncated Arnoldi (Sec. 4.2): basis ring of k + 2 vectors, twice the SpMVs")
    ap.add_argument("--batch-rhs", type=int, default=64, help="right-hand sides of the batched workload")
    ap.add_argument("--m", type=int, default=None, help="override the Krylov dimension (arnoldi mode)")
    ap.add_argument("--sketch", default="sparse_sign", choices=["sparse_sign", "srht"],
                    help="subspace embedding: sparse-sign (zeta nonzeros per column) or SRHT")
    ap.add_argument("--basis", default=None, choices=["f64", "f32", "bf16"],
                    help="basis storage (default: the workload's); f32/bf16 need an FP32 operator")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.mode == "batch":
            run_reference_batch(args, rank)
        else:
            run_reference(args, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2208_11447_gb300 as skf
    from workloads.configs import quad_scale

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    skf.set_arnoldi_mode({"auto": skf.ARNOLDI_AUTO, "persistent": skf.ARNOLDI_PERSISTENT,
                          "two_kernel": skf.ARNOLDI_TWO_KERNEL}[args.arnoldi_form])

    def barrier():
        replica_barrier(world)

    def max_over_ranks(v: float) -> float:
        return replica_max(v, world, dev)

    if args.mode == "batch":
        run_batch(args, rank, world, local, dev)
        if world > 1:
            dist.destroy_process_group()
        return

    wl, A, b = build_inputs(args.workload)
    basis = args.basis or wl.basis_dtype
    if basis != "f64" and A.values.dtype != np.float32:
        A = A.astype(np.float32)
    if basis == "f64" and A.values.dtype != np.float64:
        A = A.astype(np.float64)
    args.basis = basis
    bdt = basis_torch(basis)
    op = skf.upload_csr(A.rowptr, A.colind, A.values, device=dev)
    if args.mode == "arnoldi":
        run_arnoldi_only(args, wl, A, b, op, dev, rank, world)
        return
    if args.mode == "block":
        run_block(args, wl, A, op, dev, rank)
        return
    S = skf.Sketch(SKETCH_KIND[args.sketch](skf), A.n, wl.s, wl.zeta, 13)
    c = quad_scale(wl.func, wl.lam_lo or 0.0, op.csr.norm_inf())
    f = skf.make_func(wl.func, c)
    if wl.extra.get("ell"):
        # fixed rule: every node solved in one batch
        t_nodes, w_nodes = skf.quadrature_rule(f, int(wl.extra["ell"]))
        f = skf.make_func(wl.func, c, nodes=t_nodes, weights=w_nodes)
    p = skf.make_params(wl.m, wl.k, basis_dtype=bdt, tol=1e-10, two_pass=args.two_pass)
    b_dev = torch.as_tensor(b, device=dev)
    x_fom = torch.empty_like(b_dev)
    x_gm = torch.empty_like(b_dev)
    info_f = skf.new_info(dev)
    info_g = skf.new_info(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    # one pair = both approximants of f(A) b; they share one Arnoldi process
    # (skf_sfom_sgmres), as the reference arm's pair does, unless --separate
    # (or the two-pass mode, which the pair call does not offer)
    paired = not (args.separate or args.two_pass)

    def solve_pair(bv):
        if paired:
            skf.sfom_sgmres(op.csr, S, bv, f, p, x_fom=x_fom, x_gmres=x_gm, info_fom=info_f, info_gmres=info_g)
        else:
            skf.sfom(op.csr, S, bv, f, p, x=x_fom, info=info_f)
            skf.sgmres(op.csr, S, bv, f, p, x=x_gm, info=info_g)

    def step():
        solve_pair(b_dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st_f, st_g = skf.read_info(info_f), skf.read_info(info_g)
    accuracy = None
    if basis != "f64":
        accuracy = reference_error_fp64(skf, A, S, b_dev, f, wl, x_fom, x_gm, dev)

    # ---- timed region: device-resident inputs, L2 flushed between steps
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = skf.kernel_launch_count()
    total_ms = 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    barrier()
    launches = skf.kernel_launch_count() - launches0
    clk = clocks.stop()
    t_max = max_over_ranks(total_ms)
    value = replica_value(world, 2 * args.steps, t_max)

    # ---- dominant kernels: the truncated-Arnoldi step (spmv + update launches)
    V = torch.empty((wl.m, A.n), dtype=bdt, device=dev)
    vsc = torch.empty(wl.m, dtype=torch.float64, device=dev)
    SV = torch.empty((wl.m, wl.s), dtype=torch.float64, device=dev)
    SAV = torch.empty_like(SV)
    H = torch.empty((wl.m, wl.m + 1), dtype=torch.float64, device=dev)
    L = skf.lib()
    arn_ms = []
    for r in range(args.arnoldi_reps + 1):
        flush.zero_()
        ev0.record(stream)
        skf._check(L.skf_arnoldi_trunc(op.csr.handle, S.handle, skf._ptr(b_dev), skf.F64, wl.m, wl.k,
                                       skf._DTYPE[bdt],
                                       skf._ptr(V), A.n, skf._ptr(vsc), skf._ptr(SV), skf._ptr(SAV), skf._ptr(H),
                                       None, skf._stream(stream)))
        ev1.record(stream)
        ev1.synchronize()
        if r > 0:
            arn_ms.append(ev0.elapsed_time(ev1))
    step_us = statistics.median(arn_ms) * 1e3 / wl.m
    nnz, N, k = A.nnz, A.n, wl.k
    bv = 8 if A.values.dtype == np.float64 else 4
    bb = BASIS_BYTES[basis]
    alg_bytes = nnz * (bv + 4) + 4 * (N + 1) + (k + 1) * N * bb      # per step: A once, window, new vector
    alg_flops = 2 * nnz + (4 * k + 3) * N                             # SpMV + k dots + k axpys + norm + scale
    hbm_peak, hbm_src = measured_peaks()
    fp64_peak = skf.fp64_peak(stream)   # measured FMA throughput of this GPU (outside the timed region)
    achieved_gflops = alg_flops / (step_us * 1e-6) / 1e9
    achieved_gbs = alg_bytes / (step_us * 1e-6) / 1e9
    fp64_bound_us = alg_flops / (fp64_peak * 1e9) * 1e6
    hbm_bound_us = alg_bytes / (hbm_peak * 1e9) * 1e6
    if basis == "f64" and fp64_bound_us >= hbm_bound_us:
        roof = {"bound": "alu", "achieved": round(achieved_gflops, 1), "peak": round(fp64_peak, 1),
                "unit": "GFLOP/s", "frac": round(achieved_gflops / fp64_peak, 4), "traffic": None,
                "peak_source": "measured: skf_fp64_peak (independent FP64 FMA accumulations on every SM, this run)"}
    else:
        roof = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved_gbs / hbm_peak, 4), "traffic": None, "peak_source": hbm_src}
    persistent = basis == "f64" and args.sketch == "sparse_sign" and args.arnoldi_form != "two_kernel" and wl.k <= 4
    roof["traffic"] = NCU_TRAFFIC_PER_STEP.get((args.workload, basis, args.sketch, persistent))
    if persistent:
        kname = "k_arnoldi_persist: all m steps in one cooperative launch"
    else:
        kname = "k_arnoldi_spmv_pipe + k_arnoldi_update" if basis == "f64" else "k_arnoldi_spmv_lp + k_arnoldi_update_lp"
    if args.sketch == "srht":
        kname += " + k_srht_blocks"
    roof.update({"kernel": f"truncated-Arnoldi step ({kname})", "us_per_step": round(step_us, 2),
                 "alg_bytes_per_step": alg_bytes, "alg_flops_per_step": alg_flops,
                 "hbm": {"achieved": round(achieved_gbs, 1), "peak": hbm_peak,
                         "frac": round(achieved_gbs / hbm_peak, 4), "of": hbm_src}})

    # ---- end to end through the public API with host buffers
    b_host = torch.as_tensor(b).pin_memory()
    xf_host = torch.empty(A.n, dtype=torch.float64).pin_memory()
    xg_host = torch.empty(A.n, dtype=torch.float64).pin_memory()
    b_e2e = torch.empty_like(b_dev)
    e2e_ms = 0.0
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b_e2e.copy_(b_host, non_blocking=True)
        solve_pair(b_e2e)
        xf_host.copy_(x_fom, non_blocking=True)
        xg_host.copy_(x_gm, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_max = max_over_ranks(e2e_ms)
    e2e_value = replica_value(world, 2 * args.steps, e2e_max)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline_sample(args.workload, budget_s=args.ref_budget, sketch=args.sketch)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}

    # extra keys (single GPU, outside the timed region): the reduced-precision
    # workload's step and accuracy, and the three arms of the batched workload
    extras = None
    if world == 1 and not args.no_extras and args.workload == "cd3d_n100" and basis == "f64":
        del V, SV, SAV, H
        torch.cuda.empty_cache()
        t_ex = time.perf_counter()
        extras = {"sketch_kinds": sketch_extras(dev, op, A, b_dev, wl)}
        extras["precision"] = precision_extras(dev)
        extras["graph"] = graph_extras(dev)
        bo = batch_arms(dev, 1, 1, "16")
        extras["batch"] = {"workload": "batch_cd_8x64 (8 operators, 64 right-hand sides, m_r in [50, 400], "
                                       "sGMRES z^-1/2; one replay per arm after one warm-up)",
                           **batch_summary(bo, 1)}
        del bo
        torch.cuda.empty_cache()
        extras["seconds"] = round(time.perf_counter() - t_ex, 1)

    if rank == 0:
        line = {
            "metric": METRIC[basis], "value": round(value, 3), "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[basis],
            "data": "synthetic",
            "config": {"workload": args.workload, "N": int(A.n), "nnz": int(A.nnz), "m": wl.m, "k": wl.k,
                       "s": wl.s, "zeta": wl.zeta, "sketch": args.sketch, "f": wl.func, "quad_scale": c,
                       "quad_tol": 1e-10, "quad_rule": (f"fixed {wl.extra['ell']} nodes" if wl.extra.get("ell")
                                                        else "adaptive"),
                       "parallelism": f"replicas x{world}", "l2": "flushed between steps",
                       "ell_sfom": st_f["ell"], "ell_sgmres": st_g["ell"], "status": [st_f["status_name"],
                                                                                     st_g["status_name"]],
                       "basis": basis, "values": "f64" if A.values.dtype == np.float64 else "f32",
                       "two_pass": bool(args.two_pass),
                       "pair": ("skf_sfom_sgmres: one Arnoldi process, one whitening QR, both tails, one pass "
                                "over V_m for both recombinations" if paired else
                                "skf_sfom + skf_sgmres: two Arnoldi processes"),
                       "basis_bytes": int(BASIS_BYTES[basis] * ((A.n + 63) // 64 * 64)
                                          * (min(wl.m, wl.k + 2) if args.two_pass else wl.m))},
            "accuracy": accuracy,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 3), "unit": "solves/s", "h2d_bytes_per_step": int(b.nbytes),
                    "d2h_bytes_per_step": int(2 * b.nbytes)},
            "gpu_launches": int(launches),
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
        }
        if extras is not None:
            line["extras"] = extras
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
