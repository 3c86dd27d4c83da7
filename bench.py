#!/usr/bin/env python
"""Benchmark of the factorized Krylov solver on one GB300.

Default workload (one "step" = one full solve from X_0 = 0 to relative residual
1e-8): factorized BiCGSTAB (Algorithm 4.2) in float64 on A = 3D upwind
convection-diffusion 64^3 (n = 262,144, wind seed 1), B = the same operator on
48^3 (m = 110,592, wind seed 2), s = 4, C1, C2 ~ N(0,1) seed 0, tol 1e-8,
maxit 300.  Inputs are synthetic (``workloads``).

Prints ONE JSON line.  ``value`` = device time per solve (CUDA events on the
solve stream, inputs already in HBM); ``e2e`` = the same through the public C
ABI with host buffers (create + solve + factors back, pinned host memory);
``roofline`` = the dominant kernel class, timed by the library's CUDA-event
profiler on one more solve run on one stream (the timed solves overlap the two
bases on concurrent streams; their own figure is kept as
``achieved_in_timed_region``); ``cpu_baseline`` = the CPU FP64 oracle on the host cores (a bounded,
measured sample of the same workload, extrapolated with the algorithm's cost
structure; see ``oracle_time_to_tol``).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank solves its own replica
of the workload (the solver does not shard); the line reports the max over
ranks.  ``--impl reference`` times the CPU oracle alone (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

METRIC = "time to rel. residual 1e-8 (mixed/batched vs FP64 factorized), SpMM+Gram HBM GB/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.26


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback"}


def workload(maxit: int = 0, precision: str = "fp64"):
    p = wl.cfg_convdiff_bicgstab(64, 48, 4, tol=1e-8, maxit=maxit or 300, precision=precision)
    return p


def config_of(p):
    return {"workload": f"convdiff3d_64^3_x_48^3_s4_bicgstab_{p.precision}",
            "method": "factorized BiCGSTAB (Algorithm 4.2)",
            "n": p.A.nrows, "m": p.B.nrows, "nnzA": p.A.nnz, "nnzB": p.B.nnz, "s": p.s, "tol": p.tol,
            "maxit": p.maxit, "precision": p.precision,
            "stop": ("certified: float64 true relative residual bound <= tol with probability >= 1 - 1e-4 "
                     "(recurrence test at 0.4 tol, then a 32-column Gaussian probe of the residual)"),
            "l2": "inputs larger than L2: the basis grows to ~2 GB per side per solve (L2 = 126 MB)"}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling during the timed region (read-only query)."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        out_dir = os.environ.get("SYLV_BENCH_OUT", "/tmp")
        self.path = os.path.join(out_dir, f"sylv_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- CPU oracle timing
def oracle_time_to_tol(p, iters: int):
    """Seconds the CPU FP64 oracle needs for ``iters`` iterations of factorized
    BiCGSTAB on workload ``p``, from a bounded measured sample.

    The oracle itself is run, as it stands, on pieces of the same workload:
    (1) block Arnoldi steps (``BlockKrylovBasis.step``, BCGS2) of both bases at a
        narrow and at the final width (cost is linear in the number of blocks j:
        one SpMM plus four passes over n x js);
    (2) the small-matrix part of one iteration (two factored Sylvester
        operators, the inner products and padded updates of Algorithm 4.2) at
        half and at the final order r (cost c3 r^3 + c2 r^2);
    then sums the fitted per-step and per-iteration costs over the iteration
    structure (Arnoldi steps 1..2*iters on each side, small orders
    (2k+1)s, (2k+2)s).  Returns (seconds, sample_seconds, details).
    """
    from oracle import factorized as fz

    rng = np.random.default_rng(123)
    s = p.s
    A = p.A.to_scipy()
    Bt = p.B.to_scipy().T.tocsr()
    t_sample0 = time.perf_counter()

    def arnoldi_step_time(Op, n, j):
        b = fz.BlockKrylovBasis(Op, rng.standard_normal((n, s)), "arnoldi")
        b.blocks = [rng.standard_normal((n, s)) for _ in range(j)]  # cost-equivalent blocks
        b.H = np.zeros((j * s, (j - 1) * s))
        t = time.perf_counter()
        b.step()
        return time.perf_counter() - t

    jmax = 2 * iters
    lin = {}
    for name, Op, n in (("A", A, p.A.nrows), ("B", Bt, p.B.nrows)):
        t1 = min(arnoldi_step_time(Op, n, 2) for _ in range(2))
        t2 = arnoldi_step_time(Op, n, jmax)
        slope = (t2 - t1) / (jmax - 2)
        lin[name] = (t1 - 2 * slope, slope)
    basis = 0.0
    for j in range(1, jmax + 1):
        for a0, a1 in lin.values():
            basis += a0 + a1 * j

    def small_iter_time(k):
        r = (2 * k + 1) * s
        H = np.triu(rng.standard_normal((r + 2 * s, r + s)), -s)
        G = np.triu(rng.standard_normal((r + 2 * s, r + s)), -s)
        P, R, X = rng.standard_normal((3, r, r))
        Rt = rng.standard_normal((s, s))
        t = time.perf_counter()
        Qh = fz.small_sylvester(H[: r + s, :r], P, G[: r + s, :r])
        alpha = 1.0 / fz.inner(Rt, Qh[:s, :s])
        Sh = fz.pad(R, s) - alpha * Qh
        Th = fz.small_sylvester(H, Sh, G)
        omega = fz.inner(Th[: r + s, : r + s], Sh) / fz.inner(Th, Th)
        X2 = fz.pad(X[: r - s, : r - s], 2 * s) + fz.pad(alpha * P, s) + omega * Sh
        R2 = fz.pad(Sh, s) - omega * Th
        rn = np.sqrt(fz.inner(R2, R2))
        rho = fz.inner(Rt, R2[:s, :s])
        P2 = R2 + (rho + rn) * (fz.pad(P, 2 * s) - omega * fz.pad(Qh, s))
        del X2, P2
        return time.perf_counter() - t

    k_hi = iters - 1
    k_lo = max(1, k_hi // 2)
    th = min(small_iter_time(k_hi) for _ in range(2))
    tl = min(small_iter_time(k_lo) for _ in range(2))
    r_hi, r_lo = (2 * k_hi + 1) * s, (2 * k_lo + 1) * s
    # t(r) = c3 r^3 + c2 r^2 through the two samples
    M = np.array([[r_lo**3, r_lo**2], [r_hi**3, r_hi**2]], dtype=float)
    c3, c2 = np.linalg.solve(M, np.array([tl, th]))
    small = sum(max(0.0, c3 * ((2 * k + 1) * s) ** 3 + c2 * ((2 * k + 1) * s) ** 2) for k in range(iters))
    sample = time.perf_counter() - t_sample0
    return basis + small, sample, {"arnoldi_step_s": {k: [round(v[0], 6), round(v[1], 8)] for k, v in lin.items()},
                                   "small_iter_s": {"k_lo": k_lo, "t_lo": tl, "k_hi": k_hi, "t_hi": th}}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info

        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(v, "").isdigit():
            return int(os.environ[v])
    return os.cpu_count()


def golden_iterations():
    path = os.path.join(ROOT, "tests", "golden", "convdiff64x48_s4_bicgstab_history.txt")
    try:
        rows = [ln for ln in open(path) if ln.strip() and not ln.startswith("#")]
        return len(rows) - 1
    except OSError:
        return None


def model_check():
    """The cost model of ``oracle_time_to_tol`` against a real oracle solve timed to completion, on
    a smaller workload of the same kind (CD 24^3 x 18^3, s = 4, tol 1e-8: a few seconds)."""
    from oracle import factorized as fz

    q = wl.cfg_convdiff_bicgstab(24, 18, 4, tol=1e-8, maxit=300)
    t = time.perf_counter()
    ref = fz.factorized_bicgstab(q.A.to_scipy(), q.B.to_scipy(), q.C1, q.C2, q.tol, q.maxit)
    measured = time.perf_counter() - t
    model, sample, _ = oracle_time_to_tol(q, ref.iters)
    return {"workload": "convdiff3d_24^3_x_18^3_s4_bicgstab_fp64", "iters": ref.iters, "measured_s": measured,
            "model_s": model, "model_over_measured": model / measured, "model_sample_s": sample}


def cpu_baseline(p, iters):
    t, sample, det = oracle_time_to_tol(p, iters)
    return {"value": t, "unit": "s", "cores": blas_threads(), "kind": "oracle", "extrapolated": True,
            "sample": (f"measured {sample:.1f} s of the CPU FP64 oracle on this workload (BCGS2 Arnoldi steps of both "
                       f"bases at widths 2 and {2 * iters} blocks, small-matrix iterations at orders "
                       f"{(2 * det['small_iter_s']['k_lo'] + 1) * p.s} and {(2 * det['small_iter_s']['k_hi'] + 1) * p.s})"
                       f", summed over {iters} iterations with the per-step cost structure (extrapolated; "
                       f"model_check times a full oracle solve of a smaller case against the same model)"),
            "details": det, "model_check": model_check()}


# ----------------------------------------------------------------------------- variants
def profiled_breakdown(p, stream, precision, maxit):
    """One extra solve with every basis kernel on one stream and CUDA-event timing of
    each launch (clean per-kernel durations; the timed runs overlap the bases)."""
    import paper_2605_28274_gb300 as ps

    with ps.Solver(p.A, p.B, p.C1, p.C2, precision=precision, profile=True, stream_mode=1,
                   cuda_stream=stream.cuda_stream) as sv:
        sv.bicgstab(p.tol, maxit)
        prof = sv.profile()
    pk = peaks()
    hb = [e for e in prof if e["name"] in ("spmm", "gram", "update")]
    hb_bytes, hb_ms = sum(x["bytes"] for x in hb), sum(x["ms"] for x in hb)
    gbs = hb_bytes / (hb_ms * 1e-3) / 1e9 if hb_ms else None
    per = {e["name"]: {"ms": round(e["ms"], 2), "launches": e["launches"],
                       "gbs": round(e["bytes"] / (e["ms"] * 1e-3) / 1e9, 1) if e["ms"] and e["bytes"] else None}
           for e in sorted(prof, key=lambda e: -e["ms"])}
    return gbs, (gbs / pk["hbm_gbs"] if gbs else None), per


def timed_solves(p, stream, precision, steps, warmup, method="bicgstab"):
    import torch

    import paper_2605_28274_gb300 as ps

    with ps.Solver(p.A, p.B, p.C1, p.C2, precision=precision, cuda_stream=stream.cuda_stream) as sv:
        for _ in range(warmup):
            getattr(sv, method)(p.tol, p.maxit)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            info = getattr(sv, method)(p.tol, p.maxit)
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps / 1e3, info


def factored_rel_diff_gpu(F1, F2):
    """||V1 X1 W1^T - V2 X2 W2^T||_F / ||V2 X2 W2^T||_F without forming X: Householder QR (torch,
    on the GPU, float64) of the stacked factors [V1, V2] and [W1, W2], then the small core."""
    import torch

    (V1, X1, W1), (V2, X2, W2) = F1, F2
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    RL = torch.linalg.qr(torch.cat([t(V1), t(V2)], 1), mode="r")[1]
    RR = torch.linalg.qr(torch.cat([t(W1), t(W2)], 1), mode="r")[1]
    r1, r2 = X1.shape[0], X2.shape[0]
    D = torch.zeros((r1 + r2, r1 + r2), dtype=torch.float64, device=dev)
    D[:r1, :r1] = t(X1)
    D[r1:, r1:] = -t(X2)
    R2L = torch.linalg.qr(t(V2), mode="r")[1]
    R2R = torch.linalg.qr(t(W2), mode="r")[1]
    num = torch.linalg.norm(RL @ D @ RR.T)
    den = torch.linalg.norm(R2L @ t(X2) @ R2R.T)
    return float(num / den)


def measure_mixed(p, stream, steps, warmup, fp64_factors=None):
    """Same operators and tolerance in the mixed mode (FP32 factors, FP64 small side,
    FP64 true-residual refinement): time to a certified TRUE relative residual of p.tol, and
    the relative error of X against the FP64 solve of the same workload."""
    import paper_2605_28274_gb300 as ps

    t, info = timed_solves(p, stream, "mixed", steps, warmup)
    gbs, frac, per = profiled_breakdown(p, stream, "mixed", p.maxit)
    out = {"workload": "convdiff3d_64^3_x_48^3_s4_bicgstab_mixed", "value": t, "unit": "s",
           "status": info["status_name"], "iters_total": info["iters"], "refinements": info["refinements"],
           "true_rel_res": info["true_rel_res"], "true_rel_bound": info["true_rel_bound"], "width": info["width"],
           "spmm_gram_update_fp32_gbs": gbs, "frac_of_measured_hbm": frac,
           "kernel_profile_one_stream": per}
    if fp64_factors is not None:
        with ps.Solver(p.A, p.B, p.C1, p.C2, precision="mixed", cuda_stream=stream.cuda_stream) as sv:
            sv.bicgstab(p.tol, p.maxit)
            fm = sv.factors()
        out["rel_error_vs_fp64_solve"] = factored_rel_diff_gpu(fm, fp64_factors)
        out["rel_error_how"] = ("||X_mixed - X_fp64||_F / ||X_fp64||_F through the QR of the stacked factors; "
                                "X_fp64 = the certified FP64 solve of the timed line")
    return out


def measure_exhaustion(stream, steps, warmup):
    """The 400-unknown Laplacian with s = 8 in mixed precision (CG): the block Krylov space has
    n / s = 50 blocks, so the bases fill up; time to a certified true residual of 1e-8."""
    p = wl.cfg_laplace_cg(N=20, s=8, precision="mixed")
    t, info = timed_solves(p, stream, "mixed", steps, warmup, "cg")
    return {"workload": "laplace2d_20^2_s8_cg_mixed", "value": t, "unit": "s", "status": info["status_name"],
            "iters_total": info["iters"], "refinements": info["refinements"], "true_rel_res": info["true_rel_res"],
            "true_rel_bound": info["true_rel_bound"], "width": info["width"]}


def measure_methods(p, stream, steps, warmup):
    """The other factorized methods (Sec. 4 names CR, CGS and GPBiCG) at full size: CGS and GPBiCG on
    the benchmarked convection-diffusion operators, CG and CR on a symmetric workload of the same size class
    (A = L_512 + I/2, B = L_384 + I/2: 2D 5-point Laplacians, n = 262,144, m = 147,456, s = 4).
    Time to a relative residual of 1e-8 (mixed: true residual), FP64 and mixed."""
    out = {}
    for meth in ("cgs", "gpbicg"):
        for prec in ("fp64", "mixed"):
            t, info = timed_solves(p, stream, prec, steps, warmup, meth)
            out[f"{meth}_{prec}_convdiff3d_64^3_x_48^3_s4"] = {
                "value": t, "unit": "s", "status": info["status_name"], "iters_total": info["iters"],
                "width": info["width"], "true_rel_res": info["true_rel_res"], "true_rel_bound": info["true_rel_bound"]}
    A, B = wl.laplacian_2d(512, 0.5), wl.laplacian_2d(384, 0.5)
    C1, C2 = wl.rhs(A.nrows, B.nrows, 4, 0)
    q = wl.Problem(name="laplace2d_512x384_s4", A=A, B=B, C1=C1, C2=C2, s=4, method="cg", tol=1e-8, maxit=300)
    for meth in ("cg", "cr"):
        for prec in ("fp64", "mixed"):
            t, info = timed_solves(q, stream, prec, steps, warmup, meth)
            out[f"{meth}_{prec}_laplace2d_512^2_x_384^2_shift0.5_s4"] = {
                "value": t, "unit": "s", "status": info["status_name"], "iters_total": info["iters"],
                "width": info["width"], "true_rel_res": info["true_rel_res"], "true_rel_bound": info["true_rel_bound"]}
    return out


def measure_batched(stream, steps, warmup):
    """64 Lyapunov instances (2D Laplacian + U[0,1] shift, N ~ U{64..256}, s ~ {1,2,4}),
    batched factorized CG to 1e-8 vs the plain FP64 path looping over the instances."""
    import torch

    import paper_2605_28274_gb300 as ps

    probs = wl.cfg_batched_lyapunov(count=64)
    As, Cs = [q.A for q in probs], [q.C1 for q in probs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ps.BatchSolver(As, Cs, cuda_stream=stream.cuda_stream) as bs:
        for _ in range(warmup):
            bs.cg(1e-8, 1000)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            info = bs.cg(1e-8, 1000)
        e1.record(stream)
        torch.cuda.synchronize()
        its = [len(bs.history(i)) - 1 for i in range(len(probs))]
    t_batch = e0.elapsed_time(e1) / steps / 1e3
    svs = [ps.Solver(q.A, None, q.C1, None, lyapunov=True, cuda_stream=stream.cuda_stream) for q in probs]
    for sv in svs:
        sv.cg(1e-8, 1000)
    torch.cuda.synchronize()
    e0.record(stream)
    for sv in svs:
        sv.cg(1e-8, 1000)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    for sv in svs:
        sv.close()
    return {"workload": "batched_lyapunov_64x_laplace2d_N64-256_s124_cg_fp64", "value": t_batch, "unit": "s",
            "status": info["status_name"], "instances": len(probs), "sum_n": int(sum(q.A.nrows for q in probs)),
            "iters_min_median_max": [int(min(its)), int(np.median(its)), int(max(its))],
            "true_rel_res_max": info["true_rel_res"], "true_rel_bound_max": info["true_rel_bound"],
            "kernel_launches": info["kernel_launches"],
            "plain_fp64_sequential_s": t_seq, "speedup_vs_plain_fp64": t_seq / t_batch}


def measure_large(stream, steps, warmup):
    """Large mixed-precision BiCGSTAB: A = CD 128^3 (n = 2,097,152), B = CD 96^3
    (m = 884,736), s = 8, tol 1e-8 on the true residual."""
    p = wl.cfg_convdiff_bicgstab(128, 96, 8, tol=1e-8, maxit=400, precision="mixed")
    t, info = timed_solves(p, stream, "mixed", steps, warmup)
    gbs, frac, per = profiled_breakdown(p, stream, "mixed", p.maxit)
    return {"workload": "convdiff3d_128^3_x_96^3_s8_bicgstab_mixed", "value": t, "unit": "s",
            "status": info["status_name"], "iters_total": info["iters"], "refinements": info["refinements"],
            "true_rel_res": info["true_rel_res"], "true_rel_bound": info["true_rel_bound"], "width": info["width"],
            "error_vs_fp64": ("not formed: an FP64 solve of this workload holds ~150 GB of float64 bases; the "
                              "mixed-vs-FP64 error is measured on the 64^3 x 48^3 workload (variants.mixed)"),
            "spmm_gram_update_fp32_gbs": gbs, "frac_of_measured_hbm": frac,
            "kernel_profile_one_stream": per}


# ----------------------------------------------------------------------------- our arm
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dist=None) -> float:
    """Max of x over all ranks (replicas: the job is as slow as its slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch

    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# (kernel class, precision, tensor-core basis) -> (DRAM read + write MB, algorithmic MB, summary)
# of one ncu capture of that kernel
NCU_DRAM_PER_ALGORITHMIC = {
    ("gram", "fp64", False): (318.5, 318.8, "profiles/gram_update_fp64_convdiff64x48_s4.md"),
    ("gram", "fp64", True): (565.3, 436.2, "profiles/ob_gram_update_fp64_convdiff64x48_s4.md"),
    # the update class alternates the full (5 planes) and the second, two-plane update of a step
    ("update", "fp64", True): (605.5 + 250.9, 2 * 444.6, "profiles/ob_gram_update_fp64_convdiff64x48_s4.md"),
}


def nvtx_push(name):
    try:
        import torch

        torch.cuda.nvtx.range_push(name)
    except Exception:  # NVTX is a profiling aid only
        pass


def nvtx_pop():
    try:
        import torch

        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def run_ours(args):
    import torch

    import paper_2605_28274_gb300 as ps

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = workload(args.maxit, args.precision)
    stream = torch.cuda.Stream()
    sv = ps.Solver(p.A, p.B, p.C1, p.C2, precision=args.precision, profile=True, cuda_stream=stream.cuda_stream)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        info = sv.bicgstab(p.tol, p.maxit)
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos, prof = [], {}
    nvtx_push("timed")  # lets a profiler restrict its launch list to the timed solves
    e0.record(stream)
    for _ in range(args.steps):
        info = sv.bicgstab(p.tol, p.maxit)
        infos.append(info)
        for e in sv.profile():
            d = prof.setdefault(e["name"], {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
            for key in ("launches", "ms", "bytes", "flops"):
                d[key] += e[key]
    e1.record(stream)
    torch.cuda.synchronize()
    nvtx_pop()
    barrier()
    ms_total = e0.elapsed_time(e1)
    clocks = clk.stop()
    ms_step = max_over_ranks(ms_total / args.steps, dist)
    iters = infos[-1]["iters"]
    status = infos[-1]["status_name"]
    launches = int(sum(i["kernel_launches"] for i in infos))
    prof_timed = prof

    # The timed solves run the two bases on concurrent streams (the library's default where that
    # pays), so a kernel's event interval there includes kernels running beside it.  The roofline
    # takes per-kernel durations from one more profiled solve of the same workload on one stream
    # (stream_mode 1), right after the timed region; the timed region's own figure is kept beside it.
    svs = ps.Solver(p.A, p.B, p.C1, p.C2, precision=args.precision, profile=True, stream_mode=1,
                    cuda_stream=stream.cuda_stream)
    svs.bicgstab(p.tol, p.maxit)
    svs.bicgstab(p.tol, p.maxit)
    prof = {}
    for e in svs.profile():
        prof[e["name"]] = {key: e[key] for key in ("launches", "ms", "bytes", "flops")}
    torch.cuda.synchronize()
    svs.close()

    # roofline of the dominant kernel class (live CUDA-event timing inside the library)
    pk = peaks()
    # dominant kernel class (the residual wrapper and setup are not single kernels)
    dom = max(((k, v) for k, v in prof.items() if k not in ("true_residual", "setup")), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    ai = d["flops"] / max(d["bytes"], 1.0)
    ridge = FP64_NOMINAL_TFLOPS * 1e12 / (pk["hbm_gbs"] * 1e9)
    # the float64 Arnoldi basis on the tensor cores (its digit planes are written by the
    # "basis_split" kernels): Gram and update are bound by HBM, not by the FP64 pipe
    tensor_basis = "basis_split" in prof
    if tensor_basis and dname in ("gram", "update"):
        roof = {"bound": "hbm", "achieved": d["bytes"] / (d["ms"] * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "kernel": dname, "peak_src": f"{pk['src']} HBM copy",
                "bytes_src": "algorithmic: the float64 basis (8 B per element) and the block Y, each read once; "
                             "the kernel reads the basis as five FP16 digit planes (10 B per element)"}
    elif ai > ridge or dname.startswith("small_gemm"):
        roof = {"bound": "alu", "achieved": d["flops"] / (d["ms"] * 1e-3) / 1e12, "peak": FP64_NOMINAL_TFLOPS,
                "unit": "TFLOP/s", "kernel": dname,
                "peak_src": "FP64 nominal: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (no FP64 figure in MEASURED_PEAKS)"}
    else:
        roof = {"bound": "hbm", "achieved": d["bytes"] / (d["ms"] * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "kernel": dname, "peak_src": f"{pk['src']} HBM copy"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes per algorithmic byte from one ncu capture of the same kernel on a smaller case,
    # scaled to the average launch of this run by its algorithmic bytes (the kernel reads each
    # basis element once, so traffic grows in proportion)
    ratio = NCU_DRAM_PER_ALGORITHMIC.get((dname, args.precision, tensor_basis))
    roof["traffic"] = ratio[0] / ratio[1] * d["bytes"] / max(1, d["launches"]) if ratio else None
    roof["traffic_src"] = ratio[2] if ratio else None
    if ratio and roof["unit"] == "GB/s":  # the fraction of the copy bandwidth on what the kernel moves
        roof["frac_of_traffic"] = roof["achieved"] * ratio[0] / ratio[1] / roof["peak"]
    roof["launches"] = d["launches"]
    roof["avg_launch_us"] = d["ms"] * 1e3 / max(1, d["launches"])
    roof["timing"] = ("one profiled solve on one stream after the timed region (the timed solves run the bases on "
                      "concurrent streams, where a kernel's event interval includes the kernels beside it)")
    dt = prof_timed.get(dname)
    if dt and dt["ms"]:
        roof["achieved_in_timed_region"] = (dt["bytes"] / (dt["ms"] * 1e-3) / 1e9 if roof["unit"] == "GB/s"
                                            else dt["flops"] / (dt["ms"] * 1e-3) / 1e12)
    hb = [prof[k] for k in ("spmm", "gram", "update") if k in prof]
    hb_bytes, hb_ms = sum(x["bytes"] for x in hb), sum(x["ms"] for x in hb)
    spmm_gram = {"gbs": hb_bytes / (hb_ms * 1e-3) / 1e9 if hb_ms else None, "frac_of_measured_hbm":
                 (hb_bytes / (hb_ms * 1e-3) / 1e9 / pk["hbm_gbs"]) if hb_ms else None,
                 "tflops_fp64": sum(x["flops"] for x in hb) / (hb_ms * 1e-3) / 1e12 if hb_ms else None}
    total_ms = sum(x["ms"] for x in prof.values())
    breakdown = {k: {"share": round(v["ms"] / total_ms, 4), "ms_per_solve": v["ms"],
                     "launches_per_solve": v["launches"],
                     "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] else None,
                     "tflops": v["flops"] / (v["ms"] * 1e-3) / 1e12 if v["ms"] else None}
                 for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    # end to end through the public API with pinned host buffers
    e2e_steps = max(1, args.steps)

    def pinned(a):
        dt = torch.float64 if a.dtype == np.float64 else torch.int32
        if a.ndim == 2:  # column-major, as the C ABI takes it
            tn = torch.empty(a.shape[::-1], dtype=dt, pin_memory=True).numpy()
            tn[...] = a.T
            return tn.T
        tn = torch.empty(a.shape, dtype=dt, pin_memory=True).numpy()
        tn[...] = a
        return tn

    Ap = wl.CSR(p.A.nrows, p.A.ncols, pinned(p.A.row_ptr), pinned(p.A.col_idx), pinned(p.A.val))
    Bp = wl.CSR(p.B.nrows, p.B.ncols, pinned(p.B.row_ptr), pinned(p.B.col_idx), pinned(p.B.val))
    C1p, C2p = pinned(p.C1), pinned(p.C2)
    width = infos[-1]["width"]
    outV = torch.empty(p.A.nrows * width, dtype=torch.float64, pin_memory=True).numpy()
    outW = torch.empty(p.B.nrows * width, dtype=torch.float64, pin_memory=True).numpy()
    outX = torch.empty(width * width, dtype=torch.float64, pin_memory=True).numpy()
    h2d = (Ap.row_ptr.nbytes + Ap.col_idx.nbytes + Ap.val.nbytes + Bp.row_ptr.nbytes + Bp.col_idx.nbytes +
           Bp.val.nbytes + C1p.nbytes + C2p.nbytes)
    barrier()
    e2e_times, d2h = [], 0
    # warm-up steps as for the device timing (the first transfer into the freshly pinned output
    # buffers costs ~0.35 s once), then e2e_steps timed ones
    for step in range(args.warmup + e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with ps.Solver(Ap, Bp, C1p, C2p, precision=args.precision, cuda_stream=stream.cuda_stream) as sv2:
            inf2 = sv2.bicgstab(p.tol, p.maxit)
            V, X, W = sv2.factors(out={"V": outV, "X": outX, "W": outW})
        torch.cuda.synchronize()
        if step >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
        d2h = V.nbytes + X.nbytes + W.nbytes
    e2e_s = max_over_ranks(statistics.mean(e2e_times), dist)

    variants = {}
    if not args.no_variants:
        fp64_factors = sv.factors() if args.precision == "fp64" else None
        variants["mixed"] = measure_mixed(p, stream, args.steps, 2, fp64_factors)
        del fp64_factors
        variants["mixed"]["speedup_vs_fp64"] = (ms_step / 1e3) / variants["mixed"]["value"]
        variants["exhaustion_mixed"] = measure_exhaustion(stream, args.steps, 2)
        variants["batched"] = measure_batched(stream, args.steps, 2)
        variants["methods"] = measure_methods(p, stream, max(1, min(args.steps, 2)), 1)
        if not args.no_large:
            variants["large_mixed"] = measure_large(stream, 1, 1)
    sv.close()

    line = {"metric": METRIC, "value": ms_step / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic", "config": config_of(p),
            "iters": iters, "status": status, "rel_res": infos[-1]["rel_res"],
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "status": STATUS(inf2)},
            "true_rel_res": infos[-1]["true_rel_res"], "true_rel_bound": infos[-1]["true_rel_bound"],
            "roofline": roof, "spmm_gram_hbm": spmm_gram, "kernel_breakdown": breakdown,
            "gpu_launches": launches, "clocks": clocks, "variants": variants}
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(p, iters)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def STATUS(info):
    return info.get("status_name", str(info.get("status")))


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    p = workload()
    iters = golden_iterations() or 125
    for _ in range(args.warmup):
        oracle_time_to_tol(p, iters)
    vals, samples = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, smp, det = oracle_time_to_tol(p, iters)
        vals.append(v)
        samples.append(smp)
    wall = time.perf_counter() - t0
    v = statistics.mean(vals)
    check = model_check()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(p),
            "iters": iters,
            "cpu_baseline": {"value": v, "unit": "s", "cores": blas_threads(), "kind": "oracle", "extrapolated": True,
                             "sample": (f"each step measures {statistics.mean(samples):.1f} s of the CPU FP64 oracle "
                                        f"on this workload (Arnoldi steps at 2 and {2 * iters} blocks, small-matrix "
                                        f"iterations at two orders) and sums the fitted costs over the oracle's "
                                        f"{iters} iterations (tests/golden); model_check times a full oracle solve "
                                        f"of a smaller case against the same model"),
                             "model_check": check},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--maxit", type=int, default=0, help="override maxit (a short solve, e.g. for ncu captures)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="precision of the timed line (the variants are always measured)")
    ap.add_argument("--no-variants", action="store_true", help="skip the mixed and batched variant timings")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large mixed-precision workload (CD 128^3 x 96^3, s = 8; ~60 GB of HBM, ~40 s)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
