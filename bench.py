#!/usr/bin/env python
"""Benchmark: time to relative residual 1e-8 of block-triangular FGMRES + multigrid,
and the SG-apply HBM bandwidth, on one GB300 (replicas on N GPUs).

Default workload ("c3", the bandwidth-scale solve): 1025 x 1025 Q1 grid
(1,046,529 interior nodes), M = 6 Hermite KL terms (sigma = 0.2, separable
exponential covariance, correlation length 1), total degree p = 4 (P = 210),
219,771,090 unknowns; FGMRES(20) with the Arnoldi basis, Gram-Schmidt, Givens update
and true residual in IEEE FP64 and the block-triangular preconditioner whose V(1,1)
cycles store their levels in BF16 and compute in FP32 (stage right-hand sides and the
preconditioned vectors z_j in FP32); the outer operator A z_j of each Arnoldi step is
evaluated in double-float arithmetic from the FP32 z_j and stored in FP64; f = 1;
tolerance 1e-8 on the true relative residual, recomputed in IEEE FP64.  A step is one
full solve from U = 0 with F resident in HBM.  Every vector is 1.76 GB (> L2), so no
L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W]
                    [--workload c3|c2|c1|c4|c5|c3s|table3|table3p1|table3p1rb]
                    [--arith f64dfop|f64|df64] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead (see ``CpuSample``).
"""
import argparse
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

WORKLOADS = {
    # BF16-storage / FP32-arithmetic V-cycle (levels in BF16), FP32 stage right-hand sides and
    # preconditioned vectors z_j (sg.BF16Z); --pc-prec bf16 stores those in BF16 as well
    "c3": dict(n=1025, M=6, p=4, family=1, sigma=0.2, restart=20, pc_prec=4, tol=1e-8, f_seed=None,
               name="sg_c3_1025sq_M6_hermite_p4_P210_fgmres20_bf16pc_f32z"),
    "c2": dict(n=257, M=4, p=4, family=0, sigma=0.3, restart=30, pc_prec=1, tol=1e-8, f_seed=1,
               name="sg_c2_257sq_M4_legendre_p4_P70_sigma0.3_fgmres30_fp32pc"),
    "c1": dict(n=33, M=2, p=2, family=0, sigma=0.3, restart=30, pc_prec=0, tol=1e-8, f_seed=None,
               name="sg_c1_33sq_M2_legendre_p2_P6_gmres30_fp64"),
    # the c3 chaos space on a 513 x 513 grid with FGMRES(4): every kernel of the c3 solve on
    # vectors of 439 MB (> L2) with about 5 GB on the device, for detailed kernel profiles
    "c3s": dict(n=513, M=6, p=4, family=1, sigma=0.2, restart=4, pc_prec=4, tol=1e-8, f_seed=None,
                name="sg_c3_copy_513sq_M6_hermite_p4_P210_fgmres4_bf16pc_f32z"),
    # the paper's own experiment (Table 3) in this discretisation: h = 1/64, m = 6 Legendre, p = 4,
    # f = 2 (0.5 - x^2 - y^2) on (-0.5, 0.5)^2, sigma 0.1 .. 0.4, tol 1e-10, x0 = 0, two smoothing
    # steps before and after; the five methods of the table (context: the paper uses P1 triangles and
    # point Gauss-Seidel)
    "table3": dict(n=65, M=6, p=4, family=0, sigmas=(0.1, 0.2, 0.3, 0.4), tol=1e-10, restart=10, nu=2,
                   name="paper_table3_65sq_M6_legendre_p4_tol1e-10"),
    # the same with the paper's own discretisation: P1 triangles and point Gauss-Seidel V(2,2)
    "table3p1": dict(n=65, M=6, p=4, family=0, sigmas=(0.1, 0.2, 0.3, 0.4), tol=1e-10, restart=10, nu=2,
                     elements=1, gs_order=0, name="paper_table3_p1_65sq_M6_legendre_p4_gs_lex_tol1e-10"),
    "table3p1rb": dict(n=65, M=6, p=4, family=0, sigmas=(0.1, 0.2, 0.3, 0.4), tol=1e-10, restart=10, nu=2,
                       elements=1, gs_order=1, name="paper_table3_p1_65sq_M6_legendre_p4_gs_redblack_tol1e-10"),
    # adjoint gradient of J = E[int u] + Var[int u] / 2 w.r.t. the per-cell mean and sigma.  At sigma =
    # 0.4 the 257^2 system (lognormal mean, not coercive at the xi-box corners) makes restarted
    # GMRES(30) stagnate near 1e-6 in FP64 as well, so the timed gradient uses sigma = 0.3; the
    # 33^2 parity test keeps sigma = 0.4
    "c4": dict(n=257, M=4, p=3, family=0, sigma=0.3, restart=30, pc_prec=1, tol=1e-8, abar_seed=2,
               name="sg_c4_adjoint_257sq_M4_legendre_p3_P35_sigma0.3_lognormal_mean"),
    # 64 uneven systems (grid 65^2..513^2, M 2..6, p 2..4, sigma U[0.1, 0.5], Legendre, f = 1):
    # FGMRES(30) + block-triangular preconditioner in FP32, FP64 outer loop
    "c5": dict(count=64, batch_seed=5, family=0, restart=30, pc_prec=1, tol=1e-8, nstreams=16,
               name="sg_c5_batch64_uneven_65to513sq_M2to6_p2to4_legendre_fgmres30_fp32pc"),
}
PREC_NAME = {0: "f64", 1: "f32", 2: "bf16", 4: "bf16 storage, f32 output"}
ARITH = {"f64": 0, "df64": 1, "f64dfop": 2}                     # sg_arith of include/sg.h
ZNAME = {0: "f64", 1: "f32", 2: "bf16", 4: "f32"}              # storage of the preconditioned vectors z
METRIC = "time to rel. residual 1e-8 (block-tri GMRES+MG) and SG-apply HBM GB/s"
C4_METRIC = "time per adjoint gradient dJ/d(abar, sigma) (forward + transpose block-tri FGMRES+MG to 1e-8)"
C5_METRIC = "aggregate unknowns solved per second (64 uneven SG systems, block-tri FGMRES+MG to 1e-8)"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "_fallback": True}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(values):
    """Element-wise maximum over the ranks of the process group (the slowest replica decides a
    replica run's time); the values unchanged without one.  NCCL groups reduce on the GPU, gloo
    groups on the CPU."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def build_problem(wl, h=None):
    """KL coefficients (library host helper) and, given a handle, the device load vector
    F = e_0 (x) h^2 f from the library (f = 1, or the seeded nodal perturbation of C2)."""
    import torch
    from paper_1304_1755_gb300 import inputs, sg
    coef, _ = sg.sg_kl_coef(wl["n"], wl["M"], wl["sigma"])
    if h is None:
        return coef, None
    f = None if wl.get("f_seed") is None else torch.as_tensor(inputs.rhs_nodes(wl["f_seed"], wl["n"])).cuda()
    F = torch.empty(h.P * h.Nx, dtype=torch.float64, device="cuda")
    h.rhs(F, f)
    torch.cuda.synchronize()
    return coef, F


def k1_bytes(wl, xprec_bytes, yprec_bytes):
    n = wl["n"]
    P = math.comb(wl["M"] + wl["p"], wl["p"])
    Nx, Nc = (n - 2) ** 2, (n - 1) ** 2
    return (xprec_bytes + yprec_bytes) * Nx * P + 8 * (wl["M"] + 1) * Nc


def terms_per_row(wl):
    """Couplings per output row of A = sum_k G_k (x) K_k: the mean term plus r = 2 x lower pairs / P."""
    M, p = wl["M"], wl["p"]
    P = math.comb(M + p, p)
    return (P + 2 * M * math.comb(M + p - 1, p - 1)) / P


def k1_method_flops(wl):
    """The method's flops per SG apply: N (8 (1 + r) + r + 16) (corner mixing at 4 corners per
    coupling, per-cell weight products, the Q1 element matrix and the accumulation)."""
    n = wl["n"]
    N = (n - 2) ** 2 * math.comb(wl["M"] + wl["p"], wl["p"])
    r = terms_per_row(wl) - 1
    return N * (8 * (1 + r) + r + 16)


def gs_fp64_fmas(N, iterations, restart):
    """FP64 multiply-adds of classical Gram-Schmidt in an (F)GMRES(restart) solve of `iterations` Arnoldi
    steps over vectors of N elements: at step j of a cycle, j + 1 dot products and w.w (j + 2 per element),
    then j + 1 updates and ||w||^2 (j + 2 per element)."""
    total, left = 0, iterations
    while left > 0:
        k = min(left, restart)
        total += sum(2 * (j + 2) for j in range(k))
        left -= k
    return N * total


def time_apply(h, X, Y, prec, reps=50, warm=5):
    """Median CUDA-event time (ms) of one sg_apply (Y = A X), after warm-up launches."""
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warm):
        h.apply(X, Y, prec)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        h.apply(X, Y, prec)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def timed_solves(h, F, U, opts, steps, stream):
    """(ms per solve, last info) of `steps` solves from U = 0, CUDA events on the solve stream."""
    import torch
    h.solve(F, U, **opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        info = h.solve(F, U, **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, info


def run_apply_only(args, wl):
    """The SG apply Y = A X of the workload's problem on its own: median CUDA-event time of
    sg_apply with FP32, FP64 and double-float storage (the same launches as the operator of the
    solves), algorithmic bytes per launch and the fraction of the measured HBM bandwidth."""
    import torch
    from paper_1304_1755_gb300 import build as B
    from paper_1304_1755_gb300 import sg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    if not os.path.exists(sg.LIB_PATH):
        B.build()
    coef, _ = build_problem(wl)
    h = sg.Handle(wl["n"], wl["M"], wl["p"], wl["family"], coef, stream=torch.cuda.current_stream())
    h.autotune()
    N = h.P * h.Nx
    hbm = _peaks().get("hbm_gbs", 6800.0)
    rows = {}
    for name, prec, dt, sb, n_el in (("f32", sg.F32, torch.float32, 4, N), ("f64", sg.F64, torch.float64, 8, N),
                                     ("df64", sg.DF64, torch.float32, 8, 2 * N)):
        X = torch.rand(n_el, dtype=dt, device="cuda") * 2 - 1
        Y = torch.empty_like(X)
        ms = time_apply(h, X, Y, prec, reps=max(args.steps, 1), warm=max(args.warmup, 1))
        b = k1_bytes(wl, sb, sb)
        rows[name] = {"ms": round(ms, 4), "gbs": round(b / (ms * 1e-3) / 1e9, 1),
                      "frac_of_hbm": round(b / (ms * 1e-3) / 1e9 / hbm, 4), "bytes": b}
        del X, Y
    h.close()
    return {"metric": "SG-apply HBM GB/s", "config": {"workload": wl["name"], "unknowns": N}, "apply": rows}


def run_ours(args, wl, rank, world):
    import numpy as np
    import torch
    from paper_1304_1755_gb300 import build as B
    from paper_1304_1755_gb300 import sg
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    if not os.path.exists(sg.LIB_PATH):
        B.build()
    # a dedicated (non-default) stream: the library then replays each preconditioner application as
    # a captured CUDA graph
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    coef, _ = build_problem(wl)
    h = sg.Handle(wl["n"], wl["M"], wl["p"], wl["family"], coef, stream=stream)
    t_tune = time.perf_counter()
    h.autotune()                          # operator tile per arithmetic (set-up, outside the timed region)
    t_tune = time.perf_counter() - t_tune
    N = h.P * h.Nx
    _, F = build_problem(wl, h)
    F_host = F.cpu()
    U = torch.zeros(N, dtype=torch.float64, device="cuda")
    arith = ARITH[args.arith] if wl["pc_prec"] != sg.F64 else sg.ARITH_F64
    opts = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=wl["restart"], maxit=400, tol=wl["tol"],
                pc_prec=wl["pc_prec"], reorth=0, arith=arith)
    for _ in range(args.warmup):
        h.solve(F, U, **opts)
    torch.cuda.synchronize()
    barrier()
    infos = []
    h.timing_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(h.solve(F, U, **opts))
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms_total = e0.elapsed_time(e1)
    phase_ms, phase_launches = h.timing_read()
    h.timing_enable(False)
    clocks = clk.summary()
    t_step = max_over_ranks([ms_total / args.steps])[0]
    its = [i.iters for i in infos]
    relres = max(i.relres_true for i in infos)
    # the outer operator (dominant kernel) per launch, from the per-phase CUDA events of the timed region
    n_k1 = max(int(phase_launches[0]), 1)
    k1_launch_ms = phase_ms[0] / n_k1
    zbytes = {0: 8, 1: 4, 2: 2, 4: 4}[wl["pc_prec"]]
    ybytes = 4 * 2 if arith == sg.ARITH_DF64 else 8           # double-float w: hi + lo arrays
    bytes_k1 = k1_bytes(wl, zbytes, ybytes)
    k1_gbs = bytes_k1 / (k1_launch_ms * 1e-3) / 1e9
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "fallback 6.8 TB/s" if peaks.get("_fallback") else "measured (MEASURED_PEAKS.json hbm_gbs)"
    U_ref = U.clone()

    # end to end through the C ABI with host (pinned) buffers, copies inside the timed region
    Fh = F_host.pin_memory()
    Uh = torch.zeros(N, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    h.solve(Fh.numpy(), Uh.numpy(), **opts)      # warm-up: the first host call allocates its staging buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h.solve(Fh.numpy(), Uh.numpy(), **opts)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    del Fh, Uh

    # SG apply (K1) on its own: algorithmic bytes / median launch time, FP32 and FP64 storage
    apply_gbs = {}
    if not args.no_fp64_compare:
        for name, prec, dt, sb in (("f32", sg.F32, torch.float32, 4), ("f64", sg.F64, torch.float64, 8)):
            X = torch.rand(N, dtype=dt, device="cuda") * 2 - 1
            Y = torch.empty_like(X)
            ms = time_apply(h, X, Y, prec)
            b = k1_bytes(wl, sb, sb)
            apply_gbs[name] = {"ms": round(ms, 4), "gbs": round(b / (ms * 1e-3) / 1e9, 1),
                               "frac_of_hbm": round(b / (ms * 1e-3) / 1e9 / hbm, 4), "bytes": b,
                               "method_tflops": round(k1_method_flops(wl) / (ms * 1e-3) / 1e12, 3)}
            del X, Y

    # the other arithmetic / storage variants of the same solve (labelled context)
    variants = {}
    if args.workload == "c3" and not args.no_fp64_compare:
        for name, o2 in (("double-float Krylov basis and Gram-Schmidt (df64), bf16 levels",
                          dict(opts, arith=sg.ARITH_DF64)),
                         ("f32 levels and z, f64 Krylov", dict(opts, pc_prec=sg.F32)),
                         ("IEEE FP64 outer operator as well (arith f64), bf16 levels", dict(opts, arith=sg.ARITH_F64))):
            U2 = torch.zeros_like(U)
            ms2, i2 = timed_solves(h, F, U2, o2, args.steps, stream)
            variants[name] = {"ms_per_step": round(ms2, 3), "iterations": i2.iters, "relres_true": i2.relres_true,
                              "solution_rel_diff_to_headline": float(torch.linalg.norm(U2 - U_ref) /
                                                                     torch.linalg.norm(U_ref))}
            del U2
    # the same solve in plain FP64 (FP64 preconditioner, FP64 Krylov arithmetic and operator)
    vs64 = None
    if not args.no_fp64_compare and (wl["pc_prec"] != sg.F64 or arith != sg.ARITH_F64):
        U64 = torch.zeros_like(U)
        t64, info64 = timed_solves(h, F, U64, dict(opts, pc_prec=sg.F64, arith=sg.ARITH_F64),
                                   max(1, min(args.steps, 2)), stream)
        vs64 = {"ms_per_step": round(t64, 3), "iterations": info64.iters, "relres_true": info64.relres_true,
                "speedup_of_mixed": round(t64 / t_step, 3),
                "solution_rel_diff": float(torch.linalg.norm(U_ref - U64) / torch.linalg.norm(U64))}
        del U64
    launches_total = sum(phase_launches)
    kr = {sg.ARITH_F64: "f64", sg.ARITH_F64_DFOP: "f64 basis and Gram-Schmidt, double-float outer operator",
          sg.ARITH_DF64: "df64"}[arith]
    out = {
        "metric": METRIC,
        "value": round(t_step / 1e3, 6),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_step, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {sg.ARITH_F64: "f64", sg.ARITH_F64_DFOP: "f64 Krylov (double-float outer operator)",
                  sg.ARITH_DF64: "double-float (fp32x2) Krylov"}[arith]
                 + f", preconditioner {PREC_NAME[wl['pc_prec']]}",
        "data": "synthetic (KL coefficients of the separable exponential covariance, f = 1)",
        "config": {"workload": wl["name"], "n": wl["n"], "M": wl["M"], "p": wl["p"], "P": h.P,
                   "unknowns": N, "restart": wl["restart"], "tol": wl["tol"],
                   "krylov_arith": kr, "pc_prec": PREC_NAME[wl["pc_prec"]],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": (f"inputs larger than L2 ({8 * N / 1e9:.2f} GB per vector), no flush" if 8 * N > 129e6 else
                          "vectors fit in L2 (no flush: small-case timing)")},
        "iterations": its[-1],
        "relres_true": relres,
        "autotune_s": round(t_tune, 3),
        "sg_apply_gbs": apply_gbs or None,
        "phases_ms_per_step": {k: round(v / args.steps, 3) for k, v in
                               zip(["operator", "preconditioner", "gram_schmidt", "other"], phase_ms)},
        "gpu_launches": int(launches_total // max(args.steps, 1)),
        "gpu_launches_timed_region": int(launches_total),
        "e2e": {"value": round(e2e_s, 6), "unit": "s", "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
        "clocks": clocks,
        "vs_plain_fp64": vs64,
        # the Gram-Schmidt kernels are bound by the FP64 FMA rate (2 per SM per clock on GB300), not HBM
        "gram_schmidt_fp64": (lambda f, ms: {
            "fma_per_step": f, "ms_per_step": round(ms, 3),
            "achieved_tfma_s": round(f / (ms * 1e-3) / 1e12, 4),
            "peak_tfma_s": round(2 * 152 * 2.07e9 / 1e12, 4),
            "frac": round(f / (ms * 1e-3) / (2 * 152 * 2.07e9), 4),
            "peak_source": "derived: 2 FP64 FMA per SM per clock x 152 SMs x 2070 MHz"})(
            gs_fp64_fmas(N, its[-1], wl["restart"]) if arith != sg.ARITH_DF64 else 0,
            phase_ms[2] / args.steps) if phase_ms[2] > 0 else None,
        "variants": variants or None,
    }
    # C2's comparison: sigma in {0.1, 0.3, 0.5}, block-triangular vs block-diagonal, FP64 vs FP32
    # preconditioner inside FP64 flexible GMRES (one timed solve each, same grid and chaos space)
    if args.workload == "c2" and not args.no_fp64_compare:
        out["c2_sweep"] = c2_sweep(wl, stream)
    # roofline of the dominant kernel (the outer operator k_apply) by its algorithmic bytes: z read
    # once, w written once, the coefficient rows read once
    names = ["operator", "preconditioner", "gram_schmidt", "other"]
    dom = max(range(4), key=lambda i: phase_ms[i])
    fl = k1_method_flops(wl)
    out["roofline"] = {
        "kernel": {sg.ARITH_F64: "k_apply<ArF64> (outer SG operator, FP64)",
                   sg.ARITH_F64_DFOP: f"k_apply<ArDF, {ZNAME[wl['pc_prec']]} z, f64 w> (outer SG operator)",
                   sg.ARITH_DF64: f"k_apply<ArDF, {ZNAME[wl['pc_prec']]} z, double-float w> (outer SG operator)"}[arith],
        "dominant_phase": names[dom],
        "bound": "hbm",
        "achieved": round(k1_gbs, 1),
        "peak": round(hbm, 1),
        "unit": "GB/s",
        "frac": round(k1_gbs / hbm, 4),
        "peak_source": hbm_src,
        # DRAM bytes of one launch of this kernel in an ncu capture of the 513^2 copy (P = 210, 54,835,410
        # unknowns: 274.03 MB read + 396.30 MB written), scaled to this workload by unknowns; only for
        # the configured form, whose kernel the capture measured
        "traffic": (round(670.34e6 * N / 54835410) if arith == sg.ARITH_F64_DFOP and wl["pc_prec"] == sg.BF16Z
                    else None),
        "traffic_source": "ncu capture of the 513^2 copy, scaled by unknowns",
        "algorithmic_bytes_per_launch": bytes_k1,
        "launch_ms": round(k1_launch_ms, 4),
        "launches": n_k1,
        "diagnostics": {"method_flops_per_launch": fl,
                        "method_tflops": round(fl / (k1_launch_ms * 1e-3) / 1e12, 3),
                        "note": "the double-float operator is bound by FP32 issue (error-free transformations), "
                                "not by HBM; the method's own flops are the FP64 count of the operator"},
    }
    h.close()
    return out


def c2_sweep(wl, stream):
    import torch
    from paper_1304_1755_gb300 import sg
    rows = []
    n, M, p = wl["n"], wl["M"], wl["p"]
    for sigma in (0.1, 0.3, 0.5):
        coef, _ = sg.sg_kl_coef(n, M, sigma)
        amin = sg.sg_min_coef(coef, n, M)               # coercivity at the corners of the xi box
        h = sg.Handle(n, M, p, wl["family"], coef, stream=stream)
        _, F = build_problem(dict(wl, sigma=sigma), h)
        for pc in (sg.PC_BLOCKTRI, sg.PC_BLOCKDIAG):
            for pcp, ar in ((sg.F64, sg.ARITH_F64), (sg.F32, sg.ARITH_F64_DFOP), (sg.F32, sg.ARITH_F64)):
                U = torch.zeros_like(F)
                opts = dict(method=sg.FGMRES, precond=pc, restart=wl["restart"], maxit=400, tol=wl["tol"],
                            pc_prec=pcp, arith=ar, check=False)
                h.solve(F, U, **opts)
                U.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                info = h.solve(F, U, **opts)
                e1.record(stream)
                torch.cuda.synchronize()
                rows.append({"sigma": sigma, "min_a_at_corners": round(amin, 4),
                             "precond": "block-triangular" if pc == sg.PC_BLOCKTRI else "block-diagonal",
                             "pc_prec": {0: "f64", 1: "f32"}[pcp],
                             "krylov": {0: "f64", 2: "f64, double-float operator"}[ar],
                             "status": info.status, "iterations": info.iters, "relres_true": info.relres_true,
                             "ms": round(e0.elapsed_time(e1), 3)})
        h.close()
    return rows


def run_table3(args, wl, rank, world):
    """The five methods of the paper's Table 3 (B-GS, BD-PCG, BT-GPCG, BT-GMRes(10), BS-PCG with the flat
    and the recursive B_S), FP64, on the paper's test problem with Q1 elements and a damped-Jacobi V(2,2)
    (table3) or with the paper's own P1 triangles and point Gauss-Seidel V(2,2), lexicographic or
    red-black (table3p1, table3p1rb); iteration counts and device times, with the paper's counts (P1,
    MATLAB) beside them as context."""
    import numpy as np
    import torch
    from paper_1304_1755_gb300 import build as B
    from paper_1304_1755_gb300 import sg
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    if not os.path.exists(sg.LIB_PATH):
        B.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    paper = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_examples.json")))["table3"]
    n, M, p = wl["n"], wl["M"], wl["p"]
    h1 = 1.0 / (n - 1)
    xs = np.arange(1, n - 1) * h1 - 0.5                      # interior nodes of (-0.5, 0.5)
    X, Y = np.meshgrid(xs, xs)
    f = (2.0 * (0.5 - X ** 2 - Y ** 2)).reshape(-1)
    fdev = torch.as_tensor(f).cuda()
    methods = [("Block-GS", sg.BGS, sg.PC_BLOCKTRI), ("BD-PCG", sg.PCG, sg.PC_BLOCKDIAG),
               ("BT-GPCG", sg.GPCG, sg.PC_BLOCKTRI), ("BT-GMRes", sg.GMRES, sg.PC_BLOCKTRI),
               ("BS-PCG", sg.PCG, sg.PC_BLOCKSYM), ("BS-PCG recursive", sg.PCG, sg.PC_BLOCKSYM_REC)]
    rows, total_ms = [], 0.0
    p1 = wl.get("elements", 0) == sg.P1
    for si, sigma in enumerate(wl["sigmas"]):
        coef, _ = (sg.sg_kl_coef_p1 if p1 else sg.sg_kl_coef)(n, M, sigma)
        h = sg.Handle(n, M, p, wl["family"], coef, nu1=wl["nu"], nu2=wl["nu"], stream=stream,
                      elements=wl.get("elements", 0), gs_order=wl.get("gs_order", 0))
        F = torch.empty(h.P * h.Nx, dtype=torch.float64, device="cuda")
        h.rhs(F, fdev)
        for name, meth, pc in methods:
            U = torch.zeros_like(F)
            o = dict(method=meth, precond=pc, restart=wl["restart"], maxit=1000, tol=wl["tol"], pc_prec=sg.F64,
                     check=False)
            h.solve(F, U, **o)
            U.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            info = h.solve(F, U, **o)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            total_ms += ms
            rows.append({"sigma": sigma, "method": name, "iterations": info.iters, "status": info.status,
                         "relres_true": info.relres_true, "ms": round(ms, 3),
                         "paper_iterations": paper[name.split(" ")[0]][si][0],
                         "paper_cpu_s": paper[name.split(" ")[0]][si][1]})
        h.close()
    return {"metric": "Table 3 methods on the paper's test problem: iterations and time (context)",
            "value": round(total_ms / 1e3, 4), "unit": f"s (all {len(rows)} solves)", "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": round(total_ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (the paper's f and KL setting)",
            "config": {"workload": wl["name"],
                       "smoother": (("lexicographic" if wl["gs_order"] == 0 else "red-black") +
                                    " point Gauss-Seidel V(2,2)") if p1 else "damped Jacobi V(2,2)",
                       "elements": "P1" if p1 else "Q1"},
            "rows": rows, "gpu_launches": None, "e2e": None, "clocks": None, "roofline": None}


def c4_cpu_sample(wl, warmup=0, steps=1):
    """The oracle computing the same gradient on the 129 x 129 copy of the C4 problem: the C/OpenMP
    block-triangular FGMRES forward solve, the transposed solve with the upper sweep, then J and both
    gradients by the Python oracle; scaled to the workload by unknowns.  Returns (seconds,
    description, threads)."""
    from oracle import adjoint as oadj, csolver, kl, mg, sg as osg
    from paper_1304_1755_gb300 import inputs
    nc = 129
    unit = kl.kl_coefficients(nc, wl["M"], 1.0)
    coef = kl.kl_coefficients(nc, wl["M"], wl["sigma"], abar=inputs.lognormal_cells(wl["abar_seed"], nc, 0.2))
    sysm = osg.build(nc, wl["M"], wl["p"], wl["family"], coef)
    F = osg.rhs(sysm)
    c = csolver.CSolver(sysm, mg.Hierarchy(sysm.K[0], nc))
    times, its = [], (0, 0)
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        U, i1, _, _, _ = c.fgmres(F, restart=wl["restart"], maxit=400, tol=wl["tol"])
        _, gU = oadj.objective(sysm, U)
        Lam, i2, _, _, _ = c.fgmres(gU, restart=wl["restart"], maxit=400, tol=wl["tol"], transpose=True)
        oadj.gradients(sysm, U, Lam, unit)
        if k >= warmup:
            times.append(time.perf_counter() - t0)
        its = (i1, i2)
    N = (wl["n"] - 2) ** 2 * math.comb(wl["M"] + wl["p"], wl["p"])
    t = statistics.median(times)
    return t * N / (sysm.P * sysm.Nx), (f"oracle gradient (C/OpenMP BT-FGMRES forward {its[0]} and transposed "
                                        f"{its[1]} iterations, J and both gradients in the Python oracle) on the "
                                        f"{nc}x{nc} copy ({sysm.P * sysm.Nx} unknowns) in {t:.2f} s; scaled by "
                                        f"unknowns"), csolver.threads()


def run_c4(args, wl, rank, world):
    """Time per adjoint gradient: forward block-triangular FGMRES solve, J and dJ/dU, the transpose
    solve (upper sweep) and the gradient kernels, all on the GPU through the C ABI; against the
    plain FP64 forward solve alone."""
    import numpy as np
    import torch
    from paper_1304_1755_gb300 import build as B
    from paper_1304_1755_gb300 import inputs, sg
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    if not os.path.exists(sg.LIB_PATH):
        B.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n, M, p = wl["n"], wl["M"], wl["p"]
    coef, _ = sg.sg_kl_coef(n, M, wl["sigma"], abar=inputs.lognormal_cells(wl["abar_seed"], n, 0.2))
    h = sg.Handle(n, M, p, wl["family"], coef, stream=stream)
    N = h.P * h.Nx
    F = torch.empty(N, dtype=torch.float64, device="cuda")
    h.rhs(F)
    U, G, Lam = torch.zeros_like(F), torch.empty_like(F), torch.zeros_like(F)
    g_abar = torch.empty((n - 1) ** 2, dtype=torch.float64, device="cuda")
    opts = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=wl["restart"], maxit=400, tol=wl["tol"],
                pc_prec=wl["pc_prec"], reorth=0, arith=sg.ARITH_F64_DFOP)

    def gradient():
        fi = h.solve(F, U, **opts)
        J = h.objective(U, G)
        ai = h.solve(G, Lam, transpose=True, **opts)
        gs = h.adjoint_gradients(U, Lam, wl["sigma"], g_abar)
        return fi, ai, J, gs

    for _ in range(args.warmup):
        gradient()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.timing_enable(True)
    with ClockSampler(dev) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            fi, ai, J, gs = gradient()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    t_step = max_over_ranks([e0.elapsed_time(e1) / args.steps])[0]
    clocks = clk.summary()
    _, c4_launches = h.timing_read()
    h.timing_enable(False)
    opts64 = dict(opts, pc_prec=sg.F64, arith=sg.ARITH_F64)
    U64 = torch.zeros_like(F)
    h.solve(F, U64, **opts64)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        i64 = h.solve(F, U64, **opts64)
    e1.record(stream)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / args.steps
    # end to end: host right-hand side in, gradient out
    Fh = F.cpu().pin_memory()
    gh = torch.empty((n - 1) ** 2, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.solve(Fh.numpy(), U, **opts)
    h.objective(U, G)
    h.solve(G, Lam, transpose=True, **opts)
    h.adjoint_gradients(U, Lam, wl["sigma"], g_abar)
    gh.copy_(g_abar)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    out = {
        "metric": C4_METRIC,
        "value": round(t_step / 1e3, 6), "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_step, 3), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 Krylov (double-float outer operator), preconditioner f32",
        "data": "synthetic (lognormal mean coefficient seed 2, KL modes, f = 1)",
        "config": {"workload": wl["name"], "unknowns": N, "parameters": (n - 1) ** 2 + 1,
                   "l2": "vectors fit in L2 (no flush: small-case timing)"},
        "J": J, "dJ_dsigma": gs, "grad_abar_norm": float(torch.linalg.norm(g_abar)),
        "iterations": {"forward": fi.iters, "adjoint": ai.iters},
        "vs_plain_fp64_forward_solve": {"ms_per_step": round(t64, 3), "iterations": i64.iters,
                                        "gradient_over_fp64_solve": round(t_step / t64, 3)},
        "gpu_launches": int(sum(c4_launches)),
        "e2e": {"value": round(t_e2e, 6), "unit": "s", "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 8 * (n - 1) ** 2},
        "clocks": clocks, "roofline": None,
    }
    h.close()
    return out


def c5_systems(wl):
    """The uneven batch: per system (n, M, p, sigma) from the seeded recipe; sigma is lowered where
    needed so that the coefficient stays >= 0.05 at every corner of the xi box (the library's
    sg_min_coef of the unit-sigma fluctuation gives the bound)."""
    import numpy as np
    from paper_1304_1755_gb300 import inputs, sg
    out = []
    for s in inputs.batch_systems(wl["batch_seed"], wl["count"]):
        n, M = s["n"], s["M"]
        unit, _ = sg.sg_kl_coef(n, M, 1.0, abar=np.zeros((n - 1) ** 2))
        worst = -sg.sg_min_coef(unit, n, M)             # max over cells of sqrt3 sum_k |c_k| at sigma = 1
        sigma = min(s["sigma"], 0.95 / worst)
        coef, _ = sg.sg_kl_coef(n, M, sigma)
        out.append(dict(s, sigma=sigma, sigma_drawn=s["sigma"], coef=coef))
    return out


def run_c5(args, wl, rank, world):
    """Aggregate unknowns solved per second for the uneven batch, all systems at once
    (sg_solve_batch, nstreams worker streams) against one at a time (sg_solve in a loop)."""
    import torch
    from paper_1304_1755_gb300 import build as B
    from paper_1304_1755_gb300 import sg
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    if not os.path.exists(sg.LIB_PATH):
        B.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    systems = c5_systems(wl)
    hs = [sg.Handle(s["n"], s["M"], s["p"], wl["family"], s["coef"], stream=stream) for s in systems]
    t0 = time.perf_counter()
    for h in hs:
        h.autotune()
    tune_s = time.perf_counter() - t0
    Fs = []
    for h in hs:
        F = torch.empty(h.P * h.Nx, dtype=torch.float64, device="cuda")
        h.rhs(F)
        Fs.append(F)
    Us = [torch.zeros_like(F) for F in Fs]
    unknowns = sum(int(F.numel()) for F in Fs)
    opts = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=wl["restart"], maxit=400, tol=wl["tol"],
                pc_prec=wl["pc_prec"], reorth=0, arith=sg.ARITH_F64_DFOP)

    def one_at_a_time():
        return [h.solve(F, U, **opts) for h, F, U in zip(hs, Fs, Us)]

    def batched_streams():
        return sg.solve_batch(hs, Fs, Us, nstreams=wl["nstreams"], **opts)

    # the batch's CUDA graphs (every system's restart cycle with its Arnoldi control on the device, the
    # systems side by side) are built once, as set-up; a solve is one launch of the start graph and one
    # launch of the cycle graph per restart cycle of the whole batch
    for h in hs:
        h.timing_read()                                        # launch counters from zero
    t0 = time.perf_counter()
    batch = sg.Batch(hs, Fs, Us, **opts)
    graph_build_s = time.perf_counter() - t0
    graph_kernels = sum(sum(h.timing_read()[1]) for h in hs)   # kernel nodes captured into the graphs

    def batched():
        return batch.solve()

    for _ in range(args.warmup):
        one_at_a_time()
        batched()
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            infos = batched()
        torch.cuda.synchronize()
        barrier()
        t_batch = (time.perf_counter() - t0) / args.steps
    clocks = clk.summary()
    batch.close()
    batched_streams()
    torch.cuda.synchronize()
    for h in hs:
        h.timing_enable(True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        infos_s = batched_streams()
    torch.cuda.synchronize()
    t_streams = (time.perf_counter() - t0) / args.steps
    ph = [h.timing_read() for h in hs]
    for h in hs:
        h.timing_enable(False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        infos1 = one_at_a_time()
    torch.cuda.synchronize()
    t_seq = (time.perf_counter() - t0) / args.steps
    t_batch, t_streams, t_seq = max_over_ranks([t_batch, t_streams, t_seq])
    op_ms = sum(m[0] for m, _ in ph) / args.steps
    op_launches = sum(l[0] for _, l in ph) // args.steps
    # end to end through the C ABI with host (pinned) buffers: sg_solve stages them per system
    Fh = [F.cpu().pin_memory() for F in Fs]
    Uh = [torch.zeros_like(F).pin_memory() for F in Fh]
    batch = sg.Batch(hs, Fs, Us, **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for F, Fp in zip(Fs, Fh):                                  # host -> device, the batch solve, device -> host
        F.copy_(Fp, non_blocking=True)
    batch.solve()
    for U, Up in zip(Us, Uh):
        Up.copy_(U, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    batch.close()
    nbytes = 8 * unknowns
    out = {
        "metric": C5_METRIC,
        "value": round(world * unknowns / t_batch, 1),
        "unit": "unknowns/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_batch * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 Krylov (double-float outer operator), preconditioner f32",
        "data": "synthetic (seeded uneven batch: KL coefficients, Legendre chaos, f = 1)",
        "config": {"workload": wl["name"], "systems": len(hs), "unknowns": unknowns,
                   "batched_form": "one CUDA graph: per system a chain of conditional steps with the Arnoldi "
                                   "control on the device; one launch per restart cycle of the whole batch",
                   "sigma_lowered": sum(1 for s in systems if s["sigma"] < s["sigma_drawn"]),
                   "l2": "working set of the batch larger than L2, no flush"},
        "one_at_a_time": {"value": round(world * unknowns / t_seq, 1), "unit": "unknowns/s",
                          "ms_per_step": round(t_seq * 1e3, 3)},
        "host_streams": {"value": round(world * unknowns / t_streams, 1), "unit": "unknowns/s",
                         "ms_per_step": round(t_streams * 1e3, 3), "nstreams": wl["nstreams"],
                         "iterations_equal": all(i.iters == j.iters for i, j in zip(infos_s, infos1))},
        "batch_speedup": round(t_seq / t_batch, 3),
        "iterations": [i.iters for i in infos],
        "restart_cycles_max": max(i.restarts for i in infos) + 1,
        "relres_true_max": max(i.relres_true for i in infos),
        "iterations_within_one_of_one_at_a_time": all(abs(i.iters - j.iters) <= 1 for i, j in zip(infos, infos1)),
        "autotune_s": round(tune_s, 3),
        "graph_build_s": round(graph_build_s, 3),
        "graph_launches_per_step": 1 + max(i.restarts for i in infos) + 1,
        "gpu_launches": int(graph_kernels),
        "gpu_launches_note": "kernel nodes in the batch's two graphs (the steps a system skips are not run)",
        "e2e": {"value": round(world * unknowns / t_e2e, 1), "unit": "unknowns/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "clocks": clocks,
    }
    # the outer operator (double-float arithmetic, FP32 z in, FP64 w out): one apply per system, bytes
    # by the algorithmic count of each system, time = the mean event-timed launch over the batch
    byt = sum(k1_bytes(dict(n=s["n"], M=s["M"], p=s["p"]), 4, 8) for s in systems)
    apply_ms = op_ms / max(op_launches, 1) * len(hs)
    hbm = _peaks().get("hbm_gbs", 6800.0)
    out["roofline"] = {"kernel": "k_apply<ArDF, f32 z, f64 w> (outer SG operator), summed over the batch's systems",
                       "bound": "hbm", "achieved": round(byt / (apply_ms * 1e-3) / 1e9, 1), "peak": hbm,
                       "unit": "GB/s", "frac": round(byt / (apply_ms * 1e-3) / 1e9 / hbm, 4), "traffic": None,
                       "note": "launch time measured per system with events; concurrent streams overlap"}
    for h in hs:
        h.close()
    return out


def _cores_c():
    from oracle import csolver
    return csolver.threads()


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class CpuSampleBatch:
    """The oracle's C/OpenMP BT-FGMRES on a bounded sample of the uneven batch: its systems on
    the 65 x 65 grid, solved one after another until about 20 s have been spent; the metric is
    unknowns solved per second."""

    def __init__(self, wl, budget_s=20.0):
        from oracle import csolver, mg, sg as osg
        self.wl, self.budget_s = wl, budget_s
        self.items = []
        for s in c5_systems(wl):
            if s["n"] != 65:
                continue
            sysm = osg.build(s["n"], s["M"], s["p"], wl["family"], s["coef"])
            c = csolver.CSolver(sysm, mg.Hierarchy(sysm.K[0], s["n"]))
            self.items.append((sysm, c, osg.rhs(sysm)))

    def run(self):
        t0 = time.perf_counter()
        done = 0
        count = 0
        for sysm, c, F in self.items:
            c.fgmres(F, restart=self.wl["restart"], maxit=400, tol=self.wl["tol"])
            done += sysm.P * sysm.Nx
            count += 1
            if time.perf_counter() - t0 > self.budget_s:
                break
        dt = time.perf_counter() - t0
        return done / dt, (f"oracle C/OpenMP BT-FGMRES({self.wl['restart']}) to {self.wl['tol']:g} on {count} of "
                           f"the batch's 65x65 systems ({done} unknowns) in {dt:.1f} s, one after another")


class CpuSample:
    """The oracle's plain C/OpenMP FP64 BT-FGMRES + V(1,1) (oracle/csolve.c, the Python oracle's
    matrices, all host cores) on a bounded sample of the workload: the same M, p, family, sigma,
    right-hand side, restart and tolerance, a full solve from U = 0, on the workload's own grid
    when it has at most 513^2 vertices (C2: timed in full) and on the 513^2 copy otherwise (C3),
    scaled to the workload by unknowns (multigrid-preconditioned iteration counts do not grow
    with the grid)."""

    def __init__(self, wl):
        from oracle import csolver, kl, mg, sg as osg
        from paper_1304_1755_gb300 import inputs
        self.n = min(wl["n"], 513)
        self.wl = wl
        t0 = time.perf_counter()
        coef = kl.kl_coefficients(self.n, wl["M"], wl["sigma"])
        self.s = osg.build(self.n, wl["M"], wl["p"], wl["family"], coef)
        f = None if wl.get("f_seed") is None or self.n != wl["n"] else inputs.rhs_nodes(wl["f_seed"], self.n)
        self.F = osg.rhs(self.s, f)
        self.c = csolver.CSolver(self.s, mg.Hierarchy(self.s.K[0], self.n))
        self.cores = csolver.threads()
        self.setup_s = time.perf_counter() - t0

    def run(self):
        """One full solve; returns (seconds, iterations)."""
        _, its, rr, rc, dt = self.c.fgmres(self.F, restart=self.wl["restart"], maxit=400, tol=self.wl["tol"])
        self.relres = rr
        return dt, max(its, 1)

    @property
    def unknowns(self):
        return self.s.P * self.s.Nx

    def scaled(self, dt, unknowns):
        return dt * unknowns / self.unknowns

    def describe(self, dt, its):
        where = "the workload itself" if self.n == self.wl["n"] else f"the {self.n}x{self.n} copy, scaled by unknowns"
        return (f"oracle C/OpenMP FP64 BT-FGMRES({self.wl['restart']}) + V(1,1) to {self.wl['tol']:g} on {where} "
                f"(P={self.s.P}, {self.unknowns} unknowns): {its} iterations in {dt:.2f} s on {self.cores} threads "
                f"(+{self.setup_s:.1f} s set-up by the Python oracle)")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--arith", default="f64dfop", choices=sorted(ARITH))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--pc-prec", choices=["f64", "f32", "bf16", "bf16z"], default=None,
                    help="override the workload's preconditioner storage precision")
    ap.add_argument("--apply-only", action="store_true",
                    help="time only the SG apply (FP32, FP64 and double-float sg_apply) of the workload's "
                         "problem and print its line (for kernel profiling)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.pc_prec is not None:
        wl["pc_prec"] = {"f64": 0, "f32": 1, "bf16": 2, "bf16z": 4}[args.pc_prec]
        wl["name"] += f"_pc_{args.pc_prec}"
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload in ("table3", "table3p1", "table3p1rb", "c3s"):
            print(json.dumps({"impl": "reference", "unavailable": f"{args.workload} is a context/profiling workload "
                                                                   "without a reference timing"}))
            return
        common = {"impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                  "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                  "config": {"workload": wl["name"]}}
        if args.workload == "c4":
            v, sample, cores = c4_cpu_sample(wl, args.warmup, args.steps)
            print(json.dumps(dict(common, metric=C4_METRIC, value=round(v, 3), unit="s", higher_is_better=False,
                                  cpu_baseline={"value": round(v, 3), "unit": "s", "cores": cores, "kind": "oracle",
                                                "sample": sample},
                                  e2e={"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0})))
            return
        if args.workload == "c5":
            smp = CpuSampleBatch(wl)
            vals = []
            for k in range(args.warmup + args.steps):
                v, sample = smp.run()
                if k >= args.warmup:
                    vals.append(v)
            v = statistics.median(vals)
            print(json.dumps(dict(common, metric=C5_METRIC, value=round(v, 1), unit="unknowns/s", higher_is_better=True,
                                  cpu_baseline={"value": round(v, 1), "unit": "unknowns/s", "cores": _cores_c(),
                                                "kind": "oracle", "sample": sample},
                                  e2e={"value": round(v, 1), "unit": "unknowns/s", "h2d_bytes_per_step": 0,
                                       "d2h_bytes_per_step": 0})))
            return
        smp = CpuSample(wl)
        times = []
        for k in range(args.warmup + args.steps):
            dt, its = smp.run()
            if k >= args.warmup:
                times.append(dt)
        n, P = wl["n"], math.comb(wl["M"] + wl["p"], wl["p"])
        unknowns = (n - 2) ** 2 * P
        dt = statistics.median(times)
        v = smp.scaled(dt, unknowns)
        print(json.dumps(dict(common, metric=METRIC, value=round(v, 3), unit="s", ms_per_step=round(v * 1e3, 1),
                              higher_is_better=False,
                              data="synthetic (KL coefficients of the separable exponential covariance, f = 1)",
                              config={"workload": wl["name"], "unknowns": unknowns},
                              cpu_baseline={"value": round(v, 3), "unit": "s", "cores": smp.cores, "kind": "oracle",
                                            "sample": smp.describe(dt, its)},
                              e2e={"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0,
                                   "d2h_bytes_per_step": 0})))
        return
    if args.apply_only:
        print(json.dumps(run_apply_only(args, wl)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.workload in ("table3", "table3p1", "table3p1rb"):
        out = run_table3(args, wl, rank, world)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload == "c4":
        out = run_c4(args, wl, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            v, sample, cores = c4_cpu_sample(wl)
            out["cpu_baseline"] = {"value": round(v, 3), "unit": "s", "cores": cores, "kind": "oracle",
                                   "sample": sample}
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload == "c5":
        out = run_c5(args, wl, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            v, sample = CpuSampleBatch(wl).run()
            out["cpu_baseline"] = {"value": round(v, 1), "unit": "unknowns/s", "cores": _cores_c(), "kind": "oracle",
                                   "sample": sample}
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    out = run_ours(args, wl, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = CpuSample(wl)
        dt, its = smp.run()
        v = smp.scaled(dt, out["config"]["unknowns"])
        out["cpu_baseline"] = {"value": round(v, 3), "unit": "s", "cores": smp.cores, "kind": "oracle",
                               "sample": smp.describe(dt, its), "host_cores": _host_cores()}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
