#!/usr/bin/env python
"""Benchmark: time to relative residual 1e-8 of block-triangular FGMRES + multigrid,
and the SG-apply HBM bandwidth, on one GB300 (replicas on N GPUs).

Default workload ("c3", the bandwidth-scale solve): 1025 x 1025 Q1 grid
(1,046,529 interior nodes), M = 6 Hermite KL terms (sigma = 0.2, separable
exponential covariance, correlation length 1), total degree p = 4 (P = 210),
219,771,090 unknowns; FGMRES(20) with a double-float (FP64-class) Krylov basis and
the block-triangular preconditioner whose V(1,1) cycles store their levels in BF16
and compute in FP32 (stage right-hand sides and the preconditioned vectors z_j in
FP32); f = 1; tolerance 1e-8 on the true relative residual, recomputed in IEEE FP64.  A step is one full solve from
U = 0 with F resident in HBM.  Every vector is 1.76 GB (> L2), so no L2 flush
is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c1] [--impl ours|reference]

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


def build_problem(wl):
    import numpy as np
    from paper_1304_1755_gb300 import inputs, sg
    coef, _ = sg.sg_kl_coef(wl["n"], wl["M"], wl["sigma"])
    n = wl["n"]
    Nx = (n - 2) ** 2
    P = math.comb(wl["M"] + wl["p"], wl["p"])
    f = np.ones(Nx) if wl["f_seed"] is None else inputs.rhs_nodes(wl["f_seed"], n)
    F = np.zeros(P * Nx)
    F[:Nx] = f / (n - 1) ** 2           # F = e_0 (x) h^2 f  (lumped load vector)
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


def k1_flops(wl, df):
    """Algorithmic flops of one outer-operator launch.  FP64: N (8 (1 + r) + r + 16) (corner mixing,
    per-cell weights, element matrix and accumulation).  Double-float: the FP32 flops (add, multiply
    = 1, fused multiply-add = 2) of the exact feature-domain scheme, 83 per coupling (exact features
    38, three compensated products 45) plus 116 per unknown (features 32, node sums 84)."""
    n = wl["n"]
    N = (n - 2) ** 2 * math.comb(wl["M"] + wl["p"], wl["p"])
    t = terms_per_row(wl)
    return N * (83 * t + 116) if df else N * (8 * t + (t - 1) + 16)


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
    coef, F_host = build_problem(wl)
    h = sg.Handle(wl["n"], wl["M"], wl["p"], wl["family"], coef, stream=stream)
    t_tune = time.perf_counter()
    h.autotune()                          # operator tile per arithmetic (set-up, outside the timed region)
    t_tune = time.perf_counter() - t_tune
    N = h.P * h.Nx
    F = torch.as_tensor(F_host).cuda()
    U = torch.zeros(N, dtype=torch.float64, device="cuda")
    arith = sg.ARITH_DF64 if (args.arith == "df64" and wl["pc_prec"] != sg.F64) else sg.ARITH_F64
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
    # parity at full size: independent residual check of the last solution on sampled rows is in
    # tests/; here record the library's own recomputed FP64 residual
    its = [i.iters for i in infos]
    relres = max(i.relres_true for i in infos)
    # SG-apply (outer FP64 operator on the BF16/FP32/FP64 preconditioned vector) per launch
    n_k1 = max(int(phase_launches[0]), 1)                # operator launches in the timed region
    k1_launch_ms = phase_ms[0] / max(n_k1, 1)
    bytes_k1 = k1_bytes(wl, {0: 8, 1: 4, 2: 2, 4: 4}[wl["pc_prec"]], 8)
    k1_gbs = bytes_k1 / (k1_launch_ms * 1e-3) / 1e9
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)

    # end to end through the C ABI with host (pinned) buffers, copies inside the timed region
    Fh = torch.as_tensor(F_host).pin_memory()
    Uh = torch.zeros(N, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    h.solve(Fh.numpy(), Uh.numpy(), **opts)      # warm-up: the first host call allocates its staging buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h.solve(Fh.numpy(), Uh.numpy(), **opts)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    # the other preconditioner storage variants of the same solve (context for the precision choice)
    variants = {}
    if args.workload == "c3" and not args.no_fp64_compare:
        for name, pcp in (("bf16 levels, bf16 z", sg.BF16), ("f32 levels, f32 z", sg.F32)):
            o2 = dict(opts, pc_prec=pcp)
            U2 = torch.zeros_like(U)
            h.solve(F, U2, **o2)
            torch.cuda.synchronize()
            e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e2.record(stream)
            for _ in range(args.steps):
                i2 = h.solve(F, U2, **o2)
            e3.record(stream)
            torch.cuda.synchronize()
            variants[name] = {"ms_per_step": round(e2.elapsed_time(e3) / args.steps, 3), "iterations": i2.iters,
                              "relres_true": i2.relres_true}
            del U2
    # the same solve in plain FP64 (FP64 preconditioner, FP64 Krylov arithmetic) on the same GPU
    vs64 = None
    if not args.no_fp64_compare and (wl["pc_prec"] != sg.F64 or arith != sg.ARITH_F64):
        opts64 = dict(opts, pc_prec=sg.F64, arith=sg.ARITH_F64)
        U64 = torch.zeros_like(U)
        h.solve(F, U64, **opts64)
        torch.cuda.synchronize()
        n64 = max(1, min(args.steps, 2))
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(n64):
            info64 = h.solve(F, U64, **opts64)
        e3.record(stream)
        torch.cuda.synchronize()
        t64 = e2.elapsed_time(e3) / n64
        h.solve(F, U, **opts)
        torch.cuda.synchronize()
        vs64 = {"ms_per_step": round(t64, 3), "iterations": info64.iters, "relres_true": info64.relres_true,
                "speedup_of_mixed": round(t64 / t_step, 3),
                "solution_rel_diff": float(torch.linalg.norm(U - U64) / torch.linalg.norm(U64))}
        del U64
    launches_total = sum(phase_launches)
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
        "dtype": ("f64 storage, double-float (fp32x2) Krylov arithmetic" if arith == sg.ARITH_DF64 else "f64")
                 + f", preconditioner {PREC_NAME[wl['pc_prec']]}",
        "data": "synthetic (KL coefficients of the separable exponential covariance, f = 1)",
        "config": {"workload": wl["name"], "n": wl["n"], "M": wl["M"], "p": wl["p"], "P": h.P,
                   "unknowns": N, "restart": wl["restart"], "tol": wl["tol"],
                   "krylov_arith": "df64" if arith == sg.ARITH_DF64 else "f64",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": (f"inputs larger than L2 ({8 * N / 1e9:.2f} GB per vector), no flush" if 8 * N > 129e6 else
                          "vectors fit in L2 (no flush: small-case timing)")},
        "iterations": its[-1],
        "relres_true": relres,
        "autotune_s": round(t_tune, 3),
        "sg_apply_gbs": round(k1_gbs, 1),
        "phases_ms_per_step": {k: round(v / args.steps, 3) for k, v in
                               zip(["operator", "preconditioner", "gram_schmidt", "other"], phase_ms)},
        "gpu_launches": int(launches_total),
        "e2e": {"value": round(e2e_s, 6), "unit": "s", "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
        "clocks": clocks,
        "vs_plain_fp64": vs64,
        "preconditioner_variants": variants or None,
    }
    # C2's comparison: sigma in {0.1, 0.3, 0.5}, block-triangular vs block-diagonal, FP64 vs FP32
    # preconditioner inside FP64 flexible GMRES (one timed solve each, same grid and chaos space)
    if args.workload == "c2" and not args.no_fp64_compare:
        out["c2_sweep"] = c2_sweep(wl, stream)
    # roofline of the dominant kernel, the outer operator (k_apply): it is bound by arithmetic
    # (double-float: FP32 pipe; strict mode: FP64 units), not by HBM, on GB300
    names = ["operator", "preconditioner", "gram_schmidt", "other"]
    dom = max(range(4), key=lambda i: phase_ms[i])
    df = arith == sg.ARITH_DF64
    fl = k1_flops(wl, df)
    achieved = fl / (k1_launch_ms * 1e-3) / 1e12
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12 if df else 1.25
    out["roofline"] = {
        "kernel": (f"k_apply<ArDF, {ZNAME[wl['pc_prec']]} z, double-float w> (outer SG operator)" if df else
                   "k_apply<ArF64> (outer SG operator, FP64)"),
        "dominant_phase": names[dom],
        "bound": "alu",
        "achieved": round(achieved, 2),
        "peak": round(peak, 2),
        "unit": "TFLOP/s",
        "frac": round(achieved / peak, 4),
        # DRAM bytes of one launch from the ncu capture of this kernel on the 513^2 copy of C3
        # (profiles/k_apply_df_outer_operator_c3s_513sq_P210.md: 272.98 MB read + 391.96 MB written for
        # 54,835,410 unknowns, 12.13 B per unknown), scaled to this workload's unknowns
        "traffic": (round(12.126 * h.P * h.Nx) if df and wl["pc_prec"] in (sg.F32, sg.BF16Z) else None),
        "traffic_unit": "bytes",
        "launch_ms": round(k1_launch_ms, 4),
        "flops_per_launch": fl,
        "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock (FP32 flops of the "
                        "double-float scheme)") if df else "nominal FP64 1.25 TFLOP/s (profiling recipe)",
        "hbm_gbs": round(k1_gbs, 1),
        "hbm_frac_of_measured": round(k1_gbs / hbm, 4),
    }
    h.close()
    return out


def c2_sweep(wl, stream):
    import numpy as np
    import torch
    from paper_1304_1755_gb300 import sg
    rows = []
    n, M, p = wl["n"], wl["M"], wl["p"]
    unit, _ = sg.sg_kl_coef(n, M, 1.0)
    _, F_host = build_problem(wl)
    for sigma in (0.1, 0.3, 0.5):
        coef = unit.copy()
        coef[0] = 1.0
        coef[1:] *= sigma
        amin = float(np.min(1.0 - np.sqrt(3.0) * np.abs(coef[1:]).sum(axis=0)))
        h = sg.Handle(n, M, p, wl["family"], coef, stream=stream)
        F = torch.as_tensor(F_host).cuda()
        for pc in (sg.PC_BLOCKTRI, sg.PC_BLOCKDIAG):
            for pcp, ar in ((sg.F64, sg.ARITH_F64), (sg.F32, sg.ARITH_F64), (sg.F32, sg.ARITH_DF64)):
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
                             "pc_prec": {0: "f64", 1: "f32"}[pcp], "krylov": "df64" if ar else "f64",
                             "status": info.status, "iterations": info.iters, "relres_true": info.relres_true,
                             "ms": round(e0.elapsed_time(e1), 3)})
        h.close()
    return rows


def run_table3(args, wl, rank, world):
    """The five methods of the paper's Table 3 (B-GS, BD-PCG, BT-GPCG, BT-GMRes(10), BS-PCG), FP64, on
    this repository's Q1 / damped-Jacobi V(2,2) discretisation of the paper's test problem; iteration
    counts and device times, with the paper's counts (P1 triangles, point Gauss-Seidel V(2,2), MATLAB)
    beside them as context."""
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
    unit, _ = sg.sg_kl_coef(n, M, 1.0)
    methods = [("Block-GS", sg.BGS, sg.PC_BLOCKTRI), ("BD-PCG", sg.PCG, sg.PC_BLOCKDIAG),
               ("BT-GPCG", sg.GPCG, sg.PC_BLOCKTRI), ("BT-GMRes", sg.GMRES, sg.PC_BLOCKTRI),
               ("BS-PCG", sg.PCG, sg.PC_BLOCKSYM)]
    rows, total_ms = [], 0.0
    for si, sigma in enumerate(wl["sigmas"]):
        coef = unit.copy()
        coef[0] = 1.0
        coef[1:] *= sigma
        h = sg.Handle(n, M, p, wl["family"], coef, nu1=wl["nu"], nu2=wl["nu"], stream=stream)
        F = torch.zeros(h.P * h.Nx, dtype=torch.float64, device="cuda")
        F[:h.Nx] = torch.as_tensor(f * h1 * h1)
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
                         "paper_iterations": paper[name][si][0], "paper_cpu_s": paper[name][si][1]})
        h.close()
    return {"metric": "Table 3 methods on the paper's test problem: iterations and time (context)",
            "value": round(total_ms / 1e3, 4), "unit": "s (all 20 solves)", "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": round(total_ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (the paper's f and KL setting)",
            "config": {"workload": wl["name"], "smoother": "damped Jacobi V(2,2)", "elements": "Q1"},
            "rows": rows, "gpu_launches": None, "e2e": None, "clocks": None, "roofline": None}


def c4_cpu_sample(wl, warmup=0, steps=1):
    """The oracle (as it stands) computing the same gradient on the 129 x 129 copy of the C4 problem:
    block-triangular FGMRES forward solve, the transposed solve with the upper sweep, J and both
    gradients; scaled to the workload by unknowns.  Returns (seconds, description)."""
    from oracle import adjoint as oadj, kl, krylov, mg, precond, sg as osg
    from paper_1304_1755_gb300 import inputs
    nc = 129
    unit = kl.kl_coefficients(nc, wl["M"], 1.0)
    coef = unit.copy()
    coef[0] = inputs.lognormal_cells(wl["abar_seed"], nc, 0.2)
    coef[1:] *= wl["sigma"]
    sysm = osg.build(nc, wl["M"], wl["p"], wl["family"], coef)
    A = osg.assemble(sysm)
    F = osg.rhs(sysm)
    solver = precond.DiagSolver(sysm.K[0], mg.Hierarchy(sysm.K[0], nc))
    times, its = [], (0, 0)
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        U, i1, _ = krylov.gmres(lambda v: A @ v, lambda r: precond.block_tri_inv(sysm, solver, r), F,
                                tol=wl["tol"], restart=wl["restart"], maxit=400, flexible=True)
        _, gU = oadj.objective(sysm, U)
        Lam, i2, _ = krylov.gmres(lambda v: A.T @ v,
                                  lambda r: precond.block_tri_inv(sysm, solver, r, transpose=True), gU,
                                  tol=wl["tol"], restart=wl["restart"], maxit=400, flexible=True)
        oadj.gradients(sysm, U, Lam, unit)
        if k >= warmup:
            times.append(time.perf_counter() - t0)
        its = (i1, i2)
    N = (wl["n"] - 2) ** 2 * math.comb(wl["M"] + wl["p"], wl["p"])
    t = statistics.median(times)
    return t * N / (sysm.P * sysm.Nx), (f"oracle gradient (BT-FGMRES forward {its[0]} and transposed {its[1]} "
                                        f"iterations, J, both gradients) on the {nc}x{nc} copy "
                                        f"({sysm.P * sysm.Nx} unknowns) in {t:.2f} s; scaled by unknowns")


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
    unit, _ = sg.sg_kl_coef(n, M, 1.0)
    coef = unit.copy()
    coef[0] = inputs.lognormal_cells(wl["abar_seed"], n, 0.2)
    coef[1:] *= wl["sigma"]
    h = sg.Handle(n, M, p, wl["family"], coef, stream=stream)
    N = h.P * h.Nx
    F = torch.zeros(N, dtype=torch.float64, device="cuda")
    F[:h.Nx] = 1.0 / (n - 1) ** 2
    U, G, Lam = torch.zeros_like(F), torch.empty_like(F), torch.zeros_like(F)
    g_abar = torch.empty((n - 1) ** 2, dtype=torch.float64, device="cuda")
    opts = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=wl["restart"], maxit=400, tol=wl["tol"],
                pc_prec=wl["pc_prec"], reorth=0, arith=sg.ARITH_DF64)

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
        "dtype": "f64 storage, double-float Krylov arithmetic, preconditioner f32",
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
    needed so that the coefficient stays >= 0.05 at every corner of the xi box (Legendre:
    abar - sqrt(3) sum_k |c_k| >= 0.05 per cell)."""
    import numpy as np
    from paper_1304_1755_gb300 import inputs, sg
    out = []
    for s in inputs.batch_systems(wl["batch_seed"], wl["count"]):
        unit, _ = sg.sg_kl_coef(s["n"], s["M"], 1.0)
        worst = float(np.max(np.sqrt(3.0) * np.abs(unit[1:]).sum(axis=0)))
        sigma = min(s["sigma"], 0.95 / worst)
        coef = unit.copy()
        coef[0] = 1.0
        coef[1:] *= sigma
        n = s["n"]
        F = np.zeros(math.comb(s["M"] + s["p"], s["p"]) * (n - 2) ** 2)
        F[:(n - 2) ** 2] = 1.0 / (n - 1) ** 2
        out.append(dict(s, sigma=sigma, sigma_drawn=s["sigma"], coef=coef, F=F))
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
    Fs = [torch.as_tensor(s["F"]).cuda() for s in systems]
    Us = [torch.zeros_like(F) for F in Fs]
    unknowns = sum(int(F.numel()) for F in Fs)
    opts = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=wl["restart"], maxit=400, tol=wl["tol"],
                pc_prec=wl["pc_prec"], reorth=0, arith=sg.ARITH_F64)

    def one_at_a_time():
        return [h.solve(F, U, **opts) for h, F, U in zip(hs, Fs, Us)]

    def batched():
        return sg.solve_batch(hs, Fs, Us, nstreams=wl["nstreams"], **opts)

    for _ in range(args.warmup):
        one_at_a_time()
        batched()
    torch.cuda.synchronize()
    for h in hs:
        h.timing_enable(True)
    barrier()
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            infos = batched()
        torch.cuda.synchronize()
        barrier()
        t_batch = (time.perf_counter() - t0) / args.steps
    clocks = clk.summary()
    ph = [h.timing_read() for h in hs]
    for h in hs:
        h.timing_enable(False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        infos1 = one_at_a_time()
    torch.cuda.synchronize()
    t_seq = (time.perf_counter() - t0) / args.steps
    t_batch, t_seq = max_over_ranks([t_batch, t_seq])
    launches = sum(sum(l) for _, l in ph) // args.steps
    op_ms = sum(m[0] for m, _ in ph) / args.steps
    op_launches = sum(l[0] for _, l in ph) // args.steps
    # end to end through the C ABI with host (pinned) buffers: sg_solve stages them per system
    Fh = [torch.as_tensor(s["F"]).pin_memory() for s in systems]
    Uh = [torch.zeros_like(F).pin_memory() for F in Fh]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sg.solve_batch(hs, [F.numpy() for F in Fh], [U.numpy() for U in Uh], nstreams=wl["nstreams"], **opts)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    nbytes = 8 * unknowns
    out = {
        "metric": C5_METRIC,
        "value": round(world * unknowns / t_batch, 1),
        "unit": "unknowns/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_batch * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 Krylov, preconditioner f32",
        "data": "synthetic (seeded uneven batch: KL coefficients, Legendre chaos, f = 1)",
        "config": {"workload": wl["name"], "systems": len(hs), "unknowns": unknowns, "nstreams": wl["nstreams"],
                   "sigma_lowered": sum(1 for s in systems if s["sigma"] < s["sigma_drawn"]),
                   "l2": "working set of the batch larger than L2, no flush"},
        "one_at_a_time": {"value": round(world * unknowns / t_seq, 1), "unit": "unknowns/s",
                          "ms_per_step": round(t_seq * 1e3, 3)},
        "batch_speedup": round(t_seq / t_batch, 3),
        "iterations": [i.iters for i in infos],
        "relres_true_max": max(i.relres_true for i in infos),
        "agree_with_one_at_a_time": all(i.iters == j.iters for i, j in zip(infos, infos1)),
        "autotune_s": round(tune_s, 3),
        "gpu_launches": int(launches),
        "e2e": {"value": round(world * unknowns / t_e2e, 1), "unit": "unknowns/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "clocks": clocks,
    }
    fl = sum(k1_flops(dict(n=s["n"], M=s["M"], p=s["p"]), False) for s in systems)   # one apply per system
    apply_ms = op_ms / max(op_launches, 1) * len(hs)
    out["roofline"] = {"kernel": "k_apply<ArF64> (outer SG operator, FP64), summed over the batch's systems",
                       "bound": "alu", "achieved": round(fl / (apply_ms * 1e-3) / 1e12, 3), "peak": 1.25,
                       "unit": "TFLOP/s", "frac": round(fl / (apply_ms * 1e-3) / 1e12 / 1.25, 4), "traffic": None,
                       "peak_source": "nominal FP64 1.25 TFLOP/s (profiling recipe)",
                       "note": "launch time measured per system with events; concurrent streams overlap"}
    for h in hs:
        h.close()
    return out


class CpuSampleBatch:
    """The oracle on a bounded sample of the uneven batch: its systems on the 65 x 65 grid, solved
    one after another by the oracle's block-triangular FGMRES, until about 20 s have been spent;
    the metric is unknowns solved per second."""

    def __init__(self, wl, budget_s=20.0):
        from oracle import mg, precond, sg as osg
        self.wl, self.budget_s = wl, budget_s
        self.items = []
        for s in c5_systems(wl):
            if s["n"] != 65:
                continue
            sysm = osg.build(s["n"], s["M"], s["p"], wl["family"], s["coef"])
            A = osg.assemble(sysm)
            solver = precond.DiagSolver(sysm.K[0], mg.Hierarchy(sysm.K[0], s["n"]))
            self.items.append((sysm, A, osg.rhs(sysm), solver))

    def run(self):
        from oracle import krylov, precond
        t0 = time.perf_counter()
        done = 0
        count = 0
        for sysm, A, F, solver in self.items:
            krylov.gmres(lambda v: A @ v, lambda r: precond.block_tri_inv(sysm, solver, r), F, tol=self.wl["tol"],
                         restart=self.wl["restart"], maxit=400, flexible=True)
            done += sysm.P * sysm.Nx
            count += 1
            if time.perf_counter() - t0 > self.budget_s:
                break
        dt = time.perf_counter() - t0
        return done / dt, f"oracle BT-FGMRES({self.wl['restart']}) to {self.wl['tol']:g} on {count} of the batch's " \
                          f"65x65 systems ({done} unknowns) in {dt:.1f} s, one after another"


class CpuSample:
    """The oracle (as it stands, single-threaded scipy sparse kernels) on a bounded sample of the
    workload: the same M, p, family, sigma, restart and tolerance on a smaller grid copy
    (129 x 129 for the large workloads), a full block-triangular FGMRES solve from U = 0.
    Multigrid-preconditioned iteration counts do not grow with the grid, so the sample is scaled
    to the workload by its time per (unknown x iteration)."""

    def __init__(self, wl):
        from oracle import kl, mg, precond, sg as osg
        self.n = min(wl["n"], 129)
        self.wl = wl
        t0 = time.perf_counter()
        coef = kl.kl_coefficients(self.n, wl["M"], wl["sigma"])
        self.s = osg.build(self.n, wl["M"], wl["p"], wl["family"], coef)
        self.A = osg.assemble(self.s)
        self.F = osg.rhs(self.s)
        self.solver = precond.DiagSolver(self.s.K[0], mg.Hierarchy(self.s.K[0], self.n))
        self.setup_s = time.perf_counter() - t0

    def run(self):
        """One full solve; returns (seconds, iterations)."""
        from oracle import krylov, precond
        s, A = self.s, self.A
        t0 = time.perf_counter()
        _, its, _ = krylov.gmres(lambda v: A @ v, lambda r: precond.block_tri_inv(s, self.solver, r), self.F,
                                 tol=self.wl["tol"], restart=self.wl["restart"], maxit=400, flexible=True)
        return time.perf_counter() - t0, max(its, 1)

    @property
    def unknowns(self):
        return self.s.P * self.s.Nx

    def describe(self, dt, its):
        return (f"oracle BT-FGMRES({self.wl['restart']}) to {self.wl['tol']:g} on the {self.n}x{self.n} copy "
                f"(P={self.s.P}, {self.unknowns} unknowns): {its} iterations in {dt:.1f} s "
                f"(+{self.setup_s:.1f} s set-up); scaled by unknowns x iterations")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--arith", default="df64", choices=["f64", "df64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--pc-prec", choices=["f64", "f32", "bf16", "bf16z"], default=None,
                    help="override the workload's preconditioner storage precision")
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
        if args.workload in ("table3", "c3s"):
            print(json.dumps({"impl": "reference", "unavailable": f"{args.workload} is a context/profiling workload "
                                                                   "without a reference timing"}))
            return
        if args.workload == "c4":
            v, sample = c4_cpu_sample(wl, args.warmup, args.steps)
            print(json.dumps({"impl": "reference", "metric": C4_METRIC, "value": round(v, 3), "unit": "s",
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
                              "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                              "config": {"workload": wl["name"]},
                              "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": 1, "kind": "oracle",
                                               "sample": sample},
                              "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0,
                                      "d2h_bytes_per_step": 0}}))
            return
        if args.workload == "c5":
            smp = CpuSampleBatch(wl)
            vals = []
            for k in range(args.warmup + args.steps):
                v, sample = smp.run()
                if k >= args.warmup:
                    vals.append(v)
            v = statistics.median(vals)
            print(json.dumps({"impl": "reference", "metric": C5_METRIC, "value": round(v, 1), "unit": "unknowns/s",
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                              "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                              "config": {"workload": wl["name"]},
                              "cpu_baseline": {"value": round(v, 1), "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                                               "sample": sample},
                              "e2e": {"value": round(v, 1), "unit": "unknowns/s", "h2d_bytes_per_step": 0,
                                      "d2h_bytes_per_step": 0}}))
            return
        smp = CpuSample(wl)
        times = []
        for k in range(args.warmup + args.steps):
            dt, its = smp.run()
            if k >= args.warmup:
                times.append(dt)
        n, P = wl["n"], math.comb(wl["M"] + wl["p"], wl["p"])
        unknowns = (n - 2) ** 2 * P
        # the oracle's own iteration count at the copy, scaled to the workload's unknowns
        v = statistics.median(times) * unknowns / smp.unknowns
        sample = smp.describe(statistics.median(times), its)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1),
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic (KL coefficients of the separable exponential covariance, f = 1)",
                          "config": {"workload": wl["name"], "unknowns": unknowns},
                          "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": 1, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.workload == "table3":
        out = run_table3(args, wl, rank, world)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload == "c4":
        out = run_c4(args, wl, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            v, sample = c4_cpu_sample(wl)
            out["cpu_baseline"] = {"value": round(v, 3), "unit": "s", "cores": 1, "kind": "oracle", "sample": sample}
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload == "c5":
        out = run_c5(args, wl, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            v, sample = CpuSampleBatch(wl).run()
            out["cpu_baseline"] = {"value": round(v, 1), "unit": "unknowns/s", "cores": 1, "kind": "oracle",
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
        v = dt / (smp.unknowns * its) * out["config"]["unknowns"] * out["iterations"]
        out["cpu_baseline"] = {"value": round(v, 3), "unit": "s", "cores": 1, "kind": "oracle",
                               "sample": smp.describe(dt, its) + f" x {out['iterations']} GPU iterations "
                                                                 f"(extrapolated)"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
