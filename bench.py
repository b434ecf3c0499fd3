#!/usr/bin/env python
"""Benchmark: Jacobi-PCG solves/s of the FEM-Laplace hot path on one GB300.

Workload (one step): the two systems of the 2D jittered 1024x1024-cell mesh
(interior vertices moved by up to h/4, random cell diagonals, seed 1), P1
(1.05M unknowns) and P2 (4.19M unknowns), Dirichlet data g = x^2 - y^2 -- each
assembled on the device, converted to SELL-C-sigma (C=32, sigma=256), lifted,
and solved by fp64 Jacobi-PCG from x0 = 0 to ||b - A x|| / ||b|| <= 1e-10.
value = solves/s (2 solves per step).  Alongside: the same step with an fp32
recurrence and fp64 reliable updates, per-kernel times and the roofline of the
dominant kernel, a seeded serving mix through the continuous-batching server,
and the CPU oracle timed on this host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --profile-kernels p2 --profile-precision f64 [--profile-bj 4]   (ncu driver)

N>1 runs as torchrun ranks, one GPU each: independent replicas of the same
workload (the path has no exchange step), max-over-ranks timing.
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

TOL = 1e-10
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12  # 2 DFMA (4 flops) per SM per clock
SYSTEMS = [  # (name, dim, degree, cells, jitter, diag_mode, seed)
    ("2D-P1-jittered-1024", 2, 1, 1024, 1, 1, 1),
    ("2D-P2-jittered-1024", 2, 2, 1024, 1, 1, 1),
]
GID = 1  # g = x^2 - y^2
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of each kernel on
# this workload and the capture it comes from (ncu --set full, one launch after
# a warm-up launch, `bench.py --profile-kernels p2`); (None, why) once the
# kernel has changed since that capture
NCU_TRAFFIC = {
    "k_spmv_tma2<double,double>": (640554496, "profiles/spmv_tma2_2d_p2_1024.md"),
    "k_spmv_tma2<float,float>": (423162112, "profiles/spmv_tma2_2d_p2_1024.md"),
}
# block-Jacobi block size per system (the fastest fp64 solve in the --sweep precond runs)
BJ_BS = {"2D-P1-jittered-1024": 2, "2D-P2-jittered-1024": 4}
METRIC = "PCG solves/s at rel. residual 1e-10 (fp64 Jacobi-PCG), cfg2 P1+P2"
WORKLOAD = "cfg2: 2D unit square 1024x1024 cells, jittered +-h/4, random diagonals (seed 1), P1 + P2, g=x^2-y^2"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=48,
                    help="requests of the seeded serving mix timed after the main workload (0 = skip)")
    ap.add_argument("--no-multi-rhs", dest="multi_rhs", action="store_false",
                    help="skip the blocked multi-RHS (cfg4 shape) kernel timing")
    ap.add_argument("--no-cfg4-full", dest="cfg4_full", action="store_false",
                    help="skip the full cfg4 solve (32 right-hand sides on 2048^2 P2, fp32 recurrences with fp64 "
                         "reliable updates)")
    ap.add_argument("--profile-kernels", default=None, metavar="SYSTEM",
                    help="profiling driver only: cfg1|p1|p2|3dp1|3dp2; times the CG kernels with CUDA events")
    ap.add_argument("--profile-precision", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--sweep", default=None, choices=["eps", "rhs", "precond", "degree"],
                    help="accuracy vs stopping tolerance (eps), solve time vs number of right-hand sides (rhs), "
                         "Jacobi vs block-Jacobi block sizes (precond), or P1-P4 (degree)")
    ap.add_argument("--profile-iters", type=int, default=3)
    ap.add_argument("--profile-bj", type=int, default=0, metavar="BS",
                    help="profiling driver: time the block-Jacobi iteration with blocks of BS rows")
    ap.add_argument("--profile-solve", default=None, choices=["bicgstab", "blockcg", "persistent"],
                    help="profiling driver: one solve of the profile system with direct launches (BiCGSTAB, or "
                         "block CG with --profile-rhs columns), or fp64 CG in one persistent launch (persistent: "
                         "one cluster for n <= 8192, else a grid-tier group)")
    ap.add_argument("--profile-rhs", type=int, default=0, metavar="K",
                    help="profiling driver: time the blocked multi-RHS iteration with K harmonic right-hand sides")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples (the JSON line carries their summary): GBPCG_CLOCKS_DIR, else a temporary directory
        import tempfile
        d = os.environ.get("GBPCG_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"gbpcg_clocks_rank{gpu_index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- ranks (N > 1) --
def reduce_timing(total_s, units_per_rank, world, device):
    """Whole-job timing of N replicas: the slowest rank's time (max over
    ranks) and units of all ranks per second.  Every rank calls it."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_s)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return total_s, units_per_rank * world / total_s


# ------------------------------------------------------------- our arm --
def run_ours(args, rank, world):
    import torch
    import paper_2201_05413_gb300 as P

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    L = P.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def step(precision=P.GB_F64, host_io=None, collect=None, bj=None):
        for idx, (name, dim, deg, cells, jit, dm, seed) in enumerate(SYSTEMS):
            d = P.FemSystem(dim, deg, cells, jit, dm, seed)
            A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
            if host_io is not None:  # e2e: Dirichlet data in from pinned host memory, x out
                gB = host_io["gB"][idx].to("cuda", non_blocking=True)
            else:
                gB = d.dirichlet(GID)
            b = d.lift(gB)[:, 0]
            kw = {}
            if bj:  # block-Jacobi: setup of the block inverses inside the step
                A.block_jacobi(bj[name])
                kw["precond"] = P.GB_PC_BLOCK_JACOBI
            x, st = A.solve(b, tol=TOL, max_iter=400000, precision=precision, **kw)
            if host_io is not None:
                host_io["x"][idx].copy_(x, non_blocking=True)
            if collect is not None:
                collect.append((name, d, A, b, st))
        if host_io is not None:
            torch.cuda.current_stream().synchronize()

    def timed(nsteps, **kw):
        times = []
        for _ in range(nsteps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(**kw)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        return times

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # warm-up (also collects per-system statistics)
    info = []
    for _ in range(args.warmup):
        info = []
        step(collect=info)
    torch.cuda.synchronize()

    # ---- timed region: fp64 (the headline value)
    clk = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clk.start()
    l0 = L.gbpcg_kernel_launches()
    torch.cuda.nvtx.range_push("gbpcg_timed_f64")  # ncu --nvtx-include selects these launches
    t64 = timed(args.steps)
    torch.cuda.nvtx.range_pop()
    launches = L.gbpcg_kernel_launches() - l0
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier()
    total, value = reduce_timing(sum(t64), len(SYSTEMS) * args.steps, world, "cuda")

    # ---- mixed precision, same workload: fp32 recurrence with fp64 reliable
    # updates (RU), and fp32 inner PCG inside fp64 iterative refinement (IR)
    mixed = {}
    for pn, pv in (("f32_ru", P.GB_F32_RU), ("f32_ir", P.GB_F32_IR)):
        minfo = []
        step(precision=pv, collect=minfo)
        tm = timed(args.steps, precision=pv)
        mixed[pn] = (len(SYSTEMS) * args.steps / sum(tm), minfo)

    # ---- block-Jacobi preconditioner (fp64), same workload
    bj_info = []
    step(collect=bj_info, bj=BJ_BS)
    tbj = timed(args.steps, bj=BJ_BS)
    bj_value = len(SYSTEMS) * args.steps / sum(tbj)

    # ---- e2e through the public API with host buffers
    host_io = {"gB": [], "x": []}
    for name, d, A, b, st in info:
        host_io["gB"].append(d.dirichlet(GID).cpu().pin_memory())
        host_io["x"].append(torch.empty(d.n_free, dtype=torch.float64).pin_memory())
    h2d = sum(t.numel() * 8 for t in host_io["gB"])
    d2h = sum(t.numel() * 8 for t in host_io["x"])
    te2e = timed(args.steps, host_io=host_io)
    e2e_value = len(SYSTEMS) * args.steps * world / max(sum(te2e), 1e-12)

    # ---- x_err (Eq. 1) of every cfg2 result: P2 against the exact discrete
    # solution (g = x^2 - y^2 at the nodes), P1 against an fp64 solve at 1e-13
    refs = []
    for (name, d, A, b, st) in info:
        if "P2" in name:
            refs.append(d.dirichlet(GID, which="free")[:, 0])
        else:
            refs.append(A.solve(b, tol=1e-13, max_iter=400000)[0])

    def xerrs(collected, precision, **kw):
        out = []
        for (name, d, A, b, st), ref in zip(collected, refs):
            x, _ = A.solve(b, tol=TOL, max_iter=400000, precision=precision, **kw)
            out.append(_xerr(x, ref))
        return out

    for (name, d, A, b, st) in bj_info:
        A.block_jacobi(BJ_BS[name])
    err64 = xerrs(info, P.GB_F64)
    err_bj = xerrs(bj_info, P.GB_F64, precond=P.GB_PC_BLOCK_JACOBI)
    err_mx = {pn: xerrs(mi, pv) for pn, pv, mi in (("f32_ru", P.GB_F32_RU, mixed["f32_ru"][1]),
                                                    ("f32_ir", P.GB_F32_IR, mixed["f32_ir"][1]))}
    del refs

    # ---- per-kernel times (CUDA events per launch) on the P2 system
    name, d2, A2, b2, st2 = info[-1]
    iters_t = 100
    ms64 = A2.kernel_times(b2, P.GB_F64, iters_t)
    ms32 = A2.kernel_times(b2, P.GB_F32_IR, iters_t)
    n2, nnz2 = A2.n, A2.nnz
    # algorithmic bytes of one SpMV+dot launch (the scope table's count): values
    # + column indices once, p gathered once, q written once
    spmv_bytes64 = nnz2 * (8 + 4) + n2 * (8 + 8)
    spmv_bytes32 = nnz2 * (4 + 4) + n2 * (4 + 4)
    spmv_flops64 = 2 * (nnz2 + n2)  # one FMA per stored entry, one per row for p.q
    peak, peak_src = peaks()
    ach64 = spmv_bytes64 / (ms64[0] * 1e-3) / 1e9
    ach32 = spmv_bytes32 / (ms32[0] * 1e-3) / 1e9
    tf64 = spmv_flops64 / (ms64[0] * 1e-3) / 1e12
    iter_bytes64 = nnz2 * 12 + 7 * n2 * 8
    iter_bytes32 = nnz2 * 8 + 7 * n2 * 4
    iter_ms64, iter_ms32 = sum(ms64), sum(ms32)

    # ---- layout autotuner (untimed): its pick per system and precision against
    # the fixed layout timed above (C = 32, sigma = 256, TMA-staged SpMV)
    tuned = {}
    for (name, d, A, b, st) in info:
        for pn, pv in (("f64", P.GB_F64), ("f32", P.GB_F32_IR)):
            At, cfg = P.autotune(d, b, precision=pv)
            del At
            base = sum(A.kernel_times(b, pv, 20))
            tuned.setdefault(name, {})[pn] = {
                "C": cfg["C"], "sigma": cfg["sigma"], "spmv_variant": cfg["spmv_variant"],
                "iter_ms": round(cfg["iter_ms"], 4), "default_iter_ms": round(base, 4),
                "candidates": cfg["candidates"]}

    per_sys = []
    for (name, d, A, b, st), e in zip(info, err64):
        per_sys.append({"system": name, "n": d.n_free, "nnz": d.nnz, "iterations": st["iterations"],
                        "relres": st["relres"], "x_err": e, "solve_ms": round(st["solve_ms"], 3),
                        "effective_GBps": round(st["bytes_moved"] / (st["solve_ms"] * 1e-3) / 1e9, 1)})
    for (name, d, A, b, st), row, e in zip(bj_info, per_sys, err_bj):
        row["f64_block_jacobi"] = {"bs": BJ_BS[name], "iterations": st["iterations"], "relres": st["relres"],
                                   "x_err": e, "solve_ms": round(st["solve_ms"], 3)}
    for pn in ("f32_ru", "f32_ir"):
        for (name, d, A, b, st), row, e in zip(mixed[pn][1], per_sys, err_mx[pn]):
            row[pn] = {"iterations": st["iterations"], "outer": st["outer"],
                       "fallback_iterations": st["fallback_iterations"], "relres": st["relres"], "x_err": e,
                       "solve_ms": round(st["solve_ms"], 3)}
    mixed_value = {pn: mixed[pn][0] for pn in mixed}
    del info[:], bj_info[:], mixed
    torch.cuda.empty_cache()

    # ---- the other configurations (untimed by the step; each its own events)
    cfg3 = run_cfg3()
    cfg1 = run_cfg1()
    multi = run_multi_rhs() if args.multi_rhs else None
    cfg4 = run_cfg4_full() if args.cfg4_full else None

    out = {
        "metric": METRIC,
        "value": round(value, 4), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded jittered lattice meshes)",
        "config": {"workload": WORKLOAD, "tol": TOL, "sell": {"C": 32, "sigma": 256},
                   "parallelism": f"replicas x{world}", "l2": "flushed (512 MB write) before every timed step"},
        "e2e": {"value": round(e2e_value, 4), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": {"bound": "hbm", "achieved": round(ach64, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach64 / peak, 4), "traffic": NCU_TRAFFIC["k_spmv_tma2<double,double>"][0],
                     "traffic_source": NCU_TRAFFIC["k_spmv_tma2<double,double>"][1],
                     "kernel": "k_spmv_tma2<double,double> (2D P2 1024^2: q = A p and p.q)",
                     "bytes_per_launch": spmv_bytes64, "launch_ms": round(ms64[0], 5), "peak_source": peak_src,
                     "alu": {"achieved_TFLOPps": round(tf64, 4), "peak_TFLOPps": round(FP64_PEAK_TFLOPS, 3),
                             "frac": round(tf64 / FP64_PEAK_TFLOPS, 4)}},
        "x_err_f64": [float(f"{e:.3g}") for e in err64],
        "mixed": {pn: {"solves_per_s": round(v, 4), "vs_f64": round(v / value * world, 3),
                       "x_err": [float(f"{e:.3g}") for e in err_mx[pn]]} for pn, v in mixed_value.items()},
        "block_jacobi_f64": {"solves_per_s": round(bj_value, 4), "vs_f64": round(bj_value / value * world, 3),
                             "x_err": [float(f"{e:.3g}") for e in err_bj]},
        "iteration": {"f64": {"ms": round(iter_ms64, 4),
                              "frac_of_hbm": round(iter_bytes64 / (iter_ms64 * 1e-3) / 1e9 / peak, 4)},
                      "f32": {"ms": round(iter_ms32, 4),
                              "frac_of_hbm": round(iter_bytes32 / (iter_ms32 * 1e-3) / 1e9 / peak, 4)}},
        "cfg3": {nm: {pn: {k: (float(f"{v:.3g}") if k == "x_err" else v) for k, v in r[pn].items()
                           if k in ("solves_per_s", "its", "x_err")} for pn in ("f64", "f32_ir", "f32_ru")}
                 for nm, r in cfg3.items()},
        "cfg1": {k: cfg1[k] for k in ("iterations_per_s", "solves_per_s", "iterations", "x_err_closed_form")},
    }
    if cfg4 is not None:
        out["cfg4"] = {k: cfg4[k] for k in ("precision", "solves_per_s", "iterations", "outer", "relres_max",
                                            "x_err_vs_f64_1e-12")}
    if multi is not None:
        out["cfg4_iteration"] = {pn: {"ms": multi[pn]["iter_ms"], "frac_of_hbm": multi[pn]["frac_of_hbm_peak"],
                                      "width": multi[pn]["autotuned_width"]} for pn in ("f64", "f32")}
    details = {
        "per_system": per_sys,
        "kernel_ms": {"f64": {"spmv_pq": ms64[0], "update": ms64[1], "pupdate": ms64[2]},
                      "f32": {"spmv_pq": ms32[0], "update": ms32[1], "pupdate": ms32[2]}},
        "roofline_mixed": {"bound": "hbm", "kernel": "k_spmv_tma2<float,float> (2D P2 1024^2)",
                           "achieved": round(ach32, 1), "peak": peak, "frac": round(ach32 / peak, 4),
                           "traffic": NCU_TRAFFIC["k_spmv_tma2<float,float>"][0],
                           "traffic_source": NCU_TRAFFIC["k_spmv_tma2<float,float>"][1],
                           "bytes_per_launch": spmv_bytes32, "launch_ms": round(ms32[0], 5)},
        "autotune": tuned, "cfg3": cfg3, "cfg1": cfg1, "cfg4_full": cfg4, "multi_rhs": multi,
    }
    return out, details



# -------------------------------------------------------- oracle (CPU) --
def _oracle_counts():
    with open(os.path.join(ROOT, "oracle", "iteration_counts.json")) as f:
        return json.load(f)


def cpu_oracle_sample(budget_s):
    """Times the oracle on this host on the benchmark's workload, two ways:
    single-thread (the pinned build) and all cores (the OpenMP timing build of
    the same source, nproc threads).  Each system's oracle assembly (one
    thread) is timed in full.  All cores: the P1 solve runs to 1e-10 in full;
    the P2 solve, and every single-thread solve, is a bounded sample of PCG
    iterations whose time per iteration is scaled by the iterations the
    oracle's own full solve takes (oracle/iteration_counts.json, written by
    oracle/iteration_counts.py).  Returns solves/s per mode and the detail."""
    import oracle as O
    cores = os.cpu_count() or 1
    counts = _oracle_counts()
    per = budget_s / (2 * len(SYSTEMS))

    def sample(rp, ci, v, b, threads):
        its = 4
        while True:
            t1 = time.perf_counter()
            O.pcg(rp, ci, v, b, tol=1e-300, maxit=its, threads=threads)
            dt = time.perf_counter() - t1
            if dt > per / 2 or its >= 1 << 20:
                return dt / its, its
            its *= 2

    tot = {"single_thread": 0.0, "all_core": 0.0}
    det = []
    for name, dim, deg, cells, jit, dm, seed in SYSTEMS:
        t0 = time.perf_counter()
        sy = O.System(dim, deg, cells, jit, dm, seed).assemble()
        rp, ci, v = sy.k_ii()
        b = sy.lift(sy.eval_g(O.G_X2_Y2))[:, 0]
        t_asm = time.perf_counter() - t0
        need = counts[name]["iterations"]
        t1_it, its1 = sample(rp, ci, v, b, None)
        row = {"system": name, "assembly_s": round(t_asm, 3), "oracle_iterations": need,
               "single_thread": {"sec_per_iter": t1_it, "sample_iters": its1,
                                 "solve_s": round(t1_it * need, 2)}}
        tot["single_thread"] += t_asm + t1_it * need
        if deg == 1:  # the P1 system: one full all-core solve
            t1 = time.perf_counter()
            _, stc, itc, relc = O.pcg(rp, ci, v, b, tol=TOL, threads=cores)
            t_solve = time.perf_counter() - t1
            row["all_core"] = {"full_solve": True, "iterations": itc, "status": stc, "relres": relc,
                               "solve_s": round(t_solve, 2)}
        else:
            tn_it, itsn = sample(rp, ci, v, b, cores)
            t_solve = tn_it * need
            row["all_core"] = {"full_solve": False, "sec_per_iter": tn_it, "sample_iters": itsn,
                               "solve_s": round(t_solve, 2)}
        tot["all_core"] += t_asm + t_solve
        det.append(row)
        del sy, rp, ci, v, b
    n = len(SYSTEMS)
    return {"single_thread": n / tot["single_thread"], "all_core": n / tot["all_core"], "cores": cores,
            "detail": det}


CPU_SAMPLE = ("oracle (plain C, fp64) on this host: single-thread pinned build and the OpenMP build of the same "
              "source on all cores; oracle assembly of each system in full; all-core P1 solve in full; the other "
              "solves a bounded iteration sample x the oracle's own full-solve iteration count "
              "(oracle/iteration_counts.json)")


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on this host's cores, same config/metric
    (value = all cores; the single-thread figure alongside)."""
    vals, singles = [], []
    res = None
    for _ in range(args.warmup):
        cpu_oracle_sample(min(args.cpu_sample_s, 6.0))
    for _ in range(args.steps):
        res = cpu_oracle_sample(args.cpu_sample_s)
        vals.append(res["all_core"])
        singles.append(res["single_thread"])
    value = statistics.median(vals)
    return {
        "impl": "reference", "metric": METRIC,
        "value": round(value, 6), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded jittered lattice meshes)",
        "config": {"workload": WORKLOAD, "systems": [s[0] for s in SYSTEMS], "tol": TOL},
        "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": res["cores"], "kind": "oracle",
                         "sample": CPU_SAMPLE, "single_thread": round(statistics.median(singles), 6),
                         "detail": res["detail"]},
        "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


PROFILE_SYSTEMS = {"cfg1": (2, 1, 64, 0, 0, 0, 0), "p1": (2, 1, 1024, 1, 1, 1, 1), "p2": (2, 2, 1024, 1, 1, 1, 1),
                   "3dp1": (3, 1, 128, 0, 0, 0, 2), "3dp2": (3, 2, 64, 0, 0, 0, 2)}


def run_profile(args):
    """Profiling driver for ncu: one system, CG kernels timed with CUDA events."""
    import torch
    import paper_2201_05413_gb300 as P
    P.load()
    dim, deg, cells, jit, dm, seed, gid = PROFILE_SYSTEMS[args.profile_kernels]
    d = P.FemSystem(dim, deg, cells, jit, dm, seed)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32 | P.GB_VAL_BF16)
    prec = {"f64": P.GB_F64, "f32": P.GB_F32_IR, "bf16": P.GB_BF16_IR}[args.profile_precision]
    if args.profile_solve == "persistent":
        b = d.lift(d.dirichlet(gid))[:, 0]
        x, st = A.solve(b, tol=1e-10, persist_off=0 if A.n <= 8192 else 3, raise_on_fail=False)
        torch.cuda.synchronize()
        print(json.dumps({"system": args.profile_kernels, "solve": "persistent", "n": A.n,
                          "iterations": st["iterations"], "solve_ms": st["solve_ms"]}))
        return
    if args.profile_solve == "bicgstab":
        b = d.lift(d.dirichlet(gid))[:, 0]
        x, st = A.solve(b, tol=1e-10, method=P.GB_BICGSTAB, use_graph=0, max_iter=args.profile_iters,
                        raise_on_fail=False)
        torch.cuda.synchronize()
        print(json.dumps({"system": args.profile_kernels, "solve": "bicgstab", "n": A.n, "steps": st["iterations"]}))
        return
    if args.profile_solve == "blockcg":
        import numpy as np
        k = args.profile_rhs or 8
        coef = np.random.default_rng(3).standard_normal((k, 10))
        B = d.lift(d.dirichlet(4, coef, k))
        X, st = A.solve_block(B, tol=1e-10, precision=prec, max_iter=args.profile_iters, raise_on_fail=False)
        torch.cuda.synchronize()
        print(json.dumps({"system": args.profile_kernels, "solve": "blockcg", "n": A.n, "k": k,
                          "steps": st["iterations"]}))
        return
    if args.profile_rhs:
        import numpy as np
        k = args.profile_rhs
        coef = np.random.default_rng(3).standard_normal((k, 10))
        B = d.lift(d.dirichlet(4 if dim == 2 else 3, coef if dim == 2 else coef[:, :4], k))
        ms = P.batched_kernel_times([A], [B], prec, args.profile_iters)
        torch.cuda.synchronize()
        print(json.dumps({"system": args.profile_kernels, "precision": args.profile_precision, "n": A.n,
                          "nnz": A.nnz, "k": k, "kernel_ms": ms}))
        return
    b = d.lift(d.dirichlet(gid))[:, 0]
    if args.profile_bj:
        A.block_jacobi(args.profile_bj)
        prec |= P.gbpcg.GB_KT_BLOCK_JACOBI
    ms = A.kernel_times(b, prec, args.profile_iters)
    torch.cuda.synchronize()
    print(json.dumps({"system": args.profile_kernels, "precision": args.profile_precision, "n": A.n,
                      "nnz": A.nnz, "block_jacobi": args.profile_bj, "kernel_ms": ms}))


MULTI_SPEC = (2, 2, 2048, 1, 1, 2)  # cfg4: 2D jittered 2048^2 P2, seed 2
MULTI_K = 32


def run_multi_rhs(iters=5):
    """Blocked multi-RHS iteration at the cfg4 shape (16.8M unknowns, 32
    right-hand sides from harmonic-basis coefficients N(0,1), host seed 3):
    per-kernel CUDA-event times of the batched SpMM, X/R update and P update,
    fp64 and fp32 recurrences, with the algorithmic bytes per iteration
    (matrix once, 7 vector streams of n x k) against the HBM peak, and the
    RHS block width the autotuner picks (iteration time per width)."""
    import torch
    import paper_2201_05413_gb300 as P
    from paper_2201_05413_gb300.workloads import multi_rhs_coefficients
    d = P.FemSystem(*MULTI_SPEC)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
    B = d.lift(d.dirichlet(4, multi_rhs_coefficients(MULTI_K), MULTI_K))
    peak, src = peaks()
    out = {"workload": "cfg4: 2D jittered 2048x2048 P2 (seed 2), k=32 RHS (harmonic basis, N(0,1) coefficients, seed 3)",
           "n": A.n, "nnz": A.nnz, "k": MULTI_K, "iters_timed": iters}
    for pn, pv, sv in (("f64", P.GB_F64, 8), ("f32", P.GB_F32_IR, 4)):
        P.batched_kernel_times([A], [B], pv, 2)
        ms = P.batched_kernel_times([A], [B], pv, iters)
        it_ms = sum(ms)
        algo = A.nnz * (sv + 4) + 7 * A.n * MULTI_K * sv
        flops = (2 * A.nnz + 11 * A.n) * MULTI_K
        out[pn] = {"kernel_ms": {"spmm": round(ms[0], 4), "update": round(ms[1], 4), "pupdate": round(ms[2], 4)},
                   "iter_ms": round(it_ms, 4), "iterations_per_s": round(1e3 / it_ms, 2),
                   "algorithmic_GBps": round(algo / (it_ms * 1e-3) / 1e9, 1),
                   "frac_of_hbm_peak": round(algo / (it_ms * 1e-3) / 1e9 / peak, 4),
                   "GFLOPps": round(flops / (it_ms * 1e-3) / 1e9, 1)}
        # RHS block width autotuner: iteration time of the 32 columns cut into groups of w
        w, wms = P.autotune_rhs_width(A, B, precision=pv)
        out[pn]["autotuned_width"] = w
        out[pn]["iter_ms_by_width"] = {str(c): round(t, 4) for c, t in wms.items()}
    out["peak_source"] = src
    del B, A, d
    torch.cuda.empty_cache()
    return out


def _xerr(x, ref):
    return float((x - ref).norm() / ref.norm())


CFG3_SYSTEMS = [("3D-P1-Kuhn-128", (3, 1, 128, 0, 0, 0)), ("3D-P2-Kuhn-64", (3, 2, 64, 0, 0, 0))]


def run_cfg3():
    """cfg3: 3D Kuhn 128^3 P1 and 64^3 P2, g = x^2 + y^2 - 2 z^2, plain fp64
    PCG against the fp32 recurrence inside fp64 iterative refinement (IR) and
    with fp64 reliable updates (RU), all to Eq. 2 at 1e-10.  Solve time from
    the library's CUDA events (one warm solve first); x_err (Eq. 1) against
    the exact discrete solution (both elements reproduce this quadratic: g at
    the nodes)."""
    import paper_2201_05413_gb300 as P
    out = {}
    for name, spec in CFG3_SYSTEMS:
        d = P.FemSystem(*spec)
        A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
        b = d.lift(d.dirichlet(2))[:, 0]
        exact = d.dirichlet(2, which="free")[:, 0]
        row = {"n": A.n, "nnz": A.nnz}
        for pn, pv in (("f64", P.GB_F64), ("f32_ir", P.GB_F32_IR), ("f32_ru", P.GB_F32_RU)):
            A.solve(b, tol=TOL, max_iter=400000, precision=pv)  # warm
            x, st = A.solve(b, tol=TOL, max_iter=400000, precision=pv)
            row[pn] = {"solves_per_s": round(1e3 / st["solve_ms"], 2), "ms": round(st["solve_ms"], 2),
                       "its": st["iterations"] + st["fallback_iterations"], "relres": st["relres"],
                       "x_err": _xerr(x, exact)}
        out[name] = row
        del A, d
    return out


def run_cfg1(repeats=50):
    """cfg1: regular 64^2 P1 (the 5-point matrix), g = sin(pi x) sinh(pi y) /
    sinh(pi); fp64 PCG to 1e-10, `repeats` solves back to back (latency-bound:
    iterations/s is the figure).  x_err against the exact discrete solution
    u_ij = sin(pi i h) sinh(mu j) / sinh(64 mu), cosh mu = 2 - cos(pi h)."""
    import math

    import numpy as np
    import torch
    import paper_2201_05413_gb300 as P
    d = P.FemSystem(2, 1, 64, 0, 0, 0)
    A = d.to_sell(32, 256)
    b = d.lift(d.dirichlet(0))[:, 0]
    A.solve(b, tol=TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = 0
    for _ in range(repeats):
        x, st = A.solve(b, tol=TOL)
        its += st["iterations"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h = 1.0 / 64
    mu = math.acosh(2.0 - math.cos(math.pi * h))
    i = np.arange(1, 64)
    u = np.outer(np.sinh(mu * i) / np.sinh(64 * mu), np.sin(math.pi * i * h)).reshape(-1)  # row j, column i
    err = float(np.linalg.norm(x.cpu().numpy() - u) / np.linalg.norm(u))
    return {"n": A.n, "nnz": A.nnz, "iterations": st["iterations"], "relres": st["relres"],
            "iterations_per_s": round(its / dt, 1), "solves_per_s": round(repeats / dt, 1),
            "solve_ms": round(1e3 * dt / repeats, 3), "x_err_closed_form": err}


def run_cfg4_full(ref_columns=(0, 31)):
    """cfg4 solved in full: 2D jittered 2048^2 P2, 32 right-hand sides (the
    harmonic-basis data, N(0,1) coefficients up to degree 4), blocked
    multi-RHS PCG with fp32 recurrences and fp64 reliable updates to Eq. 2 at
    1e-10, timed with CUDA events (one launch sequence, assembly and layout
    excluded); solves/s counts each column as one solve.  x_err of two columns
    against an fp64 single-RHS solve at 1e-12."""
    import torch
    import paper_2201_05413_gb300 as P
    from paper_2201_05413_gb300.workloads import multi_rhs_coefficients
    d = P.FemSystem(*MULTI_SPEC)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
    B = d.lift(d.dirichlet(4, multi_rhs_coefficients(MULTI_K), MULTI_K))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    X, st = P.pcg_solve_batched([A], [B], tol=TOL, max_iter=400000, precision=P.GB_F32_RU)
    e1.record(stream)
    e1.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    errs = {}
    for j in ref_columns:
        xr, _ = A.solve(B[:, j].contiguous(), tol=1e-12, max_iter=400000)
        errs[str(j)] = _xerr(X[0][:, j], xr)
    out = {"precision": "f32 recurrences + f64 reliable updates", "k": MULTI_K, "n": A.n, "s": round(s, 3),
           "solves_per_s": round(MULTI_K / s, 3), "iterations": st[0]["iterations"],
           "outer": st[0]["outer"], "relres_max": st[0]["relres"],
           "x_err_vs_f64_1e-12": errs}
    del X, B, A, d
    torch.cuda.empty_cache()
    return out


def run_serving(nreq, seed=4):
    """Seeded serving mix through the continuous-batching server (assembly
    included everywhere).  (1) All requests submitted at once: saturated
    throughput, fp32 recurrences with fp64 reliable updates, and again with
    fp64 recurrences (so batching and precision show apart).  (2) The same
    requests arriving as a Poisson stream at 0.8 x the fp32 saturated
    throughput: p50/p99 latency (submit to result).  (3) The same requests one
    at a time in fp64 (pcg_solve for k = 1, pcg_solve_batched for the k
    columns of a request otherwise): throughput, and the
    p50/p99 latency a single FIFO server with these measured service times
    would give under the same arrival stream."""
    import numpy as np
    import torch
    import paper_2201_05413_gb300 as P
    from paper_2201_05413_gb300.workloads import serving_requests
    reqs = serving_requests(nreq, seed=seed)

    def submit(srv, r):
        return srv.submit(r["dim"], r["degree"], r["cells"], r["jitter"], r["diag_mode"], r["seed"],
                          k=r["k"], gid=r["gid"], coef=r["coef"])

    def saturated(precision):
        srv = P.Server(mem_budget=40 << 30, max_slots=64, precision=precision, tol=TOL)
        t0 = time.perf_counter()
        ts = [submit(srv, r) for r in reqs]
        res = srv.wait(ts, timeout_s=3600)
        wall = time.perf_counter() - t0
        stats = srv.stats()
        srv.close()
        ok = sum(1 for t in ts if res[t][0]["status"] == 0)
        lat = np.array([res[t][0]["latency_ms"] for t in ts])
        return {"ok": ok, "solves_per_s": round(nreq / wall, 3), "wall_s": round(wall, 2),
                "max_resident": stats["max_resident"], "mem_peak_GB": round(stats["mem_peak"] / 1e9, 3),
                "p50_ms": round(float(np.percentile(lat, 50)), 1)}

    sat32 = saturated(P.GB_F32_RU)
    sat64 = saturated(P.GB_F64)
    rate = 0.8 * sat32["solves_per_s"]
    gaps = np.random.default_rng(seed + 1000).exponential(1.0 / rate, nreq)
    arrive = np.cumsum(gaps) - gaps[0]
    srv = P.Server(mem_budget=40 << 30, max_slots=64, precision=P.GB_F32_RU, tol=TOL)
    t1 = time.perf_counter()
    ts2 = []
    for r, ta in zip(reqs, arrive):
        dt = ta - (time.perf_counter() - t1)
        if dt > 0:
            time.sleep(dt)
        ts2.append(submit(srv, r))
    res2 = srv.wait(ts2, timeout_s=3600)
    wall2 = time.perf_counter() - t1
    srv.close()
    lat2 = np.array([res2[t][0]["latency_ms"] for t in ts2])
    ok2 = sum(1 for t in ts2 if res2[t][0]["status"] == 0)
    # one at a time, fp64: measured service time of each request, solved by the
    # library's fastest single-request path (pcg_solve for one right-hand side,
    # the blocked multi-RHS solve of its k columns otherwise)
    service = []
    for r in reqs:
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        d = P.FemSystem(r["dim"], r["degree"], r["cells"], r["jitter"], r["diag_mode"], r["seed"])
        A = d.to_sell(32, 256, P.GB_VAL_F64)
        B = d.lift(d.dirichlet(r["gid"], r["coef"], r["k"]))
        if r["k"] == 1:
            A.solve(B[:, 0], tol=TOL, max_iter=2000000)
        else:
            P.pcg_solve_batched([A], [B], tol=TOL, max_iter=2000000)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t3)
        del A, B, d
    seq = sum(service)
    done, lat3 = 0.0, []
    for ta, sv in zip(arrive, service):  # FIFO single server under the same arrivals
        done = max(done, ta) + sv
        lat3.append(1e3 * (done - ta))
    lat3 = np.array(lat3)
    per_req = []
    for r, l2, sv in zip(reqs, lat2, service):
        side = r["degree"] * r["cells"] - 1
        per_req.append({"dim": r["dim"], "degree": r["degree"], "cells": r["cells"], "k": r["k"],
                        "n": side ** r["dim"], "poisson_latency_ms": round(float(l2), 1),
                        "alone_f64_ms": round(1e3 * sv, 1)})
    return {"requests": nreq, "of_10000": round(nreq / 10000, 4), "seed": seed, "per_request": per_req,
            "mix": "cfg5 generator (70% 2D jittered n in [32,1024], 30% 3D Kuhn n in [16,128], P1/P2, k 1-8), "
                   "mem budget 40 GB, up to 64 resident",
            "saturated_f32_ru": sat32, "saturated_f64": sat64,
            "poisson_f32_ru": {"ok": ok2, "rate_per_s": round(rate, 3), "arrival_seed": seed + 1000,
                               "solves_per_s": round(nreq / wall2, 3),
                               "p50_ms": round(float(np.percentile(lat2, 50)), 1),
                               "p99_ms": round(float(np.percentile(lat2, 99)), 1)},
            "one_at_a_time_f64": {"solves_per_s": round(nreq / seq, 3), "wall_s": round(seq, 2),
                                  "service_p50_ms": round(1e3 * float(np.percentile(service, 50)), 1),
                                  "service_p99_ms": round(1e3 * float(np.percentile(service, 99)), 1),
                                  "fifo_p50_ms": round(float(np.percentile(lat3, 50)), 1),
                                  "fifo_p99_ms": round(float(np.percentile(lat3, 99)), 1)}}


EPS_SYSTEMS = [  # (name, spec, gid, closed form available)
    ("2D-P1-jittered-1024", (2, 1, 1024, 1, 1, 1), 1, False),
    ("2D-P2-jittered-1024", (2, 2, 1024, 1, 1, 1), 1, True),
    ("3D-P1-Kuhn-128", (3, 1, 128, 0, 0, 0), 2, True),
    ("3D-P2-Kuhn-64", (3, 2, 64, 0, 0, 0), 2, True),
    ("3D-P1-Kuhn-jittered-128", (3, 1, 128, 1, 0, 7), 2, False),  # irregular tets: P1 not exact on quadratics
    ("3D-P2-Kuhn-jittered-64", (3, 2, 64, 1, 0, 7), 2, True),
]


def run_sweep_eps():
    """Accuracy and time against the stopping tolerance of Eq. (2) (the
    paper's epsilon study uses 1e-8, 1e-12 and 1e-15), fp64, fp32 recurrences
    with fp64 reliable updates, and fp32 inner PCG in fp64 iterative
    refinement; x_err (Eq. 1) against the
    exact discrete solution where the discretisation reproduces g exactly
    (P2 in 2D and 3D, the 7-point Kuhn P1 on quadratics), else against the
    fp64 solve at 1e-15 (or as far as fp64 rounding lets it go)."""
    import torch
    import paper_2201_05413_gb300 as P
    P.load()
    for name, spec, gid, exact in EPS_SYSTEMS:
        d = P.FemSystem(*spec)
        A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
        b = d.lift(d.dirichlet(gid))[:, 0]
        if exact:
            ref = d.dirichlet(gid, which="free")[:, 0]
        else:
            ref, _ = A.solve(b, tol=1e-15, max_iter=2000000, raise_on_fail=False)
        for tol in (1e-6, 1e-8, 1e-10, 1e-12, 1e-14, 1e-15):
            for pn, pv in (("f64", P.GB_F64), ("f32_ru", P.GB_F32_RU), ("f32_ir", P.GB_F32_IR)):
                x, st = A.solve(b, tol=tol, max_iter=2000000, precision=pv, raise_on_fail=False)
                torch.cuda.synchronize()
                err = float((x - ref).norm() / ref.norm())
                print(json.dumps({"sweep": "eps", "system": name, "tol": tol, "precision": pn,
                                  "status": st["status"], "iterations": st["iterations"], "relres": st["relres"],
                                  "x_err": err, "x_err_reference": "exact discrete solution" if exact else
                                  "fp64 solve at 1e-15 (or its rounding floor)", "solve_ms": round(st["solve_ms"], 2)}), flush=True)
        del A, d
        torch.cuda.empty_cache()


def run_sweep_rhs():
    """Time to solve k right-hand sides of one system (2D jittered P2 256^2,
    harmonic-basis Dirichlet data), blocked (Eq. MRH: k recurrences sharing one
    SpMM pass, in groups of up to 32 columns per system of the batch) against
    one pcg_solve per column, fp64 and fp32 recurrences; for k <= 32 also block
    CG (one Krylov space shared by the k columns, pcg_solve_block)."""
    import numpy as np
    import torch
    import paper_2201_05413_gb300 as P
    P.load()
    spec = (2, 2, 256, 1, 1, 5)
    d = P.FemSystem(*spec)
    A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
    for k in (1, 2, 4, 8, 16, 32, 64, 128, 256):
        coef = np.random.default_rng(11).standard_normal((k, 10))
        B = d.lift(d.dirichlet(4, coef, k))
        groups = [B[:, j:j + 32].contiguous() for j in range(0, k, 32)]
        row = {"sweep": "rhs", "system": "2D-P2-jittered-256", "n": A.n, "nnz": A.nnz, "k": k}
        for pn, pv, pb in (("f64", P.GB_F64, P.GB_F64), ("f32", P.GB_F32_RU, P.GB_F32_RU)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, sts = P.pcg_solve_batched([A] * len(groups), groups, tol=TOL, max_iter=2000000, precision=pb,
                                         raise_on_fail=False)
            torch.cuda.synchronize()
            tb = time.perf_counter() - t0
            t0 = time.perf_counter()
            if k <= 64:
                for j in range(k):
                    A.solve(B[:, j].contiguous(), tol=TOL, max_iter=2000000, precision=pv, raise_on_fail=False)
                torch.cuda.synchronize()
                ts = time.perf_counter() - t0
            else:
                ts = None
            row[pn] = {"blocked_s": round(tb, 4), "blocked_ms_per_rhs": round(1e3 * tb / k, 3),
                       "one_at_a_time_s": None if ts is None else round(ts, 4),
                       "one_at_a_time_ms_per_rhs": None if ts is None else round(1e3 * ts / k, 3),
                       "max_relres": max(x["relres"] for x in sts), "status": max(abs(x["status"]) for x in sts),
                       "iterations_per_column_max": max(x["iterations"] for x in sts)}
            if k <= 32:  # block CG: one Krylov space shared by the k columns
                pk = P.GB_F64 if pn == "f64" else P.GB_F32_IR
                A.solve_block(B, tol=TOL, precision=pk, raise_on_fail=False)  # warm
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, sb = A.solve_block(B, tol=TOL, precision=pk, raise_on_fail=False)
                torch.cuda.synchronize()
                tcg = time.perf_counter() - t0
                row[pn]["block_cg"] = {"s": round(tcg, 4), "ms_per_rhs": round(1e3 * tcg / k, 3),
                                       "steps": sb["iterations"], "outer": sb["outer"], "relres": sb["relres"],
                                       "status": sb["status"]}
        print(json.dumps(row), flush=True)


def run_sweep_precond():
    """Jacobi against block-Jacobi (blocks of 1..32 consecutive free dofs) on
    the sweep systems at Eq. (2)'s 1e-10: iterations, solve time (block setup
    excluded, reported apart), x/r-update kernel time, fp64 and fp32-inner
    refinement; BiCGSTAB (fp64) with Jacobi and blocks of 2 and 4; x_err
    (Eq. 1) as in the eps sweep."""
    import torch
    import paper_2201_05413_gb300 as P
    P.load()
    for name, spec, gid, exact in EPS_SYSTEMS:
        d = P.FemSystem(*spec)
        A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
        b = d.lift(d.dirichlet(gid))[:, 0]
        if exact:
            ref = d.dirichlet(gid, which="free")[:, 0]
        else:
            ref, _ = A.solve(b, tol=1e-13, max_iter=2000000, raise_on_fail=False)
        for bs in (0, 1, 2, 4, 8, 16, 32):
            row = {"sweep": "precond", "system": name, "n": A.n, "precond": "jacobi" if bs == 0 else "block_jacobi",
                   "bs": bs}
            kw, flag = {}, 0
            if bs:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                A.block_jacobi(bs)
                row["setup_ms"] = round(1e3 * (time.perf_counter() - t0), 3)
                kw, flag = {"precond": P.GB_PC_BLOCK_JACOBI}, P.gbpcg.GB_KT_BLOCK_JACOBI
            for pn, pv in (("f64", P.GB_F64), ("f32_ir", P.GB_F32_IR)):
                A.solve(b, tol=TOL, max_iter=2000000, precision=pv, raise_on_fail=False, **kw)  # warm
                x, st = A.solve(b, tol=TOL, max_iter=2000000, precision=pv, raise_on_fail=False, **kw)
                ms = A.kernel_times(b, pv | flag, 20)
                torch.cuda.synchronize()
                row[pn] = {"status": st["status"], "iterations": st["iterations"], "relres": st["relres"],
                           "solve_ms": round(st["solve_ms"], 2), "update_us": round(1e3 * ms[1], 2),
                           "iter_us": round(1e3 * sum(ms), 2),
                           "x_err": float((x - ref).norm() / ref.norm())}
            if bs in (0, 2, 4):  # BiCGSTAB, the paper's Krylov method, with the same preconditioner
                kb = dict(kw, method=P.GB_BICGSTAB)
                A.solve(b, tol=TOL, max_iter=2000000, raise_on_fail=False, **kb)  # warm
                x, st = A.solve(b, tol=TOL, max_iter=2000000, raise_on_fail=False, **kb)
                torch.cuda.synchronize()
                row["bicgstab_f64"] = {"status": st["status"], "steps": st["iterations"], "restarts": st["restarts"],
                                       "relres": st["relres"], "solve_ms": round(st["solve_ms"], 2),
                                       "x_err": float((x - ref).norm() / ref.norm())}
            print(json.dumps(row), flush=True)
        del A, d
        torch.cuda.empty_cache()


def run_sweep_degree():
    """Table 7's degree study on our meshes: P1-P4 on a regular and a jittered
    mesh per dimension (2D 128^2 cells with random diagonals, g = sin(pi x)
    sinh(pi y) / sinh(pi); 3D Kuhn 16^3 with the quartic harmonic Re (x+iy)^4,
    reproduced exactly by P4 only), solved to 1e-12 (the paper's epsilon for Table 7):
    size, nnz per row, CG iterations and time (Jacobi, block-Jacobi bs 4),
    BiCGSTAB with block-Jacobi (the paper's solver), and the nodal error
    against the exact harmonic solution."""
    import numpy as np
    import torch
    import paper_2201_05413_gb300 as P
    P.load()
    tol = 1e-12
    for dim, cells, dm, jit, gid, coef in ((2, 128, 1, 0, 0, None), (2, 128, 1, 1, 0, None), (3, 16, 0, 0, 4, "re4"),
                                           (3, 16, 0, 1, 4, "re4")):
        for deg in (1, 2, 3, 4):
            spec = (dim, deg, cells, jit, dm, 1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d = P.FemSystem(*spec)
            A = d.to_sell(32, 256)
            torch.cuda.synchronize()
            t_setup = time.perf_counter() - t0
            c = None
            if coef == "re4":
                c = np.zeros((1, 10))
                c[0, 8] = 1.0
            b = d.lift(d.dirichlet(gid, c))[:, 0]
            exact = d.dirichlet(gid, c, which="free")[:, 0]
            row = {"sweep": "degree", "dim": dim, "cells": cells, "jitter": jit, "degree": deg, "n": A.n, "nnz": A.nnz,
                   "nnz_per_row": round(A.nnz / A.n, 2), "setup_ms": round(1e3 * t_setup, 1)}
            A.block_jacobi(4)
            for name, kw in (("cg", {}), ("cg_bj4", {"precond": P.GB_PC_BLOCK_JACOBI}),
                             ("bicgstab_bj4", {"method": P.GB_BICGSTAB, "precond": P.GB_PC_BLOCK_JACOBI})):
                A.solve(b, tol=tol, max_iter=2000000, raise_on_fail=False, **kw)  # warm
                x, st = A.solve(b, tol=tol, max_iter=2000000, raise_on_fail=False, **kw)
                torch.cuda.synchronize()
                row[name] = {"status": st["status"], "iterations": st["iterations"], "solve_ms": round(st["solve_ms"], 2),
                             "relres": st["relres"],
                             "nodal_err": float((x - exact).abs().max() / exact.abs().max())}
            print(json.dumps(row), flush=True)
            del A, d
            torch.cuda.empty_cache()


def main():
    args = parse()
    if args.profile_kernels:
        run_profile(args)
        return
    if args.sweep == "eps":
        run_sweep_eps()
        return
    if args.sweep == "rhs":
        run_sweep_rhs()
        return
    if args.sweep == "precond":
        run_sweep_precond()
        return
    if args.sweep == "degree":
        run_sweep_degree()
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out, details = run_ours(args, rank, world)
    if rank == 0 and args.serve_requests > 0:
        sv = run_serving(args.serve_requests)
        details["serving"] = sv
        out["serving"] = {"requests": sv["requests"], "of_10000": sv["of_10000"],
                          "saturated_solves_per_s": {"f32_ru": sv["saturated_f32_ru"]["solves_per_s"],
                                                     "f64": sv["saturated_f64"]["solves_per_s"]},
                          "poisson_f32_ru": {k: sv["poisson_f32_ru"][k] for k in ("rate_per_s", "p50_ms", "p99_ms")},
                          "one_at_a_time_f64": {k: sv["one_at_a_time_f64"][k]
                                                for k in ("solves_per_s", "fifo_p50_ms", "fifo_p99_ms")}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_sample(args.cpu_sample_s)
        details["cpu_baseline"] = cb
        out["cpu_baseline"] = {"value": round(cb["all_core"], 6), "unit": "solves/s", "cores": cb["cores"],
                               "kind": "oracle", "sample": CPU_SAMPLE,
                               "single_thread": round(cb["single_thread"], 6)}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        import tempfile
        path = os.environ.get("GBPCG_BENCH_DETAILS") or os.path.join(tempfile.gettempdir(), "gbpcg_bench_details.json")
        with open(path, "w") as f:
            json.dump(details, f, indent=1)
        out["details_file"] = path
        print(json.dumps(out))


if __name__ == "__main__":
    main()
