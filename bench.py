#!/usr/bin/env python
"""Benchmark: Jacobi-PCG solves/s of the FEM-Laplace hot path on one GB300.

Workload (one step): the two systems of the 2D jittered 1024x1024-cell mesh
(interior vertices moved by up to h/4, random cell diagonals, seed 1), P1
(1.05M unknowns) and P2 (4.19M unknowns), Dirichlet data g = x^2 - y^2 -- each
assembled on the device, converted to SELL-C-sigma (C=32, sigma=256), lifted,
and solved by fp64 Jacobi-PCG from x0 = 0 to ||b - A x|| / ||b|| <= 1e-10.
value = solves/s (2 solves per step).  Alongside: the same step with
fp32-inner iterative refinement, per-kernel times and the HBM roofline of the
dominant kernel, and the CPU oracle timed on this host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
SYSTEMS = [  # (name, dim, degree, cells, jitter, diag_mode, seed)
    ("2D-P1-jittered-1024", 2, 1, 1024, 1, 1, 1),
    ("2D-P2-jittered-1024", 2, 2, 1024, 1, 1, 1),
]
GID = 1  # g = x^2 - y^2
WORKLOAD = "cfg2: 2D unit square 1024x1024 cells, jittered +-h/4, random diagonals (seed 1), P1 + P2, g=x^2-y^2"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

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


# ------------------------------------------------------------- our arm --
def run_ours(args, rank, world):
    import torch
    import paper_2201_05413_gb300 as P

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    L = P.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def step(precision=P.GB_F64, host_io=None, collect=None):
        for idx, (name, dim, deg, cells, jit, dm, seed) in enumerate(SYSTEMS):
            d = P.FemSystem(dim, deg, cells, jit, dm, seed)
            A = d.to_sell(32, 256, P.GB_VAL_F64 | P.GB_VAL_F32)
            if host_io is not None:  # e2e: Dirichlet data in from pinned host memory, x out
                gB = host_io["gB"][idx].to("cuda", non_blocking=True)
            else:
                gB = d.dirichlet(GID)
            b = d.lift(gB)[:, 0]
            x, st = A.solve(b, tol=TOL, max_iter=400000, precision=precision)
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
    t64 = timed(args.steps)
    launches = L.gbpcg_kernel_launches() - l0
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier()
    total = sum(t64)
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([total], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total = float(tt.item())
    solves = len(SYSTEMS) * args.steps * world
    value = solves / total

    # ---- mixed precision (fp32-inner refinement), same workload
    mixed_info = []
    step(precision=P.GB_F32_IR, collect=mixed_info)
    tmx = timed(args.steps, precision=P.GB_F32_IR)
    mixed_value = len(SYSTEMS) * args.steps / sum(tmx)

    # ---- e2e through the public API with host buffers
    host_io = {"gB": [], "x": []}
    for name, d, A, b, st in info:
        host_io["gB"].append(d.dirichlet(GID).cpu().pin_memory())
        host_io["x"].append(torch.empty(d.n_free, dtype=torch.float64).pin_memory())
    h2d = sum(t.numel() * 8 for t in host_io["gB"])
    d2h = sum(t.numel() * 8 for t in host_io["x"])
    te2e = timed(args.steps, host_io=host_io)
    e2e_value = len(SYSTEMS) * args.steps * world / max(sum(te2e), 1e-12)

    # ---- per-kernel times (CUDA events per launch) on the P2 system
    name, d2, A2, b2, st2 = info[-1]
    iters_t = 100
    ms64 = A2.kernel_times(b2, P.GB_F64, iters_t)
    ms32 = A2.kernel_times(b2, P.GB_F32_IR, iters_t)
    n2, nnz2 = A2.n, A2.nnz
    # algorithmic bytes of one SpMV+dot launch: values + indices once, row
    # lengths, p gathered once, q written once (fp64: 8-byte values/vectors)
    spmv_bytes64 = nnz2 * (8 + 4) + n2 * (4 + 8 + 8)
    spmv_bytes32 = nnz2 * (4 + 4) + n2 * (4 + 4 + 4)
    peak, peak_src = peaks()
    ach64 = spmv_bytes64 / (ms64[0] * 1e-3) / 1e9
    iter_bytes64 = nnz2 * 12 + 7 * n2 * 8
    iter_ms64 = sum(ms64)

    per_sys = []
    for (name, d, A, b, st) in info:
        per_sys.append({"system": name, "n": d.n_free, "nnz": d.nnz, "iterations": st["iterations"],
                        "relres": st["relres"], "solve_ms": round(st["solve_ms"], 3),
                        "effective_GBps": round(st["bytes_moved"] / (st["solve_ms"] * 1e-3) / 1e9, 1)})
    for (name, d, A, b, st), row in zip(mixed_info, per_sys):
        row["f32_ir"] = {"inner_iterations": st["iterations"], "outer": st["outer"],
                         "fallback_iterations": st["fallback_iterations"], "relres": st["relres"],
                         "solve_ms": round(st["solve_ms"], 3)}

    out = {
        "metric": "PCG solves/s at rel. residual 1e-10 (fp64 Jacobi-PCG), cfg2 P1+P2",
        "value": round(value, 4), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded jittered lattice meshes)",
        "config": {"workload": WORKLOAD, "systems": [s[0] for s in SYSTEMS], "tol": TOL,
                   "sell": {"C": 32, "sigma": 256}, "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MB write) before every timed step; P2 matrix 578 MB > L2"},
        "mixed_f32_ir": {"value": round(mixed_value, 4), "unit": "solves/s", "dtype": "f32 inner / f64 outer",
                         "speedup_vs_f64": round(mixed_value / value * world, 3)},
        "per_system": per_sys,
        "kernel_ms": {"f64": {"spmv_pq": ms64[0], "update": ms64[1], "pupdate": ms64[2]},
                      "f32": {"spmv_pq": ms32[0], "update": ms32[1], "pupdate": ms32[2]}},
        "iteration_GBps_f64": round(iter_bytes64 / (iter_ms64 * 1e-3) / 1e9, 1),
        "roofline": {"bound": "hbm", "kernel": "k_spmv_pq<double> (2D P2 1024^2)", "achieved": round(ach64, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(ach64 / peak, 4), "traffic": None,
                     "peak_source": peak_src, "bytes_per_launch": spmv_bytes64},
        "e2e": {"value": round(e2e_value, 4), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    return out, info


# -------------------------------------------------------- oracle (CPU) --
def cpu_oracle_sample(budget_s, gpu_iters=None):
    """Times the oracle (plain C, one thread) on the same workload: full
    assembly of each system plus a bounded number of PCG iterations, scaled to
    the iterations a full solve needs (the GPU's counts when known, else the
    oracle's own estimate from its residual decay is not attempted: the
    sample's per-iteration time times the GPU's count)."""
    import numpy as np

    import oracle as O
    res = []
    t_total = 0.0
    per = budget_s / len(SYSTEMS)
    for idx, (name, dim, deg, cells, jit, dm, seed) in enumerate(SYSTEMS):
        t0 = time.perf_counter()
        s = O.System(dim, deg, cells, jit, dm, seed).assemble()
        rp, ci, v = s.k_ii()
        b = s.lift(s.eval_g(O.G_X2_Y2))[:, 0]
        t_asm = time.perf_counter() - t0
        # bounded PCG sample: grow the iteration count until it takes ~per/2 s
        its = 4
        while True:
            t1 = time.perf_counter()
            O.pcg(rp, ci, v, b, tol=1e-300, maxit=its)
            dt = time.perf_counter() - t1
            if dt > per / 2 or its >= 1 << 20:
                break
            its *= 2
        t_it = dt / its
        need = gpu_iters[idx] if gpu_iters else its
        t_solve = t_asm + t_it * need
        t_total += t_solve
        res.append({"system": name, "assembly_s": round(t_asm, 3), "sec_per_iter": t_it,
                    "sample_iters": its, "iters_scaled_to": need, "est_solve_s": round(t_solve, 2)})
    return len(SYSTEMS) / t_total, res


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on this host's cores, same config/metric."""
    gpu_iters = None
    vals = []
    details = None
    for _ in range(args.warmup):
        cpu_oracle_sample(min(args.cpu_sample_s, 6.0), gpu_iters)
    for _ in range(args.steps):
        v, details = cpu_oracle_sample(args.cpu_sample_s, gpu_iters)
        vals.append(v)
    value = statistics.median(vals)
    sample = "oracle assembly + bounded PCG iteration sample per system; solves/s from sec/iter x own iteration count of the sample"
    return {
        "impl": "reference", "metric": "PCG solves/s at rel. residual 1e-10 (fp64 Jacobi-PCG), cfg2 P1+P2",
        "value": round(value, 6), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded jittered lattice meshes)",
        "config": {"workload": WORKLOAD, "systems": [s[0] for s in SYSTEMS], "tol": TOL},
        "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "detail": details},
        "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
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
    out, info = run_ours(args, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gpu_iters = [st["iterations"] for (_, _, _, _, st) in info]
        v, det = cpu_oracle_sample(args.cpu_sample_s, gpu_iters)
        out["cpu_baseline"] = {"value": round(v, 6), "unit": "solves/s", "cores": 1, "kind": "oracle",
                               "sample": ("oracle full assembly + a bounded PCG iteration sample per system "
                                          f"(~{args.cpu_sample_s:.0f} s total), sec/iter scaled to the GPU "
                                          "solve's iteration counts"),
                               "detail": det}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
