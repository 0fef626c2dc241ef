#!/usr/bin/env python3
"""Benchmark of the IFMM hot path on one GB300 (or N independent replicas).

Workload (default ``cube-64k``): N = 65,536 points uniform in the unit cube,
A_ij = 1/|x_i - x_j|, A_ii = 2 N^(1/3), leaves <= 64 points, Chebyshev 4x4x4,
eps = 1e-8, one standard-normal right-hand side, FP64 GMRES to a relative
residual of 1e-10 with the FMM matvec and the IFMM as right preconditioner.

A step is one pass of the whole path over the synthetic input already resident
in device memory: tree + lists + colours, operators, sigma_0, weighted bases,
elimination of every level, top LU, then GMRES (solve sweeps + FMM matvecs).
``value`` is solves/s (right-hand sides taken to 1e-10 per second of step).
The timed path uses split-TF32 Schur products on the tensor cores and the
symmetric variant (``--schur``, ``--general`` choose others); the same run
times one step of the plain FP64 general algorithm on the same input
(``plain_fp64``: "factor s vs plain FP64").  ``e2e`` repeats the step through
the C-ABI host-buffer entry points (points and b from host memory, x back to
host memory).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica (weak scaling, no collective on
the data path); rank 0 prints one JSON line.  ``--impl reference`` times the
CPU oracle on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IFMM-GMRES solves/s & p50/p99 latency to 1e-10 residual; factor s vs plain FP64"
UNIT = "solves/s"
SAMPLE_N = 4096       # oracle sample: same recipe as the workload at reduced N
FP64_PEAK_TFLOPS = 1.25  # GB300 FP64 (nominal, from the platform recipe; no measured figure)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["cube-2k", "cube-64k"], default="cube-64k")
    p.add_argument("--schur", choices=["fp64", "fp32", "tf32"], default="fp32",
                   help="Schur-product precision of the timed path (fp32: split-TF32 tensor cores)")
    p.add_argument("--general", action="store_true",
                   help="time the paper's general algorithm (two SVDs per box) instead of the "
                        "symmetric variant")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true",
                   help="skip the plain FP64 comparison step of a mixed-precision run")
    return p.parse_args()


def workload(name):
    import workloads
    return workloads.cube_2k() if name == "cube-2k" else workloads.cube_64k()


def describe(w):
    return (f"{w.name}: N={w.N} uniform in the unit cube, A_ij=1/r, A_ii=2N^(1/3), "
            f"leaves<={w.leaf_max}, Chebyshev {w.cheb_n}^3, eps={w.eps:g}, {w.nrhs} RHS, "
            "FMM matvec, right-preconditioned GMRES to 1e-10")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample_step(w_full):
    """One oracle pass (tree, operators, sigma_0, factor, GMRES) on the workload's
    recipe at N = SAMPLE_N; returns (seconds, iterations, true residual)."""
    import numpy as np

    import workloads
    from oracle.gmres import gmres
    from oracle.h2 import H2
    from oracle.ifmm import IFMM
    w = workloads.inv_r_cube(SAMPLE_N, w_full.seed, "sample", w_full.cheb_n, w_full.leaf_max,
                             w_full.eps)
    b = w.rhs(1)[:, 0]
    t0 = time.perf_counter()
    h2 = H2(w.points, w.kernel.kind, w.kernel.param, w.kernel.diag, w.cheb_n, w.leaf_max)
    f = IFMM(h2, w.eps)
    p = h2.tree.perm

    def mv(v):
        out = np.empty_like(v)
        out[p] = h2.matvec(v[p])
        return out

    x, it, _ = gmres(mv, b, f.solve, 1e-10, 500)
    dt = time.perf_counter() - t0
    res = float(np.linalg.norm(mv(x) - b) / np.linalg.norm(b))
    return dt, it, res


def sample_text(w):
    return (f"the oracle's full pass (tree, operators, sigma_0, factor, GMRES) on the same recipe "
            f"at N={SAMPLE_N} (seed {w.seed}); solves/s scaled to N={w.N} by the method's "
            f"asymptotic O(N) cost (x{SAMPLE_N}/{w.N}); the oracle's cost grows faster than N "
            "at these sizes, so the scaled figure overstates it")


def cpu_baseline(w):
    dt, it, res = oracle_sample_step(w)
    return {"value": (1.0 / dt) * (SAMPLE_N / w.N), "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle", "sample": sample_text(w), "sample_seconds": round(dt, 2),
            "sample_iters": it, "sample_true_residual": res}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    for _ in range(args.warmup):
        oracle_sample_step(w)
    times, its = [], []
    for _ in range(args.steps):
        dt, it, res = oracle_sample_step(w)
        times.append(dt)
        its.append(it)
    total = sum(times)
    value = args.steps * (SAMPLE_N / w.N) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps * (w.N / SAMPLE_N),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": describe(w)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample_text(w)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "iterations": its}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import paper_1508_01835_gb300 as ifmm
    from paper_1508_01835_gb300 import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(ifmm.LIB_PATH):
        build.build()
    w = workload(args.workload)
    dev = torch.device("cuda", local)
    pts_h = np.ascontiguousarray(w.points)
    b_h = np.ascontiguousarray(w.rhs(w.nrhs).T)        # (nrhs, N)
    pts = torch.tensor(pts_h, device=dev)
    b = torch.tensor(b_h, device=dev)
    x = torch.empty_like(b)
    ctx = ifmm.ifmm_ctx_create(local)
    schur = {"fp64": ifmm.P_FP64, "fp32": ifmm.P_FP32, "tf32": ifmm.P_TF32}[args.schur]
    opt = ifmm.make_options(dim=w.dim, cheb_n=w.cheb_n, leaf_max=w.leaf_max, eps=w.eps,
                            schur=schur, symmetric=0 if args.general else 1)
    kern = ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag)
    stream = torch.cuda.current_stream()

    def step(host=False, o=None):
        o = opt if o is None else o
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        if host:
            sys_h = ifmm.ifmm_system_create_host(ctx, pts_h, kern, o)
        else:
            sys_h = ifmm.ifmm_system_create(ctx, pts, kern, o)
        fac = ifmm.ifmm_factor(ctx, sys_h)
        ev[1].record(stream)
        if host:
            xh = np.empty_like(b_h)
            reps = ifmm.gmres_solve_host(ctx, sys_h, fac, ifmm.MV_FMM, b_h, xh, 1e-10, 500)
        else:
            reps = ifmm.gmres_solve(ctx, sys_h, fac, ifmm.MV_FMM, b, x, w.N, 1e-10, 500)
        ev[2].record(stream)
        info = ifmm.ifmm_factor_get_info(fac)
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys_h)
        return ev, reps, info

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ifmm.ifmm_profile_start(ctx)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    recs = [step() for _ in range(args.steps)]
    t_end.record(stream)
    torch.cuda.synchronize()
    stats = ifmm.ifmm_profile_stop(ctx)
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms = max_over_ranks(t_start.elapsed_time(t_end), dist, dev)
    step_ms = [ev[0].elapsed_time(ev[2]) for ev, _, _ in recs]
    factor_ms = [ev[0].elapsed_time(ev[1]) for ev, _, _ in recs]
    solve_ms = [ev[1].elapsed_time(ev[2]) for ev, _, _ in recs]
    reps = [r for _, rr, _ in recs for r in rr]
    info = recs[-1][2]
    value = whole_job_rate(args.steps * w.nrhs, world, ms)
    ok = all(r.status == 0 and r.true_rel_residual <= 1e-10 for r in reps)

    # the plain FP64 path on the same input, for "factor s vs plain FP64"
    plain = None
    if (args.schur != "fp64" or not args.general) and not args.no_plain:
        opt64 = ifmm.make_options(dim=w.dim, cheb_n=w.cheb_n, leaf_max=w.leaf_max, eps=w.eps,
                                  schur=ifmm.P_FP64)
        ev, reps64, _ = step(o=opt64)
        torch.cuda.synchronize()
        plain = {"factor_s": ev[0].elapsed_time(ev[1]) / 1e3,
                 "step_ms": ev[0].elapsed_time(ev[2]),
                 "gmres_iterations": [r.iters for r in reps64],
                 "true_rel_residual": max(r.true_rel_residual for r in reps64)}

    # end to end through the host-buffer entry points
    e2e = None
    if not args.no_e2e:
        n_e2e = min(args.steps, 2)  # bounded: each step is seconds long
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            step(host=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": n_e2e * w.nrhs / dt, "unit": UNIT, "steps": n_e2e,
               "h2d_bytes_per_step": int(pts_h.nbytes + b_h.nbytes),
               "d2h_bytes_per_step": int(b_h.nbytes)}

    # rooflines from the library's own event timings: every profiled kernel,
    # the dominant one, and the time-weighted fraction
    per_kernel, roofline, weighted = kernel_rooflines(stats, ms / 1e3, _measured_peaks())
    if roofline:
        roofline["traffic"] = _traffic(roofline["kernel"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(w), "schur": args.schur,
                   "variant": "general" if args.general else "symmetric",
                   "l2": "inputs larger than L2 (factor working set > 129 MB)",
                   "replicas": "independent per GPU"},
        "latency_ms": {"p50": _pct(step_ms, 50), "p99": _pct(step_ms, 99)},
        "solve_latency_ms": {"p50": _pct(solve_ms, 50), "p99": _pct(solve_ms, 99)},
        "factor_s": statistics.median(factor_ms) / 1e3,
        "plain_fp64": plain,
        "gmres_iterations": [r.iters for r in reps],
        "true_rel_residual": max(r.true_rel_residual for r in reps),
        "converged": ok,
        "factor_phases_s": {"init": info.seconds_init, "sigma0": info.seconds_sigma0,
                            "elim": info.seconds_elim, "top": info.seconds_top},
        "ranks": {str(l): [info.max_rank[l], round(info.avg_rank[l], 1)]
                  for l in range(2, info.levels + 1)},
        "clocks": clk, "e2e": e2e, "roofline": roofline,
        "gpu_launches": int(stats.get("(all launches)", (0,))[0]),
        "kernels": per_kernel,
        "roofline_time_weighted_frac": weighted,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ifmm.ifmm_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()


TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rates of the platform


def kernel_rooflines(stats, step_seconds, peaks):
    """Per-kernel roofline rows from the library's launch profile.

    stats: {name: (launches, seconds, flops, bytes)} (ifmm_profile_stop); names
    starting with "(" or containing ":" are totals or graph replays, not kernels.
    Bounds: block-row products (k_spmm*) are HBM-bound (bytes against the
    measured copy bandwidth); the tensor-core Schur products (k_gemm_tc*) are
    TF32 contractions (algorithmic 2MNK against the measured bf16 rate times
    the nominal TF32/BF16 ratio; the split mode issues three TF32 products per
    algorithmic product); everything else is FP64 arithmetic against the
    nominal FP64 rate.  Returns (rows by name, dominant row, time-weighted frac).
    """
    rows = {}
    for name, (launches, secs, flops, nbytes) in stats.items():
        if name.startswith("(") or ":" in name or secs <= 0:
            continue
        if name.startswith("k_spmm"):
            peak, unit, bound = peaks.get("hbm_gbs"), "GB/s", "hbm"
            achieved = nbytes / secs / 1e9
            src = "measured copy bandwidth"
        elif name.startswith("k_gemm_tc"):
            peak = peaks.get("bf16_tflops", 0.0) * TF32_PER_BF16
            unit, bound = "TFLOP/s", "tensor"
            achieved = flops / secs / 1e12
            src = "measured bf16 x nominal TF32/BF16 ratio" + (
                "; three TF32 products per algorithmic product" if "3x" in name else "")
        else:
            peak, unit, bound = FP64_PEAK_TFLOPS, "TFLOP/s", "alu"
            achieved = flops / secs / 1e12
            src = "FP64 nominal 1.25 TFLOP/s (no measured FP64 figure)"
        rows[name] = {"launches": int(launches), "s": round(secs, 4),
                      "share_of_step": secs / step_seconds if step_seconds > 0 else None,
                      "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                      "frac": achieved / peak if peak else None, "peak_source": src}
    dominant = None
    if rows:
        name = max(rows, key=lambda k: rows[k]["s"])
        r = rows[name]
        dominant = {"bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"],
                    "unit": r["unit"], "frac": r["frac"], "traffic": None, "kernel": name,
                    "peak_source": r["peak_source"], "launches": r["launches"],
                    "share_of_step": r["share_of_step"]}
    timed = [(r["s"], r["frac"]) for r in rows.values() if r["frac"] is not None]
    total = sum(t for t, _ in timed)
    weighted = sum(t * f for t, f in timed) / total if total > 0 else None
    return rows, dominant, weighted


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank runs the same replica workload)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second of the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


def _pct(v, q):
    s = sorted(v)
    if not s:
        return None
    k = min(len(s) - 1, max(0, int(math.ceil(q / 100.0 * len(s))) - 1))
    return s[k]


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        # the platform's fallback figures (one earlier measurement on a GB300)
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` at this workload's size: not captured
    (the ncu captures of the factor kernels are taken on a smaller case of the
    same recipe, and the FP64-bound kernels' time does not follow their bytes)."""
    return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
