#!/usr/bin/env python3
"""Benchmark of the IFMM hot path on one GB300 (or N independent replicas).

Default workload ``serving-cube`` (the serving configuration): 64 systems of
points uniform in the unit cube, N log-uniform in [4096, 262144], A_ij = 1/r,
A_ii = 2 N^(1/3), leaves <= 64, Chebyshev 3x3x3, eps = 1e-6, split-TF32 Schur
products, symmetric variant, every box rank capped at 2 n^D = 54 (the
prescribed-rank reading of Sec. 2.4).  The systems are factorised (batched)
and registered with the GMRES server under a 160 GB device-memory budget;
systems that do not fit are refused.  Requests arrive as a Poisson process of
2000 per second, each for a system drawn uniformly from the 64 and carrying
1..32 standard-normal right-hand sides, solved by GMRES to a true residual of
1e-10: GMRES with iterative refinement -- inner flexible GMRES whose FMM
products take the far field in FP32 (near field FP64) and whose substitution
sweeps run in FP32, outer FP64 FMM residuals (``--matvec fp64``: every product
in FP64).  A step is `--step-seconds` of arrivals; the timed
region is K consecutive steps, inputs resident on the device (requests carry
device pointers).  ``value`` = right-hand sides solved to 1e-10 within the
timed region per second; p50/p99 latency over the requests admitted in it;
shed and refused counts.  ``e2e`` repeats a window with host-buffer requests
(b copied in, x copied out by the server).  ``plain_fp64_one_at_a_time``
solves a bounded sample of the same request stream one right-hand side at a
time with plain FP64 GMRES (FP64 products and sweeps, no server, no batching)
on the same resident factorisations -- the bar the served path is measured
against.  The factorisation of the
cube-64k system (N = 65,536, Chebyshev 4^3, eps = 1e-8) is timed in the
mixed-precision symmetric form and in plain FP64 with the paper's general
algorithm ("factor s vs plain FP64").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload serving-cube|cube-64k|cube-2k]

Under torchrun each rank serves its own replica (weak scaling, no collective
on the data path); rank 0 prints one JSON line.  ``--impl reference`` times
the CPU oracle (GMRES solves with the oracle's IFMM preconditioner on the
smallest serving system) on the host cores.
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
N_SYSTEMS = 64
RATE = 2000.0              # requests per second
BUDGET = 160 * 10 ** 9     # device bytes admitted by the server
RESIDENT_SHARE = 0.7       # of the budget for resident systems; the rest for GMRES blocks
SERVE_CAP = 54             # rank cap 2 n^D of the serving systems (n = 3, D = 3)
SERVE_MAXIT = 200
RING_COLS = 96             # device output columns per system (see Load)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60,
                   help="timed steps of --step-seconds of arrivals (default 30 s: longer than "
                        "the largest systems' blocks, so the count does not hinge on which "
                        "blocks happen to finish inside the window)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["serving-cube", "cube-64k", "cube-2k"],
                   default="serving-cube")
    p.add_argument("--step-seconds", type=float, default=0.5)
    p.add_argument("--systems", type=int, default=N_SYSTEMS,
                   help="serve only the first K of the 64 systems (a reduced check of the "
                        "serving path; the full configuration is the default)")
    p.add_argument("--workers", type=int, default=8)
    p.add_argument("--schur", choices=["fp64", "fp32", "tf32"], default="fp32",
                   help="Schur-product precision of the timed path (fp32: split-TF32 tensor cores)")
    p.add_argument("--matvec", choices=["fp32", "fp64"], default="fp32",
                   help="served GMRES: fp32 = iterative refinement with the FMM far field in FP32 "
                        "(FP64 residuals); fp64 = every product in FP64")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true",
                   help="skip the cube-64k factor comparison (mixed vs plain FP64)")
    return p.parse_args()


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
# CPU oracle: served solves on the smallest serving system (baseline and the
# reference arm), and the full cube-2k pass
# ---------------------------------------------------------------------------
def _smallest_serving_index():
    import workloads
    sizes = workloads.log_uniform_sizes(N_SYSTEMS, 4096, 262144, 5000 + 999)
    return min(range(N_SYSTEMS), key=lambda s: sizes[s])


class OracleServer:
    """The oracle's IFMM of one serving system (factorised once, like a resident
    factorisation) and its GMRES solves of standard-normal right-hand sides."""

    def __init__(self):
        import numpy as np

        import workloads
        from oracle.h2 import H2
        from oracle.ifmm import IFMM
        self.np = np
        self.w = workloads.serving_cube_system(_smallest_serving_index())
        w = self.w
        t0 = time.perf_counter()
        self.h2 = H2(w.points, w.kernel.kind, w.kernel.param, w.kernel.diag, w.cheb_n, w.leaf_max)
        self.f = IFMM(self.h2, w.eps, rank_cap=SERVE_CAP)
        self.factor_s = time.perf_counter() - t0
        self.rng = np.random.default_rng(w.seed + 1)

    def solve(self):
        from oracle.gmres import gmres
        np = self.np
        p = self.h2.tree.perm
        h2 = self.h2

        def mv(v):
            out = np.empty_like(v)
            out[p] = h2.matvec(v[p])
            return out

        b = self.rng.standard_normal(self.w.N)
        t0 = time.perf_counter()
        x, it, _ = gmres(mv, b, self.f.solve, 1e-10, SERVE_MAXIT)
        dt = time.perf_counter() - t0
        res = float(np.linalg.norm(mv(x) - b) / np.linalg.norm(b))
        return dt, it, res


def _oracle_child(kind, threads):
    """Run one oracle measurement in a child process with `threads` BLAS threads."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_measure(%r)))" % (ROOT, kind))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=900)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    if out.returncode != 0 or not lines:
        return {"error": (out.stderr or out.stdout)[-300:]}
    return json.loads(lines[-1])


def _oracle_measure(kind):
    if kind == "serve":
        o = OracleServer()
        dt, it, res = o.solve()
        return {"N": o.w.N, "factor_s": o.factor_s, "solve_s": dt, "iters": it, "residual": res}
    import numpy as np

    import workloads
    from oracle.gmres import gmres
    from oracle.h2 import H2
    from oracle.ifmm import IFMM
    w = workloads.cube_2k()
    b = w.rhs(1)[:, 0]
    t0 = time.perf_counter()
    h2 = H2(w.points, w.kernel.kind, w.kernel.param, w.kernel.diag, w.cheb_n, w.leaf_max)
    f = IFMM(h2, w.eps)
    t1 = time.perf_counter()
    p = h2.tree.perm

    def mv(v):
        out = np.empty_like(v)
        out[p] = h2.matvec(v[p])
        return out

    x, it, _ = gmres(mv, b, f.solve, 1e-10, 500)
    t2 = time.perf_counter()
    return {"N": w.N, "factor_s": t1 - t0, "solve_s": t2 - t1, "iters": it,
            "residual": float(np.linalg.norm(mv(x) - b) / np.linalg.norm(b))}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        return subprocess.run(["lscpu"], capture_output=True, text=True).stdout.split(
            "Model name:")[1].splitlines()[0].strip()
    except (OSError, IndexError):
        return "unknown"


def cpu_baseline():
    cores = os.cpu_count()
    one = _oracle_child("serve", 1)
    allc = _oracle_child("serve", cores)
    c1_one = _oracle_child("cube2k", 1)
    c1_all = _oracle_child("cube2k", cores)
    val = 1.0 / allc["solve_s"] if "solve_s" in allc else None
    return {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "sample": (f"one GMRES solve to 1e-10 (1 right-hand side) with the oracle's IFMM "
                       f"preconditioner on the smallest serving system (N={allc.get('N')}), "
                       "factorisation resident (timed apart); not scaled: the serving mix's "
                       "systems are larger, so this overstates the oracle on the mix"),
            "single_thread": {"solves_per_s": 1.0 / one["solve_s"] if "solve_s" in one else None,
                              **one},
            "all_cores": allc,
            "cube_2k_full_pass": {"single_thread": c1_one, "all_cores": c1_all,
                                  "what": "tree, operators, sigma_0, factor and GMRES to 1e-10 "
                                          "on the cube-2k system (N=2048, n=3, eps=1e-6)"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    o = OracleServer()
    for _ in range(args.warmup):
        o.solve()
    times, its = [], []
    for _ in range(args.steps):
        dt, it, res = o.solve()
        times.append(dt)
        its.append(it)
    total = sum(times)
    value = args.steps / total
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": serving_description(),
                       "sample": f"one RHS of the smallest serving system (N={o.w.N}) per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": _cpu_model(),
                             "sample": f"GMRES solves (1 RHS each) with the oracle's IFMM on the "
                                       f"smallest serving system, N={o.w.N}, factorisation "
                                       f"({o.factor_s:.1f} s) resident"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "latency_ms": {"p50": 1e3 * _pct(times, 50), "p99": 1e3 * _pct(times, 99)},
            "iterations": its}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm: serving
# ---------------------------------------------------------------------------
def serving_description():
    return (f"serving-cube: {N_SYSTEMS} systems, N log-uniform in [4096, 262144] uniform in the "
            "unit cube, A_ij=1/r, A_ii=2N^(1/3), leaves<=64, Chebyshev 3^3, eps=1e-6, rank cap "
            f"{SERVE_CAP}, split-TF32 Schur, symmetric; Poisson arrivals {RATE:g}/s, 1-32 "
            "standard-normal RHS per request, GMRES to true residual 1e-10, "
            f"{BUDGET / 1e9:g} GB device budget ({RESIDENT_SHARE:.0%} for resident systems, the rest "
            "for GMRES blocks)")


class Load:
    """Poisson request stream against a server; tracks completions."""

    def __init__(self, ifmm, srv, ids, pools, rng, device_inputs, torch, N):
        self.ifmm, self.srv, self.ids, self.pools = ifmm, srv, ids, pools
        self.rng, self.device_inputs, self.torch, self.N = rng, device_inputs, torch, N
        self.pending = []
        # device outputs: per system a ring of 96 columns, allocated before any
        # timing.  At most 64 columns of a system are outstanding (one queued and
        # one running block of <= 32), and a request never wraps (<= 31 columns
        # skipped at the end), so live requests never share columns.
        self.ring, self.head = {}, {}
        self.done = []          # (submit time, completion time, nrhs, worst residual, status)
        self.shed = 0
        self.refused = 0        # requests for systems the server did not admit
        self.offered = 0

    def _submit(self, now):
        i = int(self.rng.integers(N_SYSTEMS))
        k = int(self.rng.integers(1, 33))
        self.offered += 1
        if self.ids[i] is None:
            self.refused += 1
            return
        B = self.pools[i]
        try:
            if self.device_inputs:
                h = self.head.get(i, 0)
                if h + k > RING_COLS:
                    h = 0
                x = self.ring[i][h:h + k]
                t = self.ifmm.ifmm_server_submit_device(self.srv, self.ids[i], B[:k], x, self.N[i],
                                                        1e-10, SERVE_MAXIT)
                self.head[i] = h + k
            else:
                import numpy as np
                x = np.empty((k, self.N[i]))
                t = self.ifmm.ifmm_server_submit(self.srv, self.ids[i], B[:k], x, 1e-10,
                                                 SERVE_MAXIT)
            self.pending.append((t, k, now, x, i))
        except self.ifmm.ServerError:
            self.shed += 1

    def _poll(self, block=False):
        keep = []
        for t, k, t0, x, i in self.pending:
            st, reps, lat = self.ifmm.ifmm_server_wait(self.srv, t, k, -1 if block else 0)
            if st == 6:
                keep.append((t, k, t0, x, i))
                continue
            worst = max(r.true_rel_residual for r in reps) if reps else float("nan")
            self.done.append((t0, t0 + lat, k, worst, st, max(r.iters for r in reps), i))
        self.pending = keep

    def run(self, seconds):
        t_start = time.perf_counter()
        t_next = t_start + self.rng.exponential(1.0 / RATE)
        last_poll = t_start
        while True:
            now = time.perf_counter()
            if now - t_start >= seconds:
                break
            while t_next <= now:
                self._submit(t_next)
                t_next += self.rng.exponential(1.0 / RATE)
            if now - last_poll > 0.002:
                self._poll()
                last_poll = now
            time.sleep(0.0002)
        return t_start, time.perf_counter()

    def drain(self):
        self._poll(block=True)


def run_serving(args, ifmm, torch, ctx, dev, world, rank, dist):
    import numpy as np

    import workloads
    ws = [workloads.serving_cube_system(s) for s in range(N_SYSTEMS)]
    N = [w.N for w in ws]
    n_serve = max(1, min(args.systems, N_SYSTEMS))
    schur = {"fp64": ifmm.P_FP64, "fp32": ifmm.P_FP32, "tf32": ifmm.P_TF32}[args.schur]
    opt = ifmm.make_options(dim=3, cheb_n=3, leaf_max=64, eps=1e-6, schur=schur, symmetric=1,
                            rank_cap=SERVE_CAP)
    srv = ifmm.ifmm_server_create(ctx, BUDGET, workers=args.workers)
    ifmm.ifmm_server_set_reserve(srv, int((1.0 - RESIDENT_SHARE) * BUDGET))
    ifmm.ifmm_server_set_matvec_precision(
        srv, ifmm.P_FP32 if args.matvec == "fp32" else ifmm.P_FP64)
    try:
        return _serve(args, ifmm, torch, ctx, dev, world, rank, dist, ws, N, n_serve, opt, srv)
    finally:
        ifmm.ifmm_server_destroy(srv)


def _serve(args, ifmm, torch, ctx, dev, world, rank, dist, ws, N, n_serve, opt, srv):
    import numpy as np
    # admission: factorise the systems in registration order, eight at a time
    # (batched), register each; skip those whose estimated footprint cannot fit
    systems, facs, ids = [None] * N_SYSTEMS, [None] * N_SYSTEMS, [None] * N_SYSTEMS
    t_factor, bytes_per_point, admitted_bytes = 0.0, None, 0
    order = list(range(n_serve))
    k = 0
    while k < len(order):
        group = []
        while k < len(order) and len(group) < 8:
            s = order[k]
            k += 1
            if (bytes_per_point is not None and
                    admitted_bytes + 1.05 * bytes_per_point * N[s] > RESIDENT_SHARE * BUDGET):
                continue
            group.append(s)
        if not group:
            break
        for s in group:
            w = ws[s]
            systems[s] = ifmm.ifmm_system_create(ctx, torch.tensor(w.points, device=dev),
                                                 ifmm.Kernel(w.kernel.kind, w.kernel.param,
                                                             w.kernel.diag), opt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fs = ifmm.ifmm_factor_batch(ctx, [systems[s] for s in group], allow_singular=True)
        torch.cuda.synchronize()
        t_factor += time.perf_counter() - t0
        for s, f in zip(group, fs):
            facs[s] = f
            try:
                ids[s] = ifmm.ifmm_server_register(srv, systems[s], f, maxit=SERVE_MAXIT)
            except ifmm.ServerError:
                ids[s] = None
        used = ifmm.ifmm_server_stats(srv)[0]
        admitted_bytes = used
        npts = sum(N[s] for s in range(N_SYSTEMS) if ids[s] is not None)
        if npts:
            bytes_per_point = used / npts
    admitted = [s for s in range(N_SYSTEMS) if ids[s] is not None]
    factor_info = {"systems_admitted": len(admitted), "points_admitted": sum(N[s] for s in admitted),
                   "factor_batch_s": t_factor,
                   "resident_bytes": ifmm.ifmm_server_stats(srv)[0],
                   "singular_pivot_systems": sum(
                       1 for s in admitted if ifmm.ifmm_factor_get_info(facs[s]).singular_pivots)}
    # right-hand-side pools, device and host
    pools_d, pools_h = [None] * N_SYSTEMS, [None] * N_SYSTEMS
    for s in admitted:
        B = np.ascontiguousarray(ws[s].rhs(32).T)
        pools_h[s] = B
        pools_d[s] = torch.tensor(B, device=dev)
    rng = np.random.default_rng(5999 + rank)
    load = Load(ifmm, srv, ids, pools_d, rng, True, torch, N)
    for s in admitted:
        load.ring[s] = torch.empty((RING_COLS, N[s]), dtype=torch.float64, device=dev)
    for _ in range(args.warmup):           # plans of every block width, GPU clocks up
        load.run(args.step_seconds)
    load.drain()
    load.done.clear()
    load.shed = load.refused = load.offered = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = ifmm.ifmm_launch_count()
    # While server workers run (and may capture CUDA graphs) nothing here may
    # synchronise the device or use the legacy stream: the window is bracketed
    # by events on a private non-blocking stream that carries no other work.
    mark = torch.cuda.Stream(device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(mark)
    t_start, t_end = load.run(args.steps * args.step_seconds)
    ev1.record(mark)
    ev1.synchronize()
    launches = ifmm.ifmm_launch_count() - l0
    clk = clocks.stop()
    window = ev0.elapsed_time(ev1) / 1e3
    window = max_over_ranks(window * 1e3, dist, dev) / 1e3
    load._poll()
    in_window = [d for d in load.done if d[1] <= t_end]
    solved = sum(d[2] for d in in_window if d[4] == 0)
    load.drain()
    done = load.done
    lat = sorted(d[1] - d[0] for d in done if d[4] == 0)
    worst = max((d[3] for d in done if d[4] == 0), default=float("nan"))
    failed = sum(1 for d in done if d[4] != 0)
    value = whole_job_rate(solved, world, window * 1e3)
    serve = {"offered_requests": load.offered, "admitted_requests": len(done),
             "shed_requests": load.shed, "refused_requests_unadmitted_systems": load.refused,
             "failed_requests": failed, "rhs_solved_in_window": solved,
             "window_s": window, "worst_true_rel_residual": worst,
             "gmres_iterations_p50": _pct([d[5] for d in done], 50),
             "gmres_iterations_max": max((d[5] for d in done), default=None)}
    # per-kernel profile (not timed: the event pairs cost time, and kernels of
    # concurrent workers would stretch each other's intervals): one 32-column
    # block of the largest admitted system, alone on one stream, through the
    # same GMRES the server runs
    big = max(admitted, key=lambda s_: N[s_])
    Bp = pools_d[big]
    Xp = torch.empty_like(Bp)
    gopt = dict(side=ifmm.GMRES_FLEXIBLE, precond_precision=ifmm.P_FP32)
    if args.matvec == "fp32":
        gopt.update(matvec_precision=ifmm.P_FP32, refine=10)
    ifmm.gmres_solve_ex(ctx, systems[big], facs[big], ifmm.MV_FMM, Bp, Xp, N[big], 1e-10,
                        SERVE_MAXIT, **gopt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ifmm.gmres_solve_ex(ctx, systems[big], facs[big], ifmm.MV_FMM, Bp, Xp, N[big], 1e-10,
                        SERVE_MAXIT, **gopt)
    torch.cuda.synchronize()
    block_s = time.perf_counter() - t0
    ifmm.ifmm_profile_start(ctx)
    t0 = time.perf_counter()
    preps = ifmm.gmres_solve_ex(ctx, systems[big], facs[big], ifmm.MV_FMM, Bp, Xp, N[big], 1e-10,
                                SERVE_MAXIT, **gopt)
    stats = ifmm.ifmm_profile_stop(ctx)
    prof_s = time.perf_counter() - t0
    serve["profiled_block"] = {"system_N": N[big], "columns": 32, "seconds": block_s,
                               "seconds_under_launch_profile": prof_s,
                               "gmres_iterations_max": max(r.iters for r in preps)}
    plain = None if args.no_plain else plain_one_at_a_time(ifmm, torch, ctx, systems, facs, ids,
                                                           pools_d, N)
    # end to end: host-buffer requests through ifmm_server_submit
    e2e = None
    if not args.no_e2e:
        le = Load(ifmm, srv, ids, pools_h, np.random.default_rng(7000 + rank), False, torch, N)
        n_e2e = max(2, min(args.steps, 6))
        ts, _ = le.run(n_e2e * args.step_seconds)
        te = time.perf_counter()
        solved_e = sum(d[2] for d in le.done if d[1] <= te and d[4] == 0)
        le.drain()
        moved = sum(d[2] * N[d[6]] * 8 for d in le.done)   # b in and x out, per request
        e2e = {"value": solved_e / (te - ts), "unit": UNIT, "steps": n_e2e,
               "h2d_bytes_per_step": int(moved / n_e2e), "d2h_bytes_per_step": int(moved / n_e2e),
               "what": "the same request stream with b and x in host memory (ifmm_server_submit: "
                       "the server copies b in and x out inside each request's latency)"}
    serve["plain_fp64_one_at_a_time"] = plain
    result = (value, lat, serve, factor_info, stats, prof_s, clk, e2e, launches, window)
    return result, (systems, facs)


def plain_one_at_a_time(ifmm, torch, ctx, systems, facs, ids, pools, N, budget_s=20.0):
    """The plain FP64 one-system-at-a-time path on the same request stream:
    requests drawn as the load draws them (system uniform over the 64, 1-32
    right-hand sides), each right-hand side solved alone by GMRES with FP64
    products and FP64 sweeps (right preconditioning), no server and no
    batching, on the resident factorisations; stops after budget_s seconds.
    Requests for systems the server did not admit are skipped."""
    import numpy as np
    rng = np.random.default_rng(8000)
    solved, worst, iters, reqs = 0, 0.0, [], 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        i = int(rng.integers(N_SYSTEMS))
        k = int(rng.integers(1, 33))
        if ids[i] is None:
            continue
        reqs += 1
        for c in range(k):
            b = pools[i][c]
            x = torch.empty_like(b)
            rep = ifmm.gmres_solve(ctx, systems[i], facs[i], ifmm.MV_FMM, b, x, N[i], 1e-10,
                                   SERVE_MAXIT)[0]
            if rep.status == 0:
                solved += 1
                worst = max(worst, rep.true_rel_residual)
            iters.append(rep.iters)
            if time.perf_counter() - t0 >= budget_s:
                break
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return {"value": solved / el, "unit": UNIT, "rhs_solved": solved, "requests": reqs,
            "seconds": el, "worst_true_rel_residual": worst,
            "gmres_iterations_p50": _pct(iters, 50) if iters else None,
            "what": "each right-hand side alone through gmres_solve (FP64 FMM products, FP64 "
                    "sweeps, right preconditioning), requests drawn like the served stream, on "
                    "the same factorisations, until the time budget"}


def factor_comparison(ifmm, torch, ctx, dev, schur):
    """cube-64k: factor time of the mixed-precision symmetric path, of the same
    symmetric variant in FP64 (precision alone) and of plain FP64 with the
    paper's general algorithm, plus GMRES on each."""
    import numpy as np

    import workloads
    w = workloads.cube_64k()
    kern = ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag)
    pts = torch.tensor(w.points, device=dev)
    b = torch.tensor(w.rhs(1)[:, 0], device=dev)
    out = {}
    # three legs: the timed path, the same algorithm in FP64 (the precision
    # axis alone) and the paper's general algorithm in FP64 (the plain path)
    for name, o in (("mixed_symmetric", ifmm.make_options(dim=3, cheb_n=4, leaf_max=64, eps=w.eps,
                                                          schur=schur, symmetric=1)),
                    ("fp64_symmetric", ifmm.make_options(dim=3, cheb_n=4, leaf_max=64, eps=w.eps,
                                                         schur=ifmm.P_FP64, symmetric=1)),
                    ("plain_fp64_general", ifmm.make_options(dim=3, cheb_n=4, leaf_max=64,
                                                             eps=w.eps, schur=ifmm.P_FP64))):
        s = ifmm.ifmm_system_create(ctx, pts, kern, o)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        f = ifmm.ifmm_factor(ctx, s)
        e1.record()
        x = torch.empty_like(b)
        rep = ifmm.gmres_solve(ctx, s, f, ifmm.MV_FMM, b, x, w.N, 1e-10, 500)[0]
        e2.record()
        torch.cuda.synchronize()
        out[name] = {"factor_s": e0.elapsed_time(e1) / 1e3, "gmres_ms": e1.elapsed_time(e2),
                     "gmres_iterations": rep.iters, "true_rel_residual": rep.true_rel_residual}
        out[name + "_x"] = x.cpu().numpy()
        ifmm.ifmm_factor_destroy(f)
        ifmm.ifmm_system_destroy(s)
    xa, xs, xb = (out.pop(k + "_x") for k in ("mixed_symmetric", "fp64_symmetric",
                                               "plain_fp64_general"))
    out["solution_difference"] = float(np.linalg.norm(xa - xb) / np.linalg.norm(xb))
    out["solution_difference_mixed_vs_fp64_symmetric"] = float(np.linalg.norm(xa - xs) /
                                                               np.linalg.norm(xs))
    out["workload"] = ("cube-64k: N=65536 uniform in the unit cube, 1/r, A_ii=2N^(1/3), "
                       "leaves<=64, Chebyshev 4^3, eps=1e-8, default rank cap n^D")
    return out


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
    dev = torch.device("cuda", local)
    ctx = ifmm.ifmm_ctx_create(local)
    fp64_peak, fp32_peak = ifmm.ifmm_measure_peaks(ctx)
    peaks = _measured_peaks()
    peaks["fp64_tflops"] = fp64_peak
    peaks["fp32_tflops"] = fp32_peak
    if args.workload != "serving-cube":
        line = run_case_workload(args, ifmm, torch, ctx, dev, world, rank, dist, peaks)
    else:
        res, (systems, facs) = run_serving(args, ifmm, torch, ctx, dev, world, rank, dist)
        value, lat, serve, factor_info, stats, prof_s, clk, e2e, launches, window = res
        for f in facs:             # the server is gone: free the factorisations
            if f is not None:
                ifmm.ifmm_factor_destroy(f)
        for sy in systems:
            if sy is not None:
                ifmm.ifmm_system_destroy(sy)
        per_kernel, roofline, weighted = kernel_rooflines(stats, prof_s, peaks)
        if roofline:
            roofline["traffic"] = _traffic(roofline["kernel"])
        schur = {"fp64": ifmm.P_FP64, "fp32": ifmm.P_FP32, "tf32": ifmm.P_TF32}[args.schur]
        plain = None if args.no_plain else factor_comparison(ifmm, torch, ctx, dev, schur)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * window / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f64 GMRES residuals, CGS2 and outer products with iterative refinement: "
                      "inner FMM far field f32 (near field f64), f32 substitution sweeps; "
                      if args.matvec == "fp32" else
                      "f64 GMRES (FMM products, CGS2, residuals) with f32 substitution sweeps; ")
                     + "factors with split-TF32 Schur products (f32 accumulate), f64 LU/SVD",
            "data": "synthetic",
            "config": {"workload": serving_description() + (
                           "" if args.systems >= N_SYSTEMS else
                           f" (reduced check: only the first {args.systems} systems offered for "
                           "admission)"),
                       "step": f"{args.step_seconds:g} s of arrivals; timed region = steps x step",
                       "workers": args.workers,
                       "l2": "inputs larger than L2 (resident factorisations ~100 GB)",
                       "replicas": "independent per GPU"},
            "latency_ms": {"p50": 1e3 * _pct(lat, 50) if lat else None,
                           "p99": 1e3 * _pct(lat, 99) if lat else None},
            "serving": serve, "factor": factor_info,
            "factor_vs_plain_fp64": plain,
            "clocks": clk, "e2e": e2e, "roofline": roofline,
            "gpu_launches": int(launches),
            "kernels": per_kernel, "roofline_time_weighted_frac": weighted,
            "peaks": {"fp64_tflops_measured": fp64_peak, "fp32_tflops_measured": fp32_peak,
                      "hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops")},
        }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ifmm.ifmm_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()


def run_case_workload(args, ifmm, torch, ctx, dev, world, rank, dist, peaks):
    """One system per step: creation + factorisation + FMM-GMRES to 1e-10 on one
    RHS (the cube-2k / cube-64k workloads)."""
    import numpy as np

    import workloads
    w = workloads.cube_2k() if args.workload == "cube-2k" else workloads.cube_64k()
    schur = {"fp64": ifmm.P_FP64, "fp32": ifmm.P_FP32, "tf32": ifmm.P_TF32}[args.schur]
    opt = ifmm.make_options(dim=w.dim, cheb_n=w.cheb_n, leaf_max=w.leaf_max, eps=w.eps,
                            schur=schur, symmetric=1)
    kern = ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag)
    pts = torch.tensor(w.points, device=dev)
    b = torch.tensor(np.ascontiguousarray(w.rhs(1).T), device=dev)
    x = torch.empty_like(b)

    def step():
        s = ifmm.ifmm_system_create(ctx, pts, kern, opt)
        f = ifmm.ifmm_factor(ctx, s)
        reps = ifmm.gmres_solve(ctx, s, f, ifmm.MV_FMM, b, x, w.N, 1e-10, 500)
        ifmm.ifmm_factor_destroy(f)
        ifmm.ifmm_system_destroy(s)
        return reps

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ifmm.ifmm_launch_count()
    e0.record()
    reps = [r for _ in range(args.steps) for r in step()]
    e1.record()
    torch.cuda.synchronize()
    launches = ifmm.ifmm_launch_count() - l0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ifmm.ifmm_profile_start(ctx)
    t0 = time.perf_counter()
    step()
    stats = ifmm.ifmm_profile_stop(ctx)
    per_kernel, roofline, weighted = kernel_rooflines(stats, time.perf_counter() - t0, peaks)
    return {"metric": METRIC, "value": whole_job_rate(args.steps, world, ms), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 GMRES; split-TF32 Schur products",
            "data": "synthetic",
            "config": {"workload": f"{w.name}: N={w.N}, Chebyshev {w.cheb_n}^3, eps={w.eps:g}"},
            "gmres_iterations": [r.iters for r in reps],
            "true_rel_residual": max(r.true_rel_residual for r in reps), "clocks": clk,
            "e2e": None, "roofline": roofline, "gpu_launches": int(launches),
            "kernels": per_kernel, "roofline_time_weighted_frac": weighted}


TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rates of the platform


def kernel_rooflines(stats, span_seconds, peaks):
    """Per-kernel roofline rows from the library's launch profile.

    stats: {name: (launches, seconds, flops, bytes)} (ifmm_profile_stop); names
    starting with "(" or containing ":" are totals or graph replays, not
    kernels.  Every kernel is placed against each pipe it uses -- FP64 or FP32
    arithmetic (measured FMA rates of this GPU), the tensor cores (measured
    bf16 rate x the nominal TF32/BF16 ratio; the split mode issues three TF32
    products per algorithmic product) and HBM (measured copy bandwidth) -- and
    its bound is the pipe it fills most.  Returns (rows by name, dominant row,
    time-weighted fraction of the bounding pipes)."""
    rows = {}
    for name, (launches, secs, flops, nbytes) in stats.items():
        if name.startswith("(") or ":" in name or secs <= 0:
            continue
        cands = []
        if nbytes > 0 and peaks.get("hbm_gbs"):
            cands.append(("hbm", nbytes / secs / 1e9, peaks["hbm_gbs"], "GB/s",
                          "measured copy bandwidth"))
        if flops > 0:
            if name.startswith("k_gemm_tc"):
                pk = peaks.get("bf16_tflops", 0.0) * TF32_PER_BF16
                cands.append(("tensor", flops / secs / 1e12, pk, "TFLOP/s",
                              "measured bf16 x nominal TF32/BF16 ratio" +
                              ("; three TF32 products per algorithmic product" if "3x" in name
                               else "")))
            elif "f32" in name:
                cands.append(("alu", flops / secs / 1e12, peaks["fp32_tflops"], "TFLOP/s",
                              "measured FP32 FMA rate"))
            else:
                cands.append(("alu", flops / secs / 1e12, peaks["fp64_tflops"], "TFLOP/s",
                              "measured FP64 FMA rate"))
        if not cands:
            continue
        bound, achieved, peak, unit, src = max(cands, key=lambda c: c[1] / c[2] if c[2] else 0)
        rows[name] = {"launches": int(launches), "s": round(secs, 4),
                      "share": secs / span_seconds if span_seconds > 0 else None,
                      "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                      "frac": achieved / peak if peak else None, "peak_source": src}
    dominant = None
    if rows:
        name = max(rows, key=lambda k: rows[k]["s"])
        r = rows[name]
        dominant = {"bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"],
                    "unit": r["unit"], "frac": r["frac"], "traffic": None, "kernel": name,
                    "peak_source": r["peak_source"] + " (of measured)",
                    "launches": r["launches"], "share": r["share"]}
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
    """DRAM bytes per launch of `kernel` at this workload from an ncu capture;
    None where no capture of the current kernel exists."""
    return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
