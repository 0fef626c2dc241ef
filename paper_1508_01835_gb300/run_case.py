"""Run one workload through the library and print what it took.

    python -m paper_1508_01835_gb300.run_case --workload cube-64k [--N 8192]
        [--schur fp64|fp32|tf32] [--symmetric] [--reps 2] [--no-gmres]
    python -m paper_1508_01835_gb300.run_case --mode batch [--systems 16] [--nmax 8192]
    python -m paper_1508_01835_gb300.run_case --mode serve [--systems 8] [--nmax 32768]
        [--rate 200] [--seconds 10]
    python -m paper_1508_01835_gb300.run_case --mode paper [--d 1e-3] [--orders 1,2,3,4]
        [--fmm-n 5] [--leaf 100] [--N 100000]
    python -m paper_1508_01835_gb300.run_case --mode blocks [--serving-systems 24,12]
    python -m paper_1508_01835_gb300.run_case --mode kernels [--serving-systems 12]

Each repetition: system creation (tree, lists, operators), factorisation
(sigma_0, weighted bases, elimination, top LU) and FMM-GMRES to 1e-10 on one
standard-normal right-hand side; one line per repetition with the phase
times, GMRES iterations, true residual, ranks per depth and counted flops.
``--mode batch``: independent systems on the unit sphere (the recipe of
the batched-factorisation workload: N log-uniform, A_ii = 2 sqrt(N), 4^3
Chebyshev, eps = 1e-4) with N capped at --nmax, factorised one at a time and
then with ifmm_factor_batch; prints both times.  ``--mode serve``: uniform-
cube 1/r systems (the serving workload's recipe, N log-uniform capped at
--nmax, 3^3 Chebyshev, eps = 1e-6, split-TF32 Schur products) factorised with
ifmm_factor_batch and registered with a server; requests with 1..32
standard-normal right-hand sides arrive as a Poisson process of --rate per
second for --seconds; prints p50/p99 latency, solves/s and the shed count.
``--N`` keeps the workload's recipe (distribution, kernel, leaf size,
Chebyshev order, eps, seed) at a smaller size, which is how the profiles
capture a small case of the same kernels.  IFMM_TRACE=1 adds per-level and
per-colour lines on stderr.
``--mode blocks``: serving-cube systems as the server holds them (rank cap 54,
split-TF32 Schur products, symmetric variant); per system the times of a
32-column FMM product in FP64 and with the FP32 far field, of a 32-column
substitution sweep in FP64 and FP32, and of GMRES to 1e-10 on 1 and 32
right-hand sides with FP64 products (flexible, FP32 sweeps) and with
iterative refinement (second of two runs each).  ``--mode kernels``: the
same system set-up, then one FP32 far-field product and one FP32 sweep of 32
columns, twice (a small target for ncu).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--workload", choices=["cube-2k", "cube-64k"], default="cube-64k")
    p.add_argument("--N", type=int, default=0)
    p.add_argument("--schur", choices=["fp64", "fp32", "tf32"], default="fp64")
    p.add_argument("--symmetric", action="store_true")
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--no-gmres", action="store_true")
    p.add_argument("--mode", choices=["case", "batch", "serve", "paper", "blocks", "kernels"],
                   default="case")
    p.add_argument("--serving-systems", default="24,12",
                   help="--mode blocks / kernels: indices of serving-cube systems")
    p.add_argument("--d", type=float, default=1e-3)
    p.add_argument("--orders", default="1,2,3,4")
    p.add_argument("--fmm-n", type=int, default=5)
    p.add_argument("--leaf", type=int, default=100)
    p.add_argument("--systems", type=int, default=0)
    p.add_argument("--nmax", type=int, default=0)
    p.add_argument("--rate", type=float, default=200.0)
    p.add_argument("--seconds", type=float, default=10.0)
    p.add_argument("--side", choices=["right", "left"], default="right",
                   help="--mode paper: side of the IFMM preconditioner (Appendix B)")
    p.add_argument("--rank-cap", type=int, default=0,
                   help="cap on every box rank (0: the library's default)")
    a = p.parse_args(argv)
    if a.mode == "batch":
        return batch(a)
    if a.mode == "serve":
        return serve(a)
    if a.mode == "paper":
        return paper(a)
    if a.mode in ("blocks", "kernels"):
        return blocks(a)

    import torch

    import paper_1508_01835_gb300 as ifmm
    import workloads

    w = workloads.cube_64k() if a.workload == "cube-64k" else workloads.cube_2k()
    if a.N:
        w = workloads.inv_r_cube(a.N, w.seed, f"{w.name}@N={a.N}", w.cheb_n, w.leaf_max, w.eps)
    prec = {"fp64": ifmm.P_FP64, "fp32": ifmm.P_FP32, "tf32": ifmm.P_TF32}[a.schur]
    ctx = ifmm.ifmm_ctx_create(0)
    opt = ifmm.make_options(dim=w.dim, cheb_n=w.cheb_n, leaf_max=w.leaf_max, eps=w.eps,
                            schur=prec, symmetric=1 if a.symmetric else 0, rank_cap=a.rank_cap)
    kern = ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag)
    pts = torch.tensor(w.points, device="cuda")
    b = torch.tensor(w.rhs(1)[:, 0], device="cuda")
    for rep in range(a.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = ifmm.ifmm_system_create(ctx, pts, kern, opt)
        t1 = time.perf_counter()
        f = ifmm.ifmm_factor(ctx, s)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        it, res = 0, float("nan")
        if not a.no_gmres:
            x = torch.empty_like(b)
            reps = ifmm.gmres_solve(ctx, s, f, ifmm.MV_FMM, b, x, w.N, 1e-10, 500)
            it, res = reps[0].iters, reps[0].true_rel_residual
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        info = ifmm.ifmm_factor_get_info(f)
        ranks = {l: (info.max_rank[l], round(info.avg_rank[l], 1))
                 for l in range(2, info.levels + 1)}
        print(f"[{w.name} schur={a.schur} symmetric={int(a.symmetric)} N={w.N} rep={rep}] "
              f"create {t1 - t0:.3f}s factor {t2 - t1:.3f}s gmres {t3 - t2:.3f}s it={it} "
              f"res={res:.2e} ranks={ranks} flops lu {info.flops_lu:.3g} "
              f"trsm {info.flops_trsm:.3g} schur {info.flops_schur:.3g} "
              f"lowrank {info.flops_lowrank:.3g} phases init {info.seconds_init:.3f} "
              f"sigma0 {info.seconds_sigma0:.3f} elim {info.seconds_elim:.3f} "
              f"top {info.seconds_top:.3f} bytes {info.factor_bytes / 1e9:.2f}GB", flush=True)
        ifmm.ifmm_factor_destroy(f)
        ifmm.ifmm_system_destroy(s)
    ifmm.ifmm_ctx_destroy(ctx)


def blocks(a):
    """Per-block costs on serving-cube systems (see the module docstring)."""
    import numpy as np
    import torch

    import paper_1508_01835_gb300 as ifmm
    import workloads

    ctx = ifmm.ifmm_ctx_create(0)

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / reps, out

    for si in [int(v) for v in a.serving_systems.split(",")]:
        w = workloads.serving_cube_system(si)
        opt = ifmm.make_options(dim=3, cheb_n=w.cheb_n, leaf_max=w.leaf_max, eps=w.eps,
                                schur=ifmm.P_FP32, symmetric=1, rank_cap=54)
        kern = ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag)
        t0 = time.perf_counter()
        sy = ifmm.ifmm_system_create(ctx, torch.tensor(w.points, device="cuda"), kern, opt)
        fac = ifmm.ifmm_factor(ctx, sy, allow_singular=True)
        torch.cuda.synchronize()
        print(f"[serving-cube[{si}] N={w.N}] create+factor {time.perf_counter() - t0:.2f}s",
              flush=True)
        X = torch.tensor(np.random.default_rng(4).standard_normal((32, w.N)), device="cuda")
        Y = torch.empty_like(X)
        if a.mode == "kernels":
            for _ in range(2):
                ifmm.fmm_matvec_prec(ctx, sy, ifmm.P_FP32, X, Y, w.N)
                ifmm.ifmm_solve_prec(ctx, fac, ifmm.P_FP32, X, Y, w.N)
            torch.cuda.synchronize()
        else:
            for name, prec in (("fp64", ifmm.P_FP64), ("fp32-far", ifmm.P_FP32)):
                dt, _ = timed(lambda: ifmm.fmm_matvec_prec(ctx, sy, prec, X, Y, w.N), 3)
                print(f"  matvec 32 columns {name}: {dt * 1e3:.2f} ms", flush=True)
            for name, prec in (("fp64", ifmm.P_FP64), ("fp32", ifmm.P_FP32)):
                dt, _ = timed(lambda: ifmm.ifmm_solve_prec(ctx, fac, prec, X, Y, w.N), 3)
                print(f"  sweep 32 columns {name}: {dt * 1e3:.2f} ms", flush=True)
            for width in (1, 32):
                B = X[:width].contiguous()
                Z = torch.empty_like(B)
                for name, kw in (("fp64 products", {}),
                                 ("iterative refinement", dict(matvec_precision=ifmm.P_FP32,
                                                               refine=10))):
                    dt, reps = timed(lambda: ifmm.gmres_solve_ex(
                        ctx, sy, fac, ifmm.MV_FMM, B, Z, w.N, 1e-10, 300,
                        side=ifmm.GMRES_FLEXIBLE, precond_precision=ifmm.P_FP32, **kw))
                    print(f"  GMRES {width} columns, {name}: {dt * 1e3:.1f} ms, iterations max "
                          f"{max(r.iters for r in reps)}, true residual max "
                          f"{max(r.true_rel_residual for r in reps):.2e}", flush=True)
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sy)
    ifmm.ifmm_ctx_destroy(ctx)


def paper(a):
    """The experiment of Sec. 3.2 (Table 1 for d = 1e-3, Table 2 for d = 1e-2):
    N points uniform in [-1, 1]^3 with the kernel of Eq. (K_ij), eps = 1e-3,
    leaves of at most 100 points, GMRES to 1e-10 with an FMM matvec of fixed
    order --fmm-n, unpreconditioned and with the IFMM of each order n as right
    preconditioner (the paper's general algorithm in FP64)."""
    import torch

    import paper_1508_01835_gb300 as ifmm
    import workloads
    N = a.N or 100000
    ctx = ifmm.ifmm_ctx_create(0)
    orders = [int(v) for v in a.orders.split(",")]
    if a.side == "right" and 0 not in orders:
        orders.append(0)  # the unpreconditioned run (the same on either side)
    for k, n in enumerate(orders):
        w = workloads.paper_cube(N, a.d, max(n, 1), leaf_max=a.leaf)
        opt = ifmm.make_options(dim=3, cheb_n=max(n, 1), leaf_max=w.leaf_max, eps=w.eps,
                                fmm_n=a.fmm_n, rank_cap=a.rank_cap)
        s = ifmm.ifmm_system_create(ctx, torch.tensor(w.points, device="cuda"),
                                    ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag), opt)
        b = torch.tensor(w.rhs(1)[:, 0], device="cuda")
        x = torch.empty_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = ifmm.ifmm_factor(ctx, s) if n > 0 else None
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        side = ifmm.GMRES_LEFT if a.side == "left" else ifmm.GMRES_RIGHT
        reps = ifmm.gmres_solve_ex(ctx, s, f, ifmm.MV_FMM, b, x, w.N, 1e-10, 500, side=side,
                                   refine=0)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        info = ifmm.ifmm_system_get_info(s)
        label = f"IFMM n={n} ({a.side})" if n > 0 else "no preconditioner"
        print(f"[paper d={a.d:g} N={w.N} L={info.levels} fmm_n={a.fmm_n}] {label}: "
              f"{reps[0].iters} GMRES iterations, residual estimate {reps[0].rel_residual:.2e}, "
              f"true residual {reps[0].true_rel_residual:.2e}, "
              f"factor {t1 - t0:.2f}s, GMRES {t2 - t1:.2f}s", flush=True)
        if f is not None:
            ifmm.ifmm_factor_destroy(f)
        ifmm.ifmm_system_destroy(s)
    ifmm.ifmm_ctx_destroy(ctx)


def _capped(make, count, nmax):
    import workloads
    out = []
    for k in range(count):
        w = make(k)
        if nmax and w.N > nmax:
            if w.name.startswith("sphere"):
                pts = workloads.unit_sphere(nmax, w.seed)
                w = workloads.Workload(w.name, pts, workloads.Kernel(workloads.K_INV_R, 0.0,
                                                                     2.0 * nmax ** 0.5),
                                       3, w.cheb_n, w.leaf_max, w.eps, 1, w.seed)
            else:
                w = workloads.inv_r_cube(nmax, w.seed, w.name, w.cheb_n, w.leaf_max, w.eps)
        out.append(w)
    return out


def batch(a):
    import torch

    import paper_1508_01835_gb300 as ifmm
    import workloads
    ws = _capped(workloads.sphere_system, a.systems or 16, a.nmax or 8192)
    prec = {"fp64": ifmm.P_FP64, "fp32": ifmm.P_FP32, "tf32": ifmm.P_TF32}[a.schur]
    ctx = ifmm.ifmm_ctx_create(0)
    sys = [ifmm.ifmm_system_create(ctx, torch.tensor(w.points, device="cuda"),
                                   ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag),
                                   ifmm.make_options(dim=3, cheb_n=w.cheb_n, leaf_max=w.leaf_max,
                                                     eps=w.eps, schur=prec,
                                                     symmetric=1 if a.symmetric else 0))
           for w in ws]
    for rep in range(a.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one = [ifmm.ifmm_factor(ctx, s) for s in sys]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        many = ifmm.ifmm_factor_batch(ctx, sys)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        print(f"[batch {len(ws)} sphere systems N={min(w.N for w in ws)}..{max(w.N for w in ws)} "
              f"schur={a.schur} symmetric={int(a.symmetric)} rep={rep}] one at a time "
              f"{t1 - t0:.3f}s, ifmm_factor_batch {t2 - t1:.3f}s", flush=True)
        for f in one + many:
            ifmm.ifmm_factor_destroy(f)
    for s in sys:
        ifmm.ifmm_system_destroy(s)
    ifmm.ifmm_ctx_destroy(ctx)


def serve(a):
    import numpy as np
    import torch

    import paper_1508_01835_gb300 as ifmm
    import workloads
    ws = _capped(workloads.serving_cube_system, a.systems or 8, a.nmax or 32768)
    ctx = ifmm.ifmm_ctx_create(0)
    sys = [ifmm.ifmm_system_create(ctx, torch.tensor(w.points, device="cuda"),
                                   ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag),
                                   ifmm.make_options(dim=3, cheb_n=w.cheb_n, leaf_max=w.leaf_max,
                                                     eps=w.eps, schur=ifmm.P_FP32, symmetric=1))
           for w in ws]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    facs = ifmm.ifmm_factor_batch(ctx, sys)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    srv = ifmm.ifmm_server_create(ctx, 160 << 30, workers=4)
    ids = [ifmm.ifmm_server_register(srv, s, f, maxit=100) for s, f in zip(sys, facs)]
    rng = np.random.default_rng(5999)
    pending, lats, shed, solved, worst = [], [], 0, 0, 0.0
    t_start = time.perf_counter()
    t_next = t_start
    while True:
        now = time.perf_counter()
        if now - t_start >= a.seconds:
            window = now - t_start
            break
        while t_next <= now:
            i = int(rng.integers(len(ws)))
            k = int(rng.integers(1, 33))
            b = np.ascontiguousarray(rng.standard_normal((k, ws[i].N)))
            x = np.zeros_like(b)
            try:
                pending.append((ifmm.ifmm_server_submit(srv, ids[i], b, x, 1e-10, 100), k, b, x))
            except ifmm.ServerError:
                shed += 1
            t_next += rng.exponential(1.0 / a.rate)
        keep = []
        for t, k, b, x in pending:
            st, reps, lat = ifmm.ifmm_server_wait(srv, t, k, 0)
            if st == 6:
                keep.append((t, k, b, x))
                continue
            lats.append(lat)
            solved += k
            worst = max(worst, max(r.true_rel_residual for r in reps))
        pending = keep
        time.sleep(0.0005)
    for t, k, b, x in pending:  # drain (not counted in the window's throughput)
        st, reps, lat = ifmm.ifmm_server_wait(srv, t, k, -1)
        lats.append(lat)
    used, blocks, cols, _ = ifmm.ifmm_server_stats(srv)
    lats.sort()
    p50 = lats[len(lats) // 2] if lats else float("nan")
    p99 = lats[min(len(lats) - 1, int(0.99 * len(lats)))] if lats else float("nan")
    print(f"[serve {len(ws)} cube systems N={min(w.N for w in ws)}..{max(w.N for w in ws)} "
          f"rate={a.rate}/s for {a.seconds}s] factor_batch {tf:.2f}s, admitted "
          f"{len(lats)} requests, shed {shed}, solved {solved} RHS in the window "
          f"({solved / window:.1f} solves/s), p50 {p50 * 1e3:.1f} ms, p99 {p99 * 1e3:.1f} ms, "
          f"{blocks} GMRES blocks, worst true residual {worst:.2e}, admitted device memory "
          f"{used / 2**30:.1f} GiB", flush=True)
    ifmm.ifmm_server_destroy(srv)
    for f in facs:
        ifmm.ifmm_factor_destroy(f)
    for s in sys:
        ifmm.ifmm_system_destroy(s)
    ifmm.ifmm_ctx_destroy(ctx)


if __name__ == "__main__":
    main()
