"""Python binding of the GB300 IFMM library (include/ifmm.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libifmm.so``.  PyTorch provides device memory and streams.  Vectors are
passed as CUDA tensors of shape (N,) or (nrhs, N) (contiguous, float64), i.e.
column-major N x nrhs with leading dimension N, in user point order.

The functions carry the C names; ``IFMMSolver`` bundles them for convenience.
If the library has not been built, every call raises RuntimeError -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libifmm.so")

IFMM_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
          4: "singular pivot block", 5: "GMRES did not converge", 6: "timeout",
          7: "memory budget exceeded", 8: "unsupported"}
K_INV_R, K_GAUSSIAN, K_PAPER_D = 0, 1, 2
P_FP64, P_TF32, P_BF16, P_FP32 = 0, 1, 2, 3
MV_FMM, MV_DIRECT = 0, 1
GMRES_RIGHT, GMRES_LEFT, GMRES_FLEXIBLE = 0, 1, 2


class Kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("param", C.c_double), ("diag", C.c_double)]


class Options(C.Structure):
    _fields_ = [("dim", C.c_int), ("cheb_n", C.c_int), ("leaf_max", C.c_int), ("eps", C.c_double),
                ("schur", C.c_int), ("tau_override", C.c_double), ("rank_cap", C.c_int),
                ("fmm_n", C.c_int), ("rsvd_rows", C.c_int), ("symmetric", C.c_int)]


class GmresReport(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("status", C.c_int)]


class GmresOptions(C.Structure):
    _fields_ = [("side", C.c_int), ("refine", C.c_int), ("precond_precision", C.c_int),
                ("block", C.c_int), ("matvec_precision", C.c_int)]


class SystemInfo(C.Structure):
    _fields_ = [("N", C.c_longlong), ("dim", C.c_int), ("levels", C.c_int),
                ("boxes", C.c_int * 32), ("max_leaf", C.c_int), ("lo", C.c_double * 3),
                ("edge", C.c_double)]


class FactorInfo(C.Structure):
    _fields_ = [("sigma0", C.c_double), ("sigma0_iters", C.c_int), ("tau", C.c_double),
                ("levels", C.c_int), ("top_size", C.c_int), ("max_rank", C.c_int * 32),
                ("avg_rank", C.c_double * 32), ("rank_capped", C.c_int),
                ("singular_pivots", C.c_int),
                ("flops_lu", C.c_double), ("flops_trsm", C.c_double), ("flops_schur", C.c_double),
                ("flops_lowrank", C.c_double), ("flops_top", C.c_double),
                ("seconds_init", C.c_double), ("seconds_sigma0", C.c_double),
                ("seconds_elim", C.c_double), ("seconds_top", C.c_double),
                ("factor_bytes", C.c_longlong)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_longlong), ("seconds", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


class IFMMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
P = C.c_void_p


def lib() -> C.CDLL:
    """The loaded C library; raises if it was not built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"IFMM CUDA library missing ({LIB_PATH}); build it with "
                           "`python -m paper_1508_01835_gb300.build`")
    L = C.CDLL(LIB_PATH)
    sig = {
        "ifmm_status_string": (C.c_char_p, [C.c_int]),
        "ifmm_ctx_create": (C.c_int, [C.c_int, C.POINTER(P)]),
        "ifmm_ctx_destroy": (None, [P]),
        "ifmm_last_error": (C.c_char_p, [P]),
        "ifmm_system_create": (C.c_int, [P, P, C.c_longlong, C.POINTER(Kernel),
                                         C.POINTER(Options), P, C.POINTER(P)]),
        "ifmm_system_create_host": (C.c_int, [P, P, C.c_longlong, C.POINTER(Kernel),
                                              C.POINTER(Options), P, C.POINTER(P)]),
        "ifmm_system_destroy": (None, [P]),
        "ifmm_system_get_info": (C.c_int, [P, C.POINTER(SystemInfo)]),
        "ifmm_system_get_perm": (C.c_int, [P, P]),
        "ifmm_sigma0": (C.c_int, [P, P, P, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
        "ifmm_factor": (C.c_int, [P, P, P, C.POINTER(P)]),
        "ifmm_factor_destroy": (None, [P]),
        "ifmm_factor_get_info": (C.c_int, [P, C.POINTER(FactorInfo)]),
        "ifmm_factor_get_ranks": (C.c_int, [P, C.c_int, P, C.c_int, C.POINTER(C.c_int)]),
        "ifmm_factor_footprint": (C.c_int, [P, C.POINTER(C.c_ulonglong)]),
        "ifmm_solve": (C.c_int, [P, P, P, P, C.c_int, C.c_longlong, P]),
        "ifmm_solve_prec": (C.c_int, [P, P, C.c_int, P, P, C.c_int, C.c_longlong, P]),
        "fmm_matvec": (C.c_int, [P, P, C.c_int, P, P, C.c_int, C.c_longlong, P]),
        "fmm_matvec_prec": (C.c_int, [P, P, C.c_int, P, P, C.c_int, C.c_longlong, P]),
        "gmres_solve": (C.c_int, [P, P, P, C.c_int, P, P, C.c_int, C.c_longlong, C.c_double,
                                  C.c_int, C.POINTER(GmresReport), P]),
        "gmres_solve_ex": (C.c_int, [P, P, P, C.c_int, P, P, C.c_int, C.c_longlong, C.c_double,
                                     C.c_int, C.POINTER(GmresOptions), C.POINTER(GmresReport),
                                     P]),
        "gmres_solve_host": (C.c_int, [P, P, P, C.c_int, P, P, C.c_int, C.c_longlong,
                                       C.c_double, C.c_int, C.POINTER(GmresReport), P]),
        "fmm_matvec_static": (C.c_int, [P, P, P, P, C.c_int, C.c_longlong, P]),
        "ifmm_factor_batch": (C.c_int, [P, P, C.c_int, P, P]),
        "ifmm_server_create": (C.c_int, [P, C.c_ulonglong, C.c_int, C.POINTER(P)]),
        "ifmm_server_create_ex": (C.c_int, [P, C.c_ulonglong, C.c_int, C.c_int, C.POINTER(P)]),
        "ifmm_server_submit_device": (C.c_int, [P, C.c_int, P, P, C.c_int, C.c_double, C.c_int,
                                                C.POINTER(C.c_longlong)]),
        "ifmm_server_destroy": (None, [P]),
        "ifmm_server_set_reserve": (C.c_int, [P, C.c_ulonglong]),
        "ifmm_server_set_matvec_precision": (C.c_int, [P, C.c_int]),
        "ifmm_server_register": (C.c_int, [P, P, P, C.c_int, C.POINTER(C.c_int)]),
        "ifmm_server_submit": (C.c_int, [P, C.c_int, P, P, C.c_int, C.c_double, C.c_int,
                                         C.POINTER(C.c_longlong)]),
        "ifmm_server_wait": (C.c_int, [P, C.c_longlong, C.c_int, C.POINTER(GmresReport),
                                       C.POINTER(C.c_double)]),
        "ifmm_server_stats": (C.c_int, [P, C.POINTER(C.c_ulonglong), C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "ifmm_server_last_error": (C.c_char_p, [P]),
        "ifmm_schur_product": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_int, P, C.c_int,
                                         C.c_int, P, C.c_int, C.c_int, P, C.c_int, C.c_double,
                                         C.c_double, P]),
        "ifmm_measure_peaks": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "ifmm_launch_count": (C.c_int, [C.POINTER(C.c_ulonglong)]),
        "ifmm_profile_start": (C.c_int, [P]),
        "ifmm_profile_stop": (C.c_int, [P, C.POINTER(KernelStat), C.c_int, C.POINTER(C.c_int)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(st: int, ctx=None, allow=()):
    if st != IFMM_OK and st not in allow:
        msg = lib().ifmm_last_error(ctx).decode() if ctx else ""
        raise IFMMError(st, msg)
    return st


def _stream(stream):
    if stream is None:
        import torch
        return P(torch.cuda.current_stream().cuda_stream)
    return P(int(stream))


def _vec(t, N):
    """(pointer, nrhs, ld) of a float64 CUDA tensor of shape (N,) or (nrhs, N)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError("vectors must be float64 CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("vectors must be contiguous")
    if t.dim() == 1 and t.shape[0] == N:
        return P(t.data_ptr()), 1, N
    if t.dim() == 2 and t.shape[1] == N:
        return P(t.data_ptr()), t.shape[0], N
    raise ValueError(f"expected shape ({N},) or (nrhs, {N}), got {tuple(t.shape)}")


# ---- C-named wrappers --------------------------------------------------------------
def ifmm_ctx_create(device: int = 0):
    h = P()
    _check(lib().ifmm_ctx_create(device, C.byref(h)))
    return h


def ifmm_ctx_destroy(ctx):
    lib().ifmm_ctx_destroy(ctx)


def make_options(dim=3, cheb_n=3, leaf_max=64, eps=1e-6, schur=P_FP64, tau_override=0.0,
                 rank_cap=0, fmm_n=0, rsvd_rows=0, symmetric=0) -> Options:
    return Options(dim, cheb_n, leaf_max, eps, schur, tau_override, rank_cap, fmm_n, rsvd_rows,
                   symmetric)


def ifmm_system_create(ctx, pts, kernel: Kernel, opt: Options, stream=None):
    """pts: float64 CUDA tensor (N, dim) row-major in user order."""
    import torch
    if not (pts.is_cuda and pts.dtype == torch.float64 and pts.is_contiguous()):
        raise TypeError("points must be a contiguous float64 CUDA tensor (N, dim)")
    h = P()
    _check(lib().ifmm_system_create(ctx, P(pts.data_ptr()), pts.shape[0], C.byref(kernel),
                                    C.byref(opt), _stream(stream), C.byref(h)), ctx)
    return h


def ifmm_system_create_host(ctx, pts_np, kernel: Kernel, opt: Options, stream=None):
    import numpy as np
    a = np.ascontiguousarray(pts_np, dtype=np.float64)
    h = P()
    _check(lib().ifmm_system_create_host(ctx, a.ctypes.data_as(P), a.shape[0], C.byref(kernel),
                                         C.byref(opt), _stream(stream), C.byref(h)), ctx)
    return h


def ifmm_system_destroy(sys):
    lib().ifmm_system_destroy(sys)


def ifmm_system_get_info(sys) -> SystemInfo:
    info = SystemInfo()
    _check(lib().ifmm_system_get_info(sys, C.byref(info)))
    return info


def ifmm_system_get_perm(sys, N: int):
    import numpy as np
    out = np.empty(N, dtype=np.int64)
    _check(lib().ifmm_system_get_perm(sys, out.ctypes.data_as(P)))
    return out


def ifmm_sigma0(ctx, sys, stream=None):
    s = C.c_double()
    it = C.c_int()
    _check(lib().ifmm_sigma0(ctx, sys, _stream(stream), C.byref(s), C.byref(it)), ctx)
    return s.value, it.value


def ifmm_factor(ctx, sys, stream=None, allow_singular=False):
    h = P()
    st = lib().ifmm_factor(ctx, sys, _stream(stream), C.byref(h))
    _check(st, ctx, allow=(4,) if allow_singular else ())
    return h


def ifmm_factor_destroy(fac):
    lib().ifmm_factor_destroy(fac)


def ifmm_factor_get_info(fac) -> FactorInfo:
    info = FactorInfo()
    _check(lib().ifmm_factor_get_info(fac, C.byref(info)))
    return info


def ifmm_factor_get_ranks(fac, level: int):
    n = C.c_int()
    _check(lib().ifmm_factor_get_ranks(fac, level, None, 0, C.byref(n)))
    arr = (C.c_int * max(n.value, 1))()
    _check(lib().ifmm_factor_get_ranks(fac, level, arr, n.value, C.byref(n)))
    return list(arr[:n.value])


def ifmm_factor_footprint(fac) -> int:
    b = C.c_ulonglong()
    _check(lib().ifmm_factor_footprint(fac, C.byref(b)))
    return b.value


def ifmm_solve(ctx, fac, b, x, N: int, stream=None):
    pb, k, ld = _vec(b, N)
    px, k2, _ = _vec(x, N)
    assert k == k2
    _check(lib().ifmm_solve(ctx, fac, pb, px, k, ld, _stream(stream)), ctx)


def ifmm_solve_prec(ctx, fac, prec: int, b, x, N: int, stream=None):
    pb, k, ld = _vec(b, N)
    px, k2, _ = _vec(x, N)
    assert k == k2
    _check(lib().ifmm_solve_prec(ctx, fac, prec, pb, px, k, ld, _stream(stream)), ctx)


def fmm_matvec(ctx, sys, mode: int, x, y, N: int, stream=None):
    px, k, ld = _vec(x, N)
    py, k2, _ = _vec(y, N)
    assert k == k2
    _check(lib().fmm_matvec(ctx, sys, mode, px, py, k, ld, _stream(stream)), ctx)


def fmm_matvec_prec(ctx, sys, prec: int, x, y, N: int, stream=None):
    """y = A_n x; prec P_FP32 takes the far field in FP32 (near field FP64)."""
    px, k, ld = _vec(x, N)
    py, k2, _ = _vec(y, N)
    assert k == k2
    _check(lib().fmm_matvec_prec(ctx, sys, prec, px, py, k, ld, _stream(stream)), ctx)


def fmm_matvec_static(ctx, sys, x, y, N: int, stream=None):
    """y = A_n x without any device allocation (library-owned static scratch)."""
    px, k, ld = _vec(x, N)
    py, k2, _ = _vec(y, N)
    assert k == k2
    _check(lib().fmm_matvec_static(ctx, sys, px, py, k, ld, _stream(stream)), ctx)


def gmres_solve(ctx, sys, fac, mode: int, b, x, N: int, tol=1e-10, maxit=500, stream=None):
    pb, k, ld = _vec(b, N)
    px, k2, _ = _vec(x, N)
    assert k == k2
    reps = (GmresReport * k)()
    _check(lib().gmres_solve(ctx, sys, fac, mode, pb, px, k, ld, tol, maxit, reps,
                             _stream(stream)), ctx, allow=(5,))
    return list(reps)


def gmres_solve_ex(ctx, sys, fac, mode: int, b, x, N: int, tol=1e-10, maxit=500,
                   side=GMRES_RIGHT, refine=2, precond_precision=P_FP64, block=0,
                   matvec_precision=P_FP64, stream=None):
    pb, k, ld = _vec(b, N)
    px, k2, _ = _vec(x, N)
    assert k == k2
    reps = (GmresReport * k)()
    o = GmresOptions(side, refine, precond_precision, block, matvec_precision)
    _check(lib().gmres_solve_ex(ctx, sys, fac, mode, pb, px, k, ld, tol, maxit, C.byref(o), reps,
                                _stream(stream)), ctx, allow=(5,))
    return list(reps)


def gmres_solve_host(ctx, sys, fac, mode: int, b_np, x_np, tol=1e-10, maxit=500, stream=None):
    """b_np, x_np: float64 numpy arrays of shape (nrhs, N) (C order) or (N,)."""
    import numpy as np
    assert b_np.dtype == np.float64 and x_np.dtype == np.float64
    assert b_np.flags["C_CONTIGUOUS"] and x_np.flags["C_CONTIGUOUS"]
    N = b_np.shape[-1]
    k = 1 if b_np.ndim == 1 else b_np.shape[0]
    reps = (GmresReport * k)()
    _check(lib().gmres_solve_host(ctx, sys, fac, mode, b_np.ctypes.data_as(P),
                                  x_np.ctypes.data_as(P), k, N, tol, maxit, reps,
                                  _stream(stream)), ctx, allow=(5,))
    return list(reps)


def ifmm_factor_batch(ctx, systems, stream=None, allow_singular=False):
    """Factorise several systems concurrently; returns their factorisation handles."""
    n = len(systems)
    arr = (P * max(n, 1))(*systems)
    out = (P * max(n, 1))()
    _check(lib().ifmm_factor_batch(ctx, arr, n, _stream(stream), out), ctx,
           allow=(4,) if allow_singular else ())
    return [out[i] for i in range(n)]


class ServerError(IFMMError):
    pass


def _scheck(st, srv, allow=()):
    if st != IFMM_OK and st not in allow:
        raise ServerError(st, lib().ifmm_server_last_error(srv).decode() if srv else "")
    return st


def ifmm_server_create(ctx, hbm_budget: int, workers: int = 0, precond_precision=None):
    h = P()
    if precond_precision is None:
        _check(lib().ifmm_server_create(ctx, hbm_budget, workers, C.byref(h)), ctx)
    else:
        _check(lib().ifmm_server_create_ex(ctx, hbm_budget, workers, precond_precision,
                                           C.byref(h)), ctx)
    return h


def ifmm_server_destroy(srv):
    lib().ifmm_server_destroy(srv)


def ifmm_server_set_reserve(srv, nbytes: int):
    _scheck(lib().ifmm_server_set_reserve(srv, nbytes), srv)


def ifmm_server_set_matvec_precision(srv, prec: int):
    _scheck(lib().ifmm_server_set_matvec_precision(srv, prec), srv)


def ifmm_server_register(srv, sys, fac, maxit: int = 100) -> int:
    i = C.c_int()
    _scheck(lib().ifmm_server_register(srv, sys, fac, maxit, C.byref(i)), srv)
    return i.value


def ifmm_server_submit(srv, sid: int, b_np, x_np, tol=1e-10, maxit=100) -> int:
    """b_np, x_np: float64 numpy arrays (nrhs, N) C order (or (N,)); both must
    stay alive until the ticket is waited for."""
    import numpy as np
    assert b_np.dtype == np.float64 and x_np.dtype == np.float64
    assert b_np.flags["C_CONTIGUOUS"] and x_np.flags["C_CONTIGUOUS"]
    k = 1 if b_np.ndim == 1 else b_np.shape[0]
    t = C.c_longlong()
    _scheck(lib().ifmm_server_submit(srv, sid, b_np.ctypes.data_as(P), x_np.ctypes.data_as(P), k,
                                     tol, maxit, C.byref(t)), srv)
    return t.value


def ifmm_server_submit_device(srv, sid: int, b, x, N: int, tol=1e-10, maxit=100) -> int:
    """b, x: float64 CUDA tensors (nrhs, N) or (N,); both must stay alive until
    the ticket is waited for."""
    pb, k, _ = _vec(b, N)
    px, k2, _ = _vec(x, N)
    assert k == k2
    t = C.c_longlong()
    _scheck(lib().ifmm_server_submit_device(srv, sid, pb, px, k, tol, maxit, C.byref(t)), srv)
    return t.value


def ifmm_server_wait(srv, ticket: int, nrhs: int, timeout_ms: int = -1):
    """(status, reports, latency seconds); status 6 (timeout) leaves the ticket valid."""
    reps = (GmresReport * nrhs)()
    lat = C.c_double()
    st = lib().ifmm_server_wait(srv, ticket, timeout_ms, reps, C.byref(lat))
    return st, list(reps), lat.value


def ifmm_server_stats(srv):
    """(admitted device bytes, GMRES blocks, columns solved, requests shed)."""
    u, b, c, d = C.c_ulonglong(), C.c_longlong(), C.c_longlong(), C.c_longlong()
    _scheck(lib().ifmm_server_stats(srv, C.byref(u), C.byref(b), C.byref(c), C.byref(d)), srv)
    return u.value, b.value, c.value, d.value


def ifmm_schur_product(ctx, prec: int, M: int, N: int, K: int, A, lda: int, transA: int, B,
                       ldb: int, transB: int, Cm, ldc: int, alpha=1.0, beta=0.0, stream=None):
    """C = alpha op(A) op(B) + beta C with the elimination's Schur-product kernel
    at precision `prec`.  A, B, Cm: contiguous float64 CUDA tensors whose memory
    holds column-major matrices with the given leading dimensions."""
    import torch
    for t in (A, B, Cm):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous()):
            raise TypeError("operands must be contiguous float64 CUDA tensors")
    _check(lib().ifmm_schur_product(ctx, prec, M, N, K, P(A.data_ptr()), lda, transA,
                                    P(B.data_ptr()), ldb, transB, P(Cm.data_ptr()), ldc,
                                    alpha, beta, _stream(stream)), ctx)


def ifmm_measure_peaks(ctx):
    """(FP64, FP32) TFLOP/s measured on the context's device."""
    a, b = C.c_double(), C.c_double()
    _check(lib().ifmm_measure_peaks(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def ifmm_launch_count() -> int:
    """Kernel launches the library has made in this process so far."""
    n = C.c_ulonglong()
    _check(lib().ifmm_launch_count(C.byref(n)))
    return n.value


def ifmm_profile_start(ctx):
    _check(lib().ifmm_profile_start(ctx), ctx)


def ifmm_profile_stop(ctx):
    """Per-kernel totals {name: (launches, seconds, flops, bytes)} since profile_start."""
    arr = (KernelStat * 64)()
    n = C.c_int()
    _check(lib().ifmm_profile_stop(ctx, arr, 64, C.byref(n)), ctx)
    return {arr[i].name.decode(): (arr[i].launches, arr[i].seconds, arr[i].flops, arr[i].bytes)
            for i in range(min(n.value, 64))}


class IFMMSolver:
    """Owns a context, a system and (after factor()) a factorisation."""

    def __init__(self, points, kernel: Kernel, opt: Options, device: int = 0, stream=None):
        import torch
        self.ctx = ifmm_ctx_create(device)
        self.N = int(points.shape[0])
        if isinstance(points, torch.Tensor):
            self.sys = ifmm_system_create(self.ctx, points, kernel, opt, stream)
        else:
            self.sys = ifmm_system_create_host(self.ctx, points, kernel, opt, stream)
        self.fac = None
        self.stream = stream

    def factor(self):
        if self.fac is not None:
            ifmm_factor_destroy(self.fac)
        self.fac = ifmm_factor(self.ctx, self.sys, self.stream)
        return ifmm_factor_get_info(self.fac)

    def solve(self, b, x=None):
        import torch
        x = torch.empty_like(b) if x is None else x
        ifmm_solve(self.ctx, self.fac, b, x, self.N, self.stream)
        return x

    def matvec(self, x, mode=MV_FMM, y=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        fmm_matvec(self.ctx, self.sys, mode, x, y, self.N, self.stream)
        return y

    def gmres(self, b, mode=MV_FMM, tol=1e-10, maxit=500, precondition=True, x=None):
        import torch
        x = torch.empty_like(b) if x is None else x
        reps = gmres_solve(self.ctx, self.sys, self.fac if precondition else None, mode, b, x,
                           self.N, tol, maxit, self.stream)
        return x, reps

    def close(self):
        if getattr(self, "fac", None) is not None:
            ifmm_factor_destroy(self.fac)
            self.fac = None
        if getattr(self, "sys", None) is not None:
            ifmm_system_destroy(self.sys)
            self.sys = None
        if getattr(self, "ctx", None) is not None:
            ifmm_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
