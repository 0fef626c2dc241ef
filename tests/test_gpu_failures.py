"""Failure handling through the C ABI, with every failure made on the host.

* GMRES that stops at maxit reports IFMM_ERR_NOT_CONVERGED with its report filled.
* A poisoned input -- two coincident points and a zero diagonal, so two rows
  of A (and of a leaf's pivot block) are equal -- makes the pivot test fire:
  IFMM_ERR_SINGULAR_PIVOT, the factorisation handle still valid.
* A device allocation the library cannot make (a Krylov basis for an absurd
  maxit) surfaces as IFMM_ERR_OOM and leaves the context usable.
* The server sheds a request when its system already has a full block queued,
  and ifmm_server_wait with a limit returns IFMM_ERR_TIMEOUT and keeps the
  ticket valid.
No GPU fault, trap or hang is involved: the kernels only see finite or
NaN/Inf data and every loop is bounded by sizes or iteration caps.
"""
import numpy as np
import pytest
import torch

import paper_1508_01835_gb300 as ifmm
from tests.gpu_util import cuda, kernel, opts
from workloads import Kernel, K_INV_R, cube_2k, small_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1508_01835_gb300 import build
    build.build()
    c = ifmm.ifmm_ctx_create(0)
    yield c
    ifmm.ifmm_ctx_destroy(c)


def test_gmres_not_converged_at_small_maxit(ctx):
    w = cube_2k()
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w))
    try:
        b = cuda(w.rhs(1)[:, 0])
        x = torch.empty_like(b)
        reps = (ifmm.GmresReport * 1)()          # unpreconditioned, 2 steps: C status 5
        st = ifmm.lib().gmres_solve(ctx, sys, None, ifmm.MV_FMM, ifmm.P(b.data_ptr()),
                                    ifmm.P(x.data_ptr()), 1, w.N, 1e-10, 2, reps,
                                    ifmm.P(torch.cuda.current_stream().cuda_stream))
        assert st == 5
        assert reps[0].iters == 2 and reps[0].status == 5 and reps[0].rel_residual > 1e-10
        assert np.isfinite(reps[0].true_rel_residual)
    finally:
        ifmm.ifmm_system_destroy(sys)


def test_singular_pivot_from_coincident_points(ctx):
    w = small_cube(600, 3, cheb_n=3, leaf_max=16, eps=1e-6)
    pts = w.points.copy()
    pts[1] = pts[0]                       # coincident pair: equal rows when A_ii = A_01
    k = ifmm.Kernel(K_INV_R, 0.0, 0.0)   # zero diagonal; coincident points take it too
    sys = ifmm.ifmm_system_create(ctx, cuda(pts), k, opts(w))
    try:
        with pytest.raises(ifmm.IFMMError) as e:
            ifmm.ifmm_factor(ctx, sys)
        assert e.value.status == 4
        fac = ifmm.ifmm_factor(ctx, sys, allow_singular=True)   # the handle stays valid
        assert ifmm.ifmm_factor_get_info(fac).singular_pivots >= 1
        ifmm.ifmm_factor_destroy(fac)
    finally:
        ifmm.ifmm_system_destroy(sys)
    # the context still works
    w2 = small_cube(600, 3, cheb_n=3, leaf_max=16, eps=1e-6)
    s2 = ifmm.ifmm_system_create(ctx, cuda(w2.points), kernel(w2), opts(w2))
    f2 = ifmm.ifmm_factor(ctx, s2)
    assert ifmm.ifmm_factor_get_info(f2).singular_pivots == 0
    ifmm.ifmm_factor_destroy(f2)
    ifmm.ifmm_system_destroy(s2)


def test_device_allocation_failure_is_reported(ctx):
    w = small_cube(3000, 7, cheb_n=3, leaf_max=32, eps=1e-6)
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w))
    try:
        b = cuda(w.rhs(1)[:, 0])
        x = torch.empty_like(b)
        # the Hessenberg storage of (maxit + 1) x maxit doubles is ~8e16 bytes
        with pytest.raises(ifmm.IFMMError) as e:
            ifmm.gmres_solve(ctx, sys, None, ifmm.MV_FMM, b, x, w.N, 1e-10, 100_000_000)
        assert e.value.status == 2
        y1, y2 = torch.empty_like(b), torch.empty_like(b)   # the context still works
        ifmm.fmm_matvec(ctx, sys, ifmm.MV_FMM, b, y1, w.N)
        ifmm.fmm_matvec(ctx, sys, ifmm.MV_FMM, b, y2, w.N)
        assert torch.equal(y1, y2) and bool(torch.isfinite(y1).all())
    finally:
        ifmm.ifmm_system_destroy(sys)


def test_server_sheds_and_wait_times_out(ctx):
    w = small_cube(20000, 11, cheb_n=3, leaf_max=64, eps=1e-6)
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w))
    fac = ifmm.ifmm_factor(ctx, sys)
    srv = ifmm.ifmm_server_create(ctx, 64 << 30, workers=1)
    try:
        sid = ifmm.ifmm_server_register(srv, sys, fac, maxit=200)
        rng = np.random.default_rng(2)
        bufs, tickets, shed = [], [], 0
        for _ in range(6):   # 6 blocks of 32 columns at once: at most one runs, one queues
            b = np.ascontiguousarray(rng.standard_normal((32, w.N)))
            x = np.zeros_like(b)
            bufs.append((b, x))
            try:
                tickets.append(ifmm.ifmm_server_submit(srv, sid, b, x, 1e-10, 200))
            except ifmm.ServerError as e:
                assert e.status == 7
                shed += 1
        assert shed >= 1
        assert ifmm.ifmm_server_stats(srv)[3] == shed
        st, _, _ = ifmm.ifmm_server_wait(srv, tickets[-1], 32, 0)   # not done yet
        assert st == 6
        for t in tickets:                                            # tickets stay valid
            st, reps, lat = ifmm.ifmm_server_wait(srv, t, 32, -1)
            assert st == 0 and all(r.true_rel_residual <= 1e-10 for r in reps)
    finally:
        ifmm.ifmm_server_destroy(srv)
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)
