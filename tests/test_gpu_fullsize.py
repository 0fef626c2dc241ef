"""The bench's workload at full size (N = 65,536, 1/r, Chebyshev 4^3, eps = 1e-8),
in the configurations bench.py times, checked through properties that hold at
any size and on outputs the oracle computes row by row:

* GMRES (FMM matvec, IFMM right preconditioner) reaches a true relative
  residual <= 1e-10 with the plain FP64 factorisation (the paper's general
  algorithm) and with the timed one (split-TF32 Schur products, symmetric
  variant); the two solutions agree to what that residual allows;
* sampled rows of the DIRECT product equal the oracle's kernel rows
  (Sec. 3.1) to the rounding of an N-term FP64 sum, and sampled rows of the
  FMM product (the operator A_n GMRES solves with, Sec. 3.2) stay within the
  Chebyshev interpolation error of n = 4 on each row's absolute scale
  sum_j |a_ij x_j| (the oracle's FMM at N = 8192 differs from the kernel by
  about 5e-4 of ||A x|| for a random x);
* every rank respects the n^D cap and the top system is no larger than
  64 boxes x 64.
"""
import numpy as np
import pytest
import torch

import paper_1508_01835_gb300 as ifmm
import workloads
from oracle.kernels import kernel_matrix
from tests.gpu_util import cuda, kernel, opts, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1508_01835_gb300 import build
    build.build()
    c = ifmm.ifmm_ctx_create(0)
    yield c
    ifmm.ifmm_ctx_destroy(c)


def test_bench_workload_full_size(ctx):
    w = workloads.cube_64k()
    b = cuda(w.rhs(1)[:, 0])
    xs = {}
    for name, kw in {"fp64-general": dict(schur=ifmm.P_FP64, symmetric=0),
                     "fp32-symmetric": dict(schur=ifmm.P_FP32, symmetric=1)}.items():
        sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w, **kw))
        try:
            fac = ifmm.ifmm_factor(ctx, sys)
            try:
                info = ifmm.ifmm_factor_get_info(fac)
                for l in range(2, info.levels + 1):
                    assert max(ifmm.ifmm_factor_get_ranks(fac, l)) <= 64
                assert info.top_size <= 64 * 64
                x = torch.empty_like(b)
                reps = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_FMM, b, x, w.N, 1e-10, 500)
                assert reps[0].status == 0 and reps[0].true_rel_residual <= 1e-10, \
                    (name, reps[0].iters, reps[0].true_rel_residual)
                xs[name] = x
                print(f"{name}: {reps[0].iters} GMRES iterations, true residual "
                      f"{reps[0].true_rel_residual:.2e}")
            finally:
                ifmm.ifmm_factor_destroy(fac)
            if name == "fp64-general":
                rows = np.random.default_rng(3).choice(w.N, 48, replace=False)
                xh = xs[name].cpu().numpy()
                Arows = kernel_matrix(w.kernel.kind, w.kernel.param, w.kernel.diag,
                                      w.points[rows], w.points)
                exact = Arows @ xh
                scale = np.abs(Arows) @ np.abs(xh)  # sum_j |a_ij x_j|: the rounding scale
                yd, yf = torch.empty_like(b), torch.empty_like(b)
                ifmm.fmm_matvec(ctx, sys, ifmm.MV_DIRECT, xs[name], yd, w.N)
                ifmm.fmm_matvec(ctx, sys, ifmm.MV_FMM, xs[name], yf, w.N)
                torch.cuda.synchronize()
                yd, yf = yd.cpu().numpy(), yf.cpu().numpy()
                # two FP64 sums of N terms in different orders: each is within
                # about u sqrt(N) sum_j |a_ij x_j| of the exact row (u = 2^-53)
                assert np.all(np.abs(yd[rows] - exact) <= 4 * 2.0 ** -53 * np.sqrt(w.N) * scale)
                # the FMM differs from the kernel by the Chebyshev interpolation
                # error of each far-field entry: bounded on the row's absolute
                # scale (the solution x cancels A's smooth part, so |A x| itself
                # is far smaller than that scale)
                ratio = np.max(np.abs(yf[rows] - exact) / scale)
                print(f"FMM rows: max |A_n x - A x| / sum|a x| = {ratio:.2e}")
                assert ratio < 1e-3
        finally:
            ifmm.ifmm_system_destroy(sys)
    # both residuals are <= 1e-10; kappa(A_n) is ~ 1.5e3 here (largest eigenvalue ~ N
    # times the mean of 1/r, smallest ~ the diagonal 2 N^(1/3))
    assert rel(xs["fp32-symmetric"].cpu().numpy(), xs["fp64-general"].cpu().numpy()) < 1e-6
