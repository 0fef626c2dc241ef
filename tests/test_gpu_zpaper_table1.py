"""The GMRES experiment of Sec. 3.2 on the GPU path, against the iteration
counts the paper prints in Table 1 (tests/golden/table1_gmres_d1e-3.txt).

N = 100,000 points uniform in [-1, 1]^3 (seeded; the paper's own points are
not available), kernel of Eq. (K_ij) with d = 1e-3, eps = 1e-3, leaves of at
most 100 points, the paper's general algorithm in FP64, GMRES to 1e-10 with a
fixed 5^3 Chebyshev FMM matvec.  Unpreconditioned and with the IFMM of order
n = 1 the counts must be within 2 of the printed 78 and 19 (the point
realisation differs); for every n the IFMM must cut the iteration count well
below the unpreconditioned one and GMRES must reach the residual.  (For
n >= 2 more iterations than printed are needed; the reading of sigma_0(E)
alone does not explain the difference.)
"""
import os

import numpy as np
import pytest
import torch

import paper_1508_01835_gb300 as ifmm
import workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "table1_gmres_d1e-3.txt")


def printed():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, it, res = line.split()
                rows[int(n)] = (int(it), float(res))
    return rows


@pytest.fixture(scope="module")
def ctx():
    from paper_1508_01835_gb300 import build
    build.build()
    c = ifmm.ifmm_ctx_create(0)
    yield c
    ifmm.ifmm_ctx_destroy(c)


def run(ctx, n):
    w = workloads.paper_cube(100000, 1e-3, max(n, 1), leaf_max=100)
    opt = ifmm.make_options(dim=3, cheb_n=max(n, 1), leaf_max=w.leaf_max, eps=w.eps, fmm_n=5)
    sys = ifmm.ifmm_system_create(ctx, torch.tensor(w.points, device="cuda"),
                                  ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag), opt)
    try:
        fac = ifmm.ifmm_factor(ctx, sys) if n > 0 else None
        try:
            b = torch.tensor(w.rhs(1)[:, 0], device="cuda")
            x = torch.empty_like(b)
            reps = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_FMM, b, x, w.N, 1e-10, 500)
            return reps[0]
        finally:
            if fac is not None:
                ifmm.ifmm_factor_destroy(fac)
    finally:
        ifmm.ifmm_system_destroy(sys)


def test_table1_iteration_counts(ctx):
    table = printed()
    its = {}
    for n in (0, 1, 2, 3):
        rep = run(ctx, n)
        assert rep.status == 0 and rep.true_rel_residual <= 1e-10, (n, rep.iters)
        its[n] = rep.iters
        print(f"n={n}: {rep.iters} iterations (Table 1: {table[n][0]}), "
              f"true residual {rep.true_rel_residual:.1e}")
    assert abs(its[0] - table[0][0]) <= 2
    assert abs(its[1] - table[1][0]) <= 2
    for n in (2, 3):
        assert its[n] <= its[1] and 4 * its[n] <= its[0]
