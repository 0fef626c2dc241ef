"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Every case builds the same seeded inputs on both sides.  Integer structure
(tree order, box counts, ranks) must agree exactly; floating point within the
tolerances stated per test (FP64 rounding differences only).
"""
import math

import numpy as np
import pytest
import torch

import paper_1508_01835_gb300 as ifmm
from oracle.gmres import gmres as oracle_gmres
from oracle.ifmm import IFMM, sigma0_power
from tests.gpu_util import cuda, dense_an_solve, kernel, opts, oracle_h2, rel, to_user
from workloads import Kernel, K_GAUSSIAN, K_INV_R, K_PAPER_D, cube_2k, small_cube

pytestmark = pytest.mark.gpu

CASES = {
    "cube2k": lambda: cube_2k(),                                                   # L = 2, n = 3
    "3lev": lambda: small_cube(3000, 7, cheb_n=3, leaf_max=32, eps=1e-6),  # L = 3, one merge
    "2d": lambda: small_cube(2500, 9, cheb_n=4, leaf_max=20, eps=1e-8, dim=2,
                             kernel=Kernel(K_GAUSSIAN, 0.05, 1.01)),
    "paper": lambda: small_cube(1800, 5, cheb_n=2, leaf_max=16, eps=1e-4,
                                kernel=Kernel(K_PAPER_D, 0.05, 1.0)),
    "ragged": lambda: small_cube(1001, 3, cheb_n=3, leaf_max=13, eps=1e-7),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_1508_01835_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    c = ifmm.ifmm_ctx_create(0)
    yield c
    ifmm.ifmm_ctx_destroy(c)


def make_sys(ctx, w, **kw):
    return ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w, **kw))


@pytest.mark.parametrize("name", sorted(CASES))
def test_tree_matches_oracle(ctx, name):
    w = CASES[name]()
    h2 = oracle_h2(w)
    sys = make_sys(ctx, w)
    try:
        info = ifmm.ifmm_system_get_info(sys)
        assert info.levels == h2.tree.L
        for l in range(h2.tree.L + 1):
            assert info.boxes[l] == h2.tree.levels[l].nb
        perm = ifmm.ifmm_system_get_perm(sys, w.N)
        assert np.array_equal(perm, h2.tree.perm)
    finally:
        ifmm.ifmm_system_destroy(sys)


@pytest.mark.parametrize("name", ["cube2k", "2d", "ragged", "3lev", "paper"])
def test_matvec_parity(ctx, name):
    w = CASES[name]()
    h2 = oracle_h2(w)
    sys = make_sys(ctx, w)
    try:
        X = np.random.default_rng(3).standard_normal((3, w.N))
        x = cuda(X)
        y = torch.empty_like(x)
        ifmm.fmm_matvec(ctx, sys, ifmm.MV_FMM, x, y, w.N)
        p = h2.tree.perm
        ref = np.stack([to_user(h2, h2.matvec(X[c][p])) for c in range(3)])
        assert rel(y.cpu().numpy(), ref) < 1e-13
        ifmm.fmm_matvec(ctx, sys, ifmm.MV_DIRECT, x, y, w.N)
        refd = np.stack([to_user(h2, h2.direct_matvec(X[c][p])) for c in range(3)])
        assert rel(y.cpu().numpy(), refd) < 1e-13
    finally:
        ifmm.ifmm_system_destroy(sys)


@pytest.mark.parametrize("name", ["cube2k", "3lev"])
def test_sigma0_parity(ctx, name):
    w = CASES[name]()
    h2 = oracle_h2(w)
    s_ref, it_ref = sigma0_power(h2)
    sys = make_sys(ctx, w)
    try:
        s, it = ifmm.ifmm_sigma0(ctx, sys)
        assert it == it_ref
        assert abs(s - s_ref) <= 1e-10 * s_ref
    finally:
        ifmm.ifmm_system_destroy(sys)


@pytest.mark.parametrize("N,n,leaf,dim,kern", [
    (600, 3, 16, 3, None),
    (1500, 2, 12, 3, Kernel(K_INV_R, 0.0, 3000.0)),
    (900, 3, 10, 2, Kernel(K_GAUSSIAN, 0.15, 1.01)),
])
def test_tau_zero_is_exact(ctx, N, n, leaf, dim, kern):
    """Compression disabled: the GPU factorisation is an exact block LU of E."""
    w = small_cube(N, 21, cheb_n=n, leaf_max=leaf, dim=dim, kernel=kern)
    h2 = oracle_h2(w)
    b = np.random.default_rng(1).standard_normal(N)
    x_ref, kappa = dense_an_solve(h2, b)
    sys = make_sys(ctx, w, eps=0.0)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        x = torch.empty(N, dtype=torch.float64, device="cuda:0")
        ifmm.ifmm_solve(ctx, fac, cuda(b), x, N)
        assert rel(x.cpu().numpy(), x_ref) < 1e-14 * kappa * 50
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


@pytest.mark.parametrize("name", sorted(CASES))
def test_factor_solve_parity(ctx, name):
    """Same tau on both sides: equal ranks, equal solve output to rounding."""
    w = CASES[name]()
    h2 = oracle_h2(w)
    ora = IFMM(h2, w.eps)
    sys = make_sys(ctx, w, tau=ora.tau, rank_cap=1 << 20)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        for l in range(2, h2.tree.L + 1):
            g = ifmm.ifmm_factor_get_ranks(fac, l)
            assert g == ora.ranks(l), f"ranks differ at depth {l}"
        B = w.rhs(2).T.copy()
        X = torch.empty(2, w.N, dtype=torch.float64, device="cuda:0")
        ifmm.ifmm_solve(ctx, fac, cuda(B), X, w.N)
        ref = ora.solve(B.T).T
        assert rel(X.cpu().numpy(), ref) < 1e-10
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


@pytest.mark.parametrize("name", ["cube2k", "3lev", "2d"])
def test_symmetric_variant_parity(ctx, name):
    """Reading S (one SVD per box, V side = U side) on both sides with the same
    tau: equal ranks, equal solve output to rounding."""
    w = CASES[name]()
    h2 = oracle_h2(w)
    ora = IFMM(h2, w.eps, symmetric=True)
    sys = make_sys(ctx, w, tau=ora.tau, rank_cap=1 << 20, symmetric=1)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        for l in range(2, h2.tree.L + 1):
            assert ifmm.ifmm_factor_get_ranks(fac, l) == ora.ranks(l), f"ranks differ at depth {l}"
        B = w.rhs(2).T.copy()
        X = torch.empty(2, w.N, dtype=torch.float64, device="cuda:0")
        ifmm.ifmm_solve(ctx, fac, cuda(B), X, w.N)
        assert rel(X.cpu().numpy(), ora.solve(B.T).T) < 1e-10
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


WELL = {
    "3lev": lambda: small_cube(3000, 7, cheb_n=3, leaf_max=32, eps=1e-6,
                               kernel=Kernel(K_INV_R, 0.0, 4.0 * 3000)),
    "cube2k": lambda: small_cube(2048, 1000, cheb_n=3, leaf_max=64, eps=1e-6,
                             kernel=Kernel(K_INV_R, 0.0, 4.0 * 2048)),
    "2d": lambda: small_cube(2500, 9, cheb_n=4, leaf_max=20, eps=1e-8, dim=2,
                             kernel=Kernel(K_GAUSSIAN, 0.05, 3.0)),
}


@pytest.mark.parametrize("name,cap,rows", [("3lev", 12, 20), ("cube2k", 10, 16), ("2d", 8, 16)])
def test_randomised_recompression_parity(ctx, name, cap, rows):
    """Blocks taller than `rows` under rank cap `cap` take the randomised SVD
    (Sec. 2.4) on both sides, with the same counter-based test matrix.  The
    systems are well conditioned (strong diagonal) so that the comparison
    measures the two implementations, not the amplification of rounding by
    a large condition number."""
    w = WELL[name]()
    h2 = oracle_h2(w)
    ora = IFMM(h2, w.eps, rank_cap=cap, rsvd_rows=rows)
    sys = make_sys(ctx, w, tau=ora.tau, rank_cap=cap, rsvd_rows=rows)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        for l in range(2, h2.tree.L + 1):
            assert ifmm.ifmm_factor_get_ranks(fac, l) == ora.ranks(l), f"ranks differ at depth {l}"
        b = w.rhs(1)[:, 0]
        x = torch.empty(w.N, dtype=torch.float64, device="cuda:0")
        ifmm.ifmm_solve(ctx, fac, cuda(b), x, w.N)
        assert rel(x.cpu().numpy(), ora.solve(b)) < 1e-10
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


def test_gmres_cube2k_direct_matches_dense_lu(ctx):
    """cube-2k: GMRES with the exact matvec and the IFMM preconditioner reaches
    1e-10 and agrees with the dense LU solve of A (Sec. 3.2)."""
    w = cube_2k()
    h2 = oracle_h2(w)
    b = w.rhs(1)[:, 0]
    A = h2.dense_exact()
    p = h2.tree.perm
    x_ref = to_user(h2, np.linalg.solve(A, b[p]))
    kappa = np.linalg.cond(A)
    sys = make_sys(ctx, w)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        x = torch.empty(w.N, dtype=torch.float64, device="cuda:0")
        rep = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_DIRECT, cuda(b), x, w.N, 1e-10, 500)[0]
        assert rep.status == 0 and rep.true_rel_residual <= 1e-10
        assert rel(x.cpu().numpy(), x_ref) < max(1e-8, 1e-10 * kappa * 10)
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


def _oracle_gmres(w, h2, ora, tol, side="right"):
    b = w.rhs(1)[:, 0]
    p = h2.tree.perm

    def mv(v):
        return to_user(h2, h2.matvec(v[p]))

    x, it, res = oracle_gmres(mv, b, ora.solve, tol, 500, side=side)
    return b, x, it


@pytest.mark.parametrize("name", ["cube2k", "3lev", "2d", "paper"])
def test_gmres_parity_with_oracle(ctx, name):
    """FMM matvec + IFMM right preconditioner, both sides the same
    non-restarted GMRES (refine = 0) run to tol 1e-13, so that kappa(A) ~ 1e6
    of the cube recipe does not mask a difference: same iteration count as the
    oracle's GMRES (+-1), Arnoldi estimate <= 1e-13, true residual <= 1e-10
    (without restarts the recomputed residual drifts above the estimate, by up
    to ~2e-11 on the paper-kernel case), and the same solution to 1e-10
    relative."""
    w = CASES[name]()
    h2 = oracle_h2(w)
    ora = IFMM(h2, w.eps)
    b, x_o, it_o = _oracle_gmres(w, h2, ora, 1e-13)
    sys = make_sys(ctx, w, tau=ora.tau, rank_cap=1 << 20)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        x = torch.empty(w.N, dtype=torch.float64, device="cuda:0")
        rep = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, cuda(b), x, w.N, 1e-13, 500,
                                  refine=0)[0]
        err = rel(x.cpu().numpy(), x_o)
        print(f"{name}: GMRES {rep.iters} it (oracle {it_o}), true residual "
              f"{rep.true_rel_residual:.1e}, |x - x_oracle| / |x_oracle| = {err:.1e}")
        assert rep.rel_residual <= 1e-13 and rep.true_rel_residual <= 1e-10
        assert abs(rep.iters - it_o) <= 1
        assert err < 1e-10
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


@pytest.mark.parametrize("name", ["cube2k", "3lev"])
def test_left_preconditioned_gmres_parity(ctx, name):
    """Appendix B: the IFMM as left preconditioner on both sides; the stopping
    criterion is the preconditioned residual.  Same iteration count (+-1), the
    same solution to 1e-10 at tol 1e-13, and the true residual reported."""
    w = CASES[name]()
    h2 = oracle_h2(w)
    ora = IFMM(h2, w.eps)
    b, x_o, it_o = _oracle_gmres(w, h2, ora, 1e-13, side="left")
    sys = make_sys(ctx, w, tau=ora.tau, rank_cap=1 << 20)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        x = torch.empty(w.N, dtype=torch.float64, device="cuda:0")
        rep = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, cuda(b), x, w.N, 1e-13, 500,
                                  side=ifmm.GMRES_LEFT)[0]
        err = rel(x.cpu().numpy(), x_o)
        print(f"{name} left: GMRES {rep.iters} it (oracle {it_o}), preconditioned residual "
              f"{rep.rel_residual:.1e}, true residual {rep.true_rel_residual:.1e}, error {err:.1e}")
        assert rep.status == 0 and rep.rel_residual <= 1e-13
        assert abs(rep.iters - it_o) <= 1
        assert err < 1e-10
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


def test_flexible_gmres_matches_right_gmres(ctx):
    """Flexible GMRES keeps z_k = M^-1 v_k; with the FP64 preconditioner (one
    fixed linear map) it spans the same space as right preconditioning: same
    iterations and the same solution to rounding."""
    w = CASES["3lev"]()
    sys = make_sys(ctx, w)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        B = cuda(w.rhs(2).T.copy())
        xr, xf = torch.empty_like(B), torch.empty_like(B)
        rr = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_FMM, B, xr, w.N, 1e-10, 300)
        rf = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, B, xf, w.N, 1e-10, 300,
                                 side=ifmm.GMRES_FLEXIBLE)
        assert [r.iters for r in rf] == [r.iters for r in rr]
        assert all(r.status == 0 and r.true_rel_residual <= 1e-10 for r in rf)
        assert rel(xf.cpu().numpy(), xr.cpu().numpy()) < 1e-8
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


def test_default_path_parity_on_workload_recipe(ctx):
    """The configuration the benchmark times -- the library's default rank cap
    (n^D = 64), the randomised SVD of Sec. 2.4 for tall blocks and the symmetric
    variant -- on the cube-64k recipe itself (1/r, A_ii = 2 N^(1/3), leaves <= 64,
    Chebyshev 4^3, eps = 1e-8) at N = 8192: three levels, level-2 blocks up to
    158 rows whose ranks the cap binds.  The randomised threshold is lowered to
    100 rows on both sides so that it triggers at this size (the library's
    default, 160, is reached from N ~ 2^15).  Unique results are compared:
    equal ranks at every depth, and GMRES (non-restarted, tol 1e-13) reaching
    the oracle's solution within 1e-10 in the same number of iterations (+-1).
    The preconditioner output itself is not unique here: where the cap binds it
    cuts through clustered singular values far above tau, and the oracle's own
    output moves by 2.6e-4 when the points move by 1e-13 (relative) with every
    rank unchanged; so it is checked for validity -- its normwise backward
    error against A_n within 1.5x the oracle's, and within 2e-3 of the
    oracle's output."""
    from workloads import inv_r_cube
    w = inv_r_cube(8192, 2000, "cube-64k@8192", 4, 64, 1e-8)
    h2 = oracle_h2(w)
    ora = IFMM(h2, w.eps, rank_cap=64, rsvd_rows=100, symmetric=True)
    assert max(ora.level_a[2]) > 100 and max(ora.level_r[2]) == 64
    sys = make_sys(ctx, w, tau=ora.tau, rsvd_rows=100, symmetric=1)  # rank_cap 0: default n^D
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        for l in range(2, h2.tree.L + 1):
            assert ifmm.ifmm_factor_get_ranks(fac, l) == ora.ranks(l), f"ranks differ at depth {l}"
        b = w.rhs(1)[:, 0]
        x = torch.empty(w.N, dtype=torch.float64, device="cuda:0")
        ifmm.ifmm_solve(ctx, fac, cuda(b), x, w.N)
        xg, xo = x.cpu().numpy(), ora.solve(b)
        e_solve = rel(xg, xo)
        p = h2.tree.perm
        A = h2.dense_blockwise()
        from scipy.sparse.linalg import eigsh
        smax = float(abs(eigsh(A, k=1, which="LM", return_eigenvectors=False)[0]))  # A symmetric
        eta = lambda v: np.linalg.norm(A @ v[p] - b[p]) / (smax * np.linalg.norm(v))
        x_o, it_o, _ = oracle_gmres(lambda v: to_user(h2, h2.matvec(v[p])), b, ora.solve,
                                    1e-13, 500)
        rep = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, cuda(b), x, w.N, 1e-13, 500,
                                  refine=0)[0]
        e_gmres = rel(x.cpu().numpy(), x_o)
        print(f"default path: preconditioner output vs oracle {e_solve:.1e}, backward error "
              f"{eta(xg):.2e} (oracle {eta(xo):.2e}); GMRES {rep.iters} it (oracle {it_o}), "
              f"true residual {rep.true_rel_residual:.1e}, vs oracle {e_gmres:.1e}")
        assert eta(xg) <= 1.5 * eta(xo) and e_solve < 2e-3
        assert rep.rel_residual <= 1e-13 and abs(rep.iters - it_o) <= 1
        assert e_gmres < 1e-10
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


def test_square_gauss_shape_parity(ctx):
    """The square-gauss-1m recipe (points uniform in the unit square, Gaussian
    sigma = 0.05 with A_ii = 1.01, quadtree leaves <= 128, Chebyshev 6^2,
    eps = 1e-6) at N = 8192: tree bit-exact, FMM matvec to 1e-13, equal ranks,
    solve output to 1e-10, and four right-hand sides of GMRES to the oracle's
    solutions within 1e-10 at tol 1e-13."""
    from workloads import Kernel as WK
    w = small_cube(8192, 3000, cheb_n=6, leaf_max=128, eps=1e-6, dim=2,
                   kernel=WK(K_GAUSSIAN, 0.05, 1.01))
    h2 = oracle_h2(w)
    ora = IFMM(h2, w.eps)
    sys = make_sys(ctx, w, tau=ora.tau, rank_cap=1 << 20)
    try:
        assert np.array_equal(ifmm.ifmm_system_get_perm(sys, w.N), h2.tree.perm)
        X = np.random.default_rng(4).standard_normal((4, w.N))
        y = torch.empty(4, w.N, dtype=torch.float64, device="cuda:0")
        ifmm.fmm_matvec(ctx, sys, ifmm.MV_FMM, cuda(X), y, w.N)
        p = h2.tree.perm
        ref = np.stack([to_user(h2, h2.matvec(X[c][p])) for c in range(4)])
        assert rel(y.cpu().numpy(), ref) < 1e-13
        fac = ifmm.ifmm_factor(ctx, sys)
        try:
            for l in range(2, h2.tree.L + 1):
                assert ifmm.ifmm_factor_get_ranks(fac, l) == ora.ranks(l), f"depth {l}"
            B = w.rhs(4).T.copy()
            Xs = torch.empty(4, w.N, dtype=torch.float64, device="cuda:0")
            ifmm.ifmm_solve(ctx, fac, cuda(B), Xs, w.N)
            assert rel(Xs.cpu().numpy(), ora.solve(B.T).T) < 1e-10
            reps = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, cuda(B), Xs, w.N, 1e-13, 500,
                                       refine=0)
            mv = lambda v: to_user(h2, h2.matvec(v[p]))
            for c in range(4):
                x_o, it_o, _ = oracle_gmres(mv, B[c], ora.solve, 1e-13, 500)
                assert reps[c].rel_residual <= 1e-13 and abs(reps[c].iters - it_o) <= 1
                assert rel(Xs[c].cpu().numpy(), x_o) < 1e-10, c
        finally:
            ifmm.ifmm_factor_destroy(fac)
    finally:
        ifmm.ifmm_system_destroy(sys)


def test_multi_rhs_gmres_and_host_entry(ctx):
    w = CASES["ragged"]()
    sys = make_sys(ctx, w)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        B = w.rhs(3).T.copy()
        X = torch.empty(3, w.N, dtype=torch.float64, device="cuda:0")
        reps = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_FMM, cuda(B), X, w.N, 1e-10, 200)
        assert all(r.status == 0 and r.true_rel_residual <= 1e-10 for r in reps)
        Xh = np.zeros_like(B)
        reps_h = ifmm.gmres_solve_host(ctx, sys, fac, ifmm.MV_FMM, B, Xh, 1e-10, 200)
        assert [r.iters for r in reps_h] == [r.iters for r in reps]
        assert rel(Xh, X.cpu().numpy()) < 1e-12
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


def test_dense_mode_small_n(ctx):
    w = small_cube(50, 2, cheb_n=3, leaf_max=64)
    h2 = oracle_h2(w)
    sys = make_sys(ctx, w)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        assert ifmm.ifmm_system_get_info(sys).levels == 0
        b = np.random.default_rng(0).standard_normal(50)
        x = torch.empty(50, dtype=torch.float64, device="cuda:0")
        ifmm.ifmm_solve(ctx, fac, cuda(b), x, 50)
        assert rel(x.cpu().numpy(), np.linalg.solve(h2.dense_exact(), b)) < 1e-12
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)


def test_invalid_arguments_are_rejected(ctx):
    w = small_cube(100, 1)
    pts = cuda(w.points)
    with pytest.raises(ifmm.IFMMError) as e:
        ifmm.ifmm_system_create(ctx, pts, kernel(w), opts(w, eps=-1.0))
    assert e.value.status == 1
    bad = ifmm.make_options(dim=4, cheb_n=3, leaf_max=16, eps=1e-6)
    with pytest.raises(ifmm.IFMMError):
        ifmm.ifmm_system_create(ctx, pts, kernel(w), bad)
    with pytest.raises(ifmm.IFMMError):
        ifmm.ifmm_system_create(ctx, pts, ifmm.Kernel(K_INV_R, 0.0, math.nan), opts(w))


@pytest.mark.parametrize("name", ["cube2k", "3lev"])
def test_block_gmres_parity(ctx, name):
    """Block GMRES (one Krylov space for four right-hand sides, right
    preconditioning) on both sides at tol 1e-13: the same number of block
    steps (+-1) as the oracle's block GMRES and the same solutions to 1e-10;
    no more block steps than single-vector GMRES takes per column.  The flexible
    form with FP32 sweeps reaches the true residual 1e-10 as well."""
    from oracle.gmres import block_gmres
    w = CASES[name]()
    h2 = oracle_h2(w)
    ora = IFMM(h2, w.eps)
    B = w.rhs(4)
    p = h2.tree.perm
    mv = lambda v: to_user(h2, h2.matvec(v[p]))
    X_o, steps_o, _ = block_gmres(mv, B, ora.solve, 1e-13, 200)
    sys = make_sys(ctx, w, tau=ora.tau, rank_cap=1 << 20)
    fac = ifmm.ifmm_factor(ctx, sys)
    try:
        Bt = cuda(B.T.copy())
        X = torch.empty_like(Bt)
        reps = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, Bt, X, w.N, 1e-13, 200, block=1,
                                   refine=0)
        steps = max(r.iters for r in reps)
        err = rel(X.cpu().numpy().T, X_o)
        single = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, Bt, torch.empty_like(Bt), w.N,
                                     1e-13, 200, refine=0)
        print(f"{name} block GMRES: {steps} block steps (oracle {steps_o}), single-vector "
              f"{[r.iters for r in single]}, error vs oracle {err:.1e}")
        assert abs(steps - steps_o) <= 1
        assert err < 1e-10
        assert steps <= max(r.iters for r in single)
        X32 = torch.empty_like(Bt)
        r32 = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, Bt, X32, w.N, 1e-10, 200, block=1,
                                  side=ifmm.GMRES_FLEXIBLE, precond_precision=ifmm.P_FP32)
        assert all(r.status == 0 and r.true_rel_residual <= 1e-10 for r in r32)
    finally:
        ifmm.ifmm_factor_destroy(fac)
        ifmm.ifmm_system_destroy(sys)
