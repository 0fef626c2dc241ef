"""Mixed-precision Schur products on the tcgen05 tensor cores.

1. The product kernel itself (ifmm_schur_product) against an FP64 product on
   the host, for ragged shapes spanning several 128 x 128 tiles and K slices,
   every transpose combination, and beta != 0.  The bound is the rounding of
   the inputs plus FP32 accumulation: per element
       |C - C_ref| <= (u_in + K 2^-24) * (|alpha| |op(A)| |op(B)|)_ij + |beta| 2^-52 |C|
   with u_in = 2 * 2^-11 for TF32 (both operands rounded to 10 mantissa bits),
   u_in = 4 * 2^-22 for the split product (the dropped lo*lo term and the
   rounding of the tails) and u_in = 2 * 2^-8 for BF16 (7 mantissa bits).
2. The factorisation with TF32 / split-TF32 Schur products used as the GMRES
   preconditioner: FP64 GMRES must still reach the 1e-10 residual, and its
   solution must agree with the FP64 path's to the accuracy the residual
   allows.  Iteration counts are printed for the record.
"""
import numpy as np
import pytest
import torch

import paper_1508_01835_gb300 as ifmm
from tests.gpu_util import cuda, kernel, opts, rel
from workloads import cube_2k, small_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1508_01835_gb300 import build
    build.build()
    c = ifmm.ifmm_ctx_create(0)
    yield c
    ifmm.ifmm_ctx_destroy(c)


SHAPES = [(1, 1, 1), (128, 128, 32), (200, 130, 45), (257, 300, 97), (64, 700, 33),
          (430, 430, 32), (100, 90, 0), (1500, 1300, 150)]   # the last: more tiles than SMs


@pytest.mark.parametrize("prec", [ifmm.P_TF32, ifmm.P_FP32, ifmm.P_BF16])
@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("tA,tB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_schur_product_kernel(ctx, prec, M, N, K, tA, tB):
    rng = np.random.default_rng(1000 * M + 10 * N + K + 3 * tA + tB)
    lda = (K if tA else M) + 3
    ldb = (N if tB else K) + 5
    ldc = M + 7
    A = rng.standard_normal(((M if tA else K) or 1, lda))
    B = rng.standard_normal(((K if tB else N) or 1, ldb))
    Cm = rng.standard_normal((N, ldc))
    alpha, beta = -1.25, 0.5
    opA = A[:M, :K] if tA else A[:K, :M].T
    opB = B[:K, :N] if tB else B[:N, :K].T
    C0 = Cm[:N, :M].T.copy()
    ref = alpha * opA @ opB + beta * C0
    bound_mat = abs(alpha) * np.abs(opA) @ np.abs(opB)
    dA, dB, dC = cuda(A), cuda(B), cuda(Cm)
    ifmm.ifmm_schur_product(ctx, prec, M, N, K, dA, lda, tA, dB, ldb, tB, dC, ldc, alpha, beta)
    torch.cuda.synchronize()
    out_mem = dC.cpu().numpy()
    got = out_mem[:N, :M].T
    u_in = {ifmm.P_TF32: 2 * 2.0 ** -11, ifmm.P_FP32: 4 * 2.0 ** -22,
            ifmm.P_BF16: 2 * 2.0 ** -8}[prec]
    tol = (u_in + K * 2.0 ** -24) * bound_mat + abs(beta) * 2.0 ** -52 * np.abs(C0) + 1e-300
    err = np.abs(got - ref)
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g}"
    # padding rows of C (ld > M) are untouched
    assert np.array_equal(out_mem[:N, M:], Cm[:N, M:])
    # the split product is really more accurate than plain TF32 (K > 0)
    if prec == ifmm.P_FP32 and K >= 8:
        assert np.max(err / (bound_mat + 1e-300)) < 2.0 ** -16


def test_fp64_product_kernel_matches(ctx):
    rng = np.random.default_rng(5)
    M, N, K = 150, 77, 61
    A = rng.standard_normal((K, M))
    B = rng.standard_normal((N, K))
    Cm = np.zeros((N, M))
    dC = cuda(Cm)
    ifmm.ifmm_schur_product(ctx, ifmm.P_FP64, M, N, K, cuda(A), M, 0, cuda(B), K, 0, dC, M)
    got = dC.cpu().numpy().T
    ref = A.T @ B.T
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(A.T) @ np.abs(B.T))


CASES = {
    "cube2k": lambda: cube_2k(),
    "3lev": lambda: small_cube(3000, 7, cheb_n=3, leaf_max=32, eps=1e-6),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_precision_preconditioner_reaches_fp64_residual(ctx, name):
    """Every precision of the Schur products gives a preconditioner with which
    FP64 GMRES reaches a true residual <= 1e-10; each result's distance to the
    FP64 oracle's GMRES solution (same matvec, tol 1e-10) is stated and must
    stay within what two solutions at residual 1e-10 can differ by on this
    system (kappa(A_n) x 2e-10, kappa ~ 1e6 here) and below 1e-4."""
    from oracle.gmres import gmres as oracle_gmres
    from oracle.ifmm import IFMM
    from tests.gpu_util import oracle_h2, to_user
    w = CASES[name]()
    h2 = oracle_h2(w)
    A = h2.dense_blockwise()
    kappa = np.linalg.cond(A)
    ora = IFMM(h2, w.eps)
    p = h2.tree.perm
    b_np = w.rhs(1)[:, 0]
    x_o, it_o, _ = oracle_gmres(lambda v: to_user(h2, h2.matvec(v[p])), b_np, ora.solve,
                                1e-10, 500)
    b = cuda(b_np)
    xs, its = {}, {}
    for prec in (ifmm.P_FP64, ifmm.P_FP32, ifmm.P_TF32):
        sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w, schur=prec))
        try:
            fac = ifmm.ifmm_factor(ctx, sys)
            try:
                x = torch.empty_like(b)
                reps = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_FMM, b, x, w.N, 1e-10, 300)
                assert reps[0].status == 0, (prec, reps[0].iters, reps[0].rel_residual)
                assert reps[0].true_rel_residual <= 1e-10, (prec, reps[0].true_rel_residual)
                xs[prec] = x.cpu().numpy()
                its[prec] = reps[0].iters
            finally:
                ifmm.ifmm_factor_destroy(fac)
        finally:
            ifmm.ifmm_system_destroy(sys)
    errs = {prec: rel(xs[prec], x_o) for prec in xs}
    print(f"{name}: kappa(A_n) {kappa:.1e}; GMRES iterations oracle {it_o}, fp64 "
          f"{its[ifmm.P_FP64]}, fp32 (3xTF32) {its[ifmm.P_FP32]}, tf32 {its[ifmm.P_TF32]}; "
          f"|x - x_oracle| / |x_oracle|: fp64 {errs[ifmm.P_FP64]:.1e}, fp32 "
          f"{errs[ifmm.P_FP32]:.1e}, tf32 {errs[ifmm.P_TF32]:.1e}")
    for prec in xs:
        assert errs[prec] <= min(1e-4, 2e-10 * kappa), (prec, errs[prec])
    # the split product preconditions at least as well as plain TF32, give or take one
    assert its[ifmm.P_FP32] <= its[ifmm.P_TF32] + 1


def test_tensor_core_wait_limit_reports_timeout_and_recovers(ctx, monkeypatch):
    """Failure handling of the tensor-core kernel: a pipeline wait that takes
    longer than its limit is reported as IFMM_ERR_TIMEOUT.  The test lowers the
    reporting limit to one poll (IFMM_TC_SOFT_WAIT_POLLS), so the wait for the
    last MMA commit always runs out; the kernel still waits for its own MMAs up
    to the hard bound before it frees its tensor memory, so nothing is left in
    flight.  Afterwards, with the limit restored, the same product and a
    mixed-precision factorisation succeed."""
    rng = np.random.default_rng(17)
    M, N, K = 256, 200, 160
    A, B = rng.standard_normal((K, M)), rng.standard_normal((N, K))
    dA, dB = cuda(A), cuda(B)
    dC = cuda(np.zeros((N, M)))
    monkeypatch.setenv("IFMM_TC_SOFT_WAIT_POLLS", "1")
    with pytest.raises(ifmm.IFMMError) as e:
        ifmm.ifmm_schur_product(ctx, ifmm.P_FP32, M, N, K, dA, M, 0, dB, K, 0, dC, M)
    assert e.value.status == 6
    torch.cuda.synchronize()
    monkeypatch.delenv("IFMM_TC_SOFT_WAIT_POLLS")
    ifmm.ifmm_schur_product(ctx, ifmm.P_FP32, M, N, K, dA, M, 0, dB, K, 0, dC, M)
    got = dC.cpu().numpy().T
    ref = A.T @ B.T
    assert np.max(np.abs(got - ref)) <= 2.0 ** -16 * np.max(np.abs(A.T) @ np.abs(B.T))
    w = cube_2k()
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w, schur=ifmm.P_FP32))
    try:
        fac = ifmm.ifmm_factor(ctx, sys)
        ifmm.ifmm_factor_destroy(fac)
    finally:
        ifmm.ifmm_system_destroy(sys)


@pytest.mark.parametrize("name", sorted(CASES) + ["dense"])
def test_fp32_substitution_sweeps(ctx, name):
    """The substitution sweeps with FP32 copies of the factors (and the top
    system's explicit inverse): the preconditioner output stays within FP32
    rounding amplified by the conditioning (1.2e-7 kappa(A_n)) of the FP64
    sweeps', and flexible GMRES with it reaches the FP64 residual 1e-10 in at
    most two more iterations than FP64 right preconditioning, with the same
    solution as the FP64 path within kappa(A_n) x 2e-10."""
    from tests.gpu_util import oracle_h2
    w = CASES[name]() if name != "dense" else small_cube(60, 4, cheb_n=3, leaf_max=64)
    kappa = np.linalg.cond(oracle_h2(w).dense_blockwise())
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w, schur=ifmm.P_FP32))
    try:
        fac = ifmm.ifmm_factor(ctx, sys)
        try:
            B = cuda(w.rhs(3).T.copy())
            x64, x32 = torch.empty_like(B), torch.empty_like(B)
            ifmm.ifmm_solve(ctx, fac, B, x64, w.N)
            ifmm.ifmm_solve_prec(ctx, fac, ifmm.P_FP32, B, x32, w.N)
            d = rel(x32.cpu().numpy(), x64.cpu().numpy())
            r64 = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_FMM, B, x64, w.N, 1e-10, 300)
            r32 = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, B, x32, w.N, 1e-10, 300,
                                      side=ifmm.GMRES_FLEXIBLE, precond_precision=ifmm.P_FP32)
            e = rel(x32.cpu().numpy(), x64.cpu().numpy())
            print(f"{name}: FP32 sweeps vs FP64 {d:.1e}; GMRES iterations FP64 "
                  f"{[r.iters for r in r64]}, flexible FP32 {[r.iters for r in r32]}; "
                  f"solutions differ by {e:.1e} (kappa {kappa:.1e})")
            assert d < 1.2e-7 * kappa
            assert all(r.status == 0 and r.true_rel_residual <= 1e-10 for r in r32)
            assert all(b.iters <= a.iters + 2 for a, b in zip(r64, r32))
            assert e <= max(1e-12, 2e-10 * kappa)
            with pytest.raises(ifmm.IFMMError) as err:   # FP32 sweeps need flexible GMRES
                ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, B, x32, w.N, 1e-10, 300,
                                    precond_precision=ifmm.P_FP32)
            assert err.value.status == 1
        finally:
            ifmm.ifmm_factor_destroy(fac)
    finally:
        ifmm.ifmm_system_destroy(sys)


def test_bf16_schur_products_at_loose_eps(ctx):
    """BF16 Schur products (allowed from eps = 1e-4 up): the factorisation at
    eps = 1e-3 still preconditions FP64 GMRES to a true residual of 1e-10, and
    a tighter eps is refused."""
    w = small_cube(3000, 7, cheb_n=3, leaf_max=32, eps=1e-3)
    with pytest.raises(ifmm.IFMMError) as e:
        ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w, eps=1e-6,
                                                                     schur=ifmm.P_BF16))
    assert e.value.status == 1
    b = cuda(w.rhs(1)[:, 0])
    its = {}
    for prec in (ifmm.P_FP64, ifmm.P_BF16):
        sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w, schur=prec))
        try:
            fac = ifmm.ifmm_factor(ctx, sys)
            try:
                x = torch.empty_like(b)
                rep = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_FMM, b, x, w.N, 1e-10, 300)[0]
                assert rep.status == 0 and rep.true_rel_residual <= 1e-10
                its[prec] = rep.iters
            finally:
                ifmm.ifmm_factor_destroy(fac)
        finally:
            ifmm.ifmm_system_destroy(sys)
    print(f"eps 1e-3: GMRES iterations FP64 Schur {its[ifmm.P_FP64]}, BF16 {its[ifmm.P_BF16]}")


def _far_majorant(h2, x):
    """|U| |T| ... |U^T| |x|: the far field of the FMM product with every
    operator and the vector replaced by their absolute values (the near field
    left out), from the oracle's matvec."""
    import copy
    a = copy.copy(h2)
    a.leafU = [np.abs(U) for U in h2.leafU]
    a.transfer = [np.abs(T) for T in h2.transfer]
    a.m2l = lambda l, i, q: np.abs(h2.m2l(l, i, q))
    a.p2p = lambda i, j: np.zeros((len(h2.leaf_pts(i)), len(h2.leaf_pts(j))))
    return a.matvec(np.abs(x))


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_far_field_matvec(ctx, name):
    """fmm_matvec_prec: FP64 is fmm_matvec bit for bit; FP32 takes the far
    field (P2M, M2M, M2L, L2L, L2P) in FP32 and the near field in FP64.
    Bound, per element, against the oracle's FP64 product: the far field's
    rounding is at most gamma_n |U||T|...|U^T||x| (the oracle's majorant) with
    n the longest chain of accumulated terms (leaf size + (L-2) 8 n^D for M2M
    + (L-1) 190 n^D for the M2L/L2L rows + n^D for L2P + one narrowing per
    stage), gamma_n = n 2^-24 / (1 - n 2^-24); the near field and FP64 sums add
    1e-13 of |y|.  Normwise the error must also stay below 1e-5 (the chains'
    errors are not all aligned: typically ~1e-7) and above 1e-10 (so the far
    field really ran in FP32)."""
    from tests.gpu_util import oracle_h2, to_user
    w = CASES[name]()
    h2 = oracle_h2(w)
    p = h2.tree.perm
    X = w.rhs(3)
    y_o = np.stack([to_user(h2, h2.matvec(X[p, c])) for c in range(3)], axis=1)
    F = np.stack([to_user(h2, _far_majorant(h2, X[p, c])) for c in range(3)], axis=1)
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w))
    try:
        xd = cuda(X.T.copy())
        y64, yp64, y32 = (torch.empty_like(xd) for _ in range(3))
        ifmm.fmm_matvec(ctx, sys, ifmm.MV_FMM, xd, y64, w.N)
        ifmm.fmm_matvec_prec(ctx, sys, ifmm.P_FP64, xd, yp64, w.N)
        ifmm.fmm_matvec_prec(ctx, sys, ifmm.P_FP32, xd, y32, w.N)
        torch.cuda.synchronize()
        assert torch.equal(y64, yp64)
        got = y32.cpu().numpy().T
        L, nd = h2.L, h2.nd
        lv = h2.tree.levels[L]
        mmax = int(np.max(lv.pt_end - lv.pt_begin))
        n = mmax + (L - 2) * 8 * nd + (L - 1) * 190 * nd + nd + (L + 2)
        gam = n * 2.0 ** -24 / (1 - n * 2.0 ** -24)
        err = np.abs(got - y_o)
        tol = gam * F + 1e-13 * np.abs(y_o) + 1e-300
        nerr = np.linalg.norm(got - y_o) / np.linalg.norm(y_o)
        print(f"{name}: FP32 far field, |y32 - y| / |y| = {nerr:.1e}, max err / bound "
              f"{np.max(err / tol):.1e} (gamma_n {gam:.1e}, n {n})")
        assert np.all(err <= tol)
        assert 1e-10 < nerr < 1e-5
    finally:
        ifmm.ifmm_system_destroy(sys)


@pytest.mark.parametrize("name", sorted(CASES))
def test_gmres_iterative_refinement(ctx, name):
    """GMRES-IR (matvec_precision FP32): inner products with the FP32 far
    field, FP64 true residuals.  With FP32 sweeps (flexible) and with FP64
    sweeps (right) every column reaches the true residual 1e-10 and its
    solution lies within kappa(A_n) x 2e-10 of the FP64 oracle's GMRES
    solution (tol 1e-10).  Inner iteration counts are printed next to FP64
    GMRES's.  IR with left preconditioning, the direct product or block GMRES
    is refused."""
    from oracle.gmres import gmres as oracle_gmres
    from oracle.ifmm import IFMM
    from tests.gpu_util import oracle_h2, to_user
    w = CASES[name]()
    h2 = oracle_h2(w)
    kappa = np.linalg.cond(h2.dense_blockwise())
    ora = IFMM(h2, w.eps)
    p = h2.tree.perm
    B = w.rhs(3)
    X_o = np.stack([oracle_gmres(lambda v: to_user(h2, h2.matvec(v[p])), B[:, c], ora.solve,
                                 1e-10, 500)[0] for c in range(3)], axis=1)
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w, schur=ifmm.P_FP32))
    try:
        fac = ifmm.ifmm_factor(ctx, sys)
        try:
            Bd = cuda(B.T.copy())
            x64 = torch.empty_like(Bd)
            r64 = ifmm.gmres_solve(ctx, sys, fac, ifmm.MV_FMM, Bd, x64, w.N, 1e-10, 300)
            out = {}
            for label, side, pp in (("flexible/FP32 sweeps", ifmm.GMRES_FLEXIBLE, ifmm.P_FP32),
                                    ("right/FP64 sweeps", ifmm.GMRES_RIGHT, ifmm.P_FP64)):
                x = torch.empty_like(Bd)
                reps = ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, Bd, x, w.N, 1e-10, 300,
                                           side=side, refine=10, precond_precision=pp,
                                           matvec_precision=ifmm.P_FP32)
                assert all(r.status == 0 and r.true_rel_residual <= 1e-10 for r in reps), \
                    [(r.iters, r.true_rel_residual) for r in reps]
                e = rel(x.cpu().numpy().T, X_o)
                assert e <= max(1e-12, 2e-10 * kappa), (label, e)
                out[label] = ([r.iters for r in reps], e)
            print(f"{name}: kappa {kappa:.1e}; FP64 GMRES iterations {[r.iters for r in r64]}; "
                  + "; ".join(f"IR {k}: inner iterations {v[0]}, error vs oracle {v[1]:.1e}"
                              for k, v in out.items()))
            for kw in (dict(side=ifmm.GMRES_LEFT), dict(block=1)):
                with pytest.raises(ifmm.IFMMError) as err:
                    ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_FMM, Bd, torch.empty_like(Bd), w.N,
                                        1e-10, 300, matvec_precision=ifmm.P_FP32, **kw)
                assert err.value.status == 1
            with pytest.raises(ifmm.IFMMError) as err:
                ifmm.gmres_solve_ex(ctx, sys, fac, ifmm.MV_DIRECT, Bd, torch.empty_like(Bd), w.N,
                                    1e-10, 300, matvec_precision=ifmm.P_FP32)
            assert err.value.status == 1
        finally:
            ifmm.ifmm_factor_destroy(fac)
    finally:
        ifmm.ifmm_system_destroy(sys)
