"""Pins for the IFMM oracle (Sec. 2.2-2.4, Algorithms 1-3, Appendix C)."""
import numpy as np
import pytest

from oracle.h2 import H2
from oracle.ifmm import IFMM, schur_complement
from workloads import Kernel, K_GAUSSIAN, K_INV_R, K_PAPER_D, small_cube


def setup(N, seed, n, leaf, dim=3, kernel=None):
    w = small_cube(N, seed, cheb_n=n, leaf_max=leaf, dim=dim, kernel=kernel)
    h = H2(w.points, w.kernel.kind, w.kernel.param, w.kernel.diag, n, leaf)
    return w, h


def dense_solution(h, b):
    A = h.dense_blockwise()
    p = h.tree.perm
    xt = np.linalg.solve(A, b[p])
    x = np.empty_like(xt)
    x[p] = xt
    return x


@pytest.mark.parametrize("N,n,leaf,dim,kernel", [
    (600, 3, 16, 3, None),                                  # L = 2 (leaves are the top level)
    (1500, 2, 12, 3, Kernel(K_INV_R, 0.0, 3000.0)),        # L = 3: one merge
    (900, 3, 10, 2, Kernel(K_GAUSSIAN, 0.15, 1.01)),       # quadtree, L = 3
    (700, 2, 6, 2, Kernel(K_PAPER_D, 0.05, 1.0)),         # paper kernel, L = 4
])
def test_tau_zero_is_exact_block_lu(N, n, leaf, dim, kernel):
    """With compression disabled the elimination is an exact block LU of E, so
    the IFMM solve equals the dense solve of A_n (Sec. 2.1-2.2)."""
    w, h = setup(N, 21, n, leaf, dim, kernel)
    f = IFMM(h, 0.0, tau=0.0)
    b = np.random.default_rng(1).standard_normal(N)
    x = dense_solution(h, b)
    A = h.dense_blockwise()
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(f.solve(b) - x) / np.linalg.norm(x) < 1e-14 * kappa * 50


def test_error_tracks_eps():
    """Sec. 2.4: the retained rank follows eps; the solve error falls with it."""
    N = 1200
    w, h = setup(N, 7, 4, 24, 3, Kernel(K_INV_R, 0.0, 4.0 * N))
    b = np.random.default_rng(1).standard_normal(N)
    x = dense_solution(h, b)
    errs, s0 = [], None
    for eps in (1e-2, 1e-4, 1e-6, 1e-8):
        f = IFMM(h, eps, sigma0=s0)
        s0 = f.sigma0
        errs.append(np.linalg.norm(f.solve(b) - x) / np.linalg.norm(x))
        assert errs[-1] < 10 * eps
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_ranks_bounded_and_multi_rhs():
    w, h = setup(1500, 3, 3, 16)
    f = IFMM(h, 1e-5)
    leaf = h.tree.levels[h.L]
    for i in range(leaf.nb):
        assert f.rank_log[(h.L, i)] <= leaf.pt_end[i] - leaf.pt_begin[i]
        assert f.rank_log[(h.L, i)] <= 27
    B = np.random.default_rng(2).standard_normal((1500, 3))
    X = f.solve(B)
    for c in range(3):
        assert np.allclose(X[:, c], f.solve(B[:, c]), rtol=1e-12, atol=1e-12)


def test_dense_mode_for_tiny_n():
    w, h = setup(40, 2, 3, 64)
    assert h.tree.dense
    f = IFMM(h, 1e-6)
    b = np.random.default_rng(0).standard_normal(40)
    assert np.allclose(f.solve(b), np.linalg.solve(h.dense_exact(), b), rtol=1e-12)


def test_sigma0_is_the_largest_singular_value_of_E():
    w, h = setup(300, 2, 2, 10, 3, Kernel(K_INV_R, 0.0, 600.0))
    from oracle.ifmm import sigma0_power
    s, it = sigma0_power(h)
    E = h.extended_dense()
    assert abs(s - np.linalg.svd(E, compute_uv=False)[0]) <= 1e-5 * s


def _appendix_c():
    rng = np.random.default_rng(5)
    m, r = 7, 3
    A00 = rng.standard_normal((m, m)) + 6 * np.eye(m)
    A11 = rng.standard_normal((m, m)) + 6 * np.eye(m)
    U0, U1, V0, V1 = (rng.standard_normal((m, r)) for _ in range(4))
    Z = np.zeros
    I = np.eye(r)
    E = np.block([[A00, Z((m, m)), U0, Z((m, r))],
                  [Z((m, m)), A11, Z((m, r)), U1],
                  [V0.T, Z((r, m)), Z((r, r)), -I],
                  [Z((r, m)), V1.T, -I, Z((r, r))]])
    blocks = [slice(0, m), slice(m, 2 * m), slice(2 * m, 2 * m + r), slice(2 * m + r, 2 * m + 2 * r)]
    return E, blocks, (A00, A11, U0, U1, V0, V1)


def _eliminate(E, blocks, piv):
    keep = [b for k, b in enumerate(blocks) if k not in piv]
    P = np.concatenate([np.arange(blocks[k].start, blocks[k].stop) for k in piv])
    R = np.concatenate([np.arange(b.start, b.stop) for b in keep])
    _, S = schur_complement(E[np.ix_(P, P)], E[np.ix_(P, R)], E[np.ix_(R, P)])
    return E[np.ix_(R, R)] - S


def test_appendix_c_level_by_level_closed_form():
    """Appendix C: eliminating A00 then A11 leaves
    [[-V0^T A00^-1 U0, -I], [-I, -V1^T A11^-1 U1]]."""
    E, blocks, (A00, A11, U0, U1, V0, V1) = _appendix_c()
    rest = _eliminate(E, blocks, [0, 1])
    r = U0.shape[1]
    expect = np.block([[-V0.T @ np.linalg.solve(A00, U0), -np.eye(r)],
                       [-np.eye(r), -V1.T @ np.linalg.solve(A11, U1)]])
    assert np.allclose(rest, expect, atol=1e-12)


def test_appendix_c_depth_first_closed_form():
    """Appendix C: eliminating A00, then the two auxiliary pivots, leaves the
    block-LU Schur complement A11 - U1 V0^T A00^-1 U0 V1^T; the intermediate
    after A00 is the printed 3x3 block matrix."""
    E, blocks, (A00, A11, U0, U1, V0, V1) = _appendix_c()
    m, r = A00.shape[0], U0.shape[1]
    mid = _eliminate(E, blocks, [0])
    Z = np.zeros
    expect_mid = np.block([[A11, Z((m, r)), U1],
                           [Z((r, m)), -V0.T @ np.linalg.solve(A00, U0), -np.eye(r)],
                           [V1.T, -np.eye(r), Z((r, r))]])
    assert np.allclose(mid, expect_mid, atol=1e-12)
    last = _eliminate(E, blocks, [0, 2, 3])
    expect = A11 - U1 @ V0.T @ np.linalg.solve(A00, U0) @ V1.T
    assert np.allclose(last, expect, atol=1e-11)


def test_splitmix64_reference_value():
    """The counter-based generator of the randomised SVD is SplitMix64
    (Steele, Lea, Flood 2014): its first output from state 0 is fixed."""
    from oracle.ifmm import splitmix64
    assert int(splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF


def test_rsvd_is_exact_for_low_rank_and_close_for_decaying_spectra():
    """Randomised SVD (Sec. 2.4): exact when rank <= k, accurate for the leading
    singular values of a fast-decaying spectrum."""
    from oracle.ifmm import orth, rsvd_left, rsvd_seed
    rng = np.random.default_rng(0)
    U, _ = np.linalg.qr(rng.standard_normal((200, 200)))
    V, _ = np.linalg.qr(rng.standard_normal((900, 200)))
    s = np.zeros(200)
    s[:30] = np.logspace(0, -9, 30)
    M = (U * s) @ V.T
    W, sr = rsvd_left(M, 40, rsvd_seed(3, 7, 0))
    assert np.allclose(sr[:30], s[:30], rtol=1e-6, atol=1e-14)
    assert np.linalg.norm(M - W[:, :30] @ (W[:, :30].T @ M)) < 1e-12
    s2 = 10.0 ** (-np.arange(200) / 8.0)
    M2 = (U * s2) @ V.T
    W2, sr2 = rsvd_left(M2, 48, rsvd_seed(3, 8, 1))
    assert np.allclose(sr2[:24], s2[:24], rtol=1e-8)
    Q = orth(rng.standard_normal((50, 10)))
    assert np.allclose(Q.T @ Q, np.eye(10), atol=1e-13)


# The randomised-SVD and backward-error pins run on the cube workloads' own
# conditioning carried to the plane: 1/r with A_ii = 2 N^(1/dim) (close pairs make
# A indefinite and kappa(A) ~ 1e6 here), quadtree leaves <= 48, Chebyshev 4^2.
_REC = dict(N=4096, seed=11, n=4, leaf=48, dim=2)


@pytest.fixture(scope="module")
def recipe_2d():
    w, h = setup(_REC["N"], _REC["seed"], _REC["n"], _REC["leaf"], _REC["dim"])
    A = h.dense_blockwise()
    b = np.random.default_rng(1).standard_normal(_REC["N"])
    s0 = IFMM(h, 1e-5).sigma0
    return h, A, b, s0, np.linalg.norm(A, 2)


def _backward_error(h, A, smax, b, x):
    """Normwise backward error |A_n x - b| / (|A_n|_2 |x|) in tree order."""
    p = h.tree.perm
    return np.linalg.norm(A @ x[p] - b[p]) / (smax * np.linalg.norm(x[p]))


def test_backward_error_tracks_eps_on_workload_recipe(recipe_2d):
    """Sec. 2.4: every truncation discards singular values below eps sigma_0(E),
    and sigma_0(E) is of the order of |A|, so the IFMM solve is the exact solve of
    a matrix within about eps |A| of A_n: its normwise backward error stays below
    eps (the forward error is that times kappa(A), ~1e6 on this recipe) and falls
    with eps."""
    h, A, b, s0, smax = recipe_2d
    prev = 1.0
    for eps in (1e-3, 1e-5, 1e-7):
        f = IFMM(h, eps, sigma0=s0)
        eta = _backward_error(h, A, smax, b, f.solve(b))
        assert eta < eps, (eps, eta)
        assert eta < 0.1 * prev
        prev = eta


def test_randomised_svd_equals_exact_svd_when_the_cap_does_not_bind(recipe_2d):
    """Reading R3b against reading R3: with the rank at tau below the cap, the
    randomised subspace iteration (k = cap + 16 samples, one power iteration)
    captures every singular direction above tau, so it reproduces the exact
    truncated SVD: the same ranks at every box and the same solve to rounding.
    The randomised path must actually run: blocks above rsvd_rows rows at
    levels 3 and 2, with fewer samples than rows (k < a) at level 2."""
    h, A, b, s0, smax = recipe_2d
    ex = IFMM(h, 1e-5, sigma0=s0)
    rs = IFMM(h, 1e-5, sigma0=s0, rank_cap=40, rsvd_rows=40)
    assert max(rs.level_a[3]) > 40 and max(rs.level_a[2]) > 40 + 16
    assert max(max(r) for r in ex.level_r.values()) < 40
    for l in ex.level_r:
        assert ex.level_r[l] == rs.level_r[l]
    xe, xr = ex.solve(b), rs.solve(b)
    assert np.linalg.norm(xr - xe) / np.linalg.norm(xe) < 1e-9


def test_randomised_svd_under_a_binding_cap_matches_exact_truncation(recipe_2d):
    """Reading R3b where the cap binds (ranks at tau reach 76 at eps = 1e-9, the
    cap keeps 20): the randomised SVD's rank-20 truncation is as good as the exact
    SVD's -- backward errors within 10% -- and both are limited by the cap, not
    by eps."""
    h, A, b, s0, smax = recipe_2d
    ex = IFMM(h, 1e-9, sigma0=s0, rank_cap=20)
    rs = IFMM(h, 1e-9, sigma0=s0, rank_cap=20, rsvd_rows=40)
    e_ex = _backward_error(h, A, smax, b, ex.solve(b))
    e_rs = _backward_error(h, A, smax, b, rs.solve(b))
    assert e_rs < 1.1 * e_ex and e_ex < 1.1 * e_rs
    assert e_ex > 1e-8


def test_cost_and_memory_grow_linearly_in_n():
    """Sec. 2.5 and Sec. 3.1 (linear scaling once the tree is deep): with the
    rank bounded (reading R9: a prescribed rank of 2 n^D, Sec. 2.4), quadrupling N
    in the plane adds one level with the same leaf occupancy, and the counted
    flops and stored bytes grow by 4^s with s in [0.9, 1.15] for trees of five
    and six levels.  A dense or quadratic step anywhere (lists covering all
    boxes, fill kept uncompressed, ranks growing with N) gives s near 2."""
    from workloads import uniform_cube
    res = []
    for N in (1 << 12, 1 << 14):
        pts = uniform_cube(N, 3000, 2)
        h = H2(pts, K_INV_R, 0.0, 2.0 * np.sqrt(N), 3, 16)
        f = IFMM(h, 1e-6, rank_cap=18)
        c = f.counters
        flops = sum(c.get(k, 0.0) for k in ("lu_flops", "trsm_flops", "schur_flops",
                                            "lowrank_flops", "top_flops", "init_flops"))
        res.append((h.tree.L, flops, f.stored_bytes(), max(max(r) for r in f.level_r.values())))
    (L1, f1, b1, r1), (L2, f2, b2, r2) = res
    assert (L1, L2) == (5, 6)
    s_flops = np.log(f2 / f1) / np.log(4.0)
    s_bytes = np.log(b2 / b1) / np.log(4.0)
    assert 0.9 <= s_flops <= 1.15, s_flops
    assert 0.9 <= s_bytes <= 1.15, s_bytes
    assert r1 == r2 == 18


@pytest.mark.parametrize("N,n,leaf,dim,kernel", [
    (1500, 2, 12, 3, Kernel(K_INV_R, 0.0, 3000.0)),        # L = 3: one merge
    (900, 3, 10, 2, Kernel(K_GAUSSIAN, 0.15, 1.01)),       # quadtree, L = 3
])
def test_symmetric_variant_tau_zero_is_exact(N, n, leaf, dim, kernel):
    """Reading S with compression disabled is still an exact block LU of E:
    every direction is kept, so sharing the U side's SVD changes nothing."""
    w, h = setup(N, 21, n, leaf, dim, kernel)
    f = IFMM(h, 0.0, tau=0.0, symmetric=True)
    b = np.random.default_rng(1).standard_normal(N)
    x = dense_solution(h, b)
    kappa = np.linalg.cond(h.dense_blockwise())
    assert np.linalg.norm(f.solve(b) - x) / np.linalg.norm(x) < 1e-14 * kappa * 50


def test_symmetric_variant_tracks_eps_and_matches_general():
    """Reading S at tau > 0: for a symmetric A (radial kernel, U = V) the V-side
    matrices equal the U-side ones in exact arithmetic, so the symmetric variant
    keeps the same ranks as the general algorithm (up to ties at tau) and its
    solve error follows eps like the general one (Sec. 2.4)."""
    N = 1200
    w, h = setup(N, 7, 4, 24, 3, Kernel(K_INV_R, 0.0, 4.0 * N))
    b = np.random.default_rng(1).standard_normal(N)
    x = dense_solution(h, b)
    s0 = None
    for eps in (1e-3, 1e-6, 1e-9):
        g = IFMM(h, eps, sigma0=s0)
        s0 = g.sigma0
        f = IFMM(h, eps, sigma0=s0, symmetric=True)
        eg = np.linalg.norm(g.solve(b) - x) / np.linalg.norm(x)
        es = np.linalg.norm(f.solve(b) - x) / np.linalg.norm(x)
        assert es < 10 * eps
        assert es < 3 * eg + 1e-13
        for l in range(2, h.tree.L + 1):
            rg, rs = np.array(g.ranks(l)), np.array(f.ranks(l))
            assert np.mean(rg == rs) > 0.9 and np.max(np.abs(rg - rs)) <= 2
