"""Pins for the oracle's H^2 operators, FMM matvec and extended system (Sec. 2.1)."""
import numpy as np
import pytest

from oracle.h2 import H2
from workloads import Kernel, K_GAUSSIAN, small_cube


def make(N, seed, n, leaf, dim=3, kernel=None):
    w = small_cube(N, seed, cheb_n=n, leaf_max=leaf, dim=dim, kernel=kernel)
    return w, H2(w.points, w.kernel.kind, w.kernel.param, w.kernel.diag, n, leaf)


@pytest.mark.parametrize("N,leaf,dim", [(500, 12, 3), (700, 10, 2), (900, 8, 3)])
def test_fmm_matvec_equals_blockwise_assembly(N, leaf, dim):
    _, h = make(N, 5, 3, leaf, dim)
    A = h.dense_blockwise()
    X = np.random.default_rng(1).standard_normal((N, 3))
    assert np.allclose(h.matvec(X), A @ X, rtol=1e-13, atol=1e-10)


def test_fmm_error_falls_with_n():
    w = small_cube(1500, 9, leaf_max=20)
    x = np.random.default_rng(2).standard_normal(1500)
    errs = []
    for n in (1, 2, 3, 4, 5, 6):
        h = H2(w.points, w.kernel.kind, w.kernel.param, w.kernel.diag, n, 20)
        yd = h.direct_matvec(x[h.tree.perm])
        errs.append(np.linalg.norm(h.matvec(x[h.tree.perm]) - yd) / np.linalg.norm(yd))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-4


def test_near_field_is_exact():
    # blocks between neighbouring leaves are the kernel itself (Eq. A_decomp_l3)
    w, h = make(600, 4, 2, 16)
    A = h.dense_blockwise()
    Ex = h.dense_exact()
    leaf = h.tree.levels[h.L]
    for i in range(0, leaf.nb, 7):
        ri = slice(leaf.pt_begin[i], leaf.pt_end[i])
        for j in leaf.nbrs[i]:
            rj = slice(leaf.pt_begin[j], leaf.pt_end[j])
            assert np.array_equal(A[ri, rj], Ex[ri, rj])


@pytest.mark.parametrize("N,leaf,dim", [(400, 12, 3), (500, 8, 2), (700, 6, 3)])
def test_extended_system_solves_the_h2_system(N, leaf, dim):
    _, h = make(N, 3, 2, leaf, dim)
    A = h.dense_blockwise()
    E = h.extended_dense()
    b = np.random.default_rng(4).standard_normal(N)
    rhs = np.zeros(E.shape[0])
    rhs[:N] = b
    x_ext = np.linalg.solve(E, rhs)[:N]
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(x_ext - x) / np.linalg.norm(x) < 1e-9


def test_extended_apply_matches_dense():
    _, h = make(300, 8, 2, 10, 3, Kernel(K_GAUSSIAN, 0.1, 1.01))
    E = h.extended_dense()
    v = np.random.default_rng(5).standard_normal(E.shape[0])
    assert np.allclose(h.extended_apply(v), E @ v, atol=1e-10)
    assert np.allclose(h.extended_apply(v, transpose=True), E.T @ v, atol=1e-10)
    # E is symmetric for a symmetric kernel (Sec. 2.1)
    assert np.allclose(E, E.T)


# -- the orthonormal re-representation (oracle/h2_ortho.py; Sec. 3: Chebyshev
# operators followed by an SVD, so the paper's E carries orthonormal bases) ----
def _composed_basis(o, l, i):
    """Orthonormal basis of box i at depth l over its points (tree order)."""
    h2 = o.h2
    if l == h2.L:
        return o.Q[(l, i)]
    ch = h2.tree.levels[l].children[i]
    blocks = [_composed_basis(o, l + 1, c) for c in ch]
    rows = sum(b.shape[0] for b in blocks)
    cols = sum(b.shape[1] for b in blocks)
    D = np.zeros((rows, cols))
    r0 = c0 = 0
    for b in blocks:
        D[r0:r0 + b.shape[0], c0:c0 + b.shape[1]] = b
        r0 += b.shape[0]
        c0 += b.shape[1]
    return D @ np.vstack([o.Tp[(l + 1, c)] for c in ch])


@pytest.mark.parametrize("N,leaf,dim,n", [(400, 12, 3, 2), (500, 8, 2, 3), (700, 6, 3, 2)])
def test_orthonormal_extended_system_solves_the_h2_system(N, leaf, dim, n):
    """E' (orthonormal bases) eliminated onto x is the same A_n: solving
    E' [x; z; y] = [b; 0; 0] gives the dense solve of A_n."""
    from oracle.h2_ortho import OrthonormalH2
    _, h = make(N, 3, n, leaf, dim)
    o = OrthonormalH2(h)
    E = o.extended_dense()
    b = np.random.default_rng(4).standard_normal(N)
    rhs = np.zeros(o.n)
    rhs[:N] = b
    x_ext = np.linalg.solve(E, rhs)[:N]
    x = np.linalg.solve(h.dense_blockwise(), b)
    assert np.linalg.norm(x_ext - x) / np.linalg.norm(x) < 1e-9
    v = np.random.default_rng(6).standard_normal(o.n)
    assert np.allclose(o.extended_apply(v), E @ v, atol=1e-10)
    assert np.allclose(o.extended_apply(v, transpose=True), E.T @ v, atol=1e-10)


def test_orthonormal_bases_are_orthonormal_at_every_depth():
    from oracle.h2_ortho import OrthonormalH2
    _, h = make(700, 6, 3, 2, 3)
    assert h.L >= 3   # transfers are re-represented too
    o = OrthonormalH2(h)
    for l in range(2, h.L + 1):
        for i in range(0, h.tree.levels[l].nb, 3):
            B = _composed_basis(o, l, i)
            assert np.allclose(B.T @ B, np.eye(B.shape[1]), atol=1e-12)
            assert B.shape[1] <= min(B.shape[0], h.nd)


def test_orthonormal_sigma0_is_the_largest_singular_value():
    from oracle.h2_ortho import OrthonormalH2
    _, h = make(500, 8, 2, 3)
    o = OrthonormalH2(h)
    s, it = o.sigma0_power(maxit=400, rtol=1e-9)
    s_ref = np.linalg.svd(o.extended_dense(), compute_uv=False)[0]
    assert abs(s - s_ref) <= 1e-4 * s_ref and it < 400
