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
