"""Pins for the kernel functions (Sec. 3.1, Eq. K_ij and the workloads' kernels)."""
import math

import numpy as np

from oracle.kernels import K_GAUSSIAN, K_INV_R, K_PAPER_D, kernel_of_r, kernel_matrix


def test_paper_kernel_piecewise():
    d = 1e-3
    r = np.array([0.0, 5e-4, 1e-3, 2e-3, 1.0])
    assert np.allclose(kernel_of_r(K_PAPER_D, d, math.nan, r), [1.0, 0.5, 1.0, 0.5, 1e-3])


def test_inv_r_and_gaussian_with_diagonal():
    r = np.array([0.0, 0.5, 2.0])
    assert np.allclose(kernel_of_r(K_INV_R, 0.0, 7.0, r), [7.0, 2.0, 0.5])
    s = 0.05
    g = kernel_of_r(K_GAUSSIAN, s, 1.01, r)
    assert g[0] == 1.01 and math.isclose(g[1], math.exp(-0.25 / (2 * s * s)))


def test_matrix_diagonal_and_symmetry():
    x = np.random.default_rng(0).random((20, 3))
    A = kernel_matrix(K_INV_R, 0.0, 3.0, x, x)
    assert np.allclose(np.diag(A), 3.0) and np.allclose(A, A.T)
