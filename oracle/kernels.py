"""Kernel functions a_ij = K(|r_i - r_j|) (oracle).

Paper: Sec. 3.1 (the linear system with entries defined by a kernel of the
distance, and the kernel of Eq. (K_ij): 1 at r = 0, r/d for 0 < r < d, d/r
otherwise).  The other two kernels are the workloads' own statements:
1/r with a prescribed diagonal, and the Gaussian RBF exp(-r^2 / (2 sigma^2))
with a prescribed diagonal.

Reading: a pair of coincident points (r = 0) takes the diagonal value; the
diagonal value defaults to the kernel's own value at r = 0 (1 for the paper
kernel and the Gaussian; 1/r has none, so it must be given).

Parity: pinned by closed-form values in tests.
"""
from __future__ import annotations

import math

import numpy as np

K_INV_R = 0
K_GAUSSIAN = 1
K_PAPER_D = 2


def diag_value(kind: int, param: float, diag: float) -> float:
    if not math.isnan(diag):
        return float(diag)
    if kind == K_INV_R:
        raise ValueError("1/r kernel needs an explicit diagonal value")
    return 1.0


def kernel_of_r(kind: int, param: float, diag: float, r: np.ndarray) -> np.ndarray:
    """K(r) elementwise; r == 0 gives the diagonal value."""
    r = np.asarray(r, dtype=np.float64)
    dv = diag_value(kind, param, diag) if (kind != K_INV_R or not math.isnan(diag)) else math.nan
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    if kind == K_INV_R:
        v = 1.0 / rs
    elif kind == K_GAUSSIAN:
        v = np.exp(-(rs * rs) / (2.0 * param * param))
    elif kind == K_PAPER_D:
        v = np.where(rs < param, rs / param, param / rs)
    else:
        raise ValueError(f"unknown kernel kind {kind}")
    return np.where(zero, dv, v)


def kernel_matrix(kind: int, param: float, diag: float, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Dense block K(|x_a - y_b|), shape (len(x), len(y))."""
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt(np.sum(d * d, axis=2))
    return kernel_of_r(kind, param, diag, r)
