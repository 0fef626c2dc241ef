"""Chebyshev interpolation of the black-box FMM (oracle).

Paper: Sec. 3 ("the initial low-rank approximations in the H^2-matrix are
created using interpolation based on Chebyshev polynomials", ref. fong09a)
and Sec. 2.1 (U = L2P/L2L, V^T = P2M/M2M, K = M2L).  The interpolation
formula itself is not printed in the paper; the oracle uses the standard
Chebyshev interpolant of the cited black-box FMM:

    nodes      t_a = cos((2a - 1) pi / (2n)),  a = 1..n   (on [-1, 1])
    S_n(x, t)  = 1/n + (2/n) sum_{k=1}^{n-1} T_k(x) T_k(t)

and in D dimensions the tensor product over the coordinates.  A box with
centre c and half-width h maps x to xi = (x - c) / h.  Multi-index ordering of
the n^D nodes: a = a_1 + n a_2 + n^2 a_3 (first coordinate fastest).

Parity: pinned by tests (exact interpolation of polynomials of degree < n,
partition of unity sum_a S_n(x, t_a) = 1, S_n(t_b, t_a) = delta_ab).
"""
from __future__ import annotations

from itertools import product

import numpy as np


def nodes(n: int) -> np.ndarray:
    a = np.arange(1, n + 1, dtype=np.float64)
    return np.cos((2.0 * a - 1.0) * np.pi / (2.0 * n))


def cheb_T(n: int, x: np.ndarray) -> np.ndarray:
    """T_0..T_{n-1} at x by the three-term recurrence; shape x.shape + (n,)."""
    x = np.asarray(x, dtype=np.float64)
    T = np.empty(x.shape + (n,))
    T[..., 0] = 1.0
    if n > 1:
        T[..., 1] = x
    for k in range(2, n):
        T[..., k] = 2.0 * x * T[..., k - 1] - T[..., k - 2]
    return T


def S1(n: int, x: np.ndarray) -> np.ndarray:
    """One-dimensional S_n(x, t_a) for all nodes a; shape x.shape + (n,)."""
    Tx = cheb_T(n, x)                  # (..., n)
    Tt = cheb_T(n, nodes(n))           # (n_nodes, n)
    w = np.full(n, 2.0 / n)
    w[0] = 1.0 / n
    return np.einsum("...k,ak,k->...a", Tx, Tt, w)


def node_multi_index(n: int, dim: int) -> np.ndarray:
    """(n^D, D) array: row a holds (a_1, .., a_D), first coordinate fastest."""
    idx = [tuple(reversed(t)) for t in product(range(n), repeat=dim)]
    return np.array(idx, dtype=np.int64)


def interp_matrix(n: int, xi: np.ndarray) -> np.ndarray:
    """U[p, a] = prod_d S_n(xi[p, d], t_{a_d}); xi in box-normalised coordinates."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    m, dim = xi.shape
    mi = node_multi_index(n, dim)
    U = np.ones((m, n ** dim))
    for d in range(dim):
        s = S1(n, xi[:, d])            # (m, n)
        U *= s[:, mi[:, d]]
    return U


def box_nodes(n: int, centre: np.ndarray, h: float) -> np.ndarray:
    """Physical positions of the n^D Chebyshev nodes of a box."""
    t = nodes(n)
    mi = node_multi_index(n, centre.shape[0])
    return centre[None, :] + h * t[mi]


def transfer_matrix(n: int, dim: int, child_pos: int) -> np.ndarray:
    """L2L operator U_{c->p}[a, b] = prod_d S_n(xi_d(child node a), t_{b_d}).

    child_pos bit d = 1 when the child is the upper half along dimension d.
    In the parent's normalised frame the child's node a sits at
    (2 bit_d - 1)/2 + t_{a_d}/2.  The M2M operator is its transpose.
    """
    t = nodes(n)
    mi = node_multi_index(n, dim)
    shift = np.array([((child_pos >> d) & 1) - 0.5 for d in range(dim)])
    xi = shift[None, :] + 0.5 * t[mi]
    return interp_matrix(n, xi)
