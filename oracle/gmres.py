"""Non-restarted GMRES with a right or left preconditioner (oracle).

Paper: Sec. 3.2 -- the system A x = b is solved by non-restarted GMRES
(ref. saad86a) with tolerance 1e-10 on the relative residual
||b - A x|| / ||b|| and at most 500 iterations; the FMM evaluates the
products and the IFMM is applied as a right preconditioner.  Appendix B
compares right with left preconditioning; with the preconditioner on the
left, GMRES runs on P^-1 A x = P^-1 b and the tolerance applies to
||P^-1 b - P^-1 A x|| / ||P^-1 b||.

Readings (the paper does not state them): x_0 = 0; Arnoldi with classical
Gram-Schmidt applied twice (CGS2); Givens rotations on the Hessenberg
matrix; the loop stops when the Arnoldi residual estimate |g_{k+1}| falls to
tol * ||b||; the reported true residual is recomputed with the matvec.

Parity: pinned by tests against scipy's dense solve on small systems
(exact solution within the tolerance, residual estimate = true residual) and
by the iteration count n for a matrix with n distinct eigenvalues.
"""
from __future__ import annotations

import math

import numpy as np


def gmres(matvec, b: np.ndarray, precond=None, tol: float = 1e-10, maxit: int = 500,
          side: str = "right"):
    """Returns (x, iterations, relative residual estimate).

    side "right": Krylov space of A P^-1, x = P^-1 (V y), estimate of
    ||b - A x|| / ||b||.  side "left" (Appendix B): Krylov space of P^-1 A
    started from P^-1 b, x = V y, estimate of ||P^-1 (b - A x)|| / ||P^-1 b||.
    """
    b = np.asarray(b, dtype=np.float64)
    M = precond if precond is not None else (lambda v: v)
    left = side == "left"
    r0 = M(b) if left else b
    beta = float(np.linalg.norm(r0))
    n = b.shape[0]
    if beta == 0.0:
        return np.zeros(n), 0, 0.0
    V = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    V[0] = r0 / beta
    k = 0
    res = beta
    for k in range(maxit):
        w = M(matvec(V[k])) if left else matvec(M(V[k]))
        h = V[:k + 1] @ w                       # CGS, first pass
        w = w - V[:k + 1].T @ h
        h2 = V[:k + 1] @ w                      # second pass
        w = w - V[:k + 1].T @ h2
        h = h + h2
        hn = float(np.linalg.norm(w))
        col = np.concatenate([h, [hn]])
        for j in range(k):                      # previous rotations
            t = cs[j] * col[j] + sn[j] * col[j + 1]
            col[j + 1] = -sn[j] * col[j] + cs[j] * col[j + 1]
            col[j] = t
        den = math.hypot(col[k], col[k + 1])
        cs[k] = col[k] / den if den else 1.0
        sn[k] = col[k + 1] / den if den else 0.0
        col[k] = den
        col[k + 1] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        H[:k + 2, k] = col
        res = abs(g[k + 1])
        if hn > 0.0:
            V[k + 1] = w / hn
        if res <= tol * beta or hn == 0.0:
            k += 1
            break
    else:
        k = maxit
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k]) if k else np.zeros(0)
    x = V[:k].T @ y if left else M(V[:k].T @ y)
    return x, k, res / beta


def block_gmres(matvec, B: np.ndarray, precond=None, tol: float = 1e-10, maxit: int = 500):
    """Block GMRES with a right preconditioner: one Krylov space
    span{R0, A P^-1 R0, ...} shared by the k columns of B (x_0 = 0).  Block
    Arnoldi with classical Gram-Schmidt applied twice and a QR of every new
    block; the least-squares problem min |E_1 S_0 - H Y| is solved afresh at
    each step (numpy lstsq), a column converging when its residual there is at
    most tol ||b_c||.  Returns (X, block steps, relative residual estimates)."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, k = B.shape
    M = precond if precond is not None else (lambda v: v)
    Mb = lambda V: np.column_stack([M(V[:, c]) for c in range(V.shape[1])])
    Ab = lambda V: np.column_stack([matvec(V[:, c]) for c in range(V.shape[1])])
    bn = np.linalg.norm(B, axis=0)
    V0, S0 = np.linalg.qr(B)
    Vs = [V0]
    H = np.zeros(((maxit + 1) * k, maxit * k))
    res = bn.copy()
    Y = np.zeros((0, k))
    j = 0
    for j in range(maxit):
        W = Ab(Mb(Vs[j]))
        Vall = np.hstack(Vs)
        h = Vall.T @ W
        W = W - Vall @ h
        h2 = Vall.T @ W
        W = W - Vall @ h2
        Vn, Rn = np.linalg.qr(W)
        Vs.append(Vn)
        H[:(j + 1) * k, j * k:(j + 1) * k] = h + h2
        H[(j + 1) * k:(j + 2) * k, j * k:(j + 1) * k] = Rn
        E = np.zeros(((j + 2) * k, k))
        E[:k] = S0
        Hj = H[:(j + 2) * k, :(j + 1) * k]
        Y = np.linalg.lstsq(Hj, E, rcond=None)[0]
        res = np.linalg.norm(E - Hj @ Y, axis=0)
        if np.all(res <= tol * bn):
            break
    steps = j + 1
    X = Mb(np.hstack(Vs[:steps]) @ Y)
    return X, steps, res / np.where(bn > 0, bn, 1.0)

