"""Pins for the oracle's GMRES (Sec. 3.2)."""
import numpy as np

from oracle.gmres import gmres


def test_matches_dense_solve():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((150, 150)) + 20 * np.eye(150)
    b = rng.standard_normal(150)
    x, it, res = gmres(lambda v: A @ v, b, tol=1e-12)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-11
    assert abs(res - np.linalg.norm(A @ x - b) / np.linalg.norm(b)) < 1e-10
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9)


def test_iterations_equal_distinct_eigenvalues():
    # Krylov space of a diagonalisable matrix with k distinct eigenvalues has dim k
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    ev = np.repeat([1.0, 2.0, 5.0, 7.0, 11.0], 12)
    A = Q @ np.diag(ev) @ Q.T
    b = rng.standard_normal(60)
    x, it, res = gmres(lambda v: A @ v, b, tol=1e-12)
    assert it == 5
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-10


def test_right_preconditioner_exact_inverse_converges_in_one():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((80, 80)) + 10 * np.eye(80)
    Ai = np.linalg.inv(A)
    b = rng.standard_normal(80)
    x, it, res = gmres(lambda v: A @ v, b, precond=lambda v: Ai @ v, tol=1e-10)
    assert it == 1
    assert np.allclose(A @ x, b, atol=1e-9)


def test_max_iterations_reported():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((100, 100))
    b = rng.standard_normal(100)
    x, it, res = gmres(lambda v: A @ v, b, tol=1e-14, maxit=7)
    assert it == 7 and res > 1e-14


def test_left_preconditioner_exact_inverse_converges_in_one():
    """Appendix B: with P^-1 = A^-1 on the left, P^-1 A = I and the first
    Krylov vector already holds the solution."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((80, 80)) + 10 * np.eye(80)
    Ai = np.linalg.inv(A)
    b = rng.standard_normal(80)
    x, it, res = gmres(lambda v: A @ v, b, precond=lambda v: Ai @ v, tol=1e-10, side="left")
    assert it == 1
    assert np.allclose(A @ x, b, atol=1e-9)


def test_left_residual_is_the_preconditioned_residual():
    """Appendix B: the left-preconditioned estimate measures
    ||P^-1 (b - A x)|| / ||P^-1 b||, not the true residual; a diagonal P that
    scales rows by 10^[0, 4] makes the two differ, and GMRES on the
    preconditioned system matches the dense solve of P^-1 A x = P^-1 b."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((120, 120)) + 30 * np.eye(120)
    d = 10.0 ** rng.uniform(0, 4, 120)
    b = rng.standard_normal(120)
    Pinv = lambda v: v / d
    x, it, res = gmres(lambda v: A @ v, b, precond=Pinv, tol=1e-12, side="left")
    pres = np.linalg.norm(Pinv(b - A @ x)) / np.linalg.norm(Pinv(b))
    assert abs(res - pres) < 1e-10
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-8)
    # right preconditioning builds another Krylov space; at this tolerance both
    # reach the dense solution
    xr, itr, _ = gmres(lambda v: A @ v, b, precond=Pinv, tol=1e-12, side="right")
    assert np.allclose(xr, x, rtol=1e-8)


def test_block_gmres_matches_dense_solve_and_exact_preconditioner():
    """Block GMRES: every column reaches the dense solution; with the exact
    inverse as right preconditioner one block step solves all columns; with 4
    generic right-hand sides of a 12 x 12 system the shared Krylov space gains
    4 directions per step and spans the whole space after 12 / 4 = 3 steps,
    where single-vector GMRES needs 12."""
    from oracle.gmres import block_gmres
    rng = np.random.default_rng(6)
    A = rng.standard_normal((90, 90)) + 15 * np.eye(90)
    B = rng.standard_normal((90, 3))
    X, steps, res = block_gmres(lambda v: A @ v, B, tol=1e-12)
    assert np.allclose(X, np.linalg.solve(A, B), rtol=1e-9, atol=1e-10)
    Ai = np.linalg.inv(A)
    X1, s1, _ = block_gmres(lambda v: A @ v, B, precond=lambda v: Ai @ v, tol=1e-10)
    assert s1 == 1 and np.allclose(A @ X1, B, atol=1e-9)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    As = Q @ np.diag(np.arange(1.0, 13.0)) @ Q.T
    B4 = rng.standard_normal((12, 4))
    X4, s4, _ = block_gmres(lambda v: As @ v, B4, tol=1e-12)
    assert s4 == 3 and np.allclose(As @ X4, B4, atol=1e-9)
    _, it1, _ = gmres(lambda v: As @ v, B4[:, 0], tol=1e-12)
    assert it1 == 12
