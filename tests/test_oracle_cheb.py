"""Pins for the Chebyshev interpolation operators (Sec. 3, ref. fong09a)."""
import numpy as np
import pytest

from oracle import chebyshev as cheb


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8])
def test_nodes_are_chebyshev_roots(n):
    t = cheb.nodes(n)
    # T_n(t_a) = cos(n arccos t_a) = 0 at the n roots
    assert np.allclose(np.cos(n * np.arccos(t)), 0.0, atol=1e-13)
    assert np.all(np.diff(t) < 0)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_cardinal_and_partition_of_unity(n):
    t = cheb.nodes(n)
    S = cheb.S1(n, t)
    assert np.allclose(S, np.eye(n), atol=1e-13)
    x = np.linspace(-1, 1, 37)
    assert np.allclose(cheb.S1(n, x).sum(axis=1), 1.0, atol=1e-13)


@pytest.mark.parametrize("n,dim", [(3, 3), (4, 3), (6, 2), (2, 3)])
def test_polynomials_below_degree_n_are_reproduced(n, dim):
    rng = np.random.default_rng(n * 10 + dim)
    xi = rng.uniform(-1, 1, (50, dim))
    nodes = cheb.box_nodes(n, np.zeros(dim), 1.0)
    # random tensor polynomial of degree < n in each coordinate
    coef = rng.standard_normal((n,) * dim)

    def poly(X):
        out = np.zeros(X.shape[0])
        for idx in np.ndindex(*coef.shape):
            term = coef[idx] * np.ones(X.shape[0])
            for d, e in enumerate(idx):
                term = term * X[:, d] ** e
            out += term
        return out

    U = cheb.interp_matrix(n, xi)
    assert np.allclose(U @ poly(nodes), poly(xi), atol=1e-11)


@pytest.mark.parametrize("n,dim", [(3, 3), (4, 2)])
def test_transfer_is_interpolation_to_child_nodes(n, dim):
    # L2L: values at the parent's nodes -> values at the child's nodes, exact
    # for polynomials of degree < n; check against direct evaluation.
    rng = np.random.default_rng(3)
    a = rng.standard_normal(dim)
    pnodes = cheb.box_nodes(n, np.zeros(dim), 1.0)
    f = lambda X: (X @ a) ** (n - 1) + 1.0
    for c in range(1 << dim):
        centre = np.array([0.5 if (c >> d) & 1 else -0.5 for d in range(dim)])
        cnodes = cheb.box_nodes(n, centre, 0.5)
        T = cheb.transfer_matrix(n, dim, c)
        assert np.allclose(T @ f(pnodes), f(cnodes), atol=1e-12)


def test_node_ordering_first_coordinate_fastest():
    mi = cheb.node_multi_index(3, 3)
    assert mi[:4].tolist() == [[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0]]
