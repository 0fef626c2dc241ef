"""Pins for the oracle's tree, lists and colouring (Sec. 2.3, Algorithm 1)."""
from itertools import product

import numpy as np
import pytest

from oracle.tree import build_tree, morton_key
from workloads import uniform_cube, unit_sphere


def brute_lists(lev_l, lev_p, i):
    """Neighbours: Chebyshev distance <= 1.  Interaction list: children of the
    parent's neighbours at distance >= 2 (definition in Sec. 2.2)."""
    c = lev_l.coords
    d = np.max(np.abs(c - c[i]), axis=1)
    near = sorted(np.nonzero(d <= 1)[0].tolist())
    pc = c >> 1
    pd = np.max(np.abs(pc - pc[i]), axis=1)
    far = sorted(np.nonzero((pd <= 1) & (d >= 2))[0].tolist())
    return near, far


@pytest.mark.parametrize("dim,N,leaf", [(3, 700, 16), (2, 900, 12), (3, 400, 8)])
def test_lists_match_brute_force(dim, N, leaf):
    pts = uniform_cube(N, 11 + dim, dim)
    t = build_tree(pts, leaf)
    assert t.L >= 2
    for l in range(2, t.L + 1):
        lev = t.levels[l]
        for i in range(lev.nb):
            near, far = brute_lists(lev, t.levels[l - 1], i)
            assert lev.nbrs[i] == near
            assert lev.inter[i] == far
            assert len(near) <= 3 ** dim and len(far) <= 6 ** dim - 3 ** dim


def test_list_sizes_reach_paper_bounds():
    # a full uniform level-4 octree: interior boxes have 27 neighbours, 189 interactions
    pts = uniform_cube(40000, 3, 3)
    t = build_tree(pts, 40)
    lev = t.levels[t.L]
    assert max(len(n) for n in lev.nbrs) == 27
    assert max(len(f) for f in lev.inter) == 189


def test_depth_rule_and_point_order():
    pts = uniform_cube(2048, 1000, 3)
    t = build_tree(pts, 64)
    leaf = t.levels[t.L]
    counts = leaf.pt_end - leaf.pt_begin
    assert counts.max() <= 64
    # one level less would overflow a leaf (smallest admissible depth)
    t2 = build_tree(pts, int(counts.max()) - 1)
    assert t2.L > t.L or t2.L == 0
    # points of a leaf keep input order; keys ascend
    assert np.all(np.diff(leaf.keys.astype(np.float64)) > 0)
    for i in range(leaf.nb):
        seg = t.perm[leaf.pt_begin[i]:leaf.pt_end[i]]
        assert np.all(np.diff(seg) > 0)
    assert sorted(t.perm.tolist()) == list(range(2048))


def test_dense_when_small():
    t = build_tree(uniform_cube(50, 1, 3), 64)
    assert t.dense and t.L == 0


def test_colour_classes_have_disjoint_neighbourhoods():
    pts = unit_sphere(3000, 5)
    t = build_tree(pts, 20)
    for l in range(2, t.L + 1):
        lev = t.levels[l]
        for c in range(27):
            seen = set()
            for i in np.nonzero(lev.colour == c)[0]:
                s = set(lev.nbrs[i])
                assert not (s & seen)
                seen |= s


def test_morton_interleave():
    c = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [3, 1, 2]])
    # (3,1,2): bit 0 -> x=1, y=1, z=0 (1 + 2); bit 1 -> x=1, y=0, z=1 (8 + 32)
    assert morton_key(c, 3).tolist() == [1, 2, 4, 43]
