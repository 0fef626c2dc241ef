"""Uniform 2^D-tree, neighbour and interaction lists, colouring (oracle).

Paper: Sec. 2.3 (octree: up to 3^3 = 27 neighbours including the box itself,
up to 6^3 - 3^3 = 189 boxes in the interaction list), Algorithm 1 (build an
octree of the domain), Sec. 3 (uniform tree, depth set by the points per leaf).
The interaction list I_i of a box is the set of children of its parent's
neighbours that are not neighbours of the box (Sec. 2.2, after Eq. K_jq_update).

Readings where the paper is silent (they also bind the CUDA path):
* root = the cube of edge max_d(max_d - min_d) * (1 + 1e-12) anchored at the
  per-dimension minimum of the points;
* leaf depth L = the smallest L >= 2 whose fullest leaf holds <= leaf_max
  points; N <= leaf_max means no tree (one dense block);
* a point's box index at depth l is floor(((x - lo) / edge) * 2^l), clamped;
* boxes are ordered by Morton key (x bit lowest), points inside a leaf keep
  their input order, empty boxes are dropped;
* elimination order (the paper leaves it open, Sec. 4): colour
  c = sum_d (ix_d mod 3) 3^d, colours in increasing order, boxes of one colour
  in Morton order.  Two boxes of one colour are >= 3 apart, so their neighbour
  lists are disjoint.

Parity: pinned by tests (brute-force neighbour/interaction lists on tiny
trees, list sizes <= 27 / 189, colour-class disjointness).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import product

import numpy as np

MAX_DEPTH = 20
EDGE_WIDEN = 1.0 + 1e-12


def morton_key(coords: np.ndarray, dim: int) -> np.ndarray:
    """Interleave the bits of integer box coordinates, x in the lowest bit."""
    c = np.asarray(coords, dtype=np.uint64)
    key = np.zeros(c.shape[0], dtype=np.uint64)
    for b in range(MAX_DEPTH + 1):
        for d in range(dim):
            bit = (c[:, d] >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(dim * b + d)
    return key


def box_coords(points: np.ndarray, lo: np.ndarray, edge: float, depth: int) -> np.ndarray:
    t = (points - lo) / edge
    k = np.floor(t * float(1 << depth)).astype(np.int64)
    return np.clip(k, 0, (1 << depth) - 1)


@dataclass
class Level:
    l: int
    coords: np.ndarray              # (nb, dim) int64, boxes in Morton order
    keys: np.ndarray                # (nb,) uint64 Morton keys (ascending)
    parent: np.ndarray              # (nb,) index of the parent box at level l-1 (-1 at the root)
    children: list = field(default_factory=list)   # per box: indices at level l+1 (Morton order)
    nbrs: list = field(default_factory=list)       # per box: N_i, indices, Morton order, includes i
    inter: list = field(default_factory=list)      # per box: I_i, indices, Morton order
    colour: np.ndarray | None = None
    pt_begin: np.ndarray | None = None             # leaves only: point range in tree order
    pt_end: np.ndarray | None = None

    @property
    def nb(self) -> int:
        return int(self.keys.shape[0])

    def centre_halfwidth(self, lo: np.ndarray, edge: float):
        h = edge / float(1 << (self.l + 1))
        centres = lo[None, :] + (2.0 * self.coords + 1.0) * h
        return centres, h


@dataclass
class Tree:
    dim: int
    N: int
    L: int                          # leaf depth (0 means: no tree, one dense block)
    lo: np.ndarray
    edge: float
    perm: np.ndarray                # tree order -> user index
    levels: dict                    # depth -> Level, depths 0..L
    leaf_max: int

    @property
    def dense(self) -> bool:
        return self.L == 0

    def leaf_points(self, i: int) -> np.ndarray:
        lev = self.levels[self.L]
        return np.arange(lev.pt_begin[i], lev.pt_end[i])


def _choose_depth(points, lo, edge, dim, leaf_max) -> int:
    N = points.shape[0]
    if N <= leaf_max:
        return 0
    for L in range(2, MAX_DEPTH + 1):
        keys = morton_key(box_coords(points, lo, edge, L), dim)
        _, counts = np.unique(keys, return_counts=True)
        if counts.max() <= leaf_max:
            return L
    raise ValueError("points too clustered: no depth <= 20 meets the leaf size")


def build_tree(points: np.ndarray, leaf_max: int) -> Tree:
    points = np.asarray(points, dtype=np.float64)
    N, dim = points.shape
    lo = points.min(axis=0)
    hi = points.max(axis=0)
    edge = float(np.max(hi - lo)) * EDGE_WIDEN
    if edge == 0.0:
        edge = 1.0
    L = _choose_depth(points, lo, edge, dim, leaf_max)
    if L == 0:
        lev = Level(0, np.zeros((1, dim), np.int64), np.zeros(1, np.uint64), np.array([-1]))
        lev.pt_begin = np.array([0])
        lev.pt_end = np.array([N])
        lev.nbrs = [[0]]
        lev.inter = [[]]
        lev.colour = np.zeros(1, np.int64)
        return Tree(dim, N, 0, lo, edge, np.arange(N), {0: lev}, leaf_max)

    leaf_c = box_coords(points, lo, edge, L)
    leaf_k = morton_key(leaf_c, dim)
    perm = np.argsort(leaf_k, kind="stable")
    levels: dict[int, Level] = {}
    for l in range(L, -1, -1):
        c = leaf_c >> (L - l)
        k = morton_key(c, dim)
        uk, first = np.unique(k, return_index=True)
        levels[l] = Level(l, c[first], uk, np.full(uk.shape[0], -1, np.int64))
    leaf = levels[L]
    sk = leaf_k[perm]
    leaf.pt_begin = np.searchsorted(sk, leaf.keys, side="left")
    leaf.pt_end = np.searchsorted(sk, leaf.keys, side="right")
    for l in range(1, L + 1):
        lev, par = levels[l], levels[l - 1]
        pk = lev.keys >> np.uint64(dim)
        lev.parent = np.searchsorted(par.keys, pk)
        par.children = [[] for _ in range(par.nb)]
        for i, p in enumerate(lev.parent):
            par.children[p].append(i)
    levels[L].children = [[] for _ in range(levels[L].nb)]
    for l in range(0, L + 1):
        _lists(levels, l, dim)
    return Tree(dim, N, L, lo, edge, perm, levels, leaf_max)


def _lists(levels, l, dim):
    lev = levels[l]
    index = {tuple(c): i for i, c in enumerate(lev.coords.tolist())}
    offs = list(product((-1, 0, 1), repeat=dim))
    lev.nbrs = []
    for c in lev.coords.tolist():
        nb = [index[t] for t in (tuple(a + b for a, b in zip(c, o)) for o in offs) if t in index]
        lev.nbrs.append(sorted(nb))
    lev.inter = []
    for i in range(lev.nb):
        if l < 2:
            lev.inter.append([])
            continue
        near = set(lev.nbrs[i])
        cand = []
        for pn in levels[l - 1].nbrs[lev.parent[i]]:
            cand.extend(c for c in levels[l - 1].children[pn] if c not in near)
        lev.inter.append(sorted(cand))
    w = np.array([3 ** d for d in range(dim)], dtype=np.int64)
    lev.colour = (lev.coords % 3) @ w
