"""Raw H^2 (black-box FMM) operators, FMM matvec, dense assemblies (oracle).

Paper: Sec. 2.1.  A = S^(L) + U^(L) K^(L) V^(L)T (Eq. A_decomp_l3), applied
recursively (Eq. A_decomp_l2); U = L2P/L2L, V^T = P2M/M2M, K = M2L, S = P2P.
The multipole coefficients y^(l) (Eqs. y3, y2) and local coefficients z^(l)
(Eqs. z2, z3) turn A x = b into the extended sparse system of
Eq. (Ax=b_extended).  Sec. 3.2: the black-box FMM evaluates the products
inside GMRES.

Definitions used here (Chebyshev interpolation, see ``chebyshev``):
* leaf U_i = V_i [p, a] = S_n at point p of leaf i for node a (m_i x n^D);
* transfer T_c (child c -> parent), L2L U(c, c-dagger) = T_c and M2M V = T_c;
* M2L K_iq [a, b] = K(node a of box i, node b of box q), q in I_i;
* P2P S_ij = the exact kernel block, j in N_i (leaves).
The H^2 matrix these define is written A_n (n Chebyshev nodes per dimension).

Parity: ``matvec`` is pinned against ``dense_blockwise`` (an independent
block-by-block assembly of A_n), against the direct sum with error falling as
n grows, and ``extended_dense`` is pinned by solving E [x; z; y] = [b; 0; 0]
and comparing x with the dense solve of A_n.  ``extended_apply`` and
``extended_apply_T`` are pinned against ``extended_dense``.
"""
from __future__ import annotations

import numpy as np

from . import chebyshev as cheb
from .kernels import kernel_matrix
from .tree import Tree, build_tree


class H2:
    def __init__(self, points: np.ndarray, kind: int, param: float, diag: float, n: int,
                 leaf_max: int, tree: Tree | None = None):
        self.points = np.asarray(points, dtype=np.float64)
        self.kind, self.param, self.diag = kind, param, diag
        self.n = n
        self.tree = tree if tree is not None else build_tree(self.points, leaf_max)
        t = self.tree
        self.dim = t.dim
        self.nd = n ** t.dim
        self.tp = self.points[t.perm]                  # points in tree order
        self.L = t.L
        self.transfer = [cheb.transfer_matrix(n, t.dim, c) for c in range(1 << t.dim)]
        self._m2l_cache = {}
        self._p2p_cache = {}
        self.leafU = []
        if t.L > 0:
            leaf = t.levels[t.L]
            cen, h = leaf.centre_halfwidth(t.lo, t.edge)
            for i in range(leaf.nb):
                x = self.tp[leaf.pt_begin[i]:leaf.pt_end[i]]
                self.leafU.append(cheb.interp_matrix(n, (x - cen[i]) / h))

    # -- operator blocks ---------------------------------------------------
    def kmat(self, x, y):
        return kernel_matrix(self.kind, self.param, self.diag, x, y)

    def leaf_pts(self, i):
        lev = self.tree.levels[self.L]
        return self.tp[lev.pt_begin[i]:lev.pt_end[i]]

    def p2p(self, i, j):
        if (i, j) not in self._p2p_cache:
            self._p2p_cache[(i, j)] = self.kmat(self.leaf_pts(i), self.leaf_pts(j))
        return self._p2p_cache[(i, j)]

    def child_pos(self, l, i):
        c = self.tree.levels[l].coords[i]
        return int(sum(((int(c[d]) & 1) << d) for d in range(self.dim)))

    def T(self, l, i):
        """Transfer of box i at level l to its parent (L2L; its transpose is M2M)."""
        return self.transfer[self.child_pos(l, i)]

    def m2l(self, l, i, q):
        lev = self.tree.levels[l]
        off = tuple((lev.coords[q] - lev.coords[i]).tolist())
        key = (l, off)
        if key not in self._m2l_cache:
            t = self.tree
            h = t.edge / float(1 << (l + 1))
            ci = t.lo + (2.0 * lev.coords[i] + 1.0) * h
            cq = t.lo + (2.0 * lev.coords[q] + 1.0) * h
            self._m2l_cache[key] = self.kmat(cheb.box_nodes(self.n, ci, h),
                                             cheb.box_nodes(self.n, cq, h))
        return self._m2l_cache[key]

    # -- FMM matvec ---------------------------------------------------------
    def matvec(self, x: np.ndarray) -> np.ndarray:
        """A_n x in tree order; x is (N,) or (N, k)."""
        x = np.asarray(x, dtype=np.float64)
        vec = x.ndim == 1
        X = x.reshape(x.shape[0], -1)
        t = self.tree
        if t.L == 0:
            y = self.kmat(self.tp, self.tp) @ X
            return y[:, 0] if vec else y
        L = t.L
        leaf = t.levels[L]
        mult = {L: [self.leafU[i].T @ X[leaf.pt_begin[i]:leaf.pt_end[i]] for i in range(leaf.nb)]}
        for l in range(L - 1, 1, -1):                      # M2M
            lev = t.levels[l]
            mult[l] = [sum(self.T(l + 1, c).T @ mult[l + 1][c] for c in lev.children[p])
                       for p in range(lev.nb)]
        loc = {}
        for l in range(2, L + 1):                          # M2L + L2L
            lev = t.levels[l]
            loc[l] = []
            for i in range(lev.nb):
                z = np.zeros((self.nd, X.shape[1]))
                for q in lev.inter[i]:
                    z += self.m2l(l, i, q) @ mult[l][q]
                if l > 2:
                    z += self.T(l, i) @ loc[l - 1][lev.parent[i]]
                loc[l].append(z)
        Y = np.zeros_like(X)
        for i in range(leaf.nb):                           # L2P + P2P
            r = slice(leaf.pt_begin[i], leaf.pt_end[i])
            Y[r] = self.leafU[i] @ loc[L][i]
            for j in leaf.nbrs[i]:
                Y[r] += self.p2p(i, j) @ X[leaf.pt_begin[j]:leaf.pt_end[j]]
        return Y[:, 0] if vec else Y

    def direct_matvec(self, x: np.ndarray) -> np.ndarray:
        """The exact A x in tree order (direct sum)."""
        return self.kmat(self.tp, self.tp) @ x

    # -- dense assemblies (small N only) --------------------------------------
    def dense_exact(self) -> np.ndarray:
        return self.kmat(self.tp, self.tp)

    def ancestor(self, l_from, i, l_to):
        for l in range(l_from, l_to, -1):
            i = self.tree.levels[l].parent[i]
        return i

    def up_basis(self, i, l):
        """U of leaf i carried up to level l: U_i T_{i} T_{p(i)} ... (m_i x n^D)."""
        B = self.leafU[i]
        b = i
        for lv in range(self.L, l, -1):
            B = B @ self.T(lv, b)
            b = self.tree.levels[lv].parent[b]
        return B

    def dense_blockwise(self) -> np.ndarray:
        """A_n assembled block by block from Eq. (A_decomp_l2) (independent of ``matvec``)."""
        t = self.tree
        if t.L == 0:
            return self.dense_exact()
        leaf = t.levels[self.L]
        A = np.zeros((t.N, t.N))
        for i in range(leaf.nb):
            ri = slice(leaf.pt_begin[i], leaf.pt_end[i])
            for j in range(leaf.nb):
                rj = slice(leaf.pt_begin[j], leaf.pt_end[j])
                if j in leaf.nbrs[i]:
                    A[ri, rj] = self.p2p(i, j)
                    continue
                for l in range(self.L, 1, -1):
                    ai, aj = self.ancestor(self.L, i, l), self.ancestor(self.L, j, l)
                    if aj in t.levels[l].inter[ai]:
                        A[ri, rj] = self.up_basis(i, l) @ self.m2l(l, ai, aj) @ self.up_basis(j, l).T
                        break
                else:
                    raise AssertionError("pair not covered by the H^2 partition")
        return A

    # -- extended sparse system (Eq. Ax=b_extended) ------------------------------
    def extended_layout(self):
        """Offsets of x, z^(l), y^(l) blocks; l = L..2."""
        t = self.tree
        off = {"x": 0}
        pos = t.N
        for l in range(self.L, 1, -1):
            nb = t.levels[l].nb
            off[("z", l)] = pos
            pos += nb * self.nd
            off[("y", l)] = pos
            pos += nb * self.nd
        return off, pos

    def extended_dense(self) -> np.ndarray:
        t = self.tree
        assert t.L >= 2
        off, n = self.extended_layout()
        nd = self.nd
        E = np.zeros((n, n))
        L = self.L
        leaf = t.levels[L]
        zL = off[("z", L)]
        for i in range(leaf.nb):
            ri = slice(leaf.pt_begin[i], leaf.pt_end[i])
            for j in leaf.nbrs[i]:
                E[ri, leaf.pt_begin[j]:leaf.pt_end[j]] = self.p2p(i, j)
            E[ri, zL + i * nd: zL + (i + 1) * nd] = self.leafU[i]
        for l in range(L, 1, -1):
            lev = t.levels[l]
            z0, y0 = off[("z", l)], off[("y", l)]
            for i in range(lev.nb):
                zr = slice(z0 + i * nd, z0 + (i + 1) * nd)
                yr = slice(y0 + i * nd, y0 + (i + 1) * nd)
                # Eq_z row: V_i^T xtilde_i - y_i = 0
                if l == L:
                    E[zr, leaf.pt_begin[i]:leaf.pt_end[i]] = self.leafU[i].T
                else:
                    yc0 = off[("y", l + 1)]
                    for c in lev.children[i]:
                        E[zr, yc0 + c * nd: yc0 + (c + 1) * nd] = self.T(l + 1, c).T
                E[zr, yr] = -np.eye(nd)
                # Eq_y row: -z_i + sum_q K_iq y_q + U_(i->p) z_p = 0
                E[yr, zr] = -np.eye(nd)
                for q in lev.inter[i]:
                    E[yr, y0 + q * nd: y0 + (q + 1) * nd] = self.m2l(l, i, q)
                if l > 2:
                    zp0 = off[("z", l - 1)]
                    p = lev.parent[i]
                    E[yr, zp0 + p * nd: zp0 + (p + 1) * nd] = self.T(l, i)
        return E

    def extended_apply(self, v: np.ndarray, transpose: bool = False) -> np.ndarray:
        """E v (or E^T v) block by block, without assembling E."""
        t = self.tree
        off, n = self.extended_layout()
        nd = self.nd
        L = self.L
        leaf = t.levels[L]
        out = np.zeros(n)

        def blk(kind, l, i):
            o = off[(kind, l)]
            return slice(o + i * nd, o + (i + 1) * nd)

        def pts(i):
            return slice(leaf.pt_begin[i], leaf.pt_end[i])

        def add(row, col, M):
            # row/col are slices; adds M (as stored at (row, col) of E) times v
            if transpose:
                out[col] += M.T @ v[row]
            else:
                out[row] += M @ v[col]

        for i in range(leaf.nb):
            for j in leaf.nbrs[i]:
                add(pts(i), pts(j), self.p2p(i, j))
            add(pts(i), blk("z", L, i), self.leafU[i])
        for l in range(L, 1, -1):
            lev = t.levels[l]
            for i in range(lev.nb):
                if l == L:
                    add(blk("z", l, i), pts(i), self.leafU[i].T)
                else:
                    for c in lev.children[i]:
                        add(blk("z", l, i), blk("y", l + 1, c), self.T(l + 1, c).T)
                # the two -I blocks, (z_i, y_i) and (y_i, z_i), are each other's
                # transpose, so E and E^T apply them alike
                out[blk("z", l, i)] -= v[blk("y", l, i)]
                out[blk("y", l, i)] -= v[blk("z", l, i)]
                for q in lev.inter[i]:
                    add(blk("y", l, i), blk("y", l, q), self.m2l(l, i, q))
                if l > 2:
                    add(blk("y", l, i), blk("z", l - 1, lev.parent[i]), self.T(l, i))
        return out
