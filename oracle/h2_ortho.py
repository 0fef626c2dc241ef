"""The H^2 operators of ``h2.H2`` re-represented with orthonormal bases (oracle).

Test infrastructure only (like the rest of ``oracle/``).

Paper: Sec. 3 (numerical examples) builds the initial low-rank approximations
by Chebyshev interpolation followed by an SVD that reduces the rank, so the
extended matrix E whose largest singular value sigma_0(E) sets tau = eps
sigma_0 (Eq. methods_SVD_rank_spectralnorm, Sec. 2.4) has orthonormal bases.
This module builds that representation of the same A_n without truncation:

* leaf i: U_i = Q_i R_i (thin QR; Q_i is m_i x r_i, r_i = min(m_i, n^D));
* parent p at depth l < L: W_p = [R_c T_c] stacked over its children c
  (sum r_c x n^D) = Q'_p R_p; the new transfer of child c is its row block
  of Q'_p (r_c x r_p), so Q-basis of p = blockdiag(children's bases) Q'_p;
* M2L: K'_iq = R_i K_iq R_q^T (r_i x r_q);
* near field and the -I couplings as in ``H2.extended_dense``, with the
  identity blocks of size r_i.

It is not used by the default reading of sigma_0 (raw Chebyshev operators);
it records the alternative reading and is pinned by tests: E' solved for
[b; 0] gives the dense solve of A_n, every composed basis is orthonormal, and
the power-iteration sigma_0 equals the largest singular value of dense E'.
"""
from __future__ import annotations

import math

import numpy as np

from .h2 import H2


class OrthonormalH2:
    def __init__(self, h2: H2):
        self.h2 = h2
        t = h2.tree
        L = h2.L
        assert L >= 2
        self.Q: dict = {}    # (L, i) -> leaf orthonormal basis
        self.R: dict = {}    # (l, i) -> R factor (r x n^D)
        self.Tp: dict = {}   # (l, c) -> new transfer of child c at depth l (r_c x r_parent)
        leaf = t.levels[L]
        for i in range(leaf.nb):
            q, r = np.linalg.qr(h2.leafU[i])
            self.Q[(L, i)], self.R[(L, i)] = q, r
        for l in range(L - 1, 1, -1):
            lev = t.levels[l]
            for p in range(lev.nb):
                ch = lev.children[p]
                Wp = np.vstack([self.R[(l + 1, c)] @ h2.T(l + 1, c) for c in ch])
                q, r = np.linalg.qr(Wp)
                self.R[(l, p)] = r
                o = 0
                for c in ch:
                    rc = self.R[(l + 1, c)].shape[0]
                    self.Tp[(l + 1, c)] = q[o:o + rc, :]
                    o += rc
        self.rank = {k: v.shape[0] for k, v in self.R.items()}
        self.K: dict = {}
        for l in range(2, L + 1):
            lev = t.levels[l]
            for i in range(lev.nb):
                for q in lev.inter[i]:
                    self.K[(l, i, q)] = self.R[(l, i)] @ h2.m2l(l, i, q) @ self.R[(l, q)].T
        # layout: x, then per depth L..2 the z blocks and the y blocks
        self.off: dict = {}
        pos = t.N
        for l in range(L, 1, -1):
            for kind in ("z", "y"):
                for i in range(t.levels[l].nb):
                    self.off[(kind, l, i)] = pos
                    pos += self.rank[(l, i)]
        self.n = pos

    def _blk(self, kind, l, i):
        o = self.off[(kind, l, i)]
        return slice(o, o + self.rank[(l, i)])

    def _pts(self, i):
        leaf = self.h2.tree.levels[self.h2.L]
        return slice(leaf.pt_begin[i], leaf.pt_end[i])

    def _blocks(self):
        """(row slice, column slice, matrix) of every nonzero block of E'."""
        h2, t, L = self.h2, self.h2.tree, self.h2.L
        leaf = t.levels[L]
        for i in range(leaf.nb):
            for j in leaf.nbrs[i]:
                yield self._pts(i), self._pts(j), h2.p2p(i, j)
            yield self._pts(i), self._blk("z", L, i), self.Q[(L, i)]
        for l in range(L, 1, -1):
            lev = t.levels[l]
            for i in range(lev.nb):
                zr, yr = self._blk("z", l, i), self._blk("y", l, i)
                if l == L:
                    yield zr, self._pts(i), self.Q[(L, i)].T
                else:
                    for c in lev.children[i]:
                        yield zr, self._blk("y", l + 1, c), self.Tp[(l + 1, c)].T
                r = self.rank[(l, i)]
                yield zr, yr, -np.eye(r)
                yield yr, zr, -np.eye(r)
                for q in lev.inter[i]:
                    yield yr, self._blk("y", l, q), self.K[(l, i, q)]
                if l > 2:
                    yield yr, self._blk("z", l - 1, lev.parent[i]), self.Tp[(l, i)]

    def extended_dense(self) -> np.ndarray:
        E = np.zeros((self.n, self.n))
        for r, c, M in self._blocks():
            E[r, c] += M
        return E

    def extended_apply(self, v: np.ndarray, transpose: bool = False) -> np.ndarray:
        out = np.zeros(self.n)
        for r, c, M in self._blocks():
            if transpose:
                out[c] += M.T @ v[r]
            else:
                out[r] += M @ v[c]
        return out

    def sigma0_power(self, maxit: int = 100, rtol: float = 1e-6) -> tuple[float, int]:
        """Largest singular value of E' by power iteration on E'^T E' (start
        vector all ones; stop at relative change <= rtol or maxit products),
        the same iteration the default reading applies to the raw E."""
        v = np.ones(self.n) / math.sqrt(self.n)
        prev, s, it = 0.0, 0.0, 0
        for it in range(1, maxit + 1):
            w = self.extended_apply(self.extended_apply(v), transpose=True)
            nw = float(np.linalg.norm(w))
            s = math.sqrt(nw)
            v = w / nw
            if it > 1 and abs(s - prev) <= rtol * s:
                break
            prev = s
        return s, it
