"""Inverse fast multipole method: factorisation and solve (oracle).

Paper sections followed, in order:

* Sec. 2.4, Eq. (methods_SVD_rank_spectralnorm): a fill-in keeps the singular
  values above tau = eps * sigma_0(E); sigma_0 is the largest singular value of
  the extended matrix E (here by power iteration on E^T E with the raw
  operators; the paper uses a randomised SVD for the same number).
* Footnote to Eq. (U_j_recomp) and Sec. 3: the initial bases come from the
  Chebyshev operators followed by an SVD that reduces the rank, with weights
  Sigma_U from an SVD of [ .. | U_j K_jq V_q^T | .. ] over q in I_j.
* Algorithm 1: for each level L .. 2 initialise the level's operators,
  eliminate the level, form the parent's operators; solve the top system for
  y^(2); substitute back down.
* Algorithm 2: eliminating (xtilde_i, z_i) of box i creates fill-in between
  all pairs of its neighbours; fill-in between well-separated boxes
  (j not in N_k) is compressed, all other fill-in is added to existing edges.
* Eqs. (P2P_kj)-(V_prime) and Algorithm 3: the fill is absorbed into new
  weighted bases [U Sigma_U | U' Sigma'] ~ U_hat Sigma_hat Phi, with
  r_j = U_hat^T U (the paper's r_j = Sigma_hat phi_j Sigma_U^-1) and
  t_j = V_hat^T V; every edge of the box is redirected: K(j, q) <- r_j K(j, q),
  K(q, j) <- K(q, j) t_j^T, the parent transfers U <- r_j U, V <- t_j V, and
  the fill itself lands in K(j, k) through the new bases (Eq. K_kj_update).
* Eqs. (y_merge)-(K_merge): after a level, the multipoles y of the children
  form the parent's unknowns, U/V of the parent stack the children's
  transfers and the parent's near-field blocks stack the children's K blocks.

Readings where the paper is silent or ambiguous (the CUDA path follows the
same readings):

R1  rank rule: keep exactly the singular values sigma > tau (sigma == tau is
    dropped); tau = 0 means compression disabled: every direction is kept.
R2  recompression uses the same absolute tau as the fill compression.
R3  exact truncated SVD stands in for the paper's randomised SVD and ACA, so
    results are deterministic.
R4  aggregated compression: after eliminating box i, each uneliminated
    neighbour j recompresses ONCE with all its well-separated fill of this
    elimination: SVD of [U_j Sigma_U | F_j1 | F_j2 ..] (U side) and of
    [V_j Sigma_V | F_1j^T | ..] (V side).  Taking the fill itself instead of
    its rank-revealing factor U' Sigma' gives the same left singular vectors
    and values (the right factor of an SVD is orthonormal).
R5  the U and V sides of a box keep one common rank r = max(r_U, r_V) so the
    pivot block [[S, U], [V^T, 0]] stays square.
R6  the initial weighted basis of a box: thin QR U_i = Q R, V_q = Q_q R_q;
    SVD of R [K_iq R_q^T]_{q in I_i}; U_hat = Q W_r, Sigma_U = sigma_1..r,
    r_i = W_r^T R (and the same on the V side with K_qi^T).  A box with an
    empty interaction list weights its basis by sigma_0 (R alone, scaled).
R7  parent bases are initialised after the children's level is eliminated
    (Algorithm 1 lists initialisation first; the parent's U, V depend on the
    children's r_j, t_j of Eqs. U_parent_j_update, V_parent_j_update).
R8  pivoting: partial (row) pivoting inside E(P, P) only (LAPACK getrf).
R9  an optional rank cap bounds r (default: none, the rank rule is tau
    alone).  Sec. 2.4 names two ways to fix a fill-in's rank: a prescribed
    rank, or the relative accuracy eps; the cap combines them (the rank at
    tau, but at most the prescribed rank).
R3b the randomised SVD of Sec. 2.4 (Halko, Martinsson, Tropp 2011,
    randomised subspace iteration) is an option, off by default (then the
    exact truncated SVD of reading R3 is used everywhere).  Its parameters are
    fixed readings, not tuning knobs: it needs a target rank, so it applies
    only under a rank cap, to blocks with more rows than the option
    ``rsvd_rows`` whose cap is below their height; k = min(a, cap + 16)
    sample columns (oversampling p = 16) of a uniform [-1, 1) test matrix
    drawn from a counter-based SplitMix64 stream seeded by (level, box, side),
    q = 1 power iteration, each range basis orthonormalised twice, and the
    exact SVD of the projected k-row matrix.  Any consumer that uses the same
    option draws the same test matrix.
S   symmetric variant (optional; the paper notes that its algorithm is not
    specialised to symmetric matrices and that symmetry could be exploited):
    when A is symmetric and U = V at the leaves, the V-side matrix of every
    basis SVD equals the U-side one in exact arithmetic, so the V side takes
    the U side's singular vectors and values (V_hat = U_hat, t_j = r_j) and
    only one SVD per box is computed.

Parity: pinned by tests -- with tau = 0 the factorisation is an exact block
LU of E and the solve equals the dense solve of A_n to rounding; the
two-block example of Appendix C gives the printed closed-form matrix; the
solve error tracks eps.  The exact rank profile at tau > 0 has no printed
value to pin against (parity unpinned beyond self-consistency and the error
bound).  The linear growth of cost and memory in N (Sec. 2.5, Sec. 3.1) is
pinned on counted flops and stored bytes over trees of four to six levels
(the log-log slope between N and 4N with the leaf occupancy held fixed).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .h2 import H2


# ---------------------------------------------------------------------------
# sigma_0(E) (Sec. 2.4)
# ---------------------------------------------------------------------------
def sigma0_power(h2: H2, maxit: int = 100, rtol: float = 1e-6) -> tuple[float, int]:
    """Largest singular value of E by power iteration on E^T E.

    Start vector: all ones, normalised.  Stop when the estimate changes by
    <= rtol relative, or after maxit products.
    """
    _, n = h2.extended_layout()
    v = np.ones(n) / math.sqrt(n)
    prev = 0.0
    s = 0.0
    it = 0
    for it in range(1, maxit + 1):
        w = h2.extended_apply(h2.extended_apply(v), transpose=True)
        nw = float(np.linalg.norm(w))
        s = math.sqrt(nw)
        v = w / nw
        if it > 1 and abs(s - prev) <= rtol * s:
            break
        prev = s
    return s, it


def schur_complement(EPP: np.ndarray, EPC: np.ndarray, ERP: np.ndarray):
    """Block Gaussian elimination of the pivot set P (Sec. 2.1, Fig. graph_example).

    Returns G = E(P,P)^-1 E(P,C) and the update S = E(R,P) G, so that the
    eliminated system's block E(R,C) becomes E(R,C) - S.
    """
    G = np.linalg.solve(EPP, EPC) if EPP.shape[0] else np.zeros((0, EPC.shape[1]))
    return G, ERP @ G


def left_svd(M: np.ndarray):
    """Left singular vectors (a x a) and values (a,) of M (a x w); zero-padded if w < a."""
    a, w = M.shape
    if w < a:
        M = np.hstack([M, np.zeros((a, a - w))])
    W, s, _ = np.linalg.svd(M, full_matrices=False)
    return W, s


RSVD_OVERSAMPLE = 16   # oversampling p of the randomised SVD (reading R3b)
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """SplitMix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = x + np.uint64(0x9E3779B97F4A7C15)
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def rsvd_seed(level: int, box: int, side: int) -> np.uint64:
    v = (np.uint64(level) << np.uint64(40)) ^ (np.uint64(box) << np.uint64(2)) ^ np.uint64(side)
    return splitmix64(v)


def uniform_test_matrix(rows: int, cols: int, seed) -> np.ndarray:
    """Omega[i, c] = 2 u - 1, u = (splitmix64(seed + i + c rows) >> 11) 2^-53."""
    e = np.arange(rows * cols, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = splitmix64(np.uint64(seed) + e)
    u = (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return (2.0 * u - 1.0).reshape(cols, rows).T


def _orth_once(X: np.ndarray) -> np.ndarray:
    W, s = left_svd(X.T)
    inv = np.where((s > 1e-10 * s[0]) & (s > 0), 1.0 / np.where(s > 0, s, 1.0), 0.0) if s.size else s
    return X @ (W * inv[None, :])


def orth(X: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(X) from the SVD of X^T, applied twice (the
    second pass restores orthogonality lost in small-sigma directions);
    directions with sigma <= 1e-10 sigma_max are numerically null and dropped."""
    return _orth_once(_orth_once(X))


def rsvd_left(M: np.ndarray, k: int, seed) -> tuple[np.ndarray, np.ndarray]:
    """Randomised top-k left singular vectors and values of M (reading R3b)."""
    a, w = M.shape
    Om = uniform_test_matrix(w, k, seed)
    Q = orth(M @ Om)
    Qz = orth(M.T @ Q)
    Q = orth(M @ Qz)
    Wb, s = left_svd(Q.T @ M)
    return Q @ Wb, s


def count_rank(s: np.ndarray, tau: float, full: int) -> int:
    if tau <= 0.0:
        return full
    return int(np.count_nonzero(s > tau))


@dataclass
class Record:
    """One eliminated box: what the substitution phase needs (Algorithm 1)."""
    l: int
    i: int
    a: int
    r: int
    rows: list            # [(kind, box, dim)]
    cols: list
    EPP: np.ndarray
    ERP: np.ndarray
    G: np.ndarray         # E(P,P)^-1 E(P,C)


@dataclass
class LevelState:
    l: int
    a: list
    r: list = field(default_factory=list)
    X: dict = field(default_factory=dict)     # (i, j), j in N_i: xtilde/ybar near blocks
    Y: dict = field(default_factory=dict)     # (i, q), q in N_i u I_i: ybar-ybar / M2L blocks
    U: list = field(default_factory=list)
    V: list = field(default_factory=list)
    SU: list = field(default_factory=list)
    SV: list = field(default_factory=list)
    Upar: list = field(default_factory=list)
    Vpar: list = field(default_factory=list)
    elim: list = field(default_factory=list)


class Counters(dict):
    def add(self, key, v):
        self[key] = self.get(key, 0.0) + float(v)


class IFMM:
    """Plain IFMM factorisation of the H^2 matrix A_n defined by ``h2``."""

    def __init__(self, h2: H2, eps: float, tau: float | None = None, rank_cap: int | None = None,
                 sigma0: float | None = None, rsvd_rows: int | None = None,
                 symmetric: bool = False):
        self.h2 = h2
        self.rsvd_rows = rsvd_rows
        self.symmetric = symmetric
        self.tree = h2.tree
        self.eps = eps
        self.rank_cap = rank_cap
        self.records: list[Record] = []
        self.counters = Counters()
        self.rank_log: dict = {}       # (level, box) -> rank at elimination
        self.init_rank: dict = {}      # (level, box) -> rank after the initial weighted basis
        if self.tree.dense:
            self.sigma0, self.sigma0_iters = float("nan"), 0
            self.tau = 0.0
            self.dense_lu = sla.lu_factor(h2.dense_exact())
            return
        if sigma0 is None and tau is None:
            self.sigma0, self.sigma0_iters = sigma0_power(h2)
        else:
            self.sigma0, self.sigma0_iters = (sigma0 if sigma0 is not None else float("nan")), 0
        self.tau = eps * self.sigma0 if tau is None else float(tau)
        self._factor()

    # -- helpers ------------------------------------------------------------------
    def _cap(self, k):
        return k if self.rank_cap is None else min(k, self.rank_cap)

    def _init_basis(self, st: LevelState, Uraw, Vraw):
        """Weighted initial bases of level st.l (footnote to Eq. U_j_recomp, reading R6)."""
        l = st.l
        lev = self.tree.levels[l]
        h2 = self.h2
        QU, RU, QV, RV = [], [], [], []
        for i in range(lev.nb):
            q_, r_ = np.linalg.qr(Uraw[i])
            QU.append(q_)
            RU.append(r_)
            q_, r_ = np.linalg.qr(Vraw[i])
            QV.append(q_)
            RV.append(r_)
        rt, tt = [], []
        st.r, st.U, st.V, st.SU, st.SV = [], [], [], [], []
        for i in range(lev.nb):
            k = QU[i].shape[1]
            if lev.inter[i]:
                MU = RU[i] @ np.hstack([h2.m2l(l, i, q) @ RV[q].T for q in lev.inter[i]])
                MV = RV[i] @ np.hstack([h2.m2l(l, q, i).T @ RU[q].T for q in lev.inter[i]])
            else:
                MU = self.sigma0 * RU[i]
                MV = self.sigma0 * RV[i]
            WU, sU = left_svd(MU)
            # symmetric variant (reading S): the V side reuses the U side's SVD
            WV, sV = (WU, sU) if self.symmetric else left_svd(MV)
            r = min(max(count_rank(sU, self.tau, k), count_rank(sV, self.tau, k)), k)
            r = self._cap(r)
            st.r.append(r)
            st.U.append(QU[i] @ WU[:, :r])
            st.V.append(QV[i] @ WV[:, :r])
            st.SU.append(sU[:r].copy())
            st.SV.append(sV[:r].copy())
            rt.append(WU[:, :r].T @ RU[i])
            tt.append(WV[:, :r].T @ RV[i])
            self.init_rank[(l, i)] = r
            self.counters.add("init_flops", 2.0 * MU.shape[0] * MU.shape[1] * MU.shape[0] * 2)
        for i in range(lev.nb):
            for q in lev.inter[i]:
                st.Y[(i, q)] = rt[i] @ h2.m2l(l, i, q) @ tt[q].T
            for j in lev.nbrs[i]:
                st.Y[(i, j)] = np.zeros((st.r[i], st.r[j]))
        if l > 2:
            st.Upar = [rt[i] @ h2.T(l, i) for i in range(lev.nb)]
            st.Vpar = [tt[i] @ h2.T(l, i) for i in range(lev.nb)]
        st.elim = [False] * lev.nb

    def _dim(self, st, blk):
        kind, j = blk
        return st.a[j] if kind == "x" else st.r[j]

    # -- elimination of one box (Algorithm 2) -------------------------------------------
    def _eliminate_box(self, st: LevelState, i: int):
        lev = self.tree.levels[st.l]
        nbrs = lev.nbrs
        Ni = nbrs[i]
        blocks = []
        for j in Ni:
            if j == i:
                continue
            blocks.append(("y", j) if st.elim[j] else ("x", j))
        blocks.append(("y", i))
        a, r = st.a[i], st.r[i]
        p = a + r
        dims = [self._dim(st, b) for b in blocks]
        offs = np.concatenate([[0], np.cumsum(dims)]).astype(int)
        nC = int(offs[-1])
        EPP = np.zeros((p, p))
        EPP[:a, :a] = st.X[(i, i)]
        EPP[:a, a:] = st.U[i]
        EPP[a:, :a] = st.V[i].T
        EPC = np.zeros((p, nC))
        ERP = np.zeros((nC, p))
        for b, (kind, j) in enumerate(blocks):
            s = slice(offs[b], offs[b + 1])
            if (kind, j) == ("y", i):
                EPC[a:, s] = -np.eye(r)
                ERP[s, a:] = -np.eye(r)
            else:
                EPC[:a, s] = st.X[(i, j)]
                ERP[s, :a] = st.X[(j, i)]
        G, Sch = schur_complement(EPP, EPC, ERP)      # E(R,P) E(P,P)^-1 E(P,C)
        self.counters.add("lu_flops", 2.0 / 3.0 * p ** 3)
        self.counters.add("trsm_flops", 2.0 * p * p * nC)
        self.counters.add("schur_flops", 2.0 * nC * p * nC)
        self.counters.add("factor_bytes", 8.0 * (p * p + 2 * p * nC))
        rows = [(k, j, d) for (k, j), d in zip(blocks, dims)]
        self.records.append(Record(st.l, i, a, r, rows, rows, EPP, ERP, G))
        self.rank_log[(st.l, i)] = r
        # consumed blocks
        del st.X[(i, i)]
        for (kind, j) in blocks:
            if kind == "y" and j != i:
                del st.X[(i, j)]
                del st.X[(j, i)]
        fills = {}
        for bi, rb in enumerate(blocks):
            rs = slice(offs[bi], offs[bi + 1])
            for bj, cb in enumerate(blocks):
                cs = slice(offs[bj], offs[bj + 1])
                blk = -Sch[rs, cs]
                (rk, rj), (ck, cj) = rb, cb
                if rk == "y" and ck == "y":
                    st.Y[(rj, cj)] = st.Y[(rj, cj)] + blk
                elif rk == "x" and ck == "y" and cj == i:
                    st.X[(rj, i)] = blk                 # new edge E(xtilde_j, ybar_i)
                elif rk == "y" and rj == i and ck == "x":
                    st.X[(i, cj)] = blk                 # new edge E(ybar_i, xtilde_k)
                elif cj in nbrs[rj]:
                    st.X[(rj, cj)] = st.X[(rj, cj)] + blk
                else:
                    fills[(rb, cb)] = blk               # well-separated: compress
        st.elim[i] = True
        if fills:
            self._compress(st, fills)

    # -- compression and redirection (Eqs. P2P_kj - V_prime, Algorithm 3) ----------------
    def _compress(self, st: LevelState, fills: dict):
        lev = self.tree.levels[st.l]
        recomp = sorted({j for (rb, cb) in fills for (k, j) in (rb, cb) if k == "x"})
        by_row, by_col = {}, {}
        for (rb, cb), F in fills.items():
            by_row.setdefault(rb, []).append(F)
            by_col.setdefault(cb, []).append(F.T)
        new = {}
        for j in recomp:
            FU = by_row.get(("x", j), [])
            FV = by_col.get(("x", j), [])
            MU = np.hstack([st.U[j] * st.SU[j][None, :]] + FU)
            MV = np.hstack([st.V[j] * st.SV[j][None, :]] + FV)
            aj = st.a[j]
            rcap = self._cap(aj)
            if self.rsvd_rows is not None and self.tau > 0 and aj > self.rsvd_rows and rcap < aj:
                k = min(aj, rcap + RSVD_OVERSAMPLE)
                WU, sU = rsvd_left(MU, k, rsvd_seed(st.l, j, 0))
                WV, sV = (WU, sU) if self.symmetric else rsvd_left(MV, k, rsvd_seed(st.l, j, 1))
                full = k
            else:
                WU, sU = left_svd(MU)
                WV, sV = (WU, sU) if self.symmetric else left_svd(MV)
                full = aj
            rn = min(max(count_rank(sU, self.tau, full), count_rank(sV, self.tau, full)), full)
            rn = self._cap(rn)
            Un, Vn = WU[:, :rn], WV[:, :rn]
            new[j] = (Un, Vn, sU[:rn].copy(), sV[:rn].copy(), Un.T @ st.U[j], Vn.T @ st.V[j])
            self.counters.add("lowrank_flops", 4.0 * aj * aj * (MU.shape[1] + MV.shape[1]))
        for j in recomp:
            Un, Vn, sU, sV, rj, tj = new[j]
            for q in sorted(set(lev.nbrs[j]) | set(lev.inter[j])):
                if (j, q) in st.Y:
                    st.Y[(j, q)] = rj @ st.Y[(j, q)]
                if (q, j) in st.Y:
                    st.Y[(q, j)] = st.Y[(q, j)] @ tj.T
            if st.l > 2:
                st.Upar[j] = rj @ st.Upar[j]
                st.Vpar[j] = tj @ st.Vpar[j]
            st.U[j], st.V[j], st.SU[j], st.SV[j] = Un, Vn, sU, sV
            st.r[j] = Un.shape[1]
        for ((rk, rj), (ck, cj)), F in fills.items():
            if rk == "x" and ck == "x":
                st.Y[(rj, cj)] = st.Y[(rj, cj)] + st.U[rj].T @ F @ st.V[cj]
            elif rk == "x":
                st.Y[(rj, cj)] = st.Y[(rj, cj)] + st.U[rj].T @ F
            else:
                st.Y[(rj, cj)] = st.Y[(rj, cj)] + F @ st.V[cj]

    def _eliminate_level(self, st: LevelState):
        lev = self.tree.levels[st.l]
        order = sorted(range(lev.nb), key=lambda i: (int(lev.colour[i]), i))
        for i in order:
            self._eliminate_box(st, i)

    def _merge(self, st: LevelState) -> tuple[LevelState, list, list]:
        """Form level l-1 (Eqs. y_merge, U_merge, V_merge, K_merge)."""
        par = self.tree.levels[st.l - 1]
        a = [sum(st.r[c] for c in par.children[p]) for p in range(par.nb)]
        nst = LevelState(st.l - 1, a)
        for p in range(par.nb):
            for q in par.nbrs[p]:
                nst.X[(p, q)] = np.block([[st.Y[(c, d)] for d in par.children[q]]
                                          for c in par.children[p]]) if a[p] and a[q] else \
                    np.zeros((a[p], a[q]))
        Uraw = [np.vstack([st.Upar[c] for c in par.children[p]]) for p in range(par.nb)]
        Vraw = [np.vstack([st.Vpar[c] for c in par.children[p]]) for p in range(par.nb)]
        return nst, Uraw, Vraw

    def _factor(self):
        t = self.tree
        L = t.L
        leaf = t.levels[L]
        st = LevelState(L, [int(leaf.pt_end[i] - leaf.pt_begin[i]) for i in range(leaf.nb)])
        for i in range(leaf.nb):
            for j in leaf.nbrs[i]:
                st.X[(i, j)] = self.h2.p2p(i, j)
        Uraw, Vraw = self.h2.leafU, self.h2.leafU
        self.level_r = {}
        self.level_a = {}
        for l in range(L, 1, -1):
            self._init_basis(st, Uraw, Vraw)
            self._eliminate_level(st)
            self.level_r[l] = list(st.r)
            self.level_a[l] = list(st.a)
            if l > 2:
                st, Uraw, Vraw = self._merge(st)
        lev2 = t.levels[2]
        self.top_r = list(st.r)
        T = np.block([[st.Y[(i, j)] for j in range(lev2.nb)] for i in range(lev2.nb)])
        self.top = T
        self.top_lu = sla.lu_factor(T) if T.size else None
        self.counters.add("top_flops", 2.0 / 3.0 * T.shape[0] ** 3)

    # -- substitution (the top solve and downward pass of Algorithm 1) ----------------------
    def solve(self, b: np.ndarray) -> np.ndarray:
        """x ~= A_n^-1 b, b and x in user order; b is (N,) or (N, k)."""
        b = np.asarray(b, dtype=np.float64)
        vec = b.ndim == 1
        B = b.reshape(b.shape[0], -1)
        t = self.tree
        if t.dense:
            X = sla.lu_solve(self.dense_lu, B)
            return X[:, 0] if vec else X
        k = B.shape[1]
        L = t.L
        leaf = t.levels[L]
        Bt = B[t.perm]
        xt = {L: [Bt[leaf.pt_begin[i]:leaf.pt_end[i]].copy() for i in range(leaf.nb)]}
        yb = {}
        W = []
        cur = L
        yb[L] = {}
        for rec in self.records:
            if rec.l != cur:                    # level finished: merge RHS (Eq. y_merge)
                par = t.levels[cur - 1]
                xt[cur - 1] = [np.vstack([yb[cur][c] for c in par.children[p]]) if par.children[p]
                               else np.zeros((0, k)) for p in range(par.nb)]
                cur = rec.l
                yb[cur] = {}
            i = rec.i
            bP = np.vstack([xt[cur][i], np.zeros((rec.r, k))])
            w = np.linalg.solve(rec.EPP, bP) if bP.shape[0] else bP
            W.append(w)
            yb[cur][i] = np.zeros((rec.r, k))
            off = 0
            for (kind, j, d) in rec.rows:
                upd = rec.ERP[off:off + d] @ w
                if kind == "x":
                    xt[cur][j] = xt[cur][j] - upd
                else:
                    yb[cur][j] = yb[cur][j] - upd
                off += d
        lev2 = t.levels[2]
        rhs = np.vstack([yb[2][i] for i in range(lev2.nb)])
        sol = sla.lu_solve(self.top_lu, rhs) if rhs.shape[0] else rhs
        ys = {2: {}}
        off = 0
        for i in range(lev2.nb):
            ys[2][i] = sol[off:off + self.top_r[i]]
            off += self.top_r[i]
        xs = {}
        cur = 2
        xs[2] = {}
        for rec, w in zip(reversed(self.records), reversed(W)):
            if rec.l != cur:                    # split parent unknowns into child multipoles
                par = t.levels[cur]
                ys[rec.l] = {}
                for p in range(par.nb):
                    off = 0
                    for c in par.children[p]:
                        rc = self.level_r[rec.l][c]
                        ys[rec.l][c] = xs[cur][p][off:off + rc]
                        off += rc
                cur = rec.l
                xs[cur] = {}
            xC = np.vstack([xs[cur][j] if kind == "x" else ys[cur][j] for (kind, j, d) in rec.cols]) \
                if rec.cols else np.zeros((0, k))
            xP = w - rec.G @ xC
            xs[cur][rec.i] = xP[:rec.a]
        Xt = np.vstack([xs[L][i] for i in range(leaf.nb)])
        X = np.empty_like(Xt)
        X[t.perm] = Xt
        return X[:, 0] if vec else X

    # -- reporting ------------------------------------------------------------------------
    def stored_bytes(self) -> float:
        return self.counters.get("factor_bytes", 0.0)

    def ranks(self, l: int) -> list:
        return [self.rank_log[(l, i)] for i in range(self.tree.levels[l].nb)]
