"""Helpers shared by the GPU parity tests."""
import numpy as np
import torch

import paper_1508_01835_gb300 as ifmm
from oracle.h2 import H2
from oracle.ifmm import IFMM


def opts(w, eps=None, tau=0.0, rank_cap=0, fmm_n=0, schur=0, rsvd_rows=0, symmetric=0):
    return ifmm.make_options(dim=w.dim, cheb_n=w.cheb_n, leaf_max=w.leaf_max,
                             eps=w.eps if eps is None else eps, schur=schur, tau_override=tau,
                             rank_cap=rank_cap, fmm_n=fmm_n, rsvd_rows=rsvd_rows,
                             symmetric=symmetric)


def kernel(w):
    return ifmm.Kernel(w.kernel.kind, w.kernel.param, w.kernel.diag)


def oracle_h2(w, n=None):
    return H2(w.points, w.kernel.kind, w.kernel.param, w.kernel.diag, n or w.cheb_n, w.leaf_max)


def to_user(h2, v_tree):
    out = np.empty_like(v_tree)
    out[h2.tree.perm] = v_tree
    return out


def dense_an_solve(h2, b):
    A = h2.dense_blockwise()
    p = h2.tree.perm
    xt = np.linalg.solve(A, b[p])
    return to_user(h2, xt), np.linalg.cond(A)


def cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
