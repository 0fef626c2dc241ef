"""Many systems on one GPU: batched factorisation and the GMRES server.

* ifmm_factor_batch factorises several independent systems concurrently; each
  factorisation must be the one ifmm_factor gives for that system alone (the
  kernels are deterministic, so the solves agree to rounding-free equality up
  to a tiny slack).
* The server batches queued requests of one system into one block of
  right-hand sides; every result must be the same alone and in a mix of
  systems and widths, within what the 1e-10 residual allows, and every
  residual must reach 1e-10.
* Admission: a system whose device memory exceeds the budget is refused.
"""
import numpy as np
import pytest
import torch

import paper_1508_01835_gb300 as ifmm
from tests.gpu_util import cuda, kernel, opts, rel
from workloads import small_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1508_01835_gb300 import build
    build.build()
    c = ifmm.ifmm_ctx_create(0)
    yield c
    ifmm.ifmm_ctx_destroy(c)


def workloads_mix():
    return [small_cube(2600, 11, cheb_n=3, leaf_max=32, eps=1e-6),
            small_cube(1500, 12, cheb_n=3, leaf_max=24, eps=1e-6),
            small_cube(4100, 13, cheb_n=3, leaf_max=40, eps=1e-7),
            small_cube(900, 14, cheb_n=2, leaf_max=16, eps=1e-5)]


@pytest.fixture(scope="module")
def systems(ctx):
    ws = workloads_mix()
    sys = [ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w)) for w in ws]
    yield ws, sys
    for s in sys:
        ifmm.ifmm_system_destroy(s)


def test_factor_batch_matches_one_at_a_time(ctx, systems):
    ws, sys = systems
    facs = ifmm.ifmm_factor_batch(ctx, sys)
    try:
        for w, s, f in zip(ws, sys, facs):
            single = ifmm.ifmm_factor(ctx, s)
            try:
                b = cuda(w.rhs(2).T)
                x1, x2 = torch.empty_like(b), torch.empty_like(b)
                ifmm.ifmm_solve(ctx, f, b, x1, w.N)
                ifmm.ifmm_solve(ctx, single, b, x2, w.N)
                torch.cuda.synchronize()
                assert rel(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-14
                ia, ib = ifmm.ifmm_factor_get_info(f), ifmm.ifmm_factor_get_info(single)
                assert ia.top_size == ib.top_size
                for l in range(2, ia.levels + 1):
                    assert list(ifmm.ifmm_factor_get_ranks(f, l)) == \
                        list(ifmm.ifmm_factor_get_ranks(single, l))
            finally:
                ifmm.ifmm_factor_destroy(single)
    finally:
        for f in facs:
            ifmm.ifmm_factor_destroy(f)


@pytest.mark.parametrize("mv", [ifmm.P_FP64, ifmm.P_FP32])
def test_server_results_same_alone_and_in_mix(ctx, systems, mv):
    """mv: the served GMRES's products in FP64, or iterative refinement with
    the FP32 far field (set before registration; refused afterwards)."""
    ws, sys = systems
    facs = ifmm.ifmm_factor_batch(ctx, sys)
    srv = ifmm.ifmm_server_create(ctx, 64 << 30, workers=3)
    try:
        ifmm.ifmm_server_set_matvec_precision(srv, mv)
        ids = [ifmm.ifmm_server_register(srv, s, f, maxit=100) for s, f in zip(sys, facs)]
        with pytest.raises(ifmm.ServerError):
            ifmm.ifmm_server_set_matvec_precision(srv, mv)
        rng = np.random.default_rng(77)
        reqs = []  # (system index, b)
        for k in range(14):
            i = int(rng.integers(len(ws)))
            nrhs = int(rng.integers(1, 9))
            reqs.append((i, np.ascontiguousarray(rng.standard_normal((nrhs, ws[i].N)))))
        # alone: one request at a time
        alone = []
        for i, b in reqs:
            x = np.zeros_like(b)
            t = ifmm.ifmm_server_submit(srv, ids[i], b, x, 1e-10, 100)
            st, reps, lat = ifmm.ifmm_server_wait(srv, t, b.shape[0])
            assert st == 0 and all(r.true_rel_residual <= 1e-10 for r in reps)
            alone.append(x)
        _, nb_alone, _, _ = ifmm.ifmm_server_stats(srv)
        # in a mix: everything queued at once, waited for in reverse order
        xs = [np.zeros_like(b) for _, b in reqs]
        tickets = [ifmm.ifmm_server_submit(srv, ids[i], b, x, 1e-10, 100)
                   for (i, b), x in zip(reqs, xs)]
        lats = []
        for (i, b), t in reversed(list(zip(reqs, tickets))):
            st, reps, lat = ifmm.ifmm_server_wait(srv, t, b.shape[0])
            assert st == 0 and all(r.true_rel_residual <= 1e-10 for r in reps)
            lats.append(lat)
        used, nb, cols, shed = ifmm.ifmm_server_stats(srv)
        assert nb - nb_alone < len(reqs), "the mix was not batched"
        for x_mix, x_one in zip(xs, alone):
            assert rel(x_mix, x_one) <= 1e-8
        assert used > 0 and shed == 0 and cols == 2 * sum(b.shape[0] for _, b in reqs)
        print(f"mix: {len(reqs)} requests in {nb - nb_alone} blocks, latency max {max(lats):.3f}s")
    finally:
        ifmm.ifmm_server_destroy(srv)
        for f in facs:
            ifmm.ifmm_factor_destroy(f)


def test_server_admission_refuses_over_budget(ctx, systems):
    ws, sys = systems
    fac = ifmm.ifmm_factor(ctx, sys[1])
    srv = ifmm.ifmm_server_create(ctx, 1 << 20, workers=1)
    try:
        with pytest.raises(ifmm.ServerError) as e:
            ifmm.ifmm_server_register(srv, sys[1], fac, maxit=100)
        assert e.value.status == 7 and "budget" in str(e.value)
        assert ifmm.ifmm_server_stats(srv)[0] == 0
    finally:
        ifmm.ifmm_server_destroy(srv)
        ifmm.ifmm_factor_destroy(fac)
