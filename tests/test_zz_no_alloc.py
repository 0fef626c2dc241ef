"""The allocation-free FMM product (fmm_matvec_static).

Some callers cannot allocate device memory while they run -- a host
application that owns a fixed device pool and forbids cudaMalloc, or a
real-time loop that must not stall on the allocator.  fmm_matvec_static serves them from a library-owned static
device buffer.  Here it must give the same y = A_n x as fmm_matvec on two
calls in a row (the buffer keeps the previous call's contents), for a
two-level and a deeper tree, leave the device's free memory unchanged while
it runs, and reject a request larger than its buffer.
This file is collected last so that a stop at its first failure has already
run every other test.
"""
import numpy as np
import pytest
import torch

import paper_1508_01835_gb300 as ifmm
from tests.gpu_util import cuda, kernel, opts, rel
from workloads import Kernel, K_GAUSSIAN, cube_2k, small_cube

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1508_01835_gb300 import build
    build.build()
    c = ifmm.ifmm_ctx_create(0)
    yield c
    ifmm.ifmm_ctx_destroy(c)


@pytest.mark.parametrize("make", [
    lambda: cube_2k(),
    lambda: small_cube(3000, 7, cheb_n=3, leaf_max=32, eps=1e-6),
    lambda: small_cube(2500, 9, cheb_n=4, leaf_max=20, eps=1e-8, dim=2,
                       kernel=Kernel(K_GAUSSIAN, 0.05, 1.01)),
])
def test_static_matvec_matches_fmm_matvec_twice(ctx, make):
    w = make()
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w))
    try:
        rng = np.random.default_rng(11)
        # The first call on a device loads the library's module that holds the
        # static array (CUDA loads modules at first use), which is when the
        # array's 64 MiB are taken; from then on no call changes free memory.
        X0 = cuda(rng.standard_normal((2, w.N)))
        ifmm.fmm_matvec_static(ctx, sys, X0, torch.empty_like(X0), w.N)
        for call in range(2):
            X = cuda(rng.standard_normal((2, w.N)))
            ref = torch.empty_like(X)
            out = torch.full_like(X, np.nan)
            ifmm.fmm_matvec(ctx, sys, ifmm.MV_FMM, X, ref, w.N)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]   # cudaMemGetInfo: free device bytes
            ifmm.fmm_matvec_static(ctx, sys, X, out, w.N)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0, f"call {call} allocated device memory"
            assert rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-13, f"call {call}"
    finally:
        ifmm.ifmm_system_destroy(sys)


def test_static_matvec_rejects_oversized_requests(ctx):
    w = small_cube(3000, 7, cheb_n=3, leaf_max=32, eps=1e-6)
    sys = ifmm.ifmm_system_create(ctx, cuda(w.points), kernel(w), opts(w))
    try:
        X = torch.zeros(2000, w.N, dtype=torch.float64, device="cuda:0")
        Y = torch.empty_like(X)
        with pytest.raises(ifmm.IFMMError) as e:
            ifmm.fmm_matvec_static(ctx, sys, X, Y, w.N)
        assert e.value.status == 1 and "bytes" in str(e.value)
    finally:
        ifmm.ifmm_system_destroy(sys)
