"""Host logic of bench.py (no GPU): the roofline rows built from the library's
launch profile, each kernel placed against the pipe it fills most."""
import pytest

import bench

PEAKS = {"hbm_gbs": 6685.5, "bf16_tflops": 1944.2, "fp64_tflops": 1.2, "fp32_tflops": 70.0}


def test_rooflines_bound_by_the_fullest_pipe_dominant_and_weighted():
    stats = {  # name: (launches, seconds, flops, bytes)
        "k_svd_left": (452, 10.0, 1.4e12, 0.0),
        "k_gemm_tc_3xtf32": (162, 0.8, 4.74e12, 0.0),
        "k_spmm_job": (40, 0.6, 1e9, 3.0e12),          # bytes-heavy: HBM
        "k_spmm_f32": (40, 0.5, 2.0e13, 1.0e12),       # 40 TFLOP/s FP32 vs 2 TB/s: FP32 ALU
        "k_gemm_fp64": (2812, 3.2, 1.6e12, 0.0),
        "(all launches)": (42822, 0.0, 0.0, 0.0),
        "graph:ifmm_solve": (20, 0.5, 1e9, 1e9),
    }
    rows, dom, weighted = bench.kernel_rooflines(stats, 21.0, PEAKS)
    assert set(rows) == {"k_svd_left", "k_gemm_tc_3xtf32", "k_spmm_job", "k_spmm_f32",
                         "k_gemm_fp64"}
    assert dom["kernel"] == "k_svd_left" and dom["bound"] == "alu"
    assert dom["achieved"] == pytest.approx(0.14) and dom["frac"] == pytest.approx(0.14 / 1.2)
    assert dom["share"] == pytest.approx(10.0 / 21.0)
    tc = rows["k_gemm_tc_3xtf32"]
    assert tc["bound"] == "tensor" and tc["peak"] == pytest.approx(1944.2 * 1.1 / 2.25)
    assert tc["achieved"] == pytest.approx(4.74e12 / 0.8 / 1e12)
    sp = rows["k_spmm_job"]
    assert sp["bound"] == "hbm" and sp["achieved"] == pytest.approx(5000.0)
    assert sp["frac"] == pytest.approx(5000.0 / 6685.5)
    f32 = rows["k_spmm_f32"]
    assert f32["bound"] == "alu" and f32["peak"] == 70.0 and f32["achieved"] == pytest.approx(40.0)
    fr = [(r["s"], r["frac"]) for r in rows.values()]
    assert weighted == pytest.approx(sum(t * f for t, f in fr) / sum(t for t, _ in fr))


def test_rooflines_empty_profile():
    rows, dom, weighted = bench.kernel_rooflines({"(all launches)": (0, 0.0, 0.0, 0.0)}, 1.0,
                                                 PEAKS)
    assert rows == {} and dom is None and weighted is None


def test_percentiles_and_rates():
    assert bench._pct([3.0, 1.0, 2.0], 50) == 2.0
    assert bench._pct(list(range(1, 101)), 99) == 99
    assert bench.whole_job_rate(10, 2, 2000.0) == pytest.approx(10.0)


class _FakeTorch:
    float64 = "f64"

    @staticmethod
    def empty(shape, dtype=None, device=None):
        import numpy as np
        return np.zeros(shape)


class _FakeServer:
    """Accepts requests while a system has fewer than 32 queued columns; a
    worker takes up to 32 queued columns at a time, and a block completes on
    a later poll -- the bounds the output ring relies on."""

    class ServerError(Exception):
        pass

    def __init__(self):
        self.queued, self.running, self.live, self.next = {}, {}, {}, 1

    def ifmm_server_submit_device(self, srv, sid, b, x, N, tol, maxit):
        q = self.queued.setdefault(sid, [])
        if sum(k for k, _, _ in q) + b.shape[0] > 32:
            raise self.ServerError()
        t = self.next
        self.next += 1
        q.append((b.shape[0], t, x))
        return t

    def step(self):
        for sid, q in self.queued.items():
            if self.running.get(sid):
                for _, t, _ in self.running[sid]:
                    self.live.pop(t, None)
                self.running[sid] = []
            blk, cols = [], 0
            while q and cols + q[0][0] <= 32:
                k, t, x = q.pop(0)
                blk.append((k, t, x))
                cols += k
            self.running[sid] = blk


def test_output_ring_never_hands_live_columns_to_a_new_request():
    """bench.Load's per-system output ring: every request's columns are free
    of every request not yet completed (queued or running)."""
    import numpy as np
    srv = _FakeServer()
    ifmm_ns = type("I", (), {"ServerError": _FakeServer.ServerError,
                             "ifmm_server_submit_device": srv.ifmm_server_submit_device})
    N = [5] * bench.N_SYSTEMS
    pools = {i: np.zeros((32, 5)) for i in range(bench.N_SYSTEMS)}
    load = bench.Load(ifmm_ns, None, [0] * bench.N_SYSTEMS, pools, np.random.default_rng(3), True,
                      _FakeTorch, N)
    for i in range(bench.N_SYSTEMS):
        load.ring[i] = np.zeros((bench.RING_COLS, 5))
    for step in range(4000):
        load._submit(0.0)
        if step % 7 == 0:
            srv.step()
        for i in range(bench.N_SYSTEMS):   # live = queued + running requests of system i
            live = [x for _, _, x in srv.queued.get(i, [])] + \
                   [x for _, _, x in srv.running.get(i, [])]
            spans = sorted((x.__array_interface__["data"][0],
                            x.__array_interface__["data"][0] + x.nbytes) for x in live)
            for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
                assert a1 <= b0, "two outstanding requests share output columns"
    assert load.shed > 0 and load.offered == 4000
