"""Host-side logic of the serving loop, no GPU: the Poisson request stream, slab sizing by free
device memory (through the library's host-only footprint arithmetic) and the latency summary."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import build_lib


@pytest.fixture(scope="module")
def serving():
    build_lib.build()
    from paper_1810_12707_gb300 import serving as s
    return s


def test_request_stream_is_seeded_and_has_the_stated_mix(serving):
    a = serving.make_requests(20000, rate=50.0, seed=5)
    b = serving.make_requests(20000, rate=50.0, seed=5)
    assert a == b
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) > 0)
    # exponential gaps of mean 1/rate: the sample mean is within 5 standard errors
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) <= 5 * (1 / 50.0) / np.sqrt(len(gaps))
    ns = np.array([r.n for r in a])
    for n, w in zip(serving.SIZES, serving.WEIGHTS):
        p = np.mean(ns == n)
        assert abs(p - w) <= 5 * np.sqrt(w * (1 - w) / len(a)), n
    assert {r.ic for r in a} == {"abc", "ot"}
    assert all(1e-3 <= r.nu <= 1e-2 and 1e-3 <= r.eta <= 1e-2 and 0.05 <= r.mach <= 0.5 for r in a)
    assert all(100 <= r.nsteps <= 1000 for r in a)
    assert min(r.nsteps for r in a) == 100 and max(r.nsteps for r in a) == 1000
    assert a[0].work == float(a[0].n) ** 3 * a[0].nsteps


@pytest.mark.parametrize("free_gb", [0.001, 2, 40, 250])
def test_slab_capacity_fits_the_free_memory(serving, free_gb):
    """A new slab takes as many slots as fit in the memory free at that moment (the library's
    host-only footprint arithmetic), up to the per-size cap; none when one slot does not fit."""
    from paper_1810_12707_gb300 import mhd
    free = free_gb * 1e9
    for n in serving.SIZES:
        for prec in (mhd.MHD_FP32_MIXED, mhd.MHD_FP64, mhd.MHD_FP64_DF):
            c = serving.slab_capacity(n, prec, free)
            cap = serving.SLAB_CAP[n]
            assert 0 <= c <= cap
            if c > 0:
                assert mhd.mhd_footprint_bytes(n, prec, c) <= free
            if c < cap:
                assert mhd.mhd_footprint_bytes(n, prec, c + 1) > free
    assert serving.slab_capacity(256, mhd.MHD_FP32_MIXED, 1e6) == 0
    assert serving.slab_capacity(32, mhd.MHD_FP32_MIXED, 1e12) == serving.SLAB_CAP[32]
    assert serving.slab_capacity(32, mhd.MHD_FP32_MIXED, 1e12, cap=3) == 3


def test_latency_summary(serving):
    st = serving.ServeStats(completed=3, work=6.0e9, wall=2.0, step_latency_ms=list(range(1, 101)),
                            run_latency_s=[1.0, 2.0, 3.0], queue_s=[0.0, 0.0, 1.0])
    s = st.summary()
    assert s["throughput"] == 3.0e9
    assert s["step_latency_ms_p50"] == pytest.approx(50.5)
    assert s["step_latency_ms_p99"] == pytest.approx(99.01)
    assert s["run_latency_s_p50"] == 2.0
    empty = serving.ServeStats().summary()
    assert empty["throughput"] == 0.0 and empty["step_latency_ms_p50"] is None
    st.by_size = {32: {"step_ms": [1.0, 3.0], "run_s": [2.0]}, 256: {"step_ms": [9.0], "run_s": [4.0, 6.0]}}
    per = st.summary()["per_size"]
    assert per["32"]["step_latency_ms_p50"] == 2.0 and per["256"]["run_latency_s_p50"] == 5.0
    assert per["256"]["runs"] == 2
