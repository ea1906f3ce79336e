"""Host-side logic of the serving loop, no GPU: the Poisson request stream, slot planning by free
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


@pytest.mark.parametrize("free_gb", [2, 40, 250])
def test_slot_plan_fits_memory_and_follows_the_mix(serving, free_gb):
    from paper_1810_12707_gb300 import mhd
    free = free_gb * 1e9
    slots = serving.plan_slots(free)
    used = sum(mhd.mhd_footprint_bytes(n, mhd.MHD_FP32_MIXED, s) for n, s in slots.items())
    assert all(s >= 1 for s in slots.values())
    assert all(s <= 64 for s in slots.values())
    ones = sum(mhd.mhd_footprint_bytes(n, mhd.MHD_FP32_MIXED, 1) for n in slots)
    assert used <= max(0.8 * free, ones)
    # no size can take one more slot without leaving the budget, unless it is at the cap or
    # already at or above its share
    total = sum(slots.values())
    for n, w in zip(serving.SIZES, serving.WEIGHTS):
        extra = mhd.mhd_footprint_bytes(n, mhd.MHD_FP32_MIXED, slots[n] + 1) - \
            mhd.mhd_footprint_bytes(n, mhd.MHD_FP32_MIXED, slots[n])
        if slots[n] < 64 and slots[n] < w * total:
            assert used + extra > 0.8 * free, (n, slots)
    assert slots[32] >= slots[64] >= slots[128] >= slots[256]


def test_slot_plan_is_proportional_when_memory_allows(serving):
    """With memory for every size's cap, each size gets the cap; below it, the slot counts follow
    the weights 0.4 : 0.3 : 0.2 : 0.1 to within one slot of the largest-remainder split."""
    big = serving.plan_slots(10e12)
    assert big == {n: 64 for n in serving.SIZES}
    small = serving.plan_slots(10e12, max_slots=10 ** 6, sizes=(32, 64), weights=(0.75, 0.25), fraction=1e-3)
    total = sum(small.values())
    assert abs(small[32] - 0.75 * total) <= 1 and abs(small[64] - 0.25 * total) <= 1


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
