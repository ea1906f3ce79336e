"""Serving pools and the continuous-batching loop: slot bookkeeping through the C ABI, step
budgets, compaction on retire, and the alone-versus-mix property (bitwise)."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


@pytest.mark.parametrize("precision", [0, 1])
def test_pool_budgets_compaction_and_alone_vs_mix(lib, precision):
    n = 32
    runs = [(inputs.orszag_tang(n, seed=s, mach=m, nu=nu, eta=eta), steps)
            for s, m, nu, eta, steps in ((1, 0.1, 1e-2, 2e-3, 7), (2, 0.3, 3e-3, 8e-3, 23), (3, 0.2, 5e-3, 5e-3, 15),
                                         (4, 0.4, 2e-3, 9e-3, 30), (5, 0.1, 8e-3, 1e-3, 12))]
    pool = lib.mhd_pool_create(n, 3, precision=precision)
    live, results, queue = {}, {}, list(range(len(runs)))
    while queue or live:
        while queue and len(live) < 3:
            i = queue.pop(0)
            ic, steps = runs[i]
            slot = lib.mhd_pool_admit(pool, (ic.nu, ic.eta, ic.cs), ic.rho, ic.u, ic.b, steps)
            assert slot is not None
            live[slot] = i
        if len(live) == 3:  # every slot busy: admission is refused, nothing changes
            ic0 = runs[0][0]
            assert lib.mhd_pool_admit(pool, (ic0.nu, ic0.eta, ic0.cs), ic0.rho, ic0.u, ic0.b, 5) is None
        lib.mhd_pool_step(pool, 4)
        steps, status, fin = lib.mhd_pool_progress(pool)
        for slot in list(live):
            i = live[slot]
            assert steps[slot] <= runs[i][1]
            if fin[slot]:
                assert steps[slot] == runs[i][1] and status[slot] == 0
                results[i] = lib.mhd_pool_retire(pool, slot)
                del live[slot]
    assert lib.mhd_pool_info(pool) == (0, 3)
    for i, (ic, steps) in enumerate(runs):
        ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs)], precision=precision)
        lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
        lib.mhd_step(ctx, steps)
        for g, e in zip(results[i], lib.mhd_get_state(ctx, 0)):
            assert np.array_equal(g, e)


def test_serving_loop_small(lib):
    from paper_1810_12707_gb300 import serving
    reqs = serving.make_requests(12, rate=200.0, seed=5, sizes=(16, 32), weights=(0.5, 0.5), steps=(20, 60))
    srv = serving.Server(k=5, slab_cap={16: 3, 32: 2})
    keep = [r.rid for r in reqs[:4]]
    stats = srv.run(reqs, keep_outputs=keep)
    srv.close()
    s = stats.summary()
    assert s["completed"] == len(reqs)
    assert s["step_latency_ms_p99"] >= s["step_latency_ms_p50"] > 0
    assert s["run_latency_s_p99"] >= s["run_latency_s_p50"] > 0
    for rid in keep:
        alone = serving.run_alone(reqs[rid])
        for g, e in zip(stats.outputs[rid], alone):
            assert np.array_equal(g, e)


def test_largest_run_is_admitted_once_smaller_runs_free_the_memory(lib):
    """No slot is set aside for the largest grid: with a memory budget that holds either the
    slab of small runs or one large run but not both, the large request (arriving while the small
    runs are on the device) waits, is admitted once the small runs have retired and their slab
    has been destroyed, and completes; later small requests do not overtake it."""
    from paper_1810_12707_gb300 import serving
    prec = lib.MHD_FP32_MIXED
    small, big = 16, 64
    cap = 4
    limit = lib.mhd_footprint_bytes(big, prec, 1) + 0.5 * lib.mhd_footprint_bytes(small, prec, cap)
    assert lib.mhd_footprint_bytes(small, prec, cap) + lib.mhd_footprint_bytes(big, prec, 1) > limit
    mk = lambda rid, t, n, steps: serving.Request(rid, t, n, "ot", rid % serving.IC_SEEDS, 5e-3, 5e-3, 0.2, steps)
    reqs = [mk(i, 0.0, small, 30) for i in range(4)] + [mk(4, 0.001, big, 20)] + \
           [mk(5 + i, 0.002, small, 10) for i in range(3)]
    srv = serving.Server(precision=prec, k=5, memory_limit=limit, slab_cap={small: cap, big: 1})
    stats = srv.run(reqs, keep_outputs=[4])
    srv.close()
    assert stats.completed == len(reqs)
    assert stats.peak_bytes <= limit
    first_small_done = max(stats.retired_at[i] for i in range(4))
    assert stats.admitted_at[4] >= first_small_done
    assert all(stats.admitted_at[5 + i] >= stats.admitted_at[4] for i in range(3))
    alone = serving.run_alone(reqs[4], precision=prec)
    for g, e in zip(stats.outputs[4], alone):
        assert np.array_equal(g, e)
    per = stats.summary()["per_size"]
    assert set(per) == {str(small), str(big)} and per[str(big)]["runs"] == 1
