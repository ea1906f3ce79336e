"""mhd_get_state_async: the transfer of a state into host buffers queued on a stream of its own.
Once mhd_synchronize returns the buffers hold exactly what mhd_get_state returns, in every
precision, also when the context has queued more work meanwhile (a set_state of another instance,
steps) and when several transfers are in flight at once; mhd_destroy waits for transfers still in
flight."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


def _bufs(n, pinned=False):
    if pinned:
        import torch
        return [torch.empty(s, dtype=torch.float64, pin_memory=True).numpy() for s in ((n, n, n), (3, n, n, n),
                                                                                        (3, n, n, n))]
    return [np.full((n, n, n), np.nan), np.full((3, n, n, n), np.nan), np.full((3, n, n, n), np.nan)]


def _ctx(lib, n, ics, precision):
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs) for ic in ics], precision=precision)
    for i, ic in enumerate(ics):
        lib.mhd_set_state(ctx, i, ic.rho, ic.u, ic.b)
    return ctx


def _ics(n, count, seed):
    nu, eta, mach = inputs.ensemble_params(count, seed=seed)
    return [inputs.orszag_tang(n, seed=seed + i, mach=float(mach[i]), nu=float(nu[i]), eta=float(eta[i]))
            for i in range(count)]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("n", [32, 128])
def test_async_get_equals_get(lib, precision, n):
    ics = _ics(n, 2, seed=70)
    ctx = _ctx(lib, n, ics, precision)
    lib.mhd_step(ctx, 3)
    out = _bufs(n, pinned=(n == 128))
    lib.mhd_get_state_async(ctx, 1, *out)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    ref = lib.mhd_get_state(ctx, 1)
    for a, r in zip(out, ref):
        assert np.array_equal(a, r)
    lib.mhd_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_async_get_overlapping_later_work(lib, precision):
    """get(0) in flight while instance 1 is replaced and both step, then get(1), get(0) again:
    each buffer holds the state at the moment its transfer was queued."""
    n = 64
    ics = _ics(n, 2, seed=80)
    other = _ics(n, 1, seed=90)[0]

    def run(use_async):
        ctx = _ctx(lib, n, ics, precision)
        lib.mhd_step(ctx, 2)
        outs = [_bufs(n, pinned=True) for _ in range(3)]
        get = (lambda i, o: lib.mhd_get_state_async(ctx, i, *o)) if use_async else \
            (lambda i, o: [np.copyto(d, s) for d, s in zip(o, lib.mhd_get_state(ctx, i))])
        get(0, outs[0])
        lib.mhd_set_state(ctx, 1, other.rho, other.u, other.b)
        lib.mhd_step(ctx, 2)
        get(1, outs[1])
        get(0, outs[2])
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        lib.mhd_destroy(ctx)
        return [a.copy() for o in outs for a in o]

    for a, b in zip(run(True), run(False)):
        assert np.array_equal(a, b)


def test_destroy_waits_for_async_get(lib):
    n = 64
    ics = _ics(n, 1, seed=95)
    ctx = _ctx(lib, n, ics, lib.MHD_FP64_DF)
    lib.mhd_step(ctx, 2)
    ref = lib.mhd_get_state(ctx, 0)
    out = _bufs(n, pinned=True)
    lib.mhd_get_state_async(ctx, 0, *out)
    lib.mhd_destroy(ctx)  # no synchronize: destroy waits for the copies into `out`
    for a, r in zip(out, ref):
        assert np.array_equal(a, r)


def test_async_get_checks_its_arguments(lib):
    ctx = lib.mhd_init(16, [(0.01, 0.01, 1.0)])
    good = _bufs(16)
    with pytest.raises(lib.MhdError) as err:
        lib.mhd_get_state_async(ctx, 1, *good)
    assert err.value.status == lib.MHD_EINVAL
    with pytest.raises(ValueError):
        lib.mhd_get_state_async(ctx, 0, np.zeros((16, 16, 15)), good[1], good[2])
    lib.mhd_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_host_set_waits_for_queued_steps(lib, precision):
    """A host set_state's copies into its staging slots in W1 wait for the steps queued before it
    (which use all of W1), though not for a transfer out queued after them."""
    n = 64
    ics = _ics(n, 2, seed=100)
    other = _ics(n, 1, seed=110)[0]

    def run(sync_between):
        ctx = _ctx(lib, n, ics, precision)
        lib.mhd_step(ctx, 3)
        out = _bufs(n, pinned=True)
        lib.mhd_get_state_async(ctx, 0, *out)
        if sync_between:
            assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        lib.mhd_set_state(ctx, 1, other.rho, other.u, other.b)
        lib.mhd_step(ctx, 2)
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        res = [a.copy() for a in out] + [a for i in range(2) for a in lib.mhd_get_state(ctx, i)]
        lib.mhd_destroy(ctx)
        return res

    for a, b in zip(run(False), run(True)):
        assert np.array_equal(a, b)
