"""mhd_rhs_noalloc: the right-hand side for callers that cannot allocate device memory when they
need it (a framework that already owns the memory pool, a latency-bound loop that cannot take an
allocation's device synchronisation).  Its scratch is one static device array of the library, so
the test checks, through the C ABI, that successive calls (different grids, so each call starts
from the previous call's leftovers) give what the allocating entry point mhd_rhs gives, within the
tolerance of the other RHS tests; that the first call of the process works when it is queued on a
non-blocking stream (the twiddle tables its set-up uploads must be in place for that stream); that
a later call leaves the device's free memory unchanged; and that grids above the limit are
refused.  This file sorts last so that a run stopping at the first failure has run every other
test already."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _state(n, seed):
    from paper_1810_12707_gb300 import inputs
    rng = np.random.default_rng(seed)
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + 0.2 * np.cos(X + 2 * Y) * np.sin(Z - 0.3)
    u = inputs.random_solenoidal(n, rng, kmax2=9)
    u /= inputs.rms(u)
    b = inputs.random_solenoidal(n, rng, kmax2=9)
    b *= 0.7 / inputs.rms(b)
    return rho, u, b


def _reference(mhd, n, phys, rho, u, b):
    ctx = mhd.mhd_init(n, [phys])
    mhd.mhd_set_state(ctx, 0, rho, u, b)
    ref = mhd.mhd_rhs(ctx, 0)
    mhd.mhd_destroy(ctx)
    return ref


def _close(got, ref):
    for g, e in zip(got, ref):
        g = g.cpu().numpy()
        assert np.max(np.abs(g - e)) <= 1e-12 * np.max(np.abs(e))


def test_noalloc_rhs_matches_mhd_rhs_on_successive_calls():
    import torch

    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    phys = (0.013, 0.021, 1.7)
    side = torch.cuda.Stream()  # created non-blocking: not ordered after the legacy stream
    for n, seed in ((32, 11), (16, 12)):
        rho, u, b = _state(n, seed)
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rho, u, b)]
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            got = mhd.mhd_rhs_noalloc(n, phys, *dev)
        side.synchronize()
        _close(got, _reference(mhd, n, phys, rho, u, b))

    # a later call through the raw C ABI, outputs allocated beforehand: free device memory is the
    # same before and after it
    n = 32
    rho, u, b = _state(n, 13)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rho, u, b)]
    outs = [torch.empty((n, n, n), dtype=torch.float64, device="cuda"),
            torch.empty((3, n, n, n), dtype=torch.float64, device="cuda"),
            torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")]
    ph = mhd.MhdPhys(*phys)
    lib = mhd.load_library()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st = lib.mhd_rhs_noalloc(n, ctypes.byref(ph), *[t.data_ptr() for t in dev], *[o.data_ptr() for o in outs],
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert st == mhd.MHD_OK
    assert free1 == free0
    _close(outs, _reference(mhd, n, phys, rho, u, b))


def test_noalloc_rejects_grids_above_the_limit():
    import torch

    from paper_1810_12707_gb300 import mhd
    n = 64
    rho = torch.ones((n, n, n), dtype=torch.float64, device="cuda")
    v = torch.zeros((3, n, n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(mhd.MhdError) as err:
        mhd.mhd_rhs_noalloc(n, (0.01, 0.01, 1.0), rho, v, v)
    assert err.value.status == mhd.MHD_EINVAL
