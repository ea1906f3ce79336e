"""Persistent column and flux passes (MHD_OPT_PERSISTENT): one grid of resident blocks per pass
takes tiles from a work counter that the last block resets.  Each tile is computed exactly as the
one-block-per-tile kernels compute it, so a batched run is bitwise the same either way, in every
precision, over several steps (the counters must come back to zero between launches, including
graph-replayed ones)."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("n,batch", [(32, 5), (64, 3)])
def test_persistent_passes_are_bitwise_the_regular_ones(lib, precision, n, batch):
    nu, eta, mach = inputs.ensemble_params(batch, seed=9)
    ics = [inputs.orszag_tang(n, seed=50 + i, mach=float(mach[i]), nu=float(nu[i]), eta=float(eta[i]))
           for i in range(batch)]
    out = []
    for persistent in (0, 1):
        ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs) for ic in ics], precision=precision)
        lib.mhd_set_option(ctx, lib.MHD_OPT_PERSISTENT, persistent)
        for i, ic in enumerate(ics):
            lib.mhd_set_state(ctx, i, ic.rho, ic.u, ic.b)
        lib.mhd_step(ctx, 6)  # one direct step, then graph replays
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        out.append([lib.mhd_get_state(ctx, i) for i in range(batch)] +
                   [[np.array(lib.mhd_diagnostics(ctx, i)["dt"])] for i in range(batch)])
        lib.mhd_destroy(ctx)
    for a, b in zip(out[0], out[1]):
        for g, e in zip(a, b):
            assert np.array_equal(g, e)


def test_persistent_option_is_checked(lib):
    ctx = lib.mhd_init(16, [(0.01, 0.01, 1.0)])
    with pytest.raises(lib.MhdError) as err:
        lib.mhd_set_option(ctx, lib.MHD_OPT_PERSISTENT, 2)
    assert err.value.status == lib.MHD_EINVAL
    lib.mhd_destroy(ctx)
