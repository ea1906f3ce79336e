"""The column-pass autotuner (mhd_autotune): it returns power-of-two tile widths within the launch
limits and their timings, and a run with the tuned widths is bitwise the run with the library's
default widths (tile width only regroups independent column transforms)."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


@pytest.mark.parametrize("n,batch,precision", [(32, 3, 0), (64, 2, 1), (128, 1, 1)])
def test_autotuned_run_is_bitwise_the_default_run(lib, n, batch, precision):
    ics = [inputs.orszag_tang(n, seed=s, mach=0.2) for s in range(batch)]
    out = []
    for tune in (False, True):
        ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs) for ic in ics], precision=precision)
        for i, ic in enumerate(ics):
            lib.mhd_set_state(ctx, i, ic.rho, ic.u, ic.b)
        if tune:
            r = lib.mhd_autotune(ctx, reps=3)
            for t in r["tiles"]:
                assert t in (1, 2, 4, 8, 16, 32, 64) and t * (n // 8) <= 1024
            assert all(m > 0 for m in r["ms"])
        lib.mhd_step(ctx, 12)
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        out.append([np.concatenate([np.ravel(a) for a in lib.mhd_get_state(ctx, i)]) for i in range(batch)])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_autotune_arguments(lib):
    ctx = lib.mhd_init(16, [(0.01, 0.01, 1.0)])
    with pytest.raises(lib.MhdError):
        lib.mhd_autotune(ctx, reps=0)


def test_oversized_tile_option_is_clamped(lib):
    """A tile width whose thread count the kernel's registers do not allow (64 columns x 16
    threads of an FP64 pass at 128^3) is reduced by the launcher instead of failing."""
    n = 128
    ic = inputs.orszag_tang(n, seed=1, mach=0.2)
    out = []
    for tile in (0, 64):
        ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs)])
        for opt in (lib.MHD_OPT_TILE_INV_Z, lib.MHD_OPT_TILE_INV_Y, lib.MHD_OPT_TILE_FWD_Y, lib.MHD_OPT_TILE_FWD_Z):
            lib.mhd_set_option(ctx, opt, tile)
        lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
        lib.mhd_step(ctx, 3)
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        out.append(np.concatenate([np.ravel(a) for a in lib.mhd_get_state(ctx, 0)]))
    assert np.array_equal(out[0], out[1])
