"""The column-pass autotuner (mhd_autotune) and the radix option of the mixed mode's column
passes: tuned tile widths leave results bitwise unchanged, radix 16 and radix 8 agree to FP32
rounding and with the oracle, and oversized or invalid options are handled."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


RADIX_OPTS = ("MHD_OPT_RADIX_INV_Z", "MHD_OPT_RADIX_INV_Y", "MHD_OPT_RADIX_FWD_Y", "MHD_OPT_RADIX_FWD_Z")


def run(lib, ics, n, precision, steps, tune=False, radix=None):
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs) for ic in ics], precision=precision)
    for i, ic in enumerate(ics):
        lib.mhd_set_state(ctx, i, ic.rho, ic.u, ic.b)
    tuned = lib.mhd_autotune(ctx, reps=3) if tune else None
    for name, r in zip(RADIX_OPTS, radix or ()):
        lib.mhd_set_option(ctx, getattr(lib, name), r)
    lib.mhd_step(ctx, steps)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    out = [np.concatenate([np.ravel(a) for a in lib.mhd_get_state(ctx, i)]) for i in range(len(ics))]
    lib.mhd_destroy(ctx)
    return out, tuned


@pytest.mark.parametrize("n,batch,precision", [(32, 3, 0), (64, 2, 1), (128, 1, 1)])
def test_autotuned_run_is_bitwise_the_default_tiles_run(lib, n, batch, precision):
    """Tile width only regroups independent column transforms: the tuned run equals, bit for bit,
    a run with the library's default widths and the same radices."""
    ics = [inputs.orszag_tang(n, seed=s, mach=0.2) for s in range(batch)]
    tuned_out, tuned = run(lib, ics, n, precision, 12, tune=True)
    for t, r in zip(tuned["tiles"], tuned["radix"]):
        assert t in (1, 2, 4, 8, 16, 32, 64)
        assert r in ((8, 16) if precision == 1 else (8,))
    assert all(m > 0 for m in tuned["ms"])
    ref_out, _ = run(lib, ics, n, precision, 12, radix=tuned["radix"] if precision == 1 else None)
    for a, b in zip(tuned_out, ref_out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [16, 64, 256])
def test_radix_16_and_8_agree(lib, oracle_mod, n):
    """The mixed mode's column passes with radix 16 and with radix 8 compute the same step to FP32
    rounding, and both follow the oracle to the mixed mode's bound."""
    ic = inputs.orszag_tang(n, seed=2, mach=0.2)
    a, _ = run(lib, [ic], n, 1, 10, radix=(8, 8, 8, 8))
    b, _ = run(lib, [ic], n, 1, 10, radix=(16, 16, 16, 16))
    rel = np.linalg.norm(a[0] - b[0]) / np.linalg.norm(a[0])
    assert 0 < rel <= 1e-6
    if n <= 64:
        o = oracle_mod.Oracle(n, ic.nu, ic.eta, ic.cs)
        o.set_state(ic.rho, ic.u, ic.b)
        o.step(10)
        ref = np.concatenate([np.ravel(x) for x in o.get_state()])
        for x in (a[0], b[0]):
            assert np.linalg.norm(x - ref) <= 1e-5 * np.linalg.norm(ref)


def test_autotune_arguments(lib):
    ctx = lib.mhd_init(16, [(0.01, 0.01, 1.0)])
    with pytest.raises(lib.MhdError):
        lib.mhd_autotune(ctx, reps=0)
    with pytest.raises(lib.MhdError):
        lib.mhd_set_option(ctx, lib.MHD_OPT_RADIX_FWD_Y, 4)


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
