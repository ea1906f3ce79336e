"""Adams-Bashforth steps with the assembly fused into the next step's inverse z pass
(MHD_OPT_FUSED_UPDATE).  The fused kernel updates every kept mode with the assembly
kernel's own arithmetic and transforms the new state with the inverse z pass's own transform, so
a run is bitwise the run with separate kernels, in every precision: across graph replays, across
step calls (the z buffer is reused only when nothing ran in between), after a state is replaced,
with the ABC force on, with tracers, for batches with a ragged last tile, and when the fused
block takes other tile widths."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


def _ics(n, batch, seed):
    nu, eta, mach = inputs.ensemble_params(batch, seed=seed)
    return [inputs.orszag_tang(n, seed=seed + 40 + i, mach=float(mach[i]), nu=float(nu[i]), eta=float(eta[i]))
            for i in range(batch)]


def _run(lib, n, ics, precision, fuse, script, tile=0, tracers=()):
    """Runs `script(ctx)` on a fresh context with the fused update on or off; returns every
    instance's state and time-step record, and the tracers of the instances in `tracers`."""
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs) for ic in ics], precision=precision)
    lib.mhd_set_option(ctx, lib.MHD_OPT_FUSED_UPDATE, fuse)
    if tile:
        lib.mhd_set_option(ctx, lib.MHD_OPT_TILE_FUSED, tile)
    for i, ic in enumerate(ics):
        lib.mhd_set_state(ctx, i, ic.rho, ic.u, ic.b)
    script(ctx)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    out = []
    for i in range(len(ics)):
        out += list(lib.mhd_get_state(ctx, i))
        dg = lib.mhd_diagnostics(ctx, i)
        out.append(np.array([dg["t"], dg["dt"], dg["step"]]))
    for i in tracers:
        out += list(lib.mhd_tracers_get(ctx, i))
    lib.mhd_destroy(ctx)
    return out


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(x, y), float(np.max(np.abs(x - y)))


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("n,batch", [(16, 1), (32, 5), (64, 3)])
def test_fused_update_is_bitwise_the_separate_kernels(lib, precision, n, batch):
    ics = _ics(n, batch, seed=11)

    def script(ctx):
        lib.mhd_step(ctx, 4)     # one direct step, then graph replays
        lib.mhd_step(ctx, 1)     # continues from the z buffer the last call left
        lib.mhd_diagnostics(ctx, 0)
        lib.mhd_step(ctx, 2)     # the diagnostics used the work buffers: refilled first

    _same(_run(lib, n, ics, precision, 1, script), _run(lib, n, ics, precision, 0, script))


@pytest.mark.parametrize("precision", [0, 2])
def test_fused_update_after_a_state_is_replaced(lib, precision):
    n, batch = 32, 3
    ics = _ics(n, batch, seed=21)
    other = inputs.orszag_tang(n, seed=99, mach=0.2, nu=ics[1].nu, eta=ics[1].eta)

    def script(ctx):
        lib.mhd_step(ctx, 3)
        lib.mhd_set_state(ctx, 1, other.rho, other.u, other.b)
        lib.mhd_step(ctx, 3)

    _same(_run(lib, n, ics, precision, 1, script), _run(lib, n, ics, precision, 0, script))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_fused_update_with_force_and_tracers(lib, precision):
    n, batch = 32, 2
    ics = _ics(n, batch, seed=31)
    pos = np.random.default_rng(5).uniform(0.0, 2 * np.pi, size=(40, 3))

    def script(ctx):
        lib.mhd_set_forcing(ctx, 0, 0.05)
        lib.mhd_tracers_set(ctx, 1, pos)
        lib.mhd_step(ctx, 5)

    a = _run(lib, n, ics, precision, 1, script, tracers=(1,))
    b = _run(lib, n, ics, precision, 0, script, tracers=(1,))
    _same(a, b)


@pytest.mark.parametrize("tile", [1, 2, 4, 64])
def test_fused_tile_widths_agree(lib, tile):
    n, batch = 64, 2
    ics = _ics(n, batch, seed=41)

    def script(ctx):
        lib.mhd_step(ctx, 3)

    for precision in (0, 1, 2):
        _same(_run(lib, n, ics, precision, 1, script, tile=tile), _run(lib, n, ics, precision, 0, script))


def test_fused_step_launches(lib):
    """Profiled steps (direct launches): one plain inverse z pass per step call, then every step
    runs the fused kernel in place of the assembly and the inverse z pass."""
    n = 32
    ic = _ics(n, 1, seed=51)[0]
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs)], precision=lib.MHD_FP32_MIXED)
    lib.mhd_set_option(ctx, lib.MHD_OPT_FUSED_UPDATE, 1)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    lib.mhd_profile(ctx, True)
    lib.mhd_step(ctx, 4)
    prof = lib.mhd_profile_read(ctx)
    lib.mhd_profile(ctx, False)
    assert prof["inverse_z"][1] == 1
    assert prof["assemble_iz"][1] == 4
    assert prof["assemble_ab2"][1] == 0
    assert prof["inverse_y"][1] == 4
    lib.mhd_destroy(ctx)


def test_fused_option_is_checked(lib):
    ctx = lib.mhd_init(16, [(0.01, 0.01, 1.0)])
    for opt, bad in ((lib.MHD_OPT_FUSED_UPDATE, 2), (lib.MHD_OPT_TILE_FUSED, 65), (lib.MHD_OPT_TILE_FUSED, -1)):
        with pytest.raises(lib.MhdError) as err:
            lib.mhd_set_option(ctx, opt, bad)
        assert err.value.status == lib.MHD_EINVAL
    lib.mhd_destroy(ctx)
