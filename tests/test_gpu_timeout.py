"""The one bounded device-side wait of the library: the pipelined flux pass (mixed mode, N >= 128,
MHD_OPT_FLUX_PIPELINE) waits on an mbarrier for the bulk copies that bring each row pair into
shared memory.  With the poll limit lowered to 0 (MHD_OPT_WAIT_POLLS) every such wait gives up at
once while its copy is really in flight, so the expiry path runs without any fault: the block
records the failure, waits for both of its copies still in flight and returns, and
mhd_synchronize reports MHD_ETIMEOUT.  The device stays usable: a fresh context afterwards still
gives bitwise the default pass's results."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


def run(lib, ic, pipeline, polls=None, steps=3):
    ctx = lib.mhd_init(ic.n, [(ic.nu, ic.eta, ic.cs)], precision=lib.MHD_FP32_MIXED)
    lib.mhd_set_option(ctx, lib.MHD_OPT_FLUX_PIPELINE, pipeline)
    if polls is not None:
        lib.mhd_set_option(ctx, lib.MHD_OPT_WAIT_POLLS, polls)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    lib.mhd_step(ctx, steps)
    return ctx


def test_wait_that_runs_out_reports_timeout_and_leaves_the_device_usable(lib):
    import torch

    ic = inputs.abc_dynamo(128, seed=3, b_energy=1e-2)
    ctx = run(lib, ic, pipeline=1, polls=0, steps=1)
    with pytest.raises(lib.MhdError) as err:
        lib.mhd_synchronize(ctx)
    assert err.value.status == lib.MHD_ETIMEOUT
    # both copies in flight completed within the drain's own limit
    assert "drained" in str(err.value)
    lib.mhd_destroy(ctx)
    torch.cuda.synchronize()  # no sticky error on the device

    out = []
    for pipeline in (0, 1):
        ctx = run(lib, ic, pipeline)
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        out.append(lib.mhd_get_state(ctx, 0))
        lib.mhd_destroy(ctx)
    for g, e in zip(out[1], out[0]):
        assert np.array_equal(g, e)


def test_default_poll_limit_never_runs_out(lib):
    """The same run with the limit set back explicitly to its default completes."""
    ic = inputs.abc_dynamo(128, seed=4, b_energy=1e-2)
    ctx = run(lib, ic, pipeline=1, polls=1 << 22)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    lib.mhd_destroy(ctx)


def test_poll_limit_range_is_checked(lib):
    ic = inputs.abc_dynamo(16, seed=1)
    ctx = lib.mhd_init(16, [(ic.nu, ic.eta, ic.cs)], precision=lib.MHD_FP32_MIXED)
    for bad in (-1, (1 << 22) + 1):
        with pytest.raises(lib.MhdError) as err:
            lib.mhd_set_option(ctx, lib.MHD_OPT_WAIT_POLLS, bad)
        assert err.value.status == lib.MHD_EINVAL
    lib.mhd_destroy(ctx)
