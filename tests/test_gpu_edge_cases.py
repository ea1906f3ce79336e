"""Degenerate and empty cases of the method through the C ABI, in both precisions:

* zero steps: the state, the time and the step count are untouched;
* a uniform state (constant rho and B, m = 0) is an exact steady solution: every flux is constant,
  so only the k = 0 modes are nonzero and k x (flux) vanishes; the RHS is zero, the state stays put
  over CFL steps, and the step is the advective CFL step with the fast speed sqrt(Cs^2 + |B|^2/rho);
* the ideal limit nu = eta = 0 (no viscous step limit, no damping) against the oracle;
* a tracer set emptied again: the step goes on without the push, and the flow is bitwise the run
  that never had tracers;
* grid sizes and parameters the library does not take are refused before any work.
"""
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
def test_zero_steps_is_a_no_op(lib, precision):
    ic = inputs.orszag_tang(32, seed=5)
    ctx = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=precision)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    before = lib.mhd_checkpoint(ctx, 0)
    lib.mhd_step(ctx, 0)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    assert np.array_equal(lib.mhd_checkpoint(ctx, 0), before)
    d = lib.mhd_diagnostics(ctx, 0)
    assert d["step"] == 0 and d["t"] == 0.0
    lib.mhd_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_uniform_state_is_a_fixed_point(lib, precision):
    n, cs, nu = 32, 1.1, 0.01
    rho0, b0 = 1.3, np.array([0.2, -0.1, 0.4])
    rho = np.full((n, n, n), rho0)
    b = np.broadcast_to(b0[:, None, None, None], (3, n, n, n)).copy()
    ctx = lib.mhd_init(n, [(nu, nu, cs)], precision=precision)
    lib.mhd_set_state(ctx, 0, rho, np.zeros((3, n, n, n)), b)
    for f in lib.mhd_rhs(ctx, 0):
        assert np.max(np.abs(f)) <= 1e-14
    lib.mhd_step(ctx, 5)
    r, m, bb = lib.mhd_get_state(ctx, 0)
    assert np.max(np.abs(r - rho0)) <= 1e-15 and np.max(np.abs(m)) <= 1e-15
    assert np.max(np.abs(bb - b)) <= 1e-15
    d = lib.mhd_diagnostics(ctx, 0)
    k = (n - 1) // 3
    expect = min(0.2 * (2 * np.pi / n) / np.sqrt(cs * cs + float(b0 @ b0) / rho0), 0.5 / (nu * k * k))
    # the mixed mode takes the CFL maximum from its FP32 pass
    rtol = 1e-14 if precision == 0 else 1e-6
    assert d["step"] == 5
    assert abs(d["dt"] - expect) <= rtol * expect
    assert abs(d["t"] - 5 * expect) <= 10 * rtol * expect
    lib.mhd_destroy(ctx)


def test_ideal_limit_matches_oracle(lib, oracle_mod):
    n, cs = 32, 1.4
    ic = inputs.orszag_tang(n, seed=11, mach=0.3)
    ctx = lib.mhd_init(n, [(0.0, 0.0, cs)])
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    o = oracle_mod.Oracle(n, 0.0, 0.0, cs)
    o.set_state(ic.rho, ic.u, ic.b)
    lib.mhd_step(ctx, 20)
    o.step(20)
    dg, do = lib.mhd_diagnostics(ctx, 0), o.diagnostics()
    assert abs(dg["t"] - do["t"]) <= 1e-12 * do["t"]
    for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state()):
        assert np.linalg.norm((g - e).ravel()) <= 1e-10 * np.linalg.norm(e.ravel())
    lib.mhd_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_emptied_tracer_set(lib, precision):
    n = 32
    ic = inputs.orszag_tang(n, seed=6)
    runs = []
    for with_tracers in (False, True):
        ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs)], precision=precision)
        lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
        if with_tracers:
            lib.mhd_tracers_set(ctx, 0, np.random.default_rng(0).uniform(0, 2 * np.pi, (50, 3)))
            lib.mhd_step(ctx, 3)
            lib.mhd_tracers_set(ctx, 0, np.zeros((0, 3)))
            assert lib.load_library().mhd_tracers_count(ctx.handle, 0) == 0
            pos, vel = lib.mhd_tracers_get(ctx, 0)
            assert pos.shape == (0, 3) and vel.shape == (0, 3)
            lib.mhd_step(ctx, 4)
        else:
            lib.mhd_step(ctx, 7)
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        runs.append(lib.mhd_get_state(ctx, 0))
        lib.mhd_destroy(ctx)
    for g, e in zip(*runs):
        assert np.array_equal(g, e)


def test_unsupported_sizes_and_parameters_are_refused(lib):
    for n in (8, 48, 2048):
        with pytest.raises(lib.MhdError):
            lib.mhd_init(n, [(1e-3, 1e-3, 1.0)])
    with pytest.raises(lib.MhdError):
        lib.mhd_init(32, [])                                   # no instance
    for phys in ((-1e-3, 1e-3, 1.0), (1e-3, -1e-3, 1.0), (1e-3, 1e-3, -1.0), (np.nan, 1e-3, 1.0),
                 (1e-3, np.inf, 1.0)):
        with pytest.raises(lib.MhdError):
            lib.mhd_init(32, [phys])
    ctx = lib.mhd_init(16, [(1e-3, 1e-3, 1.0)])
    lib.mhd_set_state(ctx, 0, np.ones((16, 16, 16)), np.zeros((3, 16, 16, 16)), np.zeros((3, 16, 16, 16)))
    with pytest.raises(lib.MhdError):
        lib.mhd_step(ctx, -1)
    for field in (-1, 7):
        with pytest.raises(lib.MhdError):
            lib.mhd_get_spectrum(ctx, 0, field)
    lib.mhd_destroy(ctx)


def cfl_states(n):
    """States that stress the exactness of the CFL maximum: speeds tied to 1e-9, 1e-6 and 1e-4
    relative (around the 1e-6 margin of the flux pass's FP32 screening), a peak in the last
    z-planes (reached by the last blocks of the pass), and a turbulent Orszag-Tang state."""
    X, Y, Z = inputs.grid(n)
    zl = Z.max()
    one = np.ones((n, n, n))
    zero = np.zeros((3, n, n, n))
    out = []
    for eps in (1e-9, 1e-6, 1e-4):
        u = zero.copy()
        u[0] = 1.0 + eps * np.sin(X) * np.cos(2 * Y) * np.sin(3 * Z)
        out.append((one, u, zero))
    u = zero.copy()
    u[0] = 1.0 + 0.3 * ((1.0 + np.cos(Z - zl)) / 2) ** 4  # single peak at the last z-plane
    b = zero.copy()
    b[2] = 0.5 + 0.1 * np.sin(X + Y)
    out.append((1.0 + 0.1 * np.cos(Y), u, b))
    ic = inputs.orszag_tang(n, seed=12, mach=0.5)
    out.append((ic.rho, ic.u, ic.b))
    return out


@pytest.mark.parametrize("n", [32, 64])
def test_cfl_maximum_is_exact(lib, n):
    """The step size equals the CFL formula at the exact grid maximum of |u| + c_f, taken on the
    host from the same state (FP64)."""
    cs, nu = 0.9, 1e-4
    k = (n - 1) // 3
    for rho, u, b in cfl_states(n):
        ctx = lib.mhd_init(n, [(nu, nu, cs)])
        lib.mhd_set_state(ctx, 0, rho, u, b)
        r, m, bb = lib.mhd_get_state(ctx, 0)
        speed = np.sqrt(np.sum((m / r) ** 2, axis=0)) + np.sqrt(cs * cs + np.sum(bb * bb, axis=0) / r)
        expect = min(0.2 * (2 * np.pi / n) / speed.max(), 0.5 / (nu * k * k))
        lib.mhd_step(ctx, 1)
        got = lib.mhd_diagnostics(ctx, 0)["dt"]
        lib.mhd_destroy(ctx)
        assert abs(got - expect) <= 1e-14 * expect
