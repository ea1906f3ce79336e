"""ABC body force and the paper's energy-exchange runs, through the C ABI.

* the forced RHS and 30 forced steps against the oracle (which forms rho f on the grid; the GPU
  shifts the density spectrum);
* the energy-exchange runs of section "for magnetohydrodynamic flow" (flows ABC, single-mode ABC,
  Taylor-Green, cat's eye; Mach 0.1, Re = Rm = 450, Alfven Mach 1): kinetic and magnetic energy
  exchange while the total falls monotonically, only through viscosity and resistivity.  These
  runs use RK4: at Mach 0.1 the sound modes sit on the imaginary axis, which AB2's stability
  region leaves out, and with this grid and CFL number the FP64 oracle's AB2 run grows its
  internal energy until it blows up near t = 1.4.
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def state(n, seed):
    rng = np.random.default_rng(seed)
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + 0.2 * np.cos(X + 2 * Y) * np.sin(Z - 0.3)
    u = inputs.random_solenoidal(n, rng, kmax2=9)
    u /= inputs.rms(u)
    b = inputs.random_solenoidal(n, rng, kmax2=9)
    b *= 0.7 / inputs.rms(b)
    return inputs.InitialCondition(rho, u, b, 0.013, 0.021, 1.7)


FORCE = (0.8, 1.0, 0.7, 0.4, 1)


@pytest.mark.parametrize("precision", [0, 1])
def test_forced_rhs_and_steps_match_oracle(lib, oracle_mod, precision):
    ic = state(32, 5)
    ctx = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=precision)
    lib.mhd_set_forcing(ctx, 0, *FORCE)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    o = oracle_mod.Oracle(32, ic.nu, ic.eta, ic.cs, forcing=FORCE)
    o.set_state(ic.rho, ic.u, ic.b)
    ref = o.rhs()
    scale = max(np.max(np.abs(e)) for e in ref)
    tol = 1e-12 if precision == 0 else 1e-5
    for g, e in zip(lib.mhd_rhs(ctx, 0), ref):
        assert np.max(np.abs(g - e)) <= tol * scale
    lib.mhd_step(ctx, 30)
    o.step(30)
    for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state()):
        assert rel_l2(g, e) <= (1e-10 if precision == 0 else 1e-5)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK


def test_forcing_rejects_bad_wavenumber(lib):
    ctx = lib.mhd_init(16, [(1e-2, 1e-2, 1.0)])
    with pytest.raises(lib.MhdError):
        lib.mhd_set_forcing(ctx, 0, 1.0, 1, 1, 1, 6)  # k_max = 5 at N = 16


@pytest.mark.parametrize("kind", ["abc", "abc_single", "tg_paper", "cats_eye"])
def test_energy_exchange_runs(lib, kind):
    n = 32
    ic = inputs.energy_exchange(n, kind, seed=3)
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs)], precision=lib.MHD_FP64, integrator=lib.MHD_RK4)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    d0 = lib.mhd_diagnostics(ctx, 0)
    assert abs(d0["ke"] - d0["me"]) <= 1e-3 * d0["ke"]  # Alfven Mach number 1
    ke, me, et = [d0["ke"]], [d0["me"]], [d0["etot"]]
    for _ in range(40):
        lib.mhd_step(ctx, 25)
        d = lib.mhd_diagnostics(ctx, 0)
        ke.append(d["ke"])
        me.append(d["me"])
        et.append(d["etot"])
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    assert d["t"] > 1.0
    # total energy falls, step after step (viscous and resistive losses only)
    assert all(b < a for a, b in zip(et, et[1:]))
    # the reservoirs start equal and do not decay alike: energy moves between them
    assert max(abs(k / m - 1.0) for k, m in zip(ke, me)) > 0.1


def test_abc_forcing_holds_the_beltrami_state(lib, oracle_mod):
    """Forced relaxed state: the k_f = 1 ABC flow is a Beltrami field (curl u = u), so u.grad u is
    a pure gradient and a body force of amplitude nu k_f^2 balances the viscous loss of that mode.
    Forced, the kinetic energy stays at its initial value while, unforced, it decays as
    exp(-2 nu t).  RK4 (see the module docstring); the GPU run follows the oracle to t = 5."""
    n, nu = 16, 0.02
    u = inputs.paper_flow(n, "abc")
    rho, b = np.ones((n, n, n)), np.zeros_like(u)
    for amp in (0.0, nu):
        ctx = lib.mhd_init(n, [(nu, nu, 10.0)], integrator=lib.MHD_RK4)
        lib.mhd_set_forcing(ctx, 0, amp, 1.0, 1.0, 1.0, 1)
        lib.mhd_set_state(ctx, 0, rho, u, b)
        ke0 = lib.mhd_diagnostics(ctx, 0)["ke"]
        o = oracle_mod.Oracle(n, nu, nu, 10.0, integrator=1, forcing=(amp, 1.0, 1.0, 1.0, 1))
        o.set_state(rho, u, b)
        worst = 0.0
        for _ in range(16):
            lib.mhd_step(ctx, 50)
            o.step(50)
            d, e = lib.mhd_diagnostics(ctx, 0), o.diagnostics()
            assert d["t"] == pytest.approx(e["t"], rel=1e-12)
            assert d["ke"] == pytest.approx(e["ke"], rel=1e-9)
            want = 1.0 if amp else np.exp(-2.0 * nu * d["t"])
            worst = max(worst, abs(d["ke"] / ke0 - want))
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        assert d["t"] > 4.5
        assert worst < 0.03
