"""Shell spectra, theta' and S_3 through the C ABI (paper, section "for hydrodynamic flow"),
against the oracle: element by element on the same seeded states, at grid sizes that take every
x-pass layout (8, 4, 2 and 1 row pairs per block), after steps, and in both precisions, with the
kinetic and magnetic helicities and max |div B|; plus the sum rules, bitwise repeatability, the
negative derivative skewness of decaying turbulence, and max |div B| of a field written out by
hand.
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


def mixed_state(n, seed):
    rng = np.random.default_rng(seed)
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + 0.25 * np.cos(X + 2 * Y) * np.sin(Z - 0.4) + 0.05 * np.sin(3 * Z)
    u = inputs.random_solenoidal(n, rng, kmax2=16) + 0.3 * np.stack([np.sin(2 * X), np.cos(Y + Z), 0 * X])
    u /= inputs.rms(u)
    b = inputs.random_solenoidal(n, rng, kmax2=16)
    b *= 0.5 / inputs.rms(b)
    return rho, u, b


def check_close(g, e, rtol):
    for key in ("ek", "em"):
        scale = max(np.max(np.abs(e[key])), 1e-300)
        assert np.max(np.abs(g[key] - e[key])) <= rtol * scale, key
    for key in ("theta", "d2"):
        assert g[key] == pytest.approx(e[key], rel=rtol), key
    assert abs(g["d3"] - e["d3"]) <= rtol * e["d2"] ** 1.5
    assert abs(g["s3"] - e["s3"]) <= 10 * rtol
    # helicities against their bounds: |<u . w>| <= sqrt(3) k_max <|u|^2>, |<A . B>| <= <|B|^2>
    kmax = (len(e["ek"]) - 1) / np.sqrt(3) + 1
    u2, b2 = 2 * np.sum(e["ek"]), 2 * np.sum(e["em"])
    assert abs(g["kin_hel"] - e["kin_hel"]) <= rtol * np.sqrt(3) * kmax * u2
    assert abs(g["mag_hel"] - e["mag_hel"]) <= rtol * b2
    assert abs(g["divb_max"] - e["divb_max"]) <= rtol * np.sqrt(3) * kmax * np.sqrt(b2)


@pytest.mark.parametrize("n", [16, 32, 64, 128])
def test_spectra_match_oracle(lib, oracle_mod, n):
    rho, u, b = mixed_state(n, 3)
    ctx = lib.mhd_init(n, [(0.01, 0.01, 2.0)])
    lib.mhd_set_state(ctx, 0, rho, u, b)
    o = oracle_mod.Oracle(n, 0.01, 0.01, 2.0)
    o.set_state(rho, u, b)
    g, e = lib.mhd_spectra(ctx, 0), o.spectra()
    assert len(g["ek"]) == lib.mhd_num_shells(n) == len(e["ek"])
    check_close(g, e, 1e-11)


@pytest.mark.parametrize("precision", [0, 1])
def test_spectra_after_steps(lib, oracle_mod, precision):
    n = 32
    ic = inputs.decaying_turbulence(n, 4.0, seed=7, nu=0.01)
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs)], precision=precision, integrator=lib.MHD_RK4)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    o = oracle_mod.Oracle(n, ic.nu, ic.eta, ic.cs, integrator=1)
    o.set_state(ic.rho, ic.u, ic.b)
    lib.mhd_step(ctx, 60)
    o.step(60)
    g, e = lib.mhd_spectra(ctx, 0), o.spectra()
    # FP64: round-off only; mixed: the FP32 products over 60 RK4 steps (relative 1e-6 of the state)
    check_close(g, e, 1e-9 if precision == 0 else 2e-4)
    assert np.all(g["em"] == 0.0)  # B = 0 stays 0 in both precisions


def test_sum_rules_and_repeatability(lib):
    n = 64
    rho, u, b = mixed_state(n, 5)
    ctx = lib.mhd_init(n, [(0.01, 0.01, 2.0)])
    lib.mhd_set_state(ctx, 0, np.ones((n, n, n)), u, b)
    a, c = lib.mhd_spectra(ctx, 0), lib.mhd_spectra(ctx, 0)
    for key in ("ek", "em"):
        assert np.array_equal(a[key], c[key])
    assert (a["theta"], a["s3"]) == (c["theta"], c["s3"])
    d = lib.mhd_diagnostics(ctx, 0)
    assert a["em"].sum() == pytest.approx(d["me"], rel=1e-12)
    assert a["ek"].sum() == pytest.approx(d["ke"], rel=1e-12)  # rho = 1


def test_wrong_shell_count_is_rejected(lib):
    ctx = lib.mhd_init(16, [(0.01, 0.01, 1.0)])
    lib.mhd_set_state(ctx, 0, *mixed_state(16, 1))
    import ctypes
    buf = (ctypes.c_double * 4)()
    st = lib.load_library().mhd_spectra(ctx.handle, 0, buf, buf, 4, None)
    assert st == lib.MHD_EINVAL
    assert lib.mhd_num_shells(48) == 0


def test_decaying_turbulence_develops_negative_skewness(lib):
    """From the E(k) ~ k^4 exp(-2k^2/k0^2) state (S_3 near 0, no divergence) the velocity
    derivative skewness turns negative within a fraction of an eddy turnover, energy moves to
    higher shells, and compressive motion appears (theta' > 0)."""
    n = 64
    ic = inputs.decaying_turbulence(n, 4.0, seed=9, nu=0.01)
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs)], integrator=lib.MHD_RK4)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    r0 = lib.mhd_spectra(ctx, 0)
    lib.mhd_step(ctx, 400)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    r1 = lib.mhd_spectra(ctx, 0)
    k = np.arange(len(r0["ek"]))
    assert abs(r0["s3"]) < 0.15 and r0["theta"] < 1e-10
    assert -0.7 < r1["s3"] < -0.2
    assert r1["theta"] > 1e-3
    assert (k * r1["ek"]).sum() / r1["ek"].sum() > (k * r0["ek"]).sum() / r0["ek"].sum()


@pytest.mark.parametrize("precision", [0, 1])
def test_divb_max_closed_form(lib, precision):
    """B = (a sin 2x, c cos 3y, 0): div B = 2a cos 2x - 3c sin 3y reaches 2a + 3c at the grid
    points x = 0, y = pi/2 (N = 32, 64)."""
    for n in (32, 64):
        X, Y, _ = inputs.grid(n)
        b = np.zeros((3, n, n, n))
        b[0] = 0.7 * np.sin(2 * X)
        b[1] = 0.4 * np.cos(3 * Y)
        ctx = lib.mhd_init(n, [(0.01, 0.01, 1.0)], precision=precision)
        lib.mhd_set_state(ctx, 0, np.ones((n, n, n)), np.zeros((3, n, n, n)), b)
        r = lib.mhd_spectra(ctx, 0)
        lib.mhd_destroy(ctx)
        assert abs(r["divb_max"] - 2.6) <= 1e-13
