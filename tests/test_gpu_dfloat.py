"""The double-float mode (MHD_FP64_DF) against the FP64 oracle, through the C ABI.

In this mode every value of the step is a pair of FP32 numbers (hi + lo, a 48-bit significand)
and every transform, product, RHS term and update runs in double-float arithmetic (unit roundoff
about 2^-48 = 3.6e-15, with a few more units from the lazy sums and products).  A length-N
transform then errs by about log2(N) * 2^-47 relative, so against the oracle (IEEE FP64, 2^-53)
the tolerances below are set from that bound:
  * one RHS, state round trip: max abs error <= 2e-11 of the field's largest value;
  * 100 steps: relative L2 error per physical field (rho, m, B) <= 1e-10, the FP64 target;
  * t and dt: the CFL maximum is formed in FP64 from the double-float squares at the points that
    can reach it, so dt agrees to 1e-12 relative;
  * diagnostics (taken in FP64 from the state): relative error <= 1e-10.
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
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def maxrel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def random_state(n, seed, amp=0.2):
    rng = np.random.default_rng(seed)
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + amp * np.cos(X + 2 * Y) * np.sin(Z - 0.3) + 0.05 * np.sin(3 * Y - Z)
    u = inputs.random_solenoidal(n, rng, kmax2=9)
    u /= inputs.rms(u)
    b = inputs.random_solenoidal(n, rng, kmax2=9)
    b *= 0.7 / inputs.rms(b)
    return inputs.InitialCondition(rho, u, b, 0.013, 0.021, 1.7, "random")


def make_pair(lib, oracle_mod, ic, dt=0.0, integrator=0):
    ctx = lib.mhd_init(ic.n, [(ic.nu, ic.eta, ic.cs)], dt=dt, precision=lib.MHD_FP64_DF, integrator=integrator)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    o = oracle_mod.Oracle(ic.n, ic.nu, ic.eta, ic.cs, dt=dt, integrator=integrator)
    o.set_state(ic.rho, ic.u, ic.b)
    return ctx, o


@pytest.mark.parametrize("n", [16, 32, 64])
def test_df_rhs_and_roundtrip_match_oracle(lib, oracle_mod, n):
    ic = random_state(n, 100 + n)
    ctx, o = make_pair(lib, oracle_mod, ic)
    for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state()):
        assert maxrel(g, e) <= 2e-11
    errs = [maxrel(g, e) for g, e in zip(lib.mhd_rhs(ctx, 0), o.rhs())]
    print(f"double-float RHS at {n}^3 vs oracle, max rel per field: {max(errs):.2e}")
    assert max(errs) <= 2e-11


def test_df_orszag_tang_100_fixed_steps(lib, oracle_mod):
    """N = 32, Orszag-Tang-type IC with seeded 1e-3 perturbation, Mach 0.1, nu = eta = 1e-2, fixed
    dt = 1e-3, 100 steps."""
    ic = inputs.orszag_tang(32, seed=0)
    ctx, o = make_pair(lib, oracle_mod, ic, dt=1e-3)
    lib.mhd_step(ctx, 100)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    o.step(100)
    errs = [rel_l2(g, e) for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state())]
    print(f"double-float Orszag-Tang 32^3, 100 steps, rel L2 (rho, m, B): {errs}")
    assert max(errs) <= 1e-10
    dg, do = lib.mhd_diagnostics(ctx, 0), o.diagnostics()
    assert dg["step"] == 100 and abs(dg["t"] - do["t"]) <= 1e-14
    for k in ("ke", "me", "cross_hel", "mean_speed", "mean_bmag", "smax"):
        assert abs(dg[k] - do[k]) <= 1e-10 * max(abs(do[k]), 1e-300), k


@pytest.mark.parametrize("n", [32, 64])
def test_df_cfl_steps(lib, oracle_mod, n):
    ic = random_state(n, 7 + n)
    ctx, o = make_pair(lib, oracle_mod, ic)
    lib.mhd_step(ctx, 100)
    o.step(100)
    dg, do = lib.mhd_diagnostics(ctx, 0), o.diagnostics()
    assert abs(dg["t"] - do["t"]) <= 1e-12 * do["t"]
    assert abs(dg["dt"] - do["dt"]) <= 1e-12 * do["dt"]
    errs = [rel_l2(g, e) for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state())]
    print(f"double-float random state {n}^3, 100 CFL steps, rel L2 (rho, m, B): {errs}")
    assert max(errs) <= 1e-10


@pytest.mark.parametrize("integrator", [1, 2])
def test_df_rk4_and_predictor_corrector(lib, oracle_mod, integrator):
    ic = inputs.taylor_green(32, seed=2, mach=0.3, nu=1e-3, eta=1e-3)
    ctx, o = make_pair(lib, oracle_mod, ic, integrator=integrator)
    lib.mhd_step(ctx, 50)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    o.step(50)
    for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state()):
        assert rel_l2(g, e) <= 1e-10
    assert abs(lib.mhd_diagnostics(ctx, 0)["t"] - o.diagnostics()["t"]) <= 1e-12 * o.diagnostics()["t"]


def test_df_batched_instances_match_separate_oracles(lib, oracle_mod):
    n = 32
    ics = [inputs.orszag_tang(n, seed=s, mach=m, nu=nu, eta=eta)
           for s, m, nu, eta in ((1, 0.1, 1e-2, 2e-3), (2, 0.3, 3e-3, 8e-3), (3, 0.05, 5e-3, 5e-3))]
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs) for ic in ics], precision=lib.MHD_FP64_DF)
    for i, ic in enumerate(ics):
        lib.mhd_set_state(ctx, i, ic.rho, ic.u, ic.b)
    lib.mhd_step(ctx, 40)
    for i, ic in enumerate(ics):
        o = oracle_mod.Oracle(n, ic.nu, ic.eta, ic.cs)
        o.set_state(ic.rho, ic.u, ic.b)
        o.step(40)
        for g, e in zip(lib.mhd_get_state(ctx, i), o.get_state()):
            assert rel_l2(g, e) <= 1e-10
        assert abs(lib.mhd_diagnostics(ctx, i)["t"] - o.diagnostics()["t"]) <= 1e-12 * o.diagnostics()["t"]


def test_df_checkpoint_restore_is_bitwise(lib):
    ic = random_state(32, 5)
    ctx = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=lib.MHD_FP64_DF)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    lib.mhd_step(ctx, 7)
    ck = lib.mhd_checkpoint(ctx, 0)
    lib.mhd_step(ctx, 5)
    a = lib.mhd_get_state(ctx, 0)
    lib.mhd_restore(ctx, 0, ck)
    lib.mhd_step(ctx, 5)
    for g, e in zip(lib.mhd_get_state(ctx, 0), a):
        assert np.array_equal(g, e)
    lib.mhd_destroy(ctx)


def test_df_forced_steps_match_oracle(lib, oracle_mod):
    ic = inputs.energy_exchange(32, "abc", seed=1)
    forcing = (0.2, 1.0, 1.0, 1.0, 1)
    ctx = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=lib.MHD_FP64_DF, integrator=1)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    lib.mhd_set_forcing(ctx, 0, *forcing)
    o = oracle_mod.Oracle(32, ic.nu, ic.eta, ic.cs, integrator=1, forcing=forcing)
    o.set_state(ic.rho, ic.u, ic.b)
    lib.mhd_step(ctx, 20)
    o.step(20)
    for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state()):
        assert rel_l2(g, e) <= 1e-10


def test_df_pool_run_equals_context_run(lib):
    """A run served from a double-float pool next to another run gives bitwise what a
    double-float context gives for it alone."""
    a, b = inputs.orszag_tang(32, seed=4), inputs.abc_dynamo(32, seed=5, b_energy=1e-2)
    pool = lib.mhd_pool_create(32, 3, precision=lib.MHD_FP64_DF)
    sa = lib.mhd_pool_admit(pool, (a.nu, a.eta, a.cs), a.rho, a.u, a.b, 12)
    sb = lib.mhd_pool_admit(pool, (b.nu, b.eta, b.cs), b.rho, b.u, b.b, 30)
    for _ in range(6):
        lib.mhd_pool_step(pool, 5)
    got = lib.mhd_pool_retire(pool, sa)
    lib.mhd_pool_destroy(pool)
    ctx = lib.mhd_init(32, [(a.nu, a.eta, a.cs)], precision=lib.MHD_FP64_DF)
    lib.mhd_set_state(ctx, 0, a.rho, a.u, a.b)
    lib.mhd_step(ctx, 12)
    for g, e in zip(got, lib.mhd_get_state(ctx, 0)):
        assert np.array_equal(g, e)
    lib.mhd_destroy(ctx)
