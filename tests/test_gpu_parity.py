"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP64; both sides round differently inside the FFTs, so agreement is to a small
multiple of the transform error, about log2(N^3) * 1e-16 relative per transform):
  * state round trip, spectra, one RHS: max abs error <= 1e-12 of the field's max;
  * 100 steps: relative L2 error per physical field (rho, m, B) <= 1e-10;
  * diagnostics: relative error <= 1e-11.
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


def make_pair(lib, oracle_mod, ic, dt=0.0):
    ctx = lib.mhd_init(ic.n, [(ic.nu, ic.eta, ic.cs)], dt=dt)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    o = oracle_mod.Oracle(ic.n, ic.nu, ic.eta, ic.cs, dt=dt)
    o.set_state(ic.rho, ic.u, ic.b)
    return ctx, o


def random_state(n, seed, amp=0.2):
    rng = np.random.default_rng(seed)
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + amp * np.cos(X + 2 * Y) * np.sin(Z - 0.3) + 0.05 * np.sin(3 * Y - Z)
    u = inputs.random_solenoidal(n, rng, kmax2=9)
    u /= inputs.rms(u)
    b = inputs.random_solenoidal(n, rng, kmax2=9)
    b *= 0.7 / inputs.rms(b)
    return inputs.InitialCondition(rho, u, b, 0.013, 0.021, 1.7, "random")


@pytest.mark.parametrize("n", [16, 32, 64])
def test_set_get_roundtrip_and_spectrum(lib, oracle_mod, n):
    ic = random_state(n, n)
    ctx, o = make_pair(lib, oracle_mod, ic)
    r, m, b = lib.mhd_get_state(ctx, 0)
    ro, mo, bo = o.get_state()
    for g, e in ((r, ro), (m, mo), (b, bo)):
        assert maxrel(g, e) <= 1e-12
    for f in range(7):
        spec = lib.mhd_get_spectrum(ctx, 0, f)
        ref = o.spectrum(f)[:, :, : n // 2 + 1]
        assert np.max(np.abs(spec - ref)) <= 1e-13 * max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_rhs_matches_oracle(lib, oracle_mod, n):
    ic = random_state(n, 100 + n)
    ctx, o = make_pair(lib, oracle_mod, ic)
    got = lib.mhd_rhs(ctx, 0)
    ref = o.rhs()
    for g, e in zip(got, ref):
        assert maxrel(g, e) <= 1e-12, maxrel(g, e)


def test_orszag_tang_100_fixed_steps(lib, oracle_mod):
    """N = 32, FP64, Orszag-Tang-type IC with seeded 1e-3 perturbation, Mach 0.1,
    nu = eta = 1e-2, fixed dt = 1e-3, 100 steps."""
    ic = inputs.orszag_tang(32, seed=0)
    ctx, o = make_pair(lib, oracle_mod, ic, dt=1e-3)
    lib.mhd_step(ctx, 100)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    o.step(100)
    for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state()):
        assert rel_l2(g, e) <= 1e-10
    dg, do = lib.mhd_diagnostics(ctx, 0), o.diagnostics()
    assert dg["step"] == 100 and abs(dg["t"] - do["t"]) <= 1e-14
    for k in ("ke", "me", "eint", "cross_hel", "mean_speed", "mean_bmag", "smax"):
        assert abs(dg[k] - do[k]) <= 1e-11 * max(abs(do[k]), 1e-300), k


@pytest.mark.parametrize("n", [32, 64])
def test_cfl_steps(lib, oracle_mod, n):
    ic = random_state(n, 7 + n)
    ctx, o = make_pair(lib, oracle_mod, ic, dt=0.0)
    lib.mhd_step(ctx, 30)
    o.step(30)
    dg, do = lib.mhd_diagnostics(ctx, 0), o.diagnostics()
    assert abs(dg["t"] - do["t"]) <= 1e-12 * do["t"]
    assert abs(dg["dt"] - do["dt"]) <= 1e-12 * do["dt"]
    for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state()):
        assert rel_l2(g, e) <= 1e-10


def test_batched_instances_match_separate_oracles(lib, oracle_mod):
    n = 32
    ics = [inputs.orszag_tang(n, seed=s, mach=m, nu=nu, eta=eta)
           for s, m, nu, eta in ((1, 0.1, 1e-2, 2e-3), (2, 0.3, 3e-3, 8e-3), (3, 0.05, 5e-3, 5e-3))]
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs) for ic in ics], dt=0.0)
    for i, ic in enumerate(ics):
        lib.mhd_set_state(ctx, i, ic.rho, ic.u, ic.b)
    lib.mhd_step(ctx, 20)
    for i, ic in enumerate(ics):
        o = oracle_mod.Oracle(n, ic.nu, ic.eta, ic.cs)
        o.set_state(ic.rho, ic.u, ic.b)
        o.step(20)
        for g, e in zip(lib.mhd_get_state(ctx, i), o.get_state()):
            assert rel_l2(g, e) <= 1e-10
        assert abs(lib.mhd_diagnostics(ctx, i)["t"] - o.diagnostics()["t"]) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_restore_is_bitwise(lib, precision):
    ic = inputs.orszag_tang(32, seed=5)
    a = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=precision)
    lib.mhd_set_state(a, 0, ic.rho, ic.u, ic.b)
    lib.mhd_step(a, 20)
    ref = lib.mhd_get_state(a, 0)
    b = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=precision)
    lib.mhd_set_state(b, 0, ic.rho, ic.u, ic.b)
    lib.mhd_step(b, 10)
    ck = lib.mhd_checkpoint(b, 0)
    c = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=precision)
    lib.mhd_restore(c, 0, ck)
    lib.mhd_step(c, 10)
    for g, e in zip(lib.mhd_get_state(c, 0), ref):
        assert np.array_equal(g, e)
    assert lib.mhd_diagnostics(c, 0)["step"] == 20


@pytest.mark.parametrize("precision", [0, 1])
def test_runs_are_deterministic(lib, precision):
    ic = random_state(32, 3)
    out = []
    for _ in range(2):
        ctx = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=precision)
        lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
        lib.mhd_step(ctx, 10)
        out.append(lib.mhd_get_state(ctx, 0))
    for g, e in zip(*out):
        assert np.array_equal(g, e)


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_instance_stops_and_reports(lib, precision):
    n = 16
    ic = random_state(n, 4)
    rho = ic.rho.copy()
    rho[3, 4, 5] = np.nan  # spreads to every mode of the projected state
    ctx = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs), (ic.nu, ic.eta, ic.cs)], precision=precision)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    lib.mhd_set_state(ctx, 1, rho, ic.u, ic.b)
    before = lib.mhd_checkpoint(ctx, 1)
    lib.mhd_step(ctx, 3)
    assert lib.mhd_synchronize(ctx) == lib.MHD_ENONFINITE
    assert lib.mhd_diagnostics(ctx, 0)["status"] == 0 and lib.mhd_diagnostics(ctx, 0)["step"] == 3
    d1 = lib.mhd_diagnostics(ctx, 1)
    assert d1["status"] == lib.MHD_ENONFINITE and d1["step"] == 0
    after = lib.mhd_checkpoint(ctx, 1)
    assert np.array_equal(before[:-8], after[:-8], equal_nan=True)  # state and history untouched


def test_invalid_arguments_are_rejected(lib):
    with pytest.raises(lib.MhdError):
        lib.mhd_init(48, [(1e-3, 1e-3, 1.0)])
    with pytest.raises(lib.MhdError):
        lib.mhd_init(32, [(1e-3, 1e-3, 0.0)])
    ctx = lib.mhd_init(16, [(1e-3, 1e-3, 1.0)])
    with pytest.raises(lib.MhdError):
        lib.mhd_step(ctx, 1)  # no state yet
    with pytest.raises(lib.MhdError):
        lib.mhd_get_state(ctx, 1)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_direct_launches(lib, precision):
    ic = random_state(32, 21)
    out = []
    for graph in (0, 1):
        ctx = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], precision=precision)
        lib.mhd_set_option(ctx, lib.MHD_OPT_CUDA_GRAPH, graph)
        lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
        lib.mhd_step(ctx, 3)
        lib.mhd_step(ctx, 9)
        out.append(lib.mhd_get_state(ctx, 0))
        assert lib.mhd_diagnostics(ctx, 0)["step"] == 12
    for g, e in zip(*out):
        assert np.array_equal(g, e)


def test_tile_options_leave_results_bitwise_unchanged(lib):
    ic = random_state(64, 22)
    out = []
    for tiles in ((0, 0, 0, 0), (3, 5, 7, 64), (1, 1, 1, 1)):
        ctx = lib.mhd_init(64, [(ic.nu, ic.eta, ic.cs)], precision=1)
        for opt, v in zip((lib.MHD_OPT_TILE_INV_Z, lib.MHD_OPT_TILE_INV_Y, lib.MHD_OPT_TILE_FWD_Y,
                           lib.MHD_OPT_TILE_FWD_Z), tiles):
            lib.mhd_set_option(ctx, opt, v)
        lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
        lib.mhd_step(ctx, 5)
        out.append(lib.mhd_get_state(ctx, 0))
    for other in out[1:]:
        for g, e in zip(other, out[0]):
            assert np.array_equal(g, e)
    with pytest.raises(lib.MhdError):
        lib.mhd_set_option(ctx, lib.MHD_OPT_TILE_INV_Z, 65)


@pytest.mark.parametrize("precision", [0, 1])
def test_instance_result_is_the_same_alone_and_in_a_batch(lib, precision):
    """Every kernel treats instances independently, so a run in a batch of different instances is
    bitwise the run alone."""
    n = 32
    ics = [inputs.orszag_tang(n, seed=s, mach=m, nu=nu, eta=eta)
           for s, m, nu, eta in ((7, 0.1, 1e-2, 2e-3), (8, 0.4, 3e-3, 8e-3), (9, 0.05, 5e-3, 1e-3), (10, 0.2, 1e-3, 1e-3))]
    mix = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs) for ic in ics], precision=precision)
    for i, ic in enumerate(ics):
        lib.mhd_set_state(mix, i, ic.rho, ic.u, ic.b)
    lib.mhd_step(mix, 15)
    for i, ic in enumerate(ics):
        alone = lib.mhd_init(n, [(ic.nu, ic.eta, ic.cs)], precision=precision)
        lib.mhd_set_state(alone, 0, ic.rho, ic.u, ic.b)
        lib.mhd_step(alone, 15)
        for g, e in zip(lib.mhd_get_state(mix, i), lib.mhd_get_state(alone, 0)):
            assert np.array_equal(g, e)


@pytest.mark.parametrize("integrator", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_rk4_and_predictor_corrector_match_oracle(lib, oracle_mod, integrator, precision):
    """The paper's other two time solvers, through the same kernels: FP64 to 1e-10, the mixed mode
    to 1e-5 (relative L2 per field after 30 CFL steps)."""
    ic = random_state(32, 40 + integrator)
    ctx = lib.mhd_init(32, [(ic.nu, ic.eta, ic.cs)], integrator=integrator, precision=precision)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    lib.mhd_step(ctx, 30)
    assert lib.mhd_synchronize(ctx) == lib.MHD_OK
    o = oracle_mod.Oracle(32, ic.nu, ic.eta, ic.cs, integrator=integrator)
    o.set_state(ic.rho, ic.u, ic.b)
    o.step(30)
    tol = 1e-10 if precision == 0 else 1e-5
    for g, e in zip(lib.mhd_get_state(ctx, 0), o.get_state()):
        assert rel_l2(g, e) <= tol
    dg, do = lib.mhd_diagnostics(ctx, 0), o.diagnostics()
    assert dg["step"] == 30 and abs(dg["t"] - do["t"]) <= (1e-12 if precision == 0 else 1e-6) * do["t"]
