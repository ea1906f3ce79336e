"""Pins of the oracle against properties that the paper's equations fix exactly.

* conservation form: the k = 0 modes of rho, m and B never change (their RHS is 0 * (...));
* div B = 0 is kept to round-off (the induction RHS is a curl);
* a z-independent state with u_z = B_z = 0 stays so (2D invariance of the 3D system);
* translation by one grid cell commutes with a step (no preferred position on the periodic box);
* total energy ke + me + Cs^2 <rho ln rho> decays with nu, eta > 0, and in the ideal limit its drift
  falls as the second power of dt (second-order integrator);
* the time integrator converges at second order in dt on a nonlinear state;
* the CFL step equals the formula evaluated independently on the state;
* diagnostics equal their definitions evaluated with numpy on the real-space state.
"""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs


def smooth_state(n, seed, amp_rho=0.1, b_scale=0.5):
    rng = np.random.default_rng(seed)
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + amp_rho * np.cos(X + 2 * Y) * np.sin(Z) + 0.05 * np.sin(Y - Z)
    u = inputs.random_solenoidal(n, rng, kmax2=4)
    u /= inputs.rms(u)
    b = inputs.random_solenoidal(n, rng, kmax2=4)
    b *= b_scale / inputs.rms(b)
    return rho, u, b


def test_k0_modes_are_bitwise_conserved(oracle_mod):
    n = 16
    rho, u, b = smooth_state(n, 1)
    o = oracle_mod.Oracle(n, 0.01, 0.02, 2.0, dt=0.0)
    o.set_state(rho, u, b)
    before = [o.spectrum(f)[0, 0, 0] for f in range(7)]
    o.step(15)
    after = [o.spectrum(f)[0, 0, 0] for f in range(7)]
    assert before == after
    # and they are the means of the real-space fields
    r, m, bb = o.get_state()
    assert abs(before[0] - r.mean()) < 1e-14
    assert all(abs(before[1 + d] - m[d].mean()) < 1e-14 for d in range(3))


def test_div_b_stays_at_roundoff(oracle_mod):
    n = 16
    rho, u, b = smooth_state(n, 2)
    o = oracle_mod.Oracle(n, 0.01, 0.01, 2.0, dt=0.0)
    o.set_state(rho, u, b)
    b_rms = inputs.rms(b)
    for _ in range(4):
        o.step(5)
        d = o.diagnostics()
        assert d["divb_rms"] <= 1e-13 * b_rms


def test_two_dimensional_state_stays_two_dimensional(oracle_mod):
    n = 16
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + 0.1 * np.cos(X) * np.sin(2 * Y)
    u = np.stack([-np.sin(Y), np.sin(X), np.zeros_like(X)])
    b = np.stack([-np.sin(Y), np.sin(2 * X), np.zeros_like(X)])
    o = oracle_mod.Oracle(n, 0.01, 0.01, 3.0, dt=0.0)
    o.set_state(rho, u, b)
    o.step(20)
    r, m, bb = o.get_state()
    assert np.max(np.abs(m[2])) <= 1e-15 and np.max(np.abs(bb[2])) <= 1e-15
    for f in (r, m[0], m[1], bb[0], bb[1]):
        assert np.max(np.abs(f - f[:1])) <= 1e-13 * np.max(np.abs(f))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_translation_commutes_with_step(oracle_mod, axis):
    n = 16
    rho, u, b = smooth_state(n, 3)
    ax = 2 - axis  # array axis of the coordinate
    o1 = oracle_mod.Oracle(n, 0.01, 0.02, 2.0, dt=0.0)
    o1.set_state(rho, u, b)
    o1.step(6)
    o2 = oracle_mod.Oracle(n, 0.01, 0.02, 2.0, dt=0.0)
    o2.set_state(np.roll(rho, 1, axis=ax), np.roll(u, 1, axis=ax + 1), np.roll(b, 1, axis=ax + 1))
    o2.step(6)
    for a, c in zip(o1.get_state(), o2.get_state()):
        shift_ax = ax if a.ndim == 3 else ax + 1
        assert np.max(np.abs(np.roll(a, 1, axis=shift_ax) - c)) <= 1e-12 * np.max(np.abs(a))


def test_energy_decays_with_dissipation(oracle_mod):
    n = 16
    rho, u, b = smooth_state(n, 4)
    o = oracle_mod.Oracle(n, 0.02, 0.02, 2.0, dt=0.0)
    o.set_state(rho, u, b)
    e = [o.diagnostics()["etot"]]
    for _ in range(10):
        o.step(3)
        e.append(o.diagnostics()["etot"])
    assert all(e1 < e0 for e0, e1 in zip(e, e[1:]))


def _run_fixed(oracle_mod, n, state, nu, eta, cs, dt, t_end):
    o = oracle_mod.Oracle(n, nu, eta, cs, dt=dt)
    o.set_state(*state)
    e0 = o.diagnostics()["etot"]
    o.step(int(round(t_end / dt)))
    return o, e0


def test_ab2_converges_at_second_order(oracle_mod):
    n = 16
    state = smooth_state(n, 5)
    sols = []
    for dt in (0.004, 0.002, 0.001, 0.0005):
        o, _ = _run_fixed(oracle_mod, n, state, 0.01, 0.01, 2.0, dt, 0.08)
        sols.append(np.concatenate([np.ravel(a) for a in o.get_state()]))
    d = [np.linalg.norm(a - c) for a, c in zip(sols, sols[1:])]
    ratios = [d0 / d1 for d0, d1 in zip(d, d[1:])]
    assert all(3.6 < r < 4.4 for r in ratios), ratios


def test_ideal_energy_drift_is_second_order(oracle_mod):
    """nu = eta = 0: the semi-discrete total energy is conserved up to the spatial truncation
    floor of a smooth state, so the drift of ke + me + eint over a fixed time shrinks by about 4
    per halving of dt."""
    n = 16
    state = smooth_state(n, 6, amp_rho=0.05, b_scale=0.3)
    drift = []
    for dt in (0.004, 0.002, 0.001):
        o, e0 = _run_fixed(oracle_mod, n, state, 0.0, 0.0, 2.0, dt, 0.1)
        drift.append(abs(o.diagnostics()["etot"] - e0))
    ratios = [a / b for a, b in zip(drift, drift[1:])]
    assert all(3.0 < r < 5.0 for r in ratios), (drift, ratios)


def test_cfl_step_matches_formula(oracle_mod):
    n = 16
    rho, u, b = smooth_state(n, 7)
    for nu, cs in ((0.001, 2.0), (0.3, 0.5)):  # advective limit, then viscous limit
        o = oracle_mod.Oracle(n, nu, 0.5 * nu, cs, dt=0.0, cfl_adv=0.2, cfl_visc=0.5)
        o.set_state(rho, u, b)
        r, m, bb = o.get_state()
        uu = m / r
        s = np.sqrt(np.sum(uu * uu, axis=0)) + np.sqrt(cs * cs + np.sum(bb * bb, axis=0) / r)
        kmax = (n - 1) // 3
        expect = min(0.2 * (2 * np.pi / n) / s.max(), 0.5 / (nu * kmax * kmax))
        o.step(1)
        assert abs(o.diagnostics()["dt"] - expect) <= 1e-14 * expect


def test_diagnostics_match_definitions(oracle_mod):
    n = 16
    rho, u, b = smooth_state(n, 8)
    cs = 1.5
    o = oracle_mod.Oracle(n, 0.01, 0.01, cs, dt=0.0)
    o.set_state(rho, u, b)
    o.step(3)
    d = o.diagnostics()
    r, m, bb = o.get_state()
    uu = m / r
    u2 = np.sum(uu * uu, axis=0)
    b2 = np.sum(bb * bb, axis=0)
    ref = {
        "ke": np.mean(0.5 * r * u2), "me": np.mean(0.5 * b2), "eint": np.mean(cs * cs * r * np.log(r)),
        "cross_hel": np.mean(np.sum(uu * bb, axis=0)), "mean_speed": np.mean(np.sqrt(u2)),
        "mean_bmag": np.mean(np.sqrt(b2)), "smax": np.max(np.sqrt(u2) + np.sqrt(cs * cs + b2 / r)),
        "mean_rho": r.mean(), "mean_mx": m[0].mean(), "mean_bz": bb[2].mean(),
    }
    for k, v in ref.items():
        assert abs(d[k] - v) <= 1e-13 * max(1.0, abs(v)), k
    # div B from the real-space state by the spectral derivative of numpy's FFT
    kk = np.fft.fftfreq(n, 1.0 / n)
    kk[n // 2] = 0.0
    KZ, KY, KX = np.meshgrid(kk, kk, kk, indexing="ij")
    bh = [np.fft.fftn(c) / n ** 3 for c in bb]
    div = 1j * (KX * bh[0] + KY * bh[1] + KZ * bh[2])
    assert abs(d["divb_rms"] - np.sqrt(np.sum(np.abs(div) ** 2))) <= 1e-14 + 1e-12 * d["divb_rms"]
    assert d["step"] == 3 and d["t"] > 0


def ab_weights_from_interpolant(dt, dt_prev):
    """Weights (w_n, w_{n-1}) with y^{n+1} - y^n = dt (w_n f^n + w_{n-1} f^{n-1}), obtained by
    integrating over [t_n, t_n + dt] the straight line through (t_n - dt_prev, f^{n-1}) and
    (t_n, f^n) -- the definition of the two-step Adams-Bashforth method."""
    import sympy as sp
    t, fn, fo = sp.symbols("t f_n f_o")
    line = fn + (fn - fo) * t / sp.Rational(dt_prev)
    integral = sp.integrate(line, (t, 0, sp.Rational(dt)))
    return (float(sp.diff(integral, fn)) / dt, float(sp.diff(integral, fo)) / dt)


def check_variable_step_update(om, lib=None, nsteps=6):
    """Run a nonlinear state in CFL mode and check every update against the interpolant weights
    (forward Euler on the first step).  Returns the largest relative mismatch."""
    n = 16
    rho, u, b = smooth_state(n, 9, amp_rho=0.3, b_scale=1.0)
    o = om.Oracle(n, 0.01, 0.01, 1.0, dt=0.0, lib=lib)
    o.set_state(rho, u, b)
    worst = 0.0
    f_prev = dt_prev = None
    for _ in range(nsteps):
        y0 = [o.spectrum(f) for f in range(7)]
        fn = [o.rhs_spectrum(f) for f in range(7)]
        o.step(1)
        dt = o.diagnostics()["dt"]
        if f_prev is None:
            wn, wo = 1.0, 0.0
        else:
            wn, wo = ab_weights_from_interpolant(dt, dt_prev)
        for f in range(7):
            pred = y0[f] + dt * (wn * fn[f] + wo * (f_prev[f] if f_prev else 0.0))
            scale = np.max(np.abs(dt * fn[f])) + 1e-300
            worst = max(worst, np.max(np.abs(o.spectrum(f) - pred)) / scale)
        f_prev, dt_prev = fn, dt
    return worst


def test_variable_step_ab2_is_the_interpolant_integral(oracle_mod):
    assert check_variable_step_update(oracle_mod) <= 1e-10
