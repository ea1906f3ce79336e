"""The pins catch plausible mistakes: each case plants one mistake in a copy of the oracle's source
(on the CPU, in a temporary directory), builds it, and checks that at least one pin fails on it.
The unmodified source passes the same battery."""
import os
import subprocess

import numpy as np
import pytest
import sympy as sp

import test_oracle_golden as gold
import test_oracle_integrators as integ
import test_oracle_invariants as inv
import test_oracle_linear_waves as lw
import test_oracle_rhs_closed_form as rc
import test_oracle_spectra as spec
import test_oracle_tracers as trc
from paper_1810_12707_gb300.inputs import grid

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "mhd_oracle.c")

# (name, text in the source, replacement)
MUTANTS = [
    ("continuity sign", "out[F_RHO][i] = -I *", "out[F_RHO][i] = I *"),
    ("pressure sign", "- I * k[a] * cs2 * rho", "+ I * k[a] * cs2 * rho"),
    ("magnetic pressure dropped", "m[0] * u[0] + 0.5 * b2 - B[0] * B[0]", "m[0] * u[0] - B[0] * B[0]"),
    ("magnetic tension sign", "m[0] * u[1] - B[0] * B[1]", "m[0] * u[1] + B[0] * B[1]"),
    ("emf component swapped", "u[1] * B[2] - u[2] * B[1]", "u[2] * B[1] - u[1] * B[2]"),
    ("curl index", "I * (k[1] * Eh[2] - k[2] * Eh[1])", "I * (k[2] * Eh[2] - k[1] * Eh[1])"),
    ("viscosity on m not u", "- nu * k2 * uh[a]", "- nu * k2 * mh[a]"),
    ("resistivity sign", "curlE[a] - eta * k2", "curlE[a] + eta * k2"),
    ("mask one mode too wide", "return 3 * absindex(mx, n) < n &&", "return 3 * absindex(mx, n) < n + 3 &&"),
    ("half rule instead of two-thirds", "3 * absindex(mz, n) < n;", "2 * absindex(mz, n) < n;"),
    ("AB2 variable-step weight", "a0 = -0.5 * r;", "a0 = -0.5;"),
    ("AB2 first step not Euler", "double a1 = 1.0, a0 = 0.0;", "double a1 = 1.5, a0 = 0.0;"),
    ("forward normalisation", "const double s = 1.0 / (double)n3;", "const double s = 1.0 / (double)(n3 / n);"),
    ("twiddle sign", "return cos(ang) + (double)sign * sin(ang) * I;", "return cos(ang) - (double)sign * sin(ang) * I;"),
    ("CFL uses c_s only", "const double cf = sqrt(cs2 + b2 / rho);", "const double cf = sqrt(cs2);"),
    ("RK4 stage weights", "st < 2 ? 2.0 : 1.0", "st < 2 ? 1.0 : 2.0"),
    ("RK4 stage point", "const double cstage[3] = {0.5, 0.5, 1.0};", "const double cstage[3] = {0.5, 1.0, 1.0};"),
    ("PC corrector weight", "y[i] + 0.5 * dt * (fn[i] + fs[i])", "y[i] + dt * (fn[i] + fs[i])"),
    ("force component swapped", "rho * F * (A * sin(kf * Z) + C * cos(kf * Y))", "rho * F * (C * sin(kf * Z) + A * cos(kf * Y))"),
    ("force without density", "c->rflux[1][i] = rho * F *", "c->rflux[1][i] = F *"),
    ("shell by floor not round", "sqrt(kx * kx + ky * ky + kz * kz) + 0.5)", "sqrt(kx * kx + ky * ky + kz * kz))"),
    ("spectrum of m not u", "g[i] = c->real[F_MX + a][i] / c->real[F_RHO][i];", "g[i] = c->real[F_MX + a][i];"),
    ("magnetic spectrum without 1/2", "em[sh] += 0.5 *", "em[sh] += 1.0 *"),
    ("divergence drops z", "wavenumber(y, n) * uh[1][i] + wavenumber(z, n) * uh[2][i]", "wavenumber(y, n) * uh[1][i]"),
    ("skewness exponent", "m3 / pow(m2, 1.5)", "m3 / pow(m2, 1.0)"),
    ("CIC corner weight", "G(i0, j1, k1) * ux * ly * lz", "G(i0, j1, k1) * lx * ly * uz"),
    ("CIC cell from rounding", "const int i = (int)floor(x / h)", "const int i = (int)floor(x / h + 0.5)"),
    ("Boris half step", "t[a] = B[a] * dt / 2.0;", "t[a] = B[a] * dt;"),
    ("Boris s factor", "s[a] = 2.0 * t[a] / (1.0 + t2);", "s[a] = t[a];"),
    ("Boris cross sign", "vd[1] = v[1] + (v[2] * t[0] - v[0] * t[2]);", "vd[1] = v[1] - (v[2] * t[0] - v[0] * t[2]);"),
    ("kinetic energy without 1/2", "s[0] += 0.5 * rho * u2;", "s[0] += rho * u2;"),
    ("kinetic energy without density", "s[0] += 0.5 * rho * u2;", "s[0] += 0.5 * u2;"),
    ("magnetic energy without 1/2", "s[1] += 0.5 * b2;", "s[1] += b2;"),
    ("helicity curl sign", "cplx v = I * (k[b1] * f2 - k[b2] * f1);", "cplx v = I * (k[b2] * f1 - k[b1] * f2);"),
    ("magnetic helicity without 1/k^2", "if (pass == 1) v = k2 > 0.0 ? v / k2 : 0.0;", "if (pass == 1) v = k2 > 0.0 ? v : 0.0;"),
    ("div B max drops y", "c->tmp[i] = I * (wavenumber(x, n) * c->state[F_BX][i] + wavenumber(y, n) * c->state[F_BY][i]",
     "c->tmp[i] = I * (wavenumber(x, n) * c->state[F_BX][i] + 0.0 * c->state[F_BY][i]"),
    ("internal energy without Cs^2", "s[2] += cs2 * rho * log(rho);", "s[2] += rho * log(rho);"),
    ("mean speed of m", "s[4] += sqrt(u2);", "s[4] += sqrt(u2) * rho;"),
    ("diagnostic fast speed without B", "const double v = sqrt(u2) + sqrt(cs2 + b2 / rho);",
     "const double v = sqrt(u2) + sqrt(cs2);"),
    ("position with old velocity", "v[a] = vn[a];\n      p[a] = wrap_2pi(p[a] + vn[a] * dt);",
     "p[a] = wrap_2pi(p[a] + v[a] * dt);\n      v[a] = vn[a];"),
]


def _build(tmp_path, text, repl):
    src = open(SRC).read()
    assert src.count(text) == 1, text
    path = tmp_path / "m.c"
    path.write_text(src.replace(text, repl))
    so = tmp_path / "libm.so"
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(so), str(path), "-lm"], check=True)
    return str(so)


def _battery(om, lib):
    """Return the list of pins that fail for the oracle build `lib`."""
    failed = []
    # closed-form RHS of a mixed trigonometric state
    n = 32
    cs, nu, eta = 1.7, 0.03, 0.05
    rho_e, u_e, B_e = rc.STATES["mixed"]
    exact = [rc.on_grid(e, n) for e in rc.continuum_rhs(rho_e, u_e, B_e, cs, nu, eta)]
    o = om.Oracle(n, nu, eta, cs, dt=1e-3, lib=lib)
    o.set_state(rc.on_grid(rho_e, n), np.stack([rc.on_grid(e, n) for e in u_e]),
                np.stack([rc.on_grid(e, n) for e in B_e]))
    drho, dm, db = o.rhs()
    got = [drho, *dm, *db]
    scale = max(np.max(np.abs(e)) for e in exact)
    if any(np.max(np.abs(g - e)) > 1e-12 * scale for g, e in zip(got, exact)):
        failed.append("closed form")
    # mask: a product landing on aliased indices
    n = 16
    X = grid(n)[0]
    o = om.Oracle(n, 0.01, 0.02, 1.1, dt=1e-3, lib=lib)
    u = np.zeros((3, n, n, n))
    u[0] = np.cos(4 * X) + np.cos(5 * X)
    o.set_state(np.ones((n, n, n)), u, np.zeros((3, n, n, n)))
    _, dm, _ = o.rhs()
    if np.max(np.abs(dm[0] - (np.sin(X) - 0.01 * (16 * np.cos(4 * X) + 25 * np.cos(5 * X))))) > 1e-11:
        failed.append("mask")
    # sound wave with a CFL (variable) step
    k, cs, nu = 2, 1.3, 0.02
    o = om.Oracle(n, nu, 0.01, cs, dt=0.0, lib=lib)
    o.set_state(1.0 + lw.EPS * np.cos(k * X), np.zeros((3, n, n, n)), np.zeros((3, n, n, n)))
    dts = lw.run_oracle(o, 30, False)
    A = np.array([[0, -1j * k], [-1j * k * cs ** 2, -nu * k * k]])
    y = lw.ab2_linear(A, [lw.EPS / 2, 0.0], dts)
    i = lw.idx(n, 0, k)
    gotw = np.array([o.spectrum(0)[i], o.spectrum(1)[i]])
    if not np.all(np.isfinite(gotw)) or np.max(np.abs(gotw - y)) > 1e-5 * np.max(np.abs(y)):
        failed.append("sound wave")
    # CFL formula on a magnetised state
    o = om.Oracle(n, 0.001, 0.001, 0.5, dt=0.0, lib=lib)
    b = np.zeros((3, n, n, n))
    b[2] = 2.0
    o.set_state(np.ones((n, n, n)), np.zeros((3, n, n, n)), b)
    o.step(1)
    expect = 0.2 * (2 * np.pi / n) / np.sqrt(0.25 + 4.0)
    if abs(o.diagnostics()["dt"] - expect) > 1e-12 * expect:
        failed.append("cfl")
    # RK4 and predictor-corrector on the sound wave
    for method in (integ.RK4, integ.PC):
        o = om.Oracle(n, nu, 0.01, cs, dt=0.01, lib=lib, integrator=method)
        o.set_state(1.0 + lw.EPS * np.cos(k * X), np.zeros((3, n, n, n)), np.zeros((3, n, n, n)))
        o.step(30)
        y = integ.linear_run(A, [lw.EPS / 2, 0.0], [0.01] * 30, method)
        gotm = np.array([o.spectrum(0)[i], o.spectrum(1)[i]])
        if not np.all(np.isfinite(gotm)) or np.max(np.abs(gotm - y)) > 1e-5 * np.max(np.abs(y)):
            failed.append(f"integrator {method}")
    # variable-step Adams-Bashforth against the integral of its interpolant
    if not check_variable_step(om, lib):
        failed.append("variable step")
    # ABC body force on a non-uniform density
    rho_e, u_e, B_e = rc.STATES["mixed"]
    f = rc.abc_force(0.7, 1.0, 0.6, 0.3, 1)
    ex = rc.continuum_rhs(rho_e, u_e, B_e, 1.7, 0.03, 0.05)
    ex = [rc.on_grid(e, 32) for e in [ex[0]] + [ex[1 + a] + rho_e * f[a] for a in range(3)] + ex[4:]]
    o = om.Oracle(32, 0.03, 0.05, 1.7, dt=1e-3, lib=lib, forcing=(0.7, 1.0, 0.6, 0.3, 1))
    o.set_state(rc.on_grid(rho_e, 32), np.stack([rc.on_grid(e, 32) for e in u_e]),
                np.stack([rc.on_grid(e, 32) for e in B_e]))
    drho, dm, db = o.rhs()
    if any(np.max(np.abs(g - e)) > 1e-11 * 10 for g, e in zip([drho, *dm, *db], ex)):
        failed.append("forcing")
    # the z-axis mask on aliased indices
    Z = grid(n)[2]
    o = om.Oracle(n, 0.01, 0.02, 1.1, dt=1e-3, lib=lib)
    u = np.zeros((3, n, n, n))
    u[2] = np.cos(4 * Z) + np.cos(5 * Z)
    o.set_state(np.ones((n, n, n)), u, np.zeros((3, n, n, n)))
    _, dm, _ = o.rhs()
    if np.max(np.abs(dm[2] - (np.sin(Z) - 0.01 * (16 * np.cos(4 * Z) + 25 * np.cos(5 * Z))))) > 1e-11:
        failed.append("mask z")
    # spectra, theta' and S_3
    failed += spec.closed_form_failures(om, lib)
    failed += spec.brute_force_failures(om, lib)
    # tracer particles
    failed += trc.interpolation_failures(om, lib)
    failed += trc.push_failures(om, lib)
    # exact averages of the paper's initial flows
    failed += gold.golden_failures(om, lib)
    return failed


def check_variable_step(om, lib):
    w = inv.check_variable_step_update(om, lib, nsteps=4)
    return np.isfinite(w) and w <= 1e-10


def test_unmodified_oracle_passes_battery(oracle_mod):
    assert _battery(oracle_mod, oracle_mod._load()) == []


@pytest.mark.parametrize("name,text,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle_mod, tmp_path, name, text, repl):
    lib = oracle_mod.load_library(_build(tmp_path, text, repl))
    assert _battery(oracle_mod, lib) != [], f"mistake '{name}' slipped through every pin"
