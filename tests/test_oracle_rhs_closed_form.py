"""Pins of the oracle's right-hand side against the paper's equations written out symbolically.

For trigonometric states whose every product is a trigonometric polynomial inside the 2/3 mask
(rho, u and B of low degree), the pseudo-spectral RHS equals the continuum RHS up to rounding.  The
continuum RHS is built here with sympy from the component form of the equations (section "Governing
equations", the 3D system of section "Three dimensional numerical tests", Eqs. density, velocity,
Bfield): P_tot = Cs^2 rho + |B|^2/2 with no 4 pi factors, viscosity mu lap(u), and the induction
component form with its signs exactly as printed.  Nothing here calls the oracle's arithmetic.

A second set of states puts products outside the mask (and onto aliased indices) to pin the 2/3
rule: the oracle RHS must equal the continuum RHS with every mode outside the mask removed.
"""
import numpy as np
import pytest
import sympy as sp

from paper_1810_12707_gb300.inputs import grid

x, y, z = sp.symbols("x y z", real=True)
X_ = (x, y, z)


def continuum_rhs(rho, u, B, cs, nu, eta):
    """d/dt of (rho, m_x, m_y, m_z, B_x, B_y, B_z) for the paper's 3D system, symbolically."""
    d = sp.diff
    lap = lambda f: d(f, x, 2) + d(f, y, 2) + d(f, z, 2)
    m = [rho * ui for ui in u]
    ptot = cs ** 2 * rho + (B[0] ** 2 + B[1] ** 2 + B[2] ** 2) / 2
    drho = -(d(m[0], x) + d(m[1], y) + d(m[2], z))
    dm = []
    for i in range(3):
        # paper's component form: d(rho u_i)/dt + sum_j d_j[rho u_i u_j + delta_ij P_tot - B_i B_j] = mu lap u_i
        flux = [rho * u[i] * u[j] + (ptot if i == j else 0) - B[i] * B[j] for j in range(3)]
        dm.append(-(d(flux[0], x) + d(flux[1], y) + d(flux[2], z)) + nu * lap(u[i]))
    ux, uy, uz = u
    Bx, By, Bz = B
    # induction, component form as printed (signs included)
    dBx = (d(ux * By - uy * Bx, y) + d(ux * Bz - uz * Bx, z)) + eta * lap(Bx)
    dBy = -(d(ux * By - uy * Bx, x) - d(uy * Bz - uz * By, z)) + eta * lap(By)
    dBz = -(d(ux * Bz - uz * Bx, x) + d(uy * Bz - uz * By, y)) + eta * lap(Bz)
    return [drho] + dm + [dBx, dBy, dBz]


def on_grid(expr, n):
    X, Y, Z = grid(n)
    f = sp.lambdify((x, y, z), expr, "numpy")
    return np.broadcast_to(np.asarray(f(X, Y, Z), dtype=np.float64), X.shape).copy()


STATES = {
    # every axis carries different wavenumbers and phases, so a transposed operand or a wrong
    # axis shows up; rho > 0 everywhere
    "mixed": (
        2 + sp.cos(x) * sp.sin(2 * z) / 2 + sp.sin(y) / 3,
        [sp.sin(y) + sp.cos(2 * z) / 2, sp.cos(x) * sp.sin(z), sp.sin(2 * x) / 3 + sp.cos(y)],
        [sp.cos(z) + sp.sin(y) / 2, sp.sin(x) * sp.cos(2 * y) / 2 + sp.Rational(3, 10), sp.cos(x + y) / 4],
    ),
    # the same kind of state with the roles of the axes rotated
    "rotated": (
        sp.Rational(3, 2) + sp.cos(y) * sp.sin(2 * x) / 2 + sp.sin(z) / 4,
        [sp.cos(y) * sp.sin(x), sp.sin(z) + sp.cos(2 * x) / 2, sp.sin(2 * y) / 3 + sp.cos(z)],
        [sp.sin(x) * sp.cos(2 * z) / 2 - sp.Rational(1, 5), sp.cos(x) + sp.sin(z) / 2, sp.cos(y - z) / 3],
    ),
    # Orszag-Tang type (rho = 1, so u = m exactly)
    "orszag_tang": (
        sp.Integer(1),
        [-sp.sin(y), sp.sin(x), sp.Integer(0)],
        [-sp.sin(y), sp.sin(2 * x), sp.Integer(0)],
    ),
}


@pytest.mark.parametrize("name", list(STATES))
def test_oracle_rhs_equals_continuum_rhs(oracle_mod, name):
    n = 32
    cs, nu, eta = 1.7, 0.03, 0.05
    rho_e, u_e, B_e = STATES[name]
    exact = [on_grid(e, n) for e in continuum_rhs(rho_e, u_e, B_e, cs, nu, eta)]
    o = oracle_mod.Oracle(n, nu, eta, cs, dt=1e-3)
    o.set_state(on_grid(rho_e, n), np.stack([on_grid(e, n) for e in u_e]),
                np.stack([on_grid(e, n) for e in B_e]))
    drho, dm, db = o.rhs()
    got = [drho, dm[0], dm[1], dm[2], db[0], db[1], db[2]]
    scale = max(np.max(np.abs(e)) for e in exact)
    for f, (g, e) in enumerate(zip(got, exact)):
        err = np.max(np.abs(g - e))
        assert err <= 1e-12 * scale, f"field {f}: max err {err:.3e} (scale {scale:.3e})"


def _mask_mode(n, k):
    return 3 * abs(k) < n


def test_mask_removes_products_outside_two_thirds_and_their_aliases(oracle_mod):
    """u_x = cos 4x + cos 5x on N = 16 (k_max = 5): u_x^2 holds modes 0, 1, 8, 9, 10; on this
    grid 9 and 10 alias to -7 and -6 and 8 is the Nyquist index, all outside the mask.  The RHS
    must equal the continuum RHS with those modes dropped."""
    n = 16
    nu, eta, cs = 0.01, 0.02, 1.1
    for axis in range(3):
        s = X_[axis]
        ue = [sp.Integer(0)] * 3
        ue[axis] = sp.cos(4 * s) + sp.cos(5 * s)
        o = oracle_mod.Oracle(n, nu, eta, cs, dt=1e-3)
        o.set_state(np.ones((n, n, n)), np.stack([on_grid(e, n) for e in ue]), np.zeros((3, n, n, n)))
        drho, dm, db = o.rhs()
        # continuum RHS projected on the mask, written out by hand:
        #   rho_t = -d_s u = 4 sin 4s + 5 sin 5s
        #   m_t   = -d_s (u^2) + nu lap u, and the only part of u^2 inside the mask is 1 + cos s
        exp_rho = on_grid(4 * sp.sin(4 * s) + 5 * sp.sin(5 * s), n)
        exp_m = on_grid(sp.sin(s) - nu * (16 * sp.cos(4 * s) + 25 * sp.cos(5 * s)), n)
        assert np.max(np.abs(drho - exp_rho)) <= 1e-12 * 10
        assert np.max(np.abs(dm[axis] - exp_m)) <= 1e-12 * 10
        for other in range(3):
            if other != axis:
                assert np.max(np.abs(dm[other])) <= 1e-13
        assert np.max(np.abs(db)) == 0.0


def test_mask_boundary_keeps_kmax_and_drops_kmax_plus_one(oracle_mod):
    """set_state projects onto the mask: at N = 32 (k_max = 10) mode 10 survives, mode 11 not,
    along each axis independently."""
    n = 32
    for axis in range(3):
        s = X_[axis]
        for k, keep in ((10, True), (11, False)):
            b = np.zeros((3, n, n, n))
            b[(axis + 1) % 3] = on_grid(sp.cos(k * s), n)
            o = oracle_mod.Oracle(n, 0.0, 0.0, 1.0, dt=1e-3)
            o.set_state(np.ones((n, n, n)), np.zeros((3, n, n, n)), b)
            _, _, bb = o.get_state()
            if keep:
                assert np.max(np.abs(bb - b)) <= 1e-14
            else:
                assert np.max(np.abs(bb)) <= 1e-13  # only rounding leaks
    assert oracle_mod.kmax(32) == 10 and oracle_mod.kmax(16) == 5 and oracle_mod.kmax(256) == 85


def abc_force(amp, A, B, C, kf):
    """The ABC body force as printed (section "for magnetohydrodynamic flow"), times `amp`."""
    return [amp * (A * sp.sin(kf * z) + C * sp.cos(kf * y)),
            amp * (B * sp.sin(kf * x) + A * sp.cos(kf * z)),
            amp * (C * sp.sin(kf * y) + B * sp.cos(kf * x))]


@pytest.mark.parametrize("kf", [1, 2])
def test_forced_rhs_adds_rho_times_abc_force(oracle_mod, kf):
    """Eq. velocity with its body-force term rho f: the momentum RHS gains rho f_ABC."""
    n = 32
    cs, nu, eta = 1.7, 0.03, 0.05
    amp, A, B, C = 0.7, 1.0, 0.6, 0.3
    rho_e, u_e, B_e = STATES["mixed"]
    exact = continuum_rhs(rho_e, u_e, B_e, cs, nu, eta)
    f = abc_force(amp, A, B, C, kf)
    exact = [exact[0]] + [exact[1 + a] + rho_e * f[a] for a in range(3)] + exact[4:]
    exact = [on_grid(e, n) for e in exact]
    o = oracle_mod.Oracle(n, nu, eta, cs, dt=1e-3, forcing=(amp, A, B, C, kf))
    o.set_state(on_grid(rho_e, n), np.stack([on_grid(e, n) for e in u_e]),
                np.stack([on_grid(e, n) for e in B_e]))
    got = [o.rhs()[0], *o.rhs()[1], *o.rhs()[2]]
    scale = max(np.max(np.abs(e)) for e in exact)
    for g, e in zip(got, exact):
        assert np.max(np.abs(g - e)) <= 1e-12 * scale
