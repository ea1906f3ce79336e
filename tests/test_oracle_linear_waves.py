"""Pins of the oracle's time integration against linear waves with closed-form evolution.

A small-amplitude single-Fourier-mode perturbation of a uniform state (eps = 1e-7) evolves, up to
O(eps) relative corrections, by the linearisation of the paper's 3D system (Eqs. density, velocity,
Bfield) at that wavevector, a 2x2 or 3x3 system y' = A y.  Two pins per wave:

* the discrete pin: the second-order Adams-Bashforth recursion (forward Euler first step) applied
  to A reproduces the oracle's mode amplitudes step by step, for fixed and for CFL-variable dt;
* the physics pin: the eigenvalues of A are the textbook damped dispersion relations of sound,
  Alfven and perpendicular fast waves, so A itself is not derived from the oracle's formulas.

The linearisations (uniform rho = 1, background field B0):
  sound along s:   rho_t = -i k m_s,          m_s,t = -i k Cs^2 rho - nu k^2 m_s
  Alfven along B0: m_x,t = i k B0 B_x - nu k^2 m_x,     B_x,t = i k B0 m_x - eta k^2 B_x
  fast, k perp B0: rho_t = -i k m_y,  m_y,t = -i k (Cs^2 rho + B0 B_z) - nu k^2 m_y,
                   B_z,t = -i k B0 m_y - eta k^2 B_z
"""
import numpy as np
import pytest

from paper_1810_12707_gb300.inputs import grid

EPS = 1e-7


def ab2_linear(A, y0, dts):
    """Variable-step AB2 with a forward-Euler first step for y' = A y."""
    y = np.array(y0, dtype=np.complex128)
    f_prev = None
    dt_prev = None
    for dt in dts:
        f = A @ y
        if f_prev is None:
            y = y + dt * f
        else:
            r = dt / dt_prev
            y = y + dt * ((1 + 0.5 * r) * f - 0.5 * r * f_prev)
        f_prev, dt_prev = f, dt
    return y


def by_imag(v):
    v = np.asarray(v)
    return v[np.argsort(v.imag)]


def idx(n, axis, k):
    """FFT index (kz, ky, kx) of wavevector k along `axis`."""
    i = [0, 0, 0]
    i[2 - axis] = k % n
    return tuple(i)


def run_oracle(o, nsteps, fixed_dt):
    if fixed_dt:
        o.step(nsteps)
        return [o.params.dt_fixed] * nsteps
    dts = []
    for _ in range(nsteps):
        o.step(1)
        dts.append(o.diagnostics()["dt"])
    return dts


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("fixed_dt", [True, False])
def test_sound_wave(oracle_mod, axis, fixed_dt):
    n, k, cs, nu = 16, 2, 1.3, 0.02
    X = grid(n)[axis]
    o = oracle_mod.Oracle(n, nu, 0.01, cs, dt=0.01 if fixed_dt else 0.0)
    o.set_state(1.0 + EPS * np.cos(k * X), np.zeros((3, n, n, n)), np.zeros((3, n, n, n)))
    dts = run_oracle(o, 60, fixed_dt)
    A = np.array([[0, -1j * k], [-1j * k * cs ** 2, -nu * k * k]])
    y = ab2_linear(A, [EPS / 2, 0.0], dts)
    i = idx(n, axis, k)
    got = np.array([o.spectrum(0)[i], o.spectrum(1 + axis)[i]])
    assert np.max(np.abs(got - y)) <= 1e-5 * np.max(np.abs(y)), (got, y)
    # eigenvalues of A: lambda = -nu k^2 / 2 +- i sqrt(Cs^2 k^2 - nu^2 k^4 / 4)
    lam = by_imag(np.linalg.eigvals(A))
    w = np.sqrt(cs ** 2 * k ** 2 - nu ** 2 * k ** 4 / 4)
    ref = by_imag(np.array([-nu * k * k / 2 - 1j * w, -nu * k * k / 2 + 1j * w]))
    assert np.allclose(lam, ref, rtol=1e-13, atol=1e-13)
    if not fixed_dt:
        assert len(set(dts)) > 1  # the CFL step really varies


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_alfven_wave(oracle_mod, axis):
    """B0 along `axis`, transverse perturbation B_t = eps cos(k s) along the next axis."""
    n, k, b0, nu, eta = 16, 3, 0.7, 0.015, 0.035
    tr = (axis + 1) % 3
    S = grid(n)[axis]
    b = np.zeros((3, n, n, n))
    b[axis] = b0
    b[tr] = EPS * np.cos(k * S)
    o = oracle_mod.Oracle(n, nu, eta, 2.0, dt=0.005)
    o.set_state(np.ones((n, n, n)), np.zeros((3, n, n, n)), b)
    o.step(80)
    A = np.array([[-nu * k * k, 1j * k * b0], [1j * k * b0, -eta * k * k]])
    y = ab2_linear(A, [0.0, EPS / 2], [0.005] * 80)
    i = idx(n, axis, k)
    got = np.array([o.spectrum(1 + tr)[i], o.spectrum(4 + tr)[i]])
    assert np.max(np.abs(got - y)) <= 1e-5 * np.max(np.abs(y)), (got, y)
    lam = by_imag(np.linalg.eigvals(A))
    w = np.sqrt(k * k * b0 * b0 - (nu - eta) ** 2 * k ** 4 / 4)
    ref = by_imag(np.array([-(nu + eta) * k * k / 2 - 1j * w, -(nu + eta) * k * k / 2 + 1j * w]))
    assert np.allclose(lam, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_fast_wave_perpendicular(oracle_mod, axis):
    """Wave along `axis`, B0 along the next axis: density and field compress together."""
    n, k, b0, cs, nu, eta = 16, 2, 0.9, 1.2, 0.01, 0.02
    bax = (axis + 1) % 3
    S = grid(n)[axis]
    b = np.zeros((3, n, n, n))
    b[bax] = b0 + 0.5 * EPS * np.cos(k * S)
    o = oracle_mod.Oracle(n, nu, eta, cs, dt=0.004)
    o.set_state(1.0 + EPS * np.cos(k * S), np.zeros((3, n, n, n)), b)
    o.step(100)
    A = np.array([[0, -1j * k, 0],
                  [-1j * k * cs ** 2, -nu * k * k, -1j * k * b0],
                  [0, -1j * k * b0, -eta * k * k]])
    y = ab2_linear(A, [EPS / 2, 0.0, EPS / 4], [0.004] * 100)
    i = idx(n, axis, k)
    got = np.array([o.spectrum(0)[i], o.spectrum(1 + axis)[i], o.spectrum(4 + bax)[i]])
    assert np.max(np.abs(got - y)) <= 1e-5 * np.max(np.abs(y)), (got, y)
    # ideal limit: lambda = +- i k sqrt(Cs^2 + B0^2) and 0
    A0 = A.copy()
    A0[1, 1] = A0[2, 2] = 0
    lam = np.sort(np.abs(np.linalg.eigvals(A0).imag))
    assert np.allclose(lam, [0.0, k * np.sqrt(cs ** 2 + b0 ** 2), k * np.sqrt(cs ** 2 + b0 ** 2)], atol=1e-12)
