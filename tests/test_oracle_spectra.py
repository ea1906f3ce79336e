"""Pins of the oracle's shell spectra and velocity-derivative statistics (paper, section "for
hydrodynamic flow": theta' = <(du_i/dx_i)^2>^(1/2), S_3 = <(du_1/dx_1)^3> / <(du_1/dx_1)^2>^(3/2),
and the initial spectrum E(k) = A k^4 exp(-2 k^2 / k0^2)).

* closed forms: single modes land in shell round(|k|) with energy amplitude^2/4; theta' and S_3 of
  trigonometric velocities written out by hand;
* Parseval: the shell sums add up to the oracle's grid energies (kinetic only for rho = 1);
* brute force: on a random state with non-uniform density the spectra, theta' (by Parseval, a
  different route from the oracle's grid average), S_3, the kinetic and magnetic helicities (by
  Parseval; the oracle forms them on the grid) and max |div B| from numpy's FFT of the oracle's
  own real-space fields;
* max |div B| of a trigonometric field written out by hand;
* the E(k) initial condition has, shell by shell, the requested spectrum.
"""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs


def _state(om, n, rho, u, b, lib=None):
    o = om.Oracle(n, 0.01, 0.01, 1.0, lib=lib)
    o.set_state(rho, u, b)
    return o


def closed_form_failures(om, lib=None):
    """Pins with hand-written answers; returns the names of those that fail."""
    failed = []
    n = 16
    X, Y, Z = inputs.grid(n)
    one = np.ones((n, n, n))
    zero = np.zeros((3, n, n, n))
    # single modes: u_x = a sin(2x) (shell 2); B_z = c cos(x + y) (|k| = sqrt 2, shell 1);
    # B = f (1, -1, 0) sin(x + y + z) (|k| = sqrt 3, shell 2), both solenoidal
    a, c, f = 0.9, 0.7, 0.4
    u = zero.copy()
    u[0] = a * np.sin(2 * X)
    b = zero.copy()
    b[2] = c * np.cos(X + Y)
    b[0] = f * np.sin(X + Y + Z)
    b[1] = -f * np.sin(X + Y + Z)
    r = _state(om, n, one, u, b, lib).spectra()
    want_ek = np.zeros_like(r["ek"])
    want_ek[2] = a * a / 4
    want_em = np.zeros_like(r["em"])
    want_em[1] = c * c / 4
    want_em[2] = f * f / 2
    if np.max(np.abs(r["ek"] - want_ek)) > 1e-14 or np.max(np.abs(r["em"] - want_em)) > 1e-14:
        failed.append("single modes")
    # theta' of u = (p sin 2x, q cos 3y, w sin z): div u = 2p cos 2x - 3q sin 3y + w cos z
    p, q, w = 0.8, 0.5, 1.3
    u = np.stack([p * np.sin(2 * X), q * np.cos(3 * Y), w * np.sin(Z)])
    r = _state(om, n, one, u, zero, lib).spectra()
    if abs(r["theta"] - np.sqrt((4 * p * p + 9 * q * q + w * w) / 2)) > 1e-13:
        failed.append("theta")
    # S_3 of u_x = sin x + beta sin 2x: d = cos x + 2 beta cos 2x, <d^2> = 1/2 + 2 beta^2,
    # <d^3> = 3 beta / 2 (only the cos^2 x cos 2x cross term survives the average)
    beta = 0.3
    u = zero.copy()
    u[0] = np.sin(X) + beta * np.sin(2 * X)
    u[1] = 0.6 * np.cos(Z)  # does not enter d
    r = _state(om, n, one, u, zero, lib).spectra()
    m2, m3 = 0.5 + 2 * beta * beta, 1.5 * beta
    if abs(r["d2"] - m2) > 1e-13 or abs(r["d3"] - m3) > 1e-13 or abs(r["s3"] - m3 / m2 ** 1.5) > 1e-13:
        failed.append("skewness")
    # max |div B| of B = (a sin 2x, c cos 3y, 0): div B = 2a cos 2x - 3c sin 3y reaches 2a + 3c at
    # the grid points x = 0, y = pi/2
    b = zero.copy()
    b[0] = 0.7 * np.sin(2 * X)
    b[1] = 0.4 * np.cos(3 * Y)
    r = _state(om, n, one, zero, b, lib).spectra()
    if abs(r["divb_max"] - (2 * 0.7 + 3 * 0.4)) > 1e-13:
        failed.append("div B max")
    return failed


def brute_force_failures(om, lib=None, n=16, seed=3):
    """numpy FFT of the oracle's own grid fields against the oracle's spectra."""
    failed = []
    rng = np.random.default_rng(seed)
    X, Y, Z = inputs.grid(n)
    rho = 1.0 + 0.3 * np.cos(X + 2 * Y) * np.sin(Z - 0.4) + 0.1 * np.sin(3 * Z)
    u = inputs.random_solenoidal(n, rng, kmax2=9) + 0.2 * np.stack([np.sin(2 * X), np.cos(Y), 0 * X])
    b = inputs.random_solenoidal(n, rng, kmax2=9) + 0.1 * np.stack([np.cos(X - Z), 0 * X, np.sin(2 * Z)])
    o = _state(om, n, rho, u, b, lib)
    r = o.spectra()
    rho_g, m_g, b_g = o.get_state()
    k1 = np.fft.fftfreq(n, 1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    keep = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)
    uh = np.fft.fftn(m_g / rho_g, axes=(1, 2, 3)) / n ** 3 * keep
    bh = np.fft.fftn(b_g, axes=(1, 2, 3)) / n ** 3 * keep
    shell = np.rint(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).astype(int)
    ns = len(r["ek"])
    ek = np.bincount(shell.ravel(), 0.5 * np.sum(np.abs(uh) ** 2, axis=0).ravel(), minlength=ns)[:ns]
    em = np.bincount(shell.ravel(), 0.5 * np.sum(np.abs(bh) ** 2, axis=0).ravel(), minlength=ns)[:ns]
    if np.max(np.abs(ek - r["ek"])) > 1e-13 * ek.max() or np.max(np.abs(em - r["em"])) > 1e-13 * em.max():
        failed.append("brute spectra")
    theta2 = np.sum(np.abs(KX * uh[0] + KY * uh[1] + KZ * uh[2]) ** 2)
    if abs(np.sqrt(theta2) - r["theta"]) > 1e-12 * r["theta"]:
        failed.append("brute theta")
    d = np.real(np.fft.ifftn(1j * KX * uh[0]) * n ** 3)
    m2, m3 = np.mean(d ** 2), np.mean(d ** 3)
    if abs(m2 - r["d2"]) > 1e-12 * m2 or abs(m3 - r["d3"]) > 1e-11 * m2 ** 1.5:
        failed.append("brute skewness")
    # helicities by Parseval over numpy's spectra (the oracle forms them on the grid), and
    # max |div B| from numpy's inverse transform
    def curl(fh):
        return np.stack([1j * (KY * fh[2] - KZ * fh[1]), 1j * (KZ * fh[0] - KX * fh[2]),
                         1j * (KX * fh[1] - KY * fh[0])])
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    ah = curl(bh) / np.where(k2 > 0, k2, 1.0)
    hk = float(np.real(np.sum(np.conj(uh) * curl(uh))))
    hm = float(np.real(np.sum(np.conj(ah) * bh)))
    dmax = np.max(np.abs(np.real(np.fft.ifftn(1j * (KX * bh[0] + KY * bh[1] + KZ * bh[2])) * n ** 3)))
    if abs(hk - r["kin_hel"]) > 1e-12 * np.sum(np.abs(uh) ** 2) * n:
        failed.append("brute kinetic helicity")
    if abs(hm - r["mag_hel"]) > 1e-12 * np.sum(np.abs(bh) ** 2):
        failed.append("brute magnetic helicity")
    if abs(dmax - r["divb_max"]) > 1e-12 * dmax:
        failed.append("brute div B max")
    return failed


def test_closed_forms(oracle_mod):
    assert closed_form_failures(oracle_mod) == []


def test_brute_force_numpy(oracle_mod):
    assert brute_force_failures(oracle_mod) == []


@pytest.mark.parametrize("n", [16, 32])
def test_number_of_shells(oracle_mod, n):
    k = (n - 1) // 3
    # the corner mode (k, k, k) sits in the last shell
    assert oracle_mod._load().or_num_shells(n) == int(round(np.sqrt(3) * k)) + 1


def test_shell_sums_are_the_grid_energies(oracle_mod):
    n = 32
    rng = np.random.default_rng(11)
    u = inputs.random_solenoidal(n, rng, kmax2=16)
    b = inputs.random_solenoidal(n, rng, kmax2=16)
    o = _state(oracle_mod, n, np.ones((n, n, n)), u, b)
    r, d = o.spectra(), o.diagnostics()
    assert r["ek"].sum() == pytest.approx(d["ke"], rel=1e-13)
    assert r["em"].sum() == pytest.approx(d["me"], rel=1e-13)
    # a solenoidal velocity has no divergence
    assert r["theta"] <= 1e-13 * np.sqrt(2 * d["ke"])


@pytest.mark.parametrize("k0", [2.0, 4.0])
def test_decaying_turbulence_has_the_requested_spectrum(oracle_mod, k0):
    n = 32
    ic = inputs.decaying_turbulence(n, k0, seed=7)
    o = oracle_mod.Oracle(n, ic.nu, ic.eta, ic.cs)
    o.set_state(ic.rho, ic.u, ic.b)
    r = o.spectra()
    k = np.arange(len(r["ek"]), dtype=float)
    kmax = (n - 1) // 3
    target = k ** 4 * np.exp(-2 * k * k / (k0 * k0))
    target[kmax + 1:] = 0.0
    target[0] = 0.0
    amp = r["ek"][2] / target[2]
    assert np.allclose(r["ek"], amp * target, rtol=1e-10, atol=1e-14 * r["ek"].max())
    assert r["ek"].sum() == pytest.approx(0.5, rel=1e-12)  # u_rms = 1
    assert r["theta"] <= 1e-12
    assert np.all(r["em"] == 0.0)


def test_shell_rules_agree_on_every_wavenumber():
    """The CUDA path assigns a mode to shell s by the integer bounds lo(s) <= 4|k|^2 <
    (2s + 1)^2 with lo(s) = (2s - 1)^2 for s >= 1 and lo(0) = 0, the oracle by
    floor(sqrt(|k|^2) + 0.5) in FP64.  |k|^2 is an integer and no integer lies on a boundary
    (s + 1/2)^2, so both give round(|k|); checked for every |k|^2 of the largest grid (N = 1024,
    k_max = 341)."""
    kmax = (1024 - 1) // 3
    k2 = np.arange(3 * kmax * kmax + 1, dtype=np.int64)
    s_fp = np.floor(np.sqrt(k2.astype(np.float64)) + 0.5).astype(np.int64)
    lo = np.where(s_fp == 0, 0, (2 * s_fp - 1) ** 2)
    assert np.all(lo <= 4 * k2) and np.all(4 * k2 < (2 * s_fp + 1) ** 2)
    assert np.all(k2[s_fp == 0] == 0)
