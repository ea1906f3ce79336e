"""Pins of the oracle against the golden fixture `tests/golden/paper_flows.txt`: exact volume
averages of the paper's initial flows (section "for magnetohydrodynamic flow": the ABC flow of
the kinematic dynamo runs and the four unforced flows of the energy-exchange figure), worked out
by hand from the printed formulas and parameters.

* grid diagnostics: ke = rho0 <|u|^2> / 2 of each flow (rho0 = 1 as printed, and 2), and with the
  uniform field B_x = B_y = B_z = B_0 of the dynamo runs me = 3 B_0^2 / 2, <u . B> = 0, B_hat(0) =
  B_0 and div B = 0;
* the oracle's forward transform with the curl taken as i k x u_hat gives the enstrophy and the
  kinetic helicity by Parseval (k0 = 1 as printed, and 2), and w = k0 u on the Beltrami rows;
* the oracle's helicity diagnostics (formed on the grid): <u . w> = k0 hel for the flow as
  velocity, and <A . B> = hel / k0 for the flow as magnetic field (all its modes lie at
  |k| = k0, so A = curl B / k0^2; the Taylor-Green row has hel = 0 at |k|^2 = 3 k0^2);
* on the Beltrami rows at rho = 1, B = 0 the advection u . grad u = grad(|u|^2 / 2) - u x w is a
  gradient, so the curl of the momentum RHS is exactly -nu k0^2 w;
* the energy-exchange initial states (Alfven Mach number 1) have equal kinetic and magnetic
  energies, as the paper sets them;
* circularly polarised fields, whose |u| and |B| are the same at every point, give every grid
  diagnostic in closed form.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_flows.txt")


def load_flows():
    """Rows of the fixture: dicts with name, flow, panel, ke, ens, hel (Fractions), beltrami."""
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            name, flow, panel, ke, ens, hel, bel = line
            rows.append({"name": name, "flow": flow, "panel": panel, "ke": Fraction(ke),
                         "ens": Fraction(ens), "hel": Fraction(hel), "beltrami": bel == "1"})
    return rows


def wavenumbers(n):
    k = np.fft.fftfreq(n, 1.0 / n)
    return np.meshgrid(k, k, k, indexing="ij")  # KZ, KY, KX for [z][y][x]


def curl_hat(uh, n):
    """i k x u_hat of a spectrum (3, N, N, N) indexed [z][y][x]."""
    KZ, KY, KX = wavenumbers(n)
    return np.stack([1j * (KY * uh[2] - KZ * uh[1]), 1j * (KZ * uh[0] - KX * uh[2]),
                     1j * (KX * uh[1] - KY * uh[0])])


def parseval(ah, bh):
    """<a . b> of real fields from their N^-3-normalised spectra."""
    return float(np.real(np.sum(ah * np.conj(bh))))


def golden_failures(om, lib=None):
    """The pins above; returns the names of those that fail."""
    failed = []
    n = 16
    nu = 0.02
    b0 = 0.25
    one = np.ones((n, n, n))
    for row in load_flows():
        for k0 in (1, 2):
            u = inputs.paper_flow(n, row["flow"], k0=k0)
            # grid diagnostics with the dynamo runs' uniform field, rho0 = 1 and 2
            for rho0 in (1.0, 2.0):
                o = om.Oracle(n, nu, nu, 1.0, lib=lib)
                o.set_state(rho0 * one, u, np.full((3, n, n, n), b0))
                d = o.diagnostics()
                if abs(d["ke"] - rho0 * float(row["ke"])) > 1e-14:
                    failed.append(f"{row['name']} ke")
                if abs(d["me"] - 1.5 * b0 * b0) > 1e-15 or abs(d["cross_hel"]) > 1e-14:
                    failed.append(f"{row['name']} me")
                if any(abs(d[f"mean_b{c}"] - b0) > 1e-15 for c in "xyz") or d["divb_rms"] > 1e-14:
                    failed.append(f"{row['name']} mean field")
            # enstrophy and helicity from the oracle's transform
            uh = np.stack([om.forward(c) for c in u])
            wh = curl_hat(uh, n)
            if abs(parseval(wh, wh) - k0 * k0 * float(row["ens"])) > 1e-13:
                failed.append(f"{row['name']} enstrophy")
            if abs(parseval(uh, wh) - k0 * float(row["hel"])) > 1e-13:
                failed.append(f"{row['name']} helicity")
            if row["beltrami"] and np.max(np.abs(wh - k0 * uh)) > 1e-14:
                failed.append(f"{row['name']} beltrami")
            # helicities of the oracle's spectra call: the flow as velocity gives <u . w> = k0 hel;
            # as magnetic field, all its modes at |k| = k0 (or hel = 0), <A . B> = <B . curl B> / k0^2
            o = om.Oracle(n, nu, nu, 1.0, lib=lib)
            o.set_state(one, u, u)
            r = o.spectra()
            if abs(r["kin_hel"] - k0 * float(row["hel"])) > 1e-12:
                failed.append(f"{row['name']} kinetic helicity")
            if abs(r["mag_hel"] - float(row["hel"]) / k0) > 1e-12 or r["divb_max"] > 1e-13:
                failed.append(f"{row['name']} magnetic helicity")
            # the momentum RHS of a Beltrami flow: only viscosity reaches the vorticity
            if row["beltrami"]:
                o = om.Oracle(n, nu, nu, 1.0, lib=lib)
                o.set_state(one, u, np.zeros((3, n, n, n)))
                _, dm, _ = o.rhs()
                ch = curl_hat(np.stack([np.fft.fftn(c) / n ** 3 for c in dm]), n)
                if np.max(np.abs(ch + nu * k0 * k0 * wh)) > 1e-13:
                    failed.append(f"{row['name']} viscous decay")
    failed += circular_failures(om, lib)
    # Alfven Mach number 1: equal initial energies
    for row in load_flows():
        ic = inputs.energy_exchange(n, row["flow"], seed=3)
        o = om.Oracle(n, ic.nu, ic.eta, ic.cs, lib=lib)
        o.set_state(ic.rho, ic.u, ic.b)
        d = o.diagnostics()
        if abs(d["ke"] - float(row["ke"])) > 1e-14 or abs(d["me"] - d["ke"]) > 1e-13:
            failed.append(f"{row['name']} equipartition")
    return failed


def circular_failures(om, lib=None, n=16):
    """Grid diagnostics in closed form: u = U (sin z, cos z, 0) and B = b (0, cos x, sin x) are
    solenoidal with |u| = U and |B| = b at every point, and rho = rho0 is uniform, so ke =
    rho0 U^2 / 2, me = b^2 / 2, eint = Cs^2 rho0 ln rho0, <|u|> = U, <|B|> = b, max(|u| + c_f) =
    U + sqrt(Cs^2 + b^2 / rho0) and <u . B> = U b <cos z cos x> = 0."""
    failed = []
    X, Y, Z = inputs.grid(n)
    rho0, U, b, cs = 2.0, 0.7, 0.3, 1.3
    u = U * np.stack([np.sin(Z), np.cos(Z), 0 * Z])
    B = b * np.stack([0 * X, np.cos(X), np.sin(X)])
    o = om.Oracle(n, 0.01, 0.01, cs, lib=lib)
    o.set_state(np.full((n, n, n), rho0), u, B)
    d = o.diagnostics()
    want = {"ke": rho0 * U * U / 2, "me": b * b / 2, "eint": cs * cs * rho0 * np.log(rho0), "mean_speed": U,
            "mean_bmag": b, "smax": U + np.sqrt(cs * cs + b * b / rho0), "mean_rho": rho0}
    for key, v in want.items():
        if abs(d[key] - v) > 1e-14 * max(1.0, abs(v)):
            failed.append(f"circular {key}")
    if abs(d["cross_hel"]) > 1e-15 or d["divb_rms"] > 1e-15:
        failed.append("circular cross helicity")
    return failed


def test_fixture_rows():
    rows = load_flows()
    assert [r["panel"] for r in rows] == ["a", "b", "c", "d"]
    for r in rows:
        # a Beltrami flow with w = u has ens = hel = <|u|^2> = 2 ke
        if r["beltrami"]:
            assert r["ens"] == r["hel"] == 2 * r["ke"]


def test_paper_flows_against_golden(oracle_mod):
    assert golden_failures(oracle_mod) == []


@pytest.mark.parametrize("flow", ["abc", "abc_single", "tg_paper", "cats_eye"])
def test_paper_flows_are_solenoidal_and_band_limited(flow):
    """The printed flows are divergence-free single-|k| fields (numpy's FFT, not the oracle's)."""
    n = 16
    u = inputs.paper_flow(n, flow)
    uh = np.stack([np.fft.fftn(c) / n ** 3 for c in u])
    KZ, KY, KX = wavenumbers(n)
    assert np.max(np.abs(KX * uh[0] + KY * uh[1] + KZ * uh[2])) < 1e-15
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    power = np.sum(np.abs(uh) ** 2, axis=0)
    allowed = (k2 == 1) if flow != "tg_paper" else (k2 == 3)
    assert np.sum(power[~allowed]) < 1e-28
