"""Seeded synthetic initial conditions shaped like the paper's 3D runs.

This module only generates input arrays; it holds none of the solver's arithmetic and imports
nothing else from this package, so the CPU oracle (in the tests) and the GPU library are fed the
same FP64 arrays.  Arrays follow the library's real-space convention: float64 of shape (N, N, N)
indexed [z, y, x] with x_i = 2*pi*i/N; vector fields are (3, N, N, N) with components (x, y, z).

Initial conditions (paper, section "for magnetohydrodynamic flow"):
  * ABC flow  u = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x), with k_f = 1;
  * Taylor-Green  u = (sin x cos y cos z, -cos x sin y cos z, 0);
  * Orszag-Tang type  u = (-sin y, sin x, 0), B = (-sin y, sin 2x, 0);
plus seeded random solenoidal fields built from integer wavevectors with 0 < |k|^2 <= 16, used as a
small velocity perturbation or as the seed magnetic field of a dynamo run.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def grid(n: int):
    """Coordinates (X, Y, Z), each (N, N, N) indexed [z, y, x], of the periodic 2*pi box."""
    x = 2.0 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def _low_k_vectors(kmax2: int):
    r = int(np.floor(np.sqrt(kmax2)))
    ks = [(kx, ky, kz)
          for kz in range(-r, r + 1) for ky in range(-r, r + 1) for kx in range(-r, r + 1)
          if 0 < kx * kx + ky * ky + kz * kz <= kmax2]
    return np.array(ks, dtype=np.int64)


def random_solenoidal(n: int, rng: np.random.Generator, kmax2: int = 16) -> np.ndarray:
    """A real divergence-free vector field (3, N, N, N) with modes 0 < |k|^2 <= kmax2.

    For every integer wavevector k in that shell (in a fixed order) a complex Gaussian vector a(k)
    is drawn and projected onto the plane normal to k, a - k (k.a) / |k|^2.  The field is the real
    part of sum_k a(k) exp(i k.x), which keeps k.a = 0 mode by mode.  Unnormalised.
    """
    ks = _low_k_vectors(kmax2)
    a = rng.standard_normal((len(ks), 3)) + 1j * rng.standard_normal((len(ks), 3))
    kk = ks.astype(np.float64)
    a = a - kk * (np.sum(kk * a, axis=1) / np.sum(kk * kk, axis=1))[:, None]
    spec = np.zeros((3, n, n, n), dtype=np.complex128)
    for (kx, ky, kz), v in zip(ks, a):
        spec[:, kz % n, ky % n, kx % n] += v
    # sum_k a(k) exp(i k.x) on the grid is N^3 * ifftn of the coefficient array
    f = np.real(np.fft.ifftn(spec, axes=(1, 2, 3))) * float(n) ** 3
    return np.ascontiguousarray(f)


def rms(v: np.ndarray) -> float:
    """sqrt(<|v|^2>) of a vector field (3, N, N, N)."""
    return float(np.sqrt(np.mean(np.sum(v * v, axis=0))))


@dataclass
class InitialCondition:
    """One problem instance: fields plus the physical parameters it is run with."""
    rho: np.ndarray
    u: np.ndarray
    b: np.ndarray
    nu: float
    eta: float
    cs: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.rho.shape[0])


def orszag_tang(n: int, seed: int, pert_rms: float = 1e-3, mach: float = 0.1,
                nu: float = 1e-2, eta: float = 1e-2, u0: float = 1.0) -> InitialCondition:
    """Orszag-Tang-type state with a seeded solenoidal |k| <= 4 velocity perturbation of RMS
    `pert_rms`; uniform density 1; Cs = u0 / mach."""
    X, Y, Z = grid(n)
    rng = np.random.default_rng(seed)
    du = random_solenoidal(n, rng)
    du *= pert_rms / rms(du)
    u = np.stack([-np.sin(Y), np.sin(X), np.zeros_like(X)]) * u0 + du
    b = np.stack([-np.sin(Y), np.sin(2.0 * X), np.zeros_like(X)])
    rho = np.ones((n, n, n))
    return InitialCondition(rho, np.ascontiguousarray(u), np.ascontiguousarray(b), nu, eta,
                            u0 / mach, "orszag_tang", {"seed": seed, "mach": mach})


def abc_dynamo(n: int, seed: int, b_energy: float = 1e-5, mach: float = 0.1,
               nu: float = 2e-3, eta: float = 2e-3, A: float = 1.0, B: float = 1.0,
               C: float = 1.0) -> InitialCondition:
    """ABC flow (k_f = 1) with a seeded random |k| <= 4 magnetic field of energy <|B|^2>/2 =
    `b_energy`; uniform density 1; Cs = 1 / mach."""
    X, Y, Z = grid(n)
    u = np.stack([A * np.sin(Z) + C * np.cos(Y),
                  B * np.sin(X) + A * np.cos(Z),
                  C * np.sin(Y) + B * np.cos(X)])
    rng = np.random.default_rng(seed)
    b = random_solenoidal(n, rng)
    b *= np.sqrt(2.0 * b_energy) / rms(b)
    rho = np.ones((n, n, n))
    return InitialCondition(rho, np.ascontiguousarray(u), np.ascontiguousarray(b), nu, eta,
                            1.0 / mach, "abc", {"seed": seed, "mach": mach})


def taylor_green(n: int, seed: int, b_energy: float = 1e-3, mach: float = 0.3,
                 nu: float = 1e-3, eta: float = 1e-3) -> InitialCondition:
    """Taylor-Green flow with a seeded random |k| <= 4 magnetic field of energy `b_energy`."""
    X, Y, Z = grid(n)
    u = np.stack([np.sin(X) * np.cos(Y) * np.cos(Z),
                  -np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(X)])
    rng = np.random.default_rng(seed)
    b = random_solenoidal(n, rng)
    b *= np.sqrt(2.0 * b_energy) / rms(b)
    rho = np.ones((n, n, n))
    return InitialCondition(rho, np.ascontiguousarray(u), np.ascontiguousarray(b), nu, eta,
                            1.0 / mach, "taylor_green", {"seed": seed, "mach": mach})


def ensemble_params(count: int, seed: int = 4):
    """Per-instance (nu, eta, mach) of a batched ensemble: nu, eta log-uniform in [1e-3, 1e-2],
    Mach uniform in [0.05, 0.5], drawn in that order from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    nu = 10.0 ** rng.uniform(-3.0, -2.0, count)
    eta = 10.0 ** rng.uniform(-3.0, -2.0, count)
    mach = rng.uniform(0.05, 0.5, count)
    return nu, eta, mach


def paper_flow(n: int, kind: str, A: float = 1.0, B: float = 1.0, C: float = 1.0, k0: int = 1,
               u0: float = 1.0) -> np.ndarray:
    """The unforced initial flows of the paper's energy-exchange runs, as printed
    (section "for magnetohydrodynamic flow"):
      "abc"          (A sin k0 z + C cos k0 y, B sin k0 x + A cos k0 z, C sin k0 y + B cos k0 x)
      "abc_single"   U0 (A sin k0 z, B sin k0 x, C sin k0 y)
      "tg_paper"     A U0 (cos k0 x sin k0 y cos k0 z, -sin k0 x cos k0 y cos k0 z, 0)
      "cats_eye"     U0 (B sin k0 y, A sin k0 x, A cos k0 x - B cos k0 y)"""
    X, Y, Z = grid(n)
    k = float(k0)
    if kind == "abc":
        u = [A * np.sin(k * Z) + C * np.cos(k * Y), B * np.sin(k * X) + A * np.cos(k * Z),
             C * np.sin(k * Y) + B * np.cos(k * X)]
    elif kind == "abc_single":
        u = [u0 * A * np.sin(k * Z), u0 * B * np.sin(k * X), u0 * C * np.sin(k * Y)]
    elif kind == "tg_paper":
        u = [A * u0 * np.cos(k * X) * np.sin(k * Y) * np.cos(k * Z),
             -A * u0 * np.sin(k * X) * np.cos(k * Y) * np.cos(k * Z), np.zeros_like(X)]
    elif kind == "cats_eye":
        u = [u0 * B * np.sin(k * Y), u0 * A * np.sin(k * X), u0 * (A * np.cos(k * X) - B * np.cos(k * Y))]
    else:
        raise ValueError(f"unknown flow {kind!r}")
    return np.ascontiguousarray(np.stack(u))


def energy_exchange(n: int, kind: str, seed: int = 0, mach: float = 0.1, re: float = 450.0,
                    rm: float = 450.0) -> InitialCondition:
    """Energy-exchange run: one of the paper's flows with a seeded random |k| <= 4 solenoidal
    magnetic field of the same energy as the flow (Alfven Mach number 1: equal initial kinetic and
    magnetic energies), rho = 1, Cs = 1 / mach, nu = 1 / Re, eta = 1 / Rm."""
    u = paper_flow(n, kind)
    rng = np.random.default_rng(seed)
    b = random_solenoidal(n, rng)
    b *= rms(u) / rms(b)
    return InitialCondition(np.ones((n, n, n)), u, np.ascontiguousarray(b), 1.0 / re, 1.0 / rm, 1.0 / mach,
                            f"energy_exchange_{kind}", {"seed": seed, "mach": mach})


def decaying_turbulence(n: int, k0: float, seed: int, u_rms: float = 1.0, mach: float = 0.1,
                        nu: float = 5e-3) -> InitialCondition:
    """Decaying compressible turbulence of the hydrodynamic-flow section: a seeded random
    solenoidal velocity whose shell spectrum is E(k) = A k^4 exp(-2 k^2 / k0^2) on the shells
    k = 1 .. k_max (a mode k belongs to shell round(|k|)), A fixed by the RMS speed `u_rms`;
    rho = 1, B = 0 (the induction equation then stays at B = 0), Cs = u_rms / mach, eta = nu.

    Recipe: complex Gaussian vectors on every dealiased wavevector with round(|k|) <= k_max,
    projected normal to k; the real part of their inverse transform; each shell of that field's
    spectrum rescaled to the target energy; the field rescaled to `u_rms`."""
    kmax = (n - 1) // 3
    k1 = np.fft.fftfreq(n, 1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    shell = np.floor(np.sqrt(k2) + 0.5).astype(np.int64)
    keep = ((3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n) & (shell >= 1) & (shell <= kmax))
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((3, n, n, n)) + 1j * rng.standard_normal((3, n, n, n))
    kv = np.stack([KX, KY, KZ])
    safe = np.where(k2 > 0, k2, 1.0)
    a = (a - kv * (np.sum(kv * a, axis=0) / safe)) * keep
    u = np.real(np.fft.ifftn(a, axes=(1, 2, 3)))
    uh = np.fft.fftn(u, axes=(1, 2, 3))
    e_now = np.bincount(shell.ravel(), weights=np.sum(np.abs(uh) ** 2, axis=0).ravel(), minlength=kmax + 2)
    s = np.arange(len(e_now), dtype=np.float64)
    target = s ** 4 * np.exp(-2.0 * s * s / (k0 * k0))
    gain = np.zeros_like(e_now)
    ok = (s >= 1) & (s <= kmax) & (e_now > 0)
    gain[ok] = np.sqrt(target[ok] / e_now[ok])
    uh *= gain[np.minimum(shell, len(gain) - 1)] * keep
    u = np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
    u *= u_rms / rms(u)
    return InitialCondition(np.ones((n, n, n)), np.ascontiguousarray(u), np.zeros((3, n, n, n)), nu, nu,
                            u_rms / mach, "decaying_turbulence", {"seed": seed, "k0": k0, "mach": mach})
