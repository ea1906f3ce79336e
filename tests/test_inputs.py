"""The seeded input recipes (numpy only, no GPU): each generator's field has the form, the band,
the divergence and the energy its recipe states, and the same seed gives the same arrays."""
import numpy as np
import pytest

from paper_1810_12707_gb300 import inputs


def spectrum(f):
    n = f.shape[-1]
    return np.fft.fftn(f, axes=(-3, -2, -1)) / n ** 3


def wavenumbers(n):
    k = np.fft.fftfreq(n, 1.0 / n)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    return KX, KY, KZ


@pytest.mark.parametrize("kmax2", [1, 9, 16])
def test_random_solenoidal_is_divergence_free_and_band_limited(kmax2):
    n = 16
    f = inputs.random_solenoidal(n, np.random.default_rng(7), kmax2=kmax2)
    g = inputs.random_solenoidal(n, np.random.default_rng(7), kmax2=kmax2)
    assert np.array_equal(f, g)
    fh = spectrum(f)
    KX, KY, KZ = wavenumbers(n)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    scale = np.max(np.abs(fh))
    assert np.max(np.abs(KX * fh[0] + KY * fh[1] + KZ * fh[2])) <= 1e-13 * scale
    outside = (k2 == 0) | (k2 > kmax2)
    assert np.max(np.abs(fh[:, outside])) <= 1e-15 * scale
    assert np.min(np.sum(np.abs(fh[:, ~outside]) ** 2, axis=0)) > 0  # every mode of the band drawn


def test_orszag_tang_recipe():
    n = 32
    ic = inputs.orszag_tang(n, seed=0)
    X, Y, Z = inputs.grid(n)
    base = np.stack([-np.sin(Y), np.sin(X), 0 * X])
    du = ic.u - base
    assert inputs.rms(du) == pytest.approx(1e-3, rel=1e-12)
    KX, KY, KZ = wavenumbers(n)
    dh = spectrum(du)
    assert np.max(np.abs(KX * dh[0] + KY * dh[1] + KZ * dh[2])) <= 1e-16
    assert np.array_equal(ic.b, np.stack([-np.sin(Y), np.sin(2 * X), 0 * X]))
    assert np.all(ic.rho == 1.0) and ic.cs == pytest.approx(10.0) and ic.nu == ic.eta == 1e-2
    assert np.array_equal(ic.u, inputs.orszag_tang(n, seed=0).u)
    assert not np.array_equal(ic.u, inputs.orszag_tang(n, seed=1).u)


@pytest.mark.parametrize("make,energy,mach,nu", [
    (lambda n: inputs.abc_dynamo(n, seed=1), 1e-5, 0.1, 2e-3),
    (lambda n: inputs.taylor_green(n, seed=2), 1e-3, 0.3, 1e-3),
])
def test_seed_field_recipes(make, energy, mach, nu):
    n = 32
    ic = make(n)
    X, Y, Z = inputs.grid(n)
    if ic.name == "abc":
        u = np.stack([np.sin(Z) + np.cos(Y), np.sin(X) + np.cos(Z), np.sin(Y) + np.cos(X)])
    else:
        u = np.stack([np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z), 0 * X])
    assert np.array_equal(ic.u, u)
    assert 0.5 * inputs.rms(ic.b) ** 2 == pytest.approx(energy, rel=1e-12)
    bh = spectrum(ic.b)
    KX, KY, KZ = wavenumbers(n)
    assert np.max(np.abs(KX * bh[0] + KY * bh[1] + KZ * bh[2])) <= 1e-15
    assert np.all(ic.rho == 1.0) and ic.cs == pytest.approx(1.0 / mach) and ic.nu == ic.eta == nu


def test_ensemble_parameters():
    nu, eta, mach = inputs.ensemble_params(64, seed=4)
    again = inputs.ensemble_params(64, seed=4)
    assert all(np.array_equal(a, b) for a, b in zip((nu, eta, mach), again))
    for v in (nu, eta):
        assert np.all((v >= 1e-3) & (v <= 1e-2))
        # log-uniform: log10 spread over the whole decade
        lv = np.log10(v)
        assert lv.min() < -2.8 and lv.max() > -2.2
    assert np.all((mach >= 0.05) & (mach <= 0.5)) and mach.min() < 0.1 and mach.max() > 0.45
    big = inputs.ensemble_params(20000, seed=9)
    # uniform on [-3, -2] in log10 and on [0.05, 0.5]: means within 5 standard errors
    assert abs(np.log10(big[0]).mean() + 2.5) <= 5 * (1 / np.sqrt(12)) / np.sqrt(20000)
    assert abs(big[2].mean() - 0.275) <= 5 * (0.45 / np.sqrt(12)) / np.sqrt(20000)
