"""Pins of the oracle's radix-2 FFT against definitions that do not use it.

* brute force: the DFT written out as a sum (1D), and the full 3D DFT as one N^3 x N^3 sum at
  N = 4 and 8 (every exponent exp(-i k.x) formed explicitly);
* a library special case: numpy.fft;
* Parseval's identity and the forward/inverse round trip with the N^-3 normalisation.
"""
import numpy as np
import pytest


def naive_dft(a, sign):
    n = a.size
    j = np.arange(n)
    out = np.empty(n, dtype=np.complex128)
    for k in range(n):
        out[k] = np.sum(a * np.exp(sign * 2j * np.pi * j * k / n))
    return out


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft1d_matches_direct_sum(oracle_mod, n, sign):
    rng = np.random.default_rng(n + 10 * (sign + 1))
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle_mod.fft1d(a, sign)
    ref = naive_dft(a, sign)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.linalg.norm(a))


def test_fft1d_rejects_non_power_of_two(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.fft1d(np.ones(12), -1)


@pytest.mark.parametrize("n", [4, 8])
def test_fft3d_matches_full_3d_dft(oracle_mod, n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    idx = np.arange(n)
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)  # x, y, z
    # output index (kz, ky, kx) flattened the same way as the input index (z, y, x)
    phase = -2j * np.pi * (pts @ pts.T) / n  # k . x for every (k, x) pair
    ref = (np.exp(phase) @ a.ravel()).reshape(n, n, n)
    got = oracle_mod.fft3d(a, -1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.linalg.norm(a)
    # inverse sign
    ref_inv = (np.exp(-phase) @ a.ravel()).reshape(n, n, n)
    assert np.max(np.abs(oracle_mod.fft3d(a, +1) - ref_inv)) <= 1e-12 * np.linalg.norm(a)


@pytest.mark.parametrize("n", [16, 32])
def test_fft3d_matches_numpy(oracle_mod, n):
    rng = np.random.default_rng(100 + n)
    a = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    assert np.max(np.abs(oracle_mod.fft3d(a, -1) - np.fft.fftn(a))) <= 1e-12 * np.linalg.norm(a)
    assert np.max(np.abs(oracle_mod.fft3d(a, +1) - np.fft.ifftn(a) * n ** 3)) <= 1e-12 * np.linalg.norm(a)


@pytest.mark.parametrize("n", [8, 16])
def test_forward_normalisation_parseval_and_roundtrip(oracle_mod, n):
    rng = np.random.default_rng(7 * n)
    f = rng.standard_normal((n, n, n))
    fh = oracle_mod.forward(f)
    # the k = 0 coefficient is the mean
    assert abs(fh[0, 0, 0] - f.mean()) <= 1e-15 * n ** 3
    # Parseval with the N^-3 forward normalisation: <f^2> = sum |fhat|^2
    assert abs(np.mean(f * f) - np.sum(np.abs(fh) ** 2)) <= 1e-13 * np.mean(f * f)
    # Hermitian symmetry of the spectrum of a real field
    conj_rev = np.conj(np.roll(fh[::-1, ::-1, ::-1], 1, axis=(0, 1, 2)))
    assert np.max(np.abs(fh - conj_rev)) <= 1e-15 * n
    assert np.max(np.abs(oracle_mod.inverse(fh) - f)) <= 1e-13
