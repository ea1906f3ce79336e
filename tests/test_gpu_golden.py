"""The CUDA path against the golden fixture `tests/golden/paper_flows.txt` (exact volume averages
of the paper's initial flows, section "for magnetohydrodynamic flow"), with no oracle in the loop:
the four flows as four instances of one batched context, in FP64 and in the mixed mode, at k0 = 1
(as printed) and 2:

* grid diagnostics: ke, and with the dynamo runs' uniform field B_0 (1, 1, 1) me = 3 B_0^2 / 2,
  <u . B> = 0, B_hat(0) = B_0, div B = 0;
* enstrophy and kinetic helicity by Parseval from the library's own half spectra of m (= u at
  rho = 1), and w = k0 u on the Beltrami rows;
* the helicity diagnostics: <u . w> = k0 hel and, for the flow as magnetic field, <A . B> =
  hel / k0 with div B = 0;
* the curl of the momentum RHS of a Beltrami row at rho = 1, B = 0 is -nu k0^2 w.
"""
import numpy as np
import pytest

import test_oracle_golden as gold
from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 1e-6}  # FP64, mixed (FP32 passes on a double-float state)


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


def half_parseval(ah, bh):
    """<a . b> of real fields from half spectra (3, N, N, N/2 + 1): the k_x = 0 and N/2 planes
    stand for themselves, the others for k and -k."""
    w = np.full(ah.shape[-1], 2.0)
    w[0] = 1.0
    w[-1] = 1.0
    return float(np.sum(w * np.real(ah * np.conj(bh))))


def half_curl(uh, n):
    k = np.fft.fftfreq(n, 1.0 / n)
    kx = np.arange(n // 2 + 1, dtype=np.float64)
    KZ, KY, KX = np.meshgrid(k, k, kx, indexing="ij")
    return np.stack([1j * (KY * uh[2] - KZ * uh[1]), 1j * (KZ * uh[0] - KX * uh[2]),
                     1j * (KX * uh[1] - KY * uh[0])])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k0", [1, 2])
def test_paper_flows_diagnostics_and_spectra(lib, precision, k0):
    n, nu, b0 = 32, 0.02, 0.25
    rows = gold.load_flows()
    tol = TOL[precision]
    ctx = lib.mhd_init(n, [(nu, nu, 1.0)] * len(rows), precision=precision)
    one = np.ones((n, n, n))
    for i, row in enumerate(rows):
        lib.mhd_set_state(ctx, i, one, inputs.paper_flow(n, row["flow"], k0=k0), np.full((3, n, n, n), b0))
    for i, row in enumerate(rows):
        d = lib.mhd_diagnostics(ctx, i)
        assert abs(d["ke"] - float(row["ke"])) <= tol, row["name"]
        assert abs(d["me"] - 1.5 * b0 * b0) <= tol and abs(d["cross_hel"]) <= tol, row["name"]
        assert all(abs(v - b0) <= tol for v in d["mean_b"]) and d["divb_rms"] <= tol, row["name"]
        uh = np.stack([lib.mhd_get_spectrum(ctx, i, 1 + a) for a in range(3)])
        wh = half_curl(uh, n)
        assert abs(half_parseval(wh, wh) - k0 * k0 * float(row["ens"])) <= 10 * tol, row["name"]
        assert abs(half_parseval(uh, wh) - k0 * float(row["hel"])) <= 10 * tol, row["name"]
        if row["beltrami"]:
            assert np.max(np.abs(wh - k0 * uh)) <= tol, row["name"]
    lib.mhd_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k0", [1, 2])
def test_paper_flows_helicities(lib, precision, k0):
    """The library's helicity diagnostics: the flow as velocity gives <u . w> = k0 hel; the flow as
    magnetic field (all modes at |k| = k0, or hel = 0) gives <A . B> = hel / k0 and div B = 0."""
    n = 32
    rows = gold.load_flows()
    ctx = lib.mhd_init(n, [(0.02, 0.02, 1.0)] * len(rows), precision=precision)
    for i, row in enumerate(rows):
        u = inputs.paper_flow(n, row["flow"], k0=k0)
        lib.mhd_set_state(ctx, i, np.ones((n, n, n)), u, u)
    for i, row in enumerate(rows):
        r = lib.mhd_spectra(ctx, i)
        assert abs(r["kin_hel"] - k0 * float(row["hel"])) <= 1e-12, row["name"]
        assert abs(r["mag_hel"] - float(row["hel"]) / k0) <= 1e-12, row["name"]
        assert r["divb_max"] <= 1e-12, row["name"]
    lib.mhd_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k0", [1, 2])
def test_beltrami_rhs_viscous_decay(lib, precision, k0):
    n, nu = 32, 0.02
    rows = [r for r in gold.load_flows() if r["beltrami"]]
    ctx = lib.mhd_init(n, [(nu, nu, 1.0)] * len(rows), precision=precision)
    flows = [inputs.paper_flow(n, r["flow"], k0=k0) for r in rows]
    for i, u in enumerate(flows):
        lib.mhd_set_state(ctx, i, np.ones((n, n, n)), u, np.zeros((3, n, n, n)))
    for i, (row, u) in enumerate(zip(rows, flows)):
        _, dm, _ = lib.mhd_rhs(ctx, i)
        ch = gold.curl_hat(np.stack([np.fft.fftn(c) / n ** 3 for c in dm]), n)
        wh = gold.curl_hat(np.stack([np.fft.fftn(c) / n ** 3 for c in u]), n)
        assert np.max(np.abs(ch + nu * k0 * k0 * wh)) <= 10 * TOL[precision], row["name"]
    lib.mhd_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_circular_fields_diagnostics(lib, precision):
    """Grid diagnostics in closed form (u = U (sin z, cos z, 0), B = b (0, cos x, sin x), uniform
    rho0: |u| = U and |B| = b everywhere), with the library's Mach numbers and Alfven speed."""
    n = 32
    X, Y, Z = inputs.grid(n)
    rho0, U, b, cs = 2.0, 0.7, 0.3, 1.3
    ctx = lib.mhd_init(n, [(0.01, 0.01, cs)], precision=precision)
    lib.mhd_set_state(ctx, 0, np.full((n, n, n), rho0), U * np.stack([np.sin(Z), np.cos(Z), 0 * Z]),
                      b * np.stack([0 * X, np.cos(X), np.sin(X)]))
    d = lib.mhd_diagnostics(ctx, 0)
    lib.mhd_destroy(ctx)
    va = b / np.sqrt(rho0)
    want = {"ke": rho0 * U * U / 2, "me": b * b / 2, "eint": cs * cs * rho0 * np.log(rho0), "mean_speed": U,
            "mean_bmag": b, "smax": U + np.sqrt(cs * cs + b * b / rho0), "mean_rho": rho0,
            "mach_s": U / cs, "v_a": va, "mach_a": U / va}
    for key, v in want.items():
        assert abs(d[key] - v) <= 1e-13 * max(1.0, abs(v)), key
    assert abs(d["cross_hel"]) <= 1e-14 and d["divb_rms"] <= 1e-14
