"""FP64-tolerance parity at 512^3 (the FP64 path and the double-float mode), the size of the
Taylor-Green configuration (N = 512, Mach 0.3, seeded
random B at <|B|^2>/2 = 1e-3, nu = eta = 1e-3), through the kernels the library instantiates for
N = 512 (their own flux block size and tile widths), where the oracle cannot be run directly (it
holds about fifty full N^3 complex arrays: some 130 GB of host memory).

* RHS: for trigonometric states whose products all lie inside the 2/3 mask, the pseudo-spectral
  RHS equals the continuum RHS (sympy, the paper's component form) up to rounding; checked at
  20000 sampled grid points to 1e-12 of the field scale.
* Two CFL steps of the Taylor-Green state, every mode compared.  The state is band-limited
  (|k_i| <= 4), rho = 1 and m = u is solenoidal, so the first step leaves rho = 1 up to rounding
  and both RHS evaluations of two steps see a constant density, where u = m / rho is band-limited
  and every product (|k_i| <= 16 at most) lies inside the 2/3 mask of a 64^3 grid as well.  The
  pseudo-spectral method then computes the same Fourier coefficients on both grids (no product
  aliases on either), so the 512^3 run must equal the oracle run on the 64^3 grid (every 8th grid
  value of the same fields), zero-padded, at every one of its modes.  The CFL step sizes are the
  512^3 grid's: the host forms them from the fields on that grid (the initial arrays, and the
  oracle's state after one step evaluated on the 512^3 grid) and the oracle replays them.
"""
import numpy as np
import pytest
import sympy as sp

import test_oracle_rhs_closed_form as rc
from paper_1810_12707_gb300 import inputs

pytestmark = pytest.mark.gpu

N = 512


@pytest.fixture(scope="module")
def lib():
    from paper_1810_12707_gb300 import build_lib, mhd
    build_lib.build()
    return mhd


# FP64, and the double-float mode, whose 48-bit significand has 32 times FP64's unit roundoff:
# bounds 20 and 10 times looser (precision, RHS bound, every-mode bound)
PRECISIONS = [(0, 1e-12, 1e-13), (2, 2e-11, 1e-12)]


@pytest.mark.parametrize("prec,rhs_tol,mode_tol", PRECISIONS)
@pytest.mark.parametrize("name", ["mixed", "rotated"])
def test_fp64_512_rhs_equals_continuum_rhs(lib, name, prec, rhs_tol, mode_tol):
    torch = pytest.importorskip("torch")
    n = N
    rho_e, u_e, B_e = rc.STATES[name]
    cs, nu, eta = 1.7, 0.03, 0.05
    h = 2 * np.pi / n
    c = torch.arange(n, dtype=torch.float64, device="cuda") * h
    Zc, Yc, Xc = c.view(n, 1, 1), c.view(1, n, 1), c.view(1, 1, n)

    def on_device(expr, out):
        f = sp.lambdify((rc.x, rc.y, rc.z), expr, modules=[{"sin": torch.sin, "cos": torch.cos}])
        out.copy_(torch.as_tensor(f(Xc, Yc, Zc), dtype=torch.float64, device="cuda").expand(n, n, n))

    rho = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    u = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    b = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    on_device(rho_e, rho)
    for a in range(3):
        on_device(u_e[a], u[a])
        on_device(B_e[a], b[a])
    ctx = lib.mhd_init(n, [(nu, eta, cs)], precision=prec)
    lib.mhd_set_state(ctx, 0, rho, u, b)
    del rho, u, b
    rng = np.random.default_rng(1)
    idx = rng.integers(0, n, (20000, 3))  # (z, y, x)
    iz, iy, ix = (torch.as_tensor(idx[:, k], device="cuda") for k in range(3))
    pz, py, px = (h * idx[:, k] for k in range(3))
    drho, dm, db = lib.mhd_rhs(ctx, 0, device=True)
    got = [t[iz, iy, ix].cpu().numpy() for t in (drho, dm[0], dm[1], dm[2], db[0], db[1], db[2])]
    lib.mhd_destroy(ctx)
    del drho, dm, db
    torch.cuda.empty_cache()
    worst = 0.0
    for g, e in zip(got, rc.continuum_rhs(rho_e, u_e, B_e, cs, nu, eta)):
        want = np.broadcast_to(sp.lambdify((rc.x, rc.y, rc.z), e, "numpy")(px, py, pz), g.shape)
        scale = max(1.0, float(np.max(np.abs(want))))
        err = float(np.max(np.abs(g - want))) / scale
        worst = max(worst, err)
        assert err <= rhs_tol
    print(f"512^3 precision {prec} RHS ({name}) vs continuum: worst {worst:.2e} of the field scale")


def _cfl_dt(rho, m, b, cs, nu, eta, n):
    """The CFL step of the library and the oracle, from fields on the n^3 grid (host, FP64)."""
    u2 = np.zeros_like(rho)
    for a in range(3):
        u2 += (m[a] / rho) ** 2
    b2 = np.zeros_like(rho)
    for a in range(3):
        b2 += b[a] * b[a]
    smax = float(np.max(np.sqrt(u2) + np.sqrt(cs * cs + b2 / rho)))
    k = (n - 1) // 3
    dt = 0.2 * (2 * np.pi / n) / smax
    return min(dt, 0.5 / (max(nu, eta) * k * k))


def _on_fine_grid(spec, ns, n):
    """Real field on the n^3 grid of the truncated spectrum `spec` ((ns, ns, ns), FFT order,
    forward-normalised), modes |k_i| <= (ns - 1) // 3 only."""
    import scipy.fft
    k = (ns - 1) // 3
    sel = np.r_[0:k + 1, ns - k:ns]
    dst = np.r_[0:k + 1, n - k:n]
    half = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    half[np.ix_(dst, dst, np.arange(k + 1))] = spec[np.ix_(sel, sel, np.arange(k + 1))]
    return scipy.fft.irfftn(half, s=(n, n, n), axes=(0, 1, 2), workers=-1) * float(n) ** 3


@pytest.mark.parametrize("prec,rhs_tol,mode_tol", PRECISIONS)
def test_taylor_green_512_two_cfl_steps_match_oracle_at_every_mode(lib, oracle_mod, prec, rhs_tol, mode_tol):
    n, ns = N, 64
    ic = inputs.taylor_green(n, seed=2, b_energy=1e-3, mach=0.3, nu=1e-3, eta=1e-3)
    cs, nu, eta = ic.cs, ic.nu, ic.eta
    ctx = lib.mhd_init(n, [(nu, eta, cs)], precision=prec)
    lib.mhd_set_state(ctx, 0, ic.rho, ic.u, ic.b)
    gpu_dt = []
    for _ in range(2):
        lib.mhd_step(ctx, 1)
        assert lib.mhd_synchronize(ctx) == lib.MHD_OK
        gpu_dt.append(lib.mhd_diagnostics(ctx, 0)["dt"])

    # oracle on the 64^3 grid: the same band-limited fields sampled at every 8th point
    sub = (slice(None, None, n // ns),) * 3
    o = oracle_mod.Oracle(ns, nu, eta, cs)
    o.set_state(ic.rho[sub], ic.u[(slice(None),) + sub], ic.b[(slice(None),) + sub])
    dt0 = _cfl_dt(ic.rho, ic.rho[None] * ic.u, ic.b, cs, nu, eta, n)
    del ic
    o.set_fixed_dt(dt0)
    o.step(1)
    rho1 = _on_fine_grid(o.spectrum(0), ns, n)
    assert np.max(np.abs(rho1 - 1.0)) <= 1e-13  # the density stays uniform over the first step
    m1 = [_on_fine_grid(o.spectrum(1 + a), ns, n) for a in range(3)]
    b1 = [_on_fine_grid(o.spectrum(4 + a), ns, n) for a in range(3)]
    dt1 = _cfl_dt(rho1, m1, b1, cs, nu, eta, n)
    del rho1, m1, b1
    o.set_fixed_dt(dt1)
    o.step(1)
    print(f"512^3 TG CFL steps: GPU {gpu_dt}, host {[dt0, dt1]}")
    assert abs(gpu_dt[0] - dt0) <= 1e-12 * dt0
    assert abs(gpu_dt[1] - dt1) <= 1e-12 * dt1

    # per physical field (rho; m and B as vectors): differences relative to the field's largest
    # Fourier coefficient
    k = (ns - 1) // 3
    sel = np.r_[0:k + 1, ns - k:ns]
    dst = np.r_[0:k + 1, n - k:n]
    box = np.ix_(dst, dst, np.arange(k + 1))
    d_in, d_out, scale = np.zeros(7), np.zeros(7), np.zeros(7)
    for f in range(7):
        g = lib.mhd_get_spectrum(ctx, 0, f)  # (n, n, n/2 + 1)
        e = o.spectrum(f)[np.ix_(sel, sel, np.arange(k + 1))]
        scale[f] = float(np.max(np.abs(e)))
        d_in[f] = float(np.max(np.abs(g[box] - e)))
        g[box] = 0.0
        d_out[f] = float(np.max(np.abs(g)))
        del g
    lib.mhd_destroy(ctx)
    for name, fs in (("rho", [0]), ("m", [1, 2, 3]), ("B", [4, 5, 6])):
        s = max(scale[f] for f in fs)
        ein, eout = max(d_in[f] for f in fs) / s, max(d_out[f] for f in fs) / s
        print(f"512^3 TG precision {prec} after 2 CFL steps vs padded 64^3 oracle, {name}: kept modes "
              f"{ein:.2e}, modes outside {eout:.2e} of the largest coefficient")
        assert ein <= mode_tol
        assert eout <= mode_tol
