/*
 * mhd_oracle.c -- plain FP64 CPU oracle for the 3D pseudo-spectral isothermal compressible MHD
 * right-hand side and the explicit Adams-Bashforth step that consumes it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links, includes or calls this file; only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark load it (through ctypes).
 * It is deliberately slow and unfused: every stage of one time step is a separate full-grid pass
 * over full complex N^3 spectra, in the order the paper's method prescribes, so that a reader can
 * check it against the paper by eye.
 *
 * What is computed (paper, "Three dimensional numerical tests", Eqs. density, velocity, Bfield):
 *   d(rho)/dt  = -div(rho u)
 *   d(rho u)/dt = -div[ rho u(x)u + (P + |B|^2/2) I - B(x)B ] + mu lap(u),   P = Cs^2 rho
 *   dB/dt      = -div( u(x)B - B(x)u ) + eta lap(B)
 * in the component form the paper writes out for the momentum and induction equations
 * (section "Governing equations"), with no energy equation (isothermal closure), plus the
 * optional ABC body force rho f of section "for magnetohydrodynamic flow" in the momentum
 * equation.  Diagnostics: grid energies and means, and the shell spectra, theta' and S_3 of the
 * hydrodynamic-flow section with the kinetic and magnetic helicities and max |div B|
 * (or_spectra).  Tracer particles of section "Tracer Particles" (cloud-in-cell interpolation and
 * a Boris push, or_tracers_*).
 *
 * Spatial discretisation (paper, section "Code G-MHD3D"; Table I): pseudo-spectral.  Derivatives
 * are products with i k in Fourier space, nonlinear products are formed in real space.  Products
 * are dealiased with the 2/3 rule: a mode survives iff 3|k_x| < N, 3|k_y| < N and 3|k_z| < N.
 * The derivative multiplier of the Nyquist index N/2 is zero (that mode is masked anyway).
 *
 * Conventions (the readings this oracle takes where the paper is silent):
 *   grid          x_i = 2 pi i / N on the periodic box [0, 2 pi)^3, real index (z*N + y)*N + x
 *   forward FFT   fhat(k) = N^-3 sum_x f(x) exp(-i k.x)     (so fhat(0) is the mean)
 *   inverse FFT   f(x) = sum_k fhat(k) exp(+i k.x)          (unscaled)
 *   wavenumber    FFT index m -> m for m < N/2, m - N for m > N/2, and 0 (derivative) at N/2
 *   viscosity     +nu lap(u) with u = m / rho, as in Eq. velocity (mu there is nu here)
 *   magnetic      Heaviside-Lorentz units: B^2/2 and B(x)B, as in Eq. velocity
 *   pressure      -grad P = -i k Cs^2 rho_hat, taken from the (already dealiased) density spectrum
 *   integrator    Adams-Bashforth of order 2 with variable step (forward Euler on the first step):
 *                 y^{n+1} = y^n + dt_n [ (1 + r/2) f^n - (r/2) f^{n-1} ],  r = dt_n / dt_{n-1};
 *                 also the classical fourth-order Runge-Kutta method and a predictor-corrector
 *                 (the paper lists Adams-Bashforth, RK4 and predictor-corrector solvers; its
 *                 results use Adams-Bashforth).  The predictor-corrector is read as the AB2
 *                 predictor above followed by one trapezoidal (Adams-Moulton order 2) correction,
 *                 y^{n+1} = y^n + dt/2 [ f^n + f(y*) ].  Every method takes dt from the CFL
 *                 condition at y^n.
 *   CFL           dt = min( C_a dx / max_x(|u| + c_f),  C_v / (max(nu, eta) k_max^2) ),
 *                 dx = 2 pi / N, c_f = sqrt(Cs^2 + |B|^2 / rho), k_max = floor((N-1)/3);
 *                 a fixed dt is used instead when one is given.
 *
 * Everything is IEEE double precision; no -ffast-math.  Results do not depend on the number of
 * OpenMP threads: every parallel loop writes disjoint outputs and every sum is taken in a fixed
 * serial order over per-plane partials.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------------------------ */
/* Radix-2 FFT                                                                                */
/* ------------------------------------------------------------------------------------------ */

static int is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

/* exp(sign * 2 pi i * j / n), each value computed directly from cos/sin of its own angle. */
static cplx twiddle(int j, int n, int sign) {
  const double ang = 2.0 * M_PI * (double)j / (double)n;
  return cos(ang) + (double)sign * sin(ang) * I;
}

/*
 * In-place iterative radix-2 decimation-in-time FFT of length n (a power of two):
 *   a[k] <- sum_j a[j] exp(sign * 2 pi i j k / n),   unscaled.
 * Step 1 permutes the input into bit-reversed order; step 2 merges sub-transforms of length
 * len/2 into transforms of length len with the butterfly (u, w v) -> (u + w v, u - w v).
 * `w` holds exp(sign 2 pi i j / n) for j < n/2.
 */
void or_fft1d_tw(cplx *a, int n, const cplx *w) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1;
    const int step = n / len; /* w_len^j = w_n^(j * n / len) */
    for (int s = 0; s < n; s += len) {
      for (int j = 0; j < half; ++j) {
        const cplx u = a[s + j];
        const cplx v = a[s + j + half] * w[j * step];
        a[s + j] = u + v;
        a[s + j + half] = u - v;
      }
    }
  }
}

static cplx *make_twiddles(int n, int sign) {
  cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)(n / 2 > 0 ? n / 2 : 1));
  for (int j = 0; j < n / 2; ++j) w[j] = twiddle(j, n, sign);
  return w;
}

/* 1D transform of a contiguous array; returns 0 on success, -1 if n is not a power of two. */
int or_fft1d(cplx *a, int n, int sign) {
  if (!is_pow2(n)) return -1;
  cplx *w = make_twiddles(n, sign);
  or_fft1d_tw(a, n, w);
  free(w);
  return 0;
}

/*
 * 3D transform of an N^3 complex array with index (z*N + y)*N + x, unscaled, applied as three
 * passes of 1D transforms: along x (contiguous rows), then y, then z.  Each strided pencil is
 * gathered into a contiguous buffer, transformed and scattered back.
 */
int or_fft3d(cplx *a, int n, int sign) {
  if (!is_pow2(n)) return -1;
  cplx *w = make_twiddles(n, sign);
  const size_t N = (size_t)n;
#pragma omp parallel
  {
    cplx *buf = (cplx *)malloc(sizeof(cplx) * N);
    /* x pass */
#pragma omp for schedule(static)
    for (long r = 0; r < (long)(N * N); ++r) or_fft1d_tw(a + (size_t)r * N, n, w);
    /* y pass */
#pragma omp for schedule(static)
    for (long p = 0; p < (long)(N * N); ++p) {
      const size_t z = (size_t)p / N, x = (size_t)p % N;
      for (size_t y = 0; y < N; ++y) buf[y] = a[(z * N + y) * N + x];
      or_fft1d_tw(buf, n, w);
      for (size_t y = 0; y < N; ++y) a[(z * N + y) * N + x] = buf[y];
    }
    /* z pass */
#pragma omp for schedule(static)
    for (long p = 0; p < (long)(N * N); ++p) {
      const size_t y = (size_t)p / N, x = (size_t)p % N;
      for (size_t z = 0; z < N; ++z) buf[z] = a[(z * N + y) * N + x];
      or_fft1d_tw(buf, n, w);
      for (size_t z = 0; z < N; ++z) a[(z * N + y) * N + x] = buf[z];
    }
    free(buf);
  }
  free(w);
  return 0;
}

/* fhat = N^-3 FFT(f) for a real field f. */
int or_forward(const double *f, cplx *fhat, int n) {
  const size_t n3 = (size_t)n * n * n;
  for (size_t i = 0; i < n3; ++i) fhat[i] = f[i];
  if (or_fft3d(fhat, n, -1)) return -1;
  const double s = 1.0 / (double)n3;
  for (size_t i = 0; i < n3; ++i) fhat[i] *= s;
  return 0;
}

/* f = Re IFFT(fhat), unscaled.  `tmp` is N^3 complex scratch (may alias nothing else). */
static int or_inverse_tmp(const cplx *fhat, double *f, int n, cplx *tmp) {
  const size_t n3 = (size_t)n * n * n;
  memcpy(tmp, fhat, sizeof(cplx) * n3);
  if (or_fft3d(tmp, n, +1)) return -1;
  for (size_t i = 0; i < n3; ++i) f[i] = creal(tmp[i]);
  return 0;
}

int or_inverse(const cplx *fhat, double *f, int n) {
  const size_t n3 = (size_t)n * n * n;
  cplx *tmp = (cplx *)malloc(sizeof(cplx) * n3);
  if (!tmp) return -2;
  int rc = or_inverse_tmp(fhat, f, n, tmp);
  free(tmp);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Wavenumbers and the 2/3 dealiasing mask                                                     */
/* ------------------------------------------------------------------------------------------ */

/* Signed wavenumber of FFT index m used in derivatives; the Nyquist index gets 0. */
static double wavenumber(int m, int n) {
  if (2 * m < n) return (double)m;
  if (2 * m == n) return 0.0;
  return (double)(m - n);
}

/* Magnitude of the signed index of FFT index m (the Nyquist index counts as n/2). */
static int absindex(int m, int n) { return (2 * m <= n) ? m : n - m; }

/* D(k) of the 2/3 rule: 1 iff 3|k_x| < N, 3|k_y| < N and 3|k_z| < N. */
static int mask23(int mx, int my, int mz, int n) {
  return 3 * absindex(mx, n) < n && 3 * absindex(my, n) < n && 3 * absindex(mz, n) < n;
}

int or_kmax(int n) { return (n - 1) / 3; }

/* ------------------------------------------------------------------------------------------ */
/* Solver state                                                                               */
/* ------------------------------------------------------------------------------------------ */

enum { F_RHO = 0, F_MX, F_MY, F_MZ, F_BX, F_BY, F_BZ, NSTATE };
/* flux fields, in this order: T_xx T_yy T_zz T_xy T_xz T_yz, E_x E_y E_z, u_x u_y u_z */
enum { T_XX = 0, T_YY, T_ZZ, T_XY, T_XZ, T_YZ, E_X, E_Y, E_Z, U_X, U_Y, U_Z, NFLUX };

typedef struct {
  int n;
  double nu, eta, cs;   /* viscosity (mu), resistivity, isothermal sound speed */
  double dt_fixed;      /* > 0: fixed step; <= 0: CFL step */
  double cfl_adv, cfl_visc;
  int integrator;       /* 0 Adams-Bashforth 2, 1 Runge-Kutta 4, 2 predictor-corrector */
  /* ABC body force rho f (paper, section "for magnetohydrodynamic flow"): f = famp *
   * (A sin(kf z) + C cos(kf y), B sin(kf x) + A cos(kf z), C sin(kf y) + B cos(kf x));
   * off when famp == 0 */
  double famp, fa, fb, fc;
  int fkf;
} or_params;

typedef struct {
  or_params p;
  size_t n3;
  cplx *state[NSTATE]; /* masked spectra of rho, m, B */
  cplx *hist[NSTATE];  /* f^{n-1}: the RHS of the previous step */
  cplx *rhs[NSTATE];
  cplx *ystage[NSTATE]; /* intermediate states of the multi-stage methods */
  cplx *kacc[NSTATE];   /* RK4 weighted sum of the stage derivatives */
  cplx *flux[NFLUX];
  cplx *force[3];       /* spectra of rho f */
  double *real[NSTATE];
  double *rflux[NFLUX];
  cplx *tmp;
  double t, dt_prev, dt_last;
  int64_t step;
  /* tracer particles (section "Tracer Particles"): ntr particles, tr[m][6] = x y z vx vy vz;
   * bgrid: the grid magnetic field they are pushed with (3 N^3) */
  int64_t ntr;
  double *tr;
  double *bgrid;
} or_ctx;

static void ctx_free(or_ctx *c) {
  if (!c) return;
  for (int f = 0; f < NSTATE; ++f) {
    free(c->state[f]);
    free(c->hist[f]);
    free(c->rhs[f]);
    free(c->ystage[f]);
    free(c->kacc[f]);
    free(c->real[f]);
  }
  for (int f = 0; f < NFLUX; ++f) {
    free(c->flux[f]);
    free(c->rflux[f]);
  }
  for (int d = 0; d < 3; ++d) free(c->force[d]);
  free(c->tmp);
  free(c->tr);
  free(c->bgrid);
  free(c);
}

or_ctx *or_create(const or_params *p) {
  if (!p || !is_pow2(p->n) || p->n < 4 || p->integrator < 0 || p->integrator > 2) return NULL;
  or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
  if (!c) return NULL;
  c->p = *p;
  c->n3 = (size_t)p->n * p->n * p->n;
  int ok = 1;
  for (int f = 0; f < NSTATE; ++f) {
    ok &= (c->state[f] = (cplx *)calloc(c->n3, sizeof(cplx))) != NULL;
    ok &= (c->hist[f] = (cplx *)calloc(c->n3, sizeof(cplx))) != NULL;
    ok &= (c->rhs[f] = (cplx *)calloc(c->n3, sizeof(cplx))) != NULL;
    ok &= (c->ystage[f] = (cplx *)calloc(c->n3, sizeof(cplx))) != NULL;
    ok &= (c->kacc[f] = (cplx *)calloc(c->n3, sizeof(cplx))) != NULL;
    ok &= (c->real[f] = (double *)calloc(c->n3, sizeof(double))) != NULL;
  }
  for (int f = 0; f < NFLUX; ++f) {
    ok &= (c->flux[f] = (cplx *)calloc(c->n3, sizeof(cplx))) != NULL;
    ok &= (c->rflux[f] = (double *)calloc(c->n3, sizeof(double))) != NULL;
  }
  for (int d = 0; d < 3; ++d) ok &= (c->force[d] = (cplx *)calloc(c->n3, sizeof(cplx))) != NULL;
  ok &= (c->tmp = (cplx *)calloc(c->n3, sizeof(cplx))) != NULL;
  if (!ok) {
    ctx_free(c);
    return NULL;
  }
  return c;
}

void or_destroy(or_ctx *c) { ctx_free(c); }

static void apply_mask(cplx *a, int n) {
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x)
        if (!mask23(x, y, z, n)) a[((size_t)z * n + y) * n + x] = 0.0;
}

/*
 * Initial state from real-space rho, u = (u_x, u_y, u_z), B = (B_x, B_y, B_z) (each N^3, the
 * components of u and B stacked).  The evolved variable is the momentum density m = rho u; every
 * field is transformed and projected onto the dealiased modes.  Resets time, step and history.
 */
int or_set_state(or_ctx *c, const double *rho, const double *u, const double *b) {
  const size_t n3 = c->n3;
  const int n = c->p.n;
  double *m = (double *)malloc(sizeof(double) * n3);
  if (!m) return -2;
  if (or_forward(rho, c->state[F_RHO], n)) return -1;
  for (int d = 0; d < 3; ++d) {
    for (size_t i = 0; i < n3; ++i) m[i] = rho[i] * u[d * n3 + i];
    or_forward(m, c->state[F_MX + d], n);
    or_forward(b + d * n3, c->state[F_BX + d], n);
  }
  free(m);
  for (int f = 0; f < NSTATE; ++f) {
    apply_mask(c->state[f], n);
    memset(c->hist[f], 0, sizeof(cplx) * n3);
  }
  c->t = 0.0;
  c->dt_prev = 0.0;
  c->dt_last = 0.0;
  c->step = 0;
  return 0;
}

/* Real-space rho, m, B of the current state (each N^3; m and B components stacked). */
int or_get_state(or_ctx *c, double *rho, double *m, double *b) {
  const size_t n3 = c->n3;
  const int n = c->p.n;
  or_inverse_tmp(c->state[F_RHO], rho, n, c->tmp);
  for (int d = 0; d < 3; ++d) {
    or_inverse_tmp(c->state[F_MX + d], m + d * n3, n, c->tmp);
    or_inverse_tmp(c->state[F_BX + d], b + d * n3, n, c->tmp);
  }
  return 0;
}

/* Copy of one state spectrum (full N^3 complex layout, zeros outside the mask). */
int or_get_spectrum(or_ctx *c, int field, cplx *out) {
  if (field < 0 || field >= NSTATE) return -1;
  memcpy(out, c->state[field], sizeof(cplx) * c->n3);
  return 0;
}

/* Replace one state spectrum (the caller's spectrum is masked on the way in). */
int or_set_spectrum(or_ctx *c, int field, const cplx *in) {
  if (field < 0 || field >= NSTATE) return -1;
  memcpy(c->state[field], in, sizeof(cplx) * c->n3);
  apply_mask(c->state[field], c->p.n);
  return 0;
}

/*
 * The right-hand side f(y) of the 3D system, in the order of the pseudo-spectral method:
 *   1. inverse transforms of rho_hat, m_hat, B_hat to the grid;
 *   2. u = m / rho, |B|^2, and the products on the grid:
 *        T_ij = m_i u_j + delta_ij |B|^2 / 2 - B_i B_j       (momentum flux without P)
 *        E    = u x B                                       (so that -div(uB - Bu) = curl E)
 *        u                                                  (for the viscous term)
 *   3. forward transforms of the 12 products;
 *   4. in Fourier space:
 *        rho_t   = -i k . m_hat
 *        m_t,i   = -i sum_j k_j T_ij_hat - i k_i Cs^2 rho_hat - nu |k|^2 u_i_hat
 *        B_t     =  i k x E_hat - eta |k|^2 B_hat
 *   5. multiplication of every RHS spectrum by the 2/3 mask D(k).
 * The state is `y` and the RHS goes to `out` (7 spectra each).  Also returns max_x(|u| + c_f)
 * over the grid (for the CFL step) in *smax.
 */
static int compute_rhs_of(or_ctx *c, cplx *const *y, cplx *const *out, double *smax) {
  const int n = c->p.n;
  const size_t n3 = c->n3;
  const double cs2 = c->p.cs * c->p.cs;

  /* 1. */
  for (int f = 0; f < NSTATE; ++f) or_inverse_tmp(y[f], c->real[f], n, c->tmp);

  /* 2. */
  double *plane_max = (double *)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int z = 0; z < n; ++z) {
    double pm = 0.0;
    for (size_t i = (size_t)z * n * n; i < (size_t)(z + 1) * n * n; ++i) {
      const double rho = c->real[F_RHO][i];
      const double m[3] = {c->real[F_MX][i], c->real[F_MY][i], c->real[F_MZ][i]};
      const double B[3] = {c->real[F_BX][i], c->real[F_BY][i], c->real[F_BZ][i]};
      const double u[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
      const double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
      c->rflux[T_XX][i] = m[0] * u[0] + 0.5 * b2 - B[0] * B[0];
      c->rflux[T_YY][i] = m[1] * u[1] + 0.5 * b2 - B[1] * B[1];
      c->rflux[T_ZZ][i] = m[2] * u[2] + 0.5 * b2 - B[2] * B[2];
      c->rflux[T_XY][i] = m[0] * u[1] - B[0] * B[1];
      c->rflux[T_XZ][i] = m[0] * u[2] - B[0] * B[2];
      c->rflux[T_YZ][i] = m[1] * u[2] - B[1] * B[2];
      c->rflux[E_X][i] = u[1] * B[2] - u[2] * B[1];
      c->rflux[E_Y][i] = u[2] * B[0] - u[0] * B[2];
      c->rflux[E_Z][i] = u[0] * B[1] - u[1] * B[0];
      c->rflux[U_X][i] = u[0];
      c->rflux[U_Y][i] = u[1];
      c->rflux[U_Z][i] = u[2];
      const double speed = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      const double cf = sqrt(cs2 + b2 / rho);
      const double s = speed + cf;
      if (!(s <= pm)) pm = s; /* propagates NaN */
    }
    plane_max[z] = pm;
  }
  double sm = 0.0;
  for (int z = 0; z < n; ++z)
    if (!(plane_max[z] <= sm)) sm = plane_max[z];
  free(plane_max);
  if (smax) *smax = sm;

  /* 3. */
  for (int f = 0; f < NFLUX; ++f) or_forward(c->rflux[f], c->flux[f], n);

  /* body force: rho f on the grid, transformed (reuses the first three flux grids) */
  const int forced = c->p.famp != 0.0;
  if (forced) {
    const double kf = (double)c->p.fkf, A = c->p.fa, B = c->p.fb, C = c->p.fc, F = c->p.famp;
    for (int z = 0; z < n; ++z) {
      for (int y = 0; y < n; ++y) {
        for (int x = 0; x < n; ++x) {
          const size_t i = ((size_t)z * n + y) * n + x;
          const double X = 2.0 * M_PI * x / n, Y = 2.0 * M_PI * y / n, Z = 2.0 * M_PI * z / n;
          const double rho = c->real[F_RHO][i];
          c->rflux[0][i] = rho * F * (A * sin(kf * Z) + C * cos(kf * Y));
          c->rflux[1][i] = rho * F * (B * sin(kf * X) + A * cos(kf * Z));
          c->rflux[2][i] = rho * F * (C * sin(kf * Y) + B * cos(kf * X));
        }
      }
    }
    for (int d = 0; d < 3; ++d) or_forward(c->rflux[d], c->force[d], n);
  }

  /* 4. and 5. */
  const double nu = c->p.nu, eta = c->p.eta;
  cplx *const *yv = y;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < n; ++z) {
    for (int y = 0; y < n; ++y) {
      for (int x = 0; x < n; ++x) {
        const size_t i = ((size_t)z * n + y) * n + x;
        if (!mask23(x, y, z, n)) {
          for (int f = 0; f < NSTATE; ++f) out[f][i] = 0.0;
          continue;
        }
        const double k[3] = {wavenumber(x, n), wavenumber(y, n), wavenumber(z, n)};
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        const cplx rho = yv[F_RHO][i];
        const cplx mh[3] = {yv[F_MX][i], yv[F_MY][i], yv[F_MZ][i]};
        const cplx Bh[3] = {yv[F_BX][i], yv[F_BY][i], yv[F_BZ][i]};
        /* symmetric momentum-flux tensor T_ij_hat */
        const cplx Txx = c->flux[T_XX][i], Tyy = c->flux[T_YY][i], Tzz = c->flux[T_ZZ][i];
        const cplx Txy = c->flux[T_XY][i], Txz = c->flux[T_XZ][i], Tyz = c->flux[T_YZ][i];
        const cplx T[3][3] = {{Txx, Txy, Txz}, {Txy, Tyy, Tyz}, {Txz, Tyz, Tzz}};
        const cplx Eh[3] = {c->flux[E_X][i], c->flux[E_Y][i], c->flux[E_Z][i]};
        const cplx uh[3] = {c->flux[U_X][i], c->flux[U_Y][i], c->flux[U_Z][i]};

        /* continuity */
        out[F_RHO][i] = -I * (k[0] * mh[0] + k[1] * mh[1] + k[2] * mh[2]);
        /* momentum */
        for (int a = 0; a < 3; ++a) {
          cplx divT = k[0] * T[a][0] + k[1] * T[a][1] + k[2] * T[a][2];
          out[F_MX + a][i] = -I * divT - I * k[a] * cs2 * rho - nu * k2 * uh[a] + (forced ? c->force[a][i] : 0.0);
        }
        /* induction: curl E with E = u x B */
        const cplx curlE[3] = {I * (k[1] * Eh[2] - k[2] * Eh[1]), I * (k[2] * Eh[0] - k[0] * Eh[2]),
                               I * (k[0] * Eh[1] - k[1] * Eh[0])};
        for (int a = 0; a < 3; ++a) out[F_BX + a][i] = curlE[a] - eta * k2 * Bh[a];
      }
    }
  }
  return 0;
}

static int compute_rhs(or_ctx *c, double *smax) { return compute_rhs_of(c, c->state, c->rhs, smax); }

/* Real-space RHS of the current state: drho (N^3), dm (3 N^3), dB (3 N^3).  State unchanged. */
int or_rhs(or_ctx *c, double *drho, double *dm, double *db) {
  compute_rhs(c, NULL);
  const size_t n3 = c->n3;
  or_inverse_tmp(c->rhs[F_RHO], drho, c->p.n, c->tmp);
  for (int d = 0; d < 3; ++d) {
    or_inverse_tmp(c->rhs[F_MX + d], dm + d * n3, c->p.n, c->tmp);
    or_inverse_tmp(c->rhs[F_BX + d], db + d * n3, c->p.n, c->tmp);
  }
  return 0;
}

/* RHS spectrum of one field (full N^3 complex layout) for the current state. */
int or_rhs_spectrum(or_ctx *c, int field, cplx *out) {
  if (field < 0 || field >= NSTATE) return -1;
  compute_rhs(c, NULL);
  memcpy(out, c->rhs[field], sizeof(cplx) * c->n3);
  return 0;
}

/* The CFL step of the current state given max_x(|u| + c_f). */
static double cfl_dt(const or_ctx *c, double smax) {
  const int n = c->p.n;
  const double dx = 2.0 * M_PI / (double)n;
  double dt = c->p.cfl_adv * dx / smax;
  const double diff = c->p.nu > c->p.eta ? c->p.nu : c->p.eta;
  const int km = or_kmax(n);
  if (diff > 0.0 && km > 0) {
    const double dtv = c->p.cfl_visc / (diff * (double)km * (double)km);
    if (dtv < dt) dt = dtv;
  }
  return dt;
}

/* dst = a + w * b for all 7 fields (b may be NULL: dst = a). */
static void axpy7(cplx *const *dst, cplx *const *a, double w, cplx *const *b, size_t n3) {
  for (int f = 0; f < NSTATE; ++f) {
    cplx *d = dst[f];
    const cplx *x = a[f], *y = b ? b[f] : NULL;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)n3; ++i) d[i] = y ? x[i] + w * y[i] : x[i];
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Tracer particles (section "Tracer Particles": CIC interpolation, Eq. tracer_eq; Boris push,   */
/* Eq. boris; position update, Eq. euler)                                                       */
/* ------------------------------------------------------------------------------------------ */

/* Position wrapped into the periodic box [0, 2 pi). */
static double wrap_2pi(double x) {
  const double L = 2.0 * M_PI;
  double w = x - L * floor(x / L);
  if (w >= L) w -= L; /* x just below a multiple of L can round up to L */
  return w;
}

/*
 * Cloud-in-cell value of the periodic grid field g (N^3, index (z*N + y)*N + x) at (x, y, z), as
 * Eq. tracer_eq: the particle's cell has its bottom-left-front corner at grid index (i, j, k);
 * each of the 8 corners is weighted by the volume of the sub-cell opposite to it.  Reading: the
 * volumes are divided by the cell volume h^3 (weights summing to 1) and the printed factor dt is
 * not applied.  Periodic: index N is index 0.
 */
static double cic(const double *g, int n, double x, double y, double z) {
  const double h = 2.0 * M_PI / (double)n;
  const int i = (int)floor(x / h), j = (int)floor(y / h), k = (int)floor(z / h);
  /* distances from the lower faces (p - x_g^i) and to the upper faces (x_g^{i+1} - p), in cells */
  const double lx = x / h - i, ly = y / h - j, lz = z / h - k;
  const double ux = 1.0 - lx, uy = 1.0 - ly, uz = 1.0 - lz;
  const int i0 = ((i % n) + n) % n, j0 = ((j % n) + n) % n, k0 = ((k % n) + n) % n;
  const int i1 = (i0 + 1) % n, j1 = (j0 + 1) % n, k1 = (k0 + 1) % n;
#define G(a, b, c) g[((size_t)(c) * n + (b)) * n + (a)]
  return G(i0, j0, k0) * ux * uy * uz + G(i1, j0, k0) * lx * uy * uz + G(i0, j1, k0) * ux * ly * uz +
         G(i1, j1, k0) * lx * ly * uz + G(i0, j0, k1) * ux * uy * lz + G(i1, j0, k1) * lx * uy * lz +
         G(i0, j1, k1) * ux * ly * lz + G(i1, j1, k1) * lx * ly * lz;
#undef G
}

/* Grid u = m / rho (which = 1) or B (which = 0) of the current state into out[3][N^3]. */
static void grid_field(or_ctx *c, int which, double *out) {
  const int n = c->p.n;
  const size_t n3 = c->n3;
  if (which == 0) {
    for (int a = 0; a < 3; ++a) or_inverse_tmp(c->state[F_BX + a], out + a * n3, n, c->tmp);
    return;
  }
  or_inverse_tmp(c->state[F_RHO], c->real[F_RHO], n, c->tmp);
  for (int a = 0; a < 3; ++a) {
    or_inverse_tmp(c->state[F_MX + a], out + a * n3, n, c->tmp);
    for (size_t i = 0; i < n3; ++i) out[a * n3 + i] /= c->real[F_RHO][i];
  }
}

/* CIC value of B (which = 0) or u (which = 1) at `count` positions pos[m][3] into out[m][3]. */
int or_tracer_field(or_ctx *c, int which, int64_t count, const double *pos, double *out) {
  double *g = (double *)malloc(sizeof(double) * 3 * c->n3);
  if (!g) return -2;
  grid_field(c, which, g);
  for (int64_t m = 0; m < count; ++m) {
    const double x = wrap_2pi(pos[3 * m]), y = wrap_2pi(pos[3 * m + 1]), z = wrap_2pi(pos[3 * m + 2]);
    for (int a = 0; a < 3; ++a) out[3 * m + a] = cic(g + a * c->n3, c->p.n, x, y, z);
  }
  free(g);
  return 0;
}

/* Place `count` tracers at pos[m][3] (wrapped into the box) with the CIC-interpolated grid
 * velocity as their initial velocity; count = 0 removes them. */
int or_tracers_set(or_ctx *c, int64_t count, const double *pos) {
  free(c->tr);
  c->tr = NULL;
  c->ntr = 0;
  if (count <= 0) return 0;
  c->tr = (double *)malloc(sizeof(double) * 6 * (size_t)count);
  if (!c->bgrid) c->bgrid = (double *)malloc(sizeof(double) * 3 * c->n3);
  if (!c->tr || !c->bgrid) return -2;
  double *v = (double *)malloc(sizeof(double) * 3 * (size_t)count);
  if (!v) return -2;
  or_tracer_field(c, 1, count, pos, v);
  for (int64_t m = 0; m < count; ++m)
    for (int a = 0; a < 3; ++a) {
      c->tr[6 * m + a] = wrap_2pi(pos[3 * m + a]);
      c->tr[6 * m + 3 + a] = v[3 * m + a];
    }
  free(v);
  c->ntr = count;
  return 0;
}

/* Positions and velocities of the tracers, [m][3] each (either may be NULL). */
int or_tracers_get(or_ctx *c, double *pos, double *vel) {
  for (int64_t m = 0; m < c->ntr; ++m)
    for (int a = 0; a < 3; ++a) {
      if (pos) pos[3 * m + a] = c->tr[6 * m + a];
      if (vel) vel[3 * m + a] = c->tr[6 * m + 3 + a];
    }
  return 0;
}

/* One push of every tracer over dt in the grid magnetic field of the current state, in the
 * paper's order: (1) the cell, (2) B at the particle by CIC, (3) the Boris velocity update with
 * q = M = 1 and no electric field, (4) the position update with the new velocity, wrapped. */
static void push_tracers(or_ctx *c, double dt) {
  grid_field(c, 0, c->bgrid);
  const size_t n3 = c->n3;
#pragma omp parallel for schedule(static)
  for (long m = 0; m < (long)c->ntr; ++m) {
    double *p = c->tr + 6 * m, *v = p + 3;
    double B[3];
    for (int a = 0; a < 3; ++a) B[a] = cic(c->bgrid + a * n3, c->p.n, p[0], p[1], p[2]);
    double t[3], s[3], vd[3];
    for (int a = 0; a < 3; ++a) t[a] = B[a] * dt / 2.0;
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + t2);
    vd[0] = v[0] + (v[1] * t[2] - v[2] * t[1]);
    vd[1] = v[1] + (v[2] * t[0] - v[0] * t[2]);
    vd[2] = v[2] + (v[0] * t[1] - v[1] * t[0]);
    const double vn[3] = {v[0] + (vd[1] * s[2] - vd[2] * s[1]), v[1] + (vd[2] * s[0] - vd[0] * s[2]),
                          v[2] + (vd[0] * s[1] - vd[1] * s[0])};
    for (int a = 0; a < 3; ++a) {
      v[a] = vn[a];
      p[a] = wrap_2pi(p[a] + vn[a] * dt);
    }
  }
}

/*
 * Advance `nsteps` steps of the configured method.  Returns 0, or 1 if a non-finite value
 * appeared in max(|u| + c_f) or dt at the start of a step (the state is then left at the last
 * finite step).
 *   AB2  y^{n+1} = y^n + dt [(1 + r/2) f^n - (r/2) f^{n-1}]   (Euler when there is no f^{n-1})
 *   RK4  k1 = f(y), k2 = f(y + dt/2 k1), k3 = f(y + dt/2 k2), k4 = f(y + dt k3),
 *        y^{n+1} = y^n + dt/6 (k1 + 2 k2 + 2 k3 + k4)
 *   PC   y* = AB2 predictor, y^{n+1} = y^n + dt/2 [f^n + f(y*)]
 */
int or_step(or_ctx *c, int nsteps) {
  const size_t n3 = c->n3;
  for (int s = 0; s < nsteps; ++s) {
    double smax = 0.0;
    compute_rhs(c, &smax); /* f^n = f(y^n) in c->rhs */
    const double dt = c->p.dt_fixed > 0.0 ? c->p.dt_fixed : cfl_dt(c, smax);
    if (!isfinite(smax) || !isfinite(dt) || dt <= 0.0) return 1;
    /* tracers move over [t_n, t_n + dt] in the magnetic field of y^n */
    if (c->ntr > 0) push_tracers(c, dt);
    double a1 = 1.0, a0 = 0.0; /* AB2 coefficients of f^n and f^{n-1} */
    if (c->step > 0) {
      const double r = dt / c->dt_prev;
      a1 = 1.0 + 0.5 * r;
      a0 = -0.5 * r;
    }
    if (c->p.integrator == 1) {
      /* k1 in c->rhs; kacc accumulates k1 + 2 k2 + 2 k3 + k4 */
      axpy7(c->kacc, c->rhs, 0.0, NULL, n3);
      const double cstage[3] = {0.5, 0.5, 1.0};
      for (int st = 0; st < 3; ++st) {
        axpy7(c->ystage, c->state, cstage[st] * dt, c->rhs, n3);
        compute_rhs_of(c, c->ystage, c->rhs, NULL);
        axpy7(c->kacc, c->kacc, st < 2 ? 2.0 : 1.0, c->rhs, n3);
      }
      axpy7(c->state, c->state, dt / 6.0, c->kacc, n3);
    } else {
      for (int f = 0; f < NSTATE; ++f) {
        cplx *y = (c->p.integrator == 2) ? c->ystage[f] : c->state[f];
        const cplx *y0 = c->state[f], *fn = c->rhs[f];
        cplx *fo = c->hist[f];
#pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)n3; ++i) {
          y[i] = y0[i] + dt * (a1 * fn[i] + a0 * fo[i]);
          fo[i] = fn[i];
        }
      }
      if (c->p.integrator == 2) {
        /* corrector: f(y*) into c->rhs, then y^{n+1} = y^n + dt/2 (f^n + f(y*)); f^n is in hist */
        compute_rhs_of(c, c->ystage, c->rhs, NULL);
        for (int f = 0; f < NSTATE; ++f) {
          cplx *y = c->state[f];
          const cplx *fn = c->hist[f], *fs = c->rhs[f];
#pragma omp parallel for schedule(static)
          for (long i = 0; i < (long)n3; ++i) y[i] = y[i] + 0.5 * dt * (fn[i] + fs[i]);
        }
      }
    }
    c->dt_prev = dt;
    c->dt_last = dt;
    c->t += dt;
    c->step += 1;
  }
  return 0;
}

/* Fix the step size of the following steps (dt > 0), or go back to the CFL step (dt <= 0).  For
 * tests that replay a step-size sequence decided elsewhere; the history is kept, so the next AB2
 * step uses r = dt / (the previous step's dt) as usual. */
int or_set_fixed_dt(or_ctx *c, double dt) {
  if (!c || !isfinite(dt)) return -1;
  c->p.dt_fixed = dt > 0.0 ? dt : 0.0;
  return 0;
}

/* History (f^{n-1}) access for checkpoint tests. */
int or_get_history(or_ctx *c, int field, cplx *out, double *dt_prev, double *t, int64_t *step) {
  if (field < 0 || field >= NSTATE) return -1;
  memcpy(out, c->hist[field], sizeof(cplx) * c->n3);
  if (dt_prev) *dt_prev = c->dt_prev;
  if (t) *t = c->t;
  if (step) *step = c->step;
  return 0;
}

/*
 * Scalar diagnostics of the current state (volume averages <.> over the grid):
 *   out[0]  ke        <|m|^2 / (2 rho)>
 *   out[1]  me        <|B|^2 / 2>
 *   out[2]  eint      <Cs^2 rho ln rho>  (isothermal internal energy, conserved with ke + me
 *                                         in the ideal limit)
 *   out[3]  cross_hel <u . B>
 *   out[4]  mean_speed <|u|>
 *   out[5]  mean_bmag  <|B|>
 *   out[6]  smax       max(|u| + c_f)
 *   out[7]  mean_rho   rho_hat(0)
 *   out[8..10]  mean_m   m_hat(0)
 *   out[11..13] mean_b   B_hat(0)
 *   out[14] divb_rms  sqrt(<(div B)^2>), from Parseval over the spectrum
 *   out[15] t, out[16] dt of the last step, out[17] step
 * Sums are taken per z-plane, then over planes in order.
 */
int or_diagnostics(or_ctx *c, double *out) {
  const int n = c->p.n;
  const size_t n3 = c->n3;
  const double cs2 = c->p.cs * c->p.cs;
  for (int f = 0; f < NSTATE; ++f) or_inverse_tmp(c->state[f], c->real[f], n, c->tmp);
  double *acc = (double *)calloc((size_t)n * 7, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int z = 0; z < n; ++z) {
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (size_t i = (size_t)z * n * n; i < (size_t)(z + 1) * n * n; ++i) {
      const double rho = c->real[F_RHO][i];
      const double m[3] = {c->real[F_MX][i], c->real[F_MY][i], c->real[F_MZ][i]};
      const double B[3] = {c->real[F_BX][i], c->real[F_BY][i], c->real[F_BZ][i]};
      const double u[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
      const double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
      const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
      s[0] += 0.5 * rho * u2;
      s[1] += 0.5 * b2;
      s[2] += cs2 * rho * log(rho);
      s[3] += u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
      s[4] += sqrt(u2);
      s[5] += sqrt(b2);
      const double v = sqrt(u2) + sqrt(cs2 + b2 / rho);
      if (!(v <= s[6])) s[6] = v;
    }
    for (int q = 0; q < 7; ++q) acc[(size_t)z * 7 + q] = s[q];
  }
  double tot[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int z = 0; z < n; ++z) {
    for (int q = 0; q < 6; ++q) tot[q] += acc[(size_t)z * 7 + q];
    if (!(acc[(size_t)z * 7 + 6] <= tot[6])) tot[6] = acc[(size_t)z * 7 + 6];
  }
  free(acc);
  for (int q = 0; q < 6; ++q) out[q] = tot[q] / (double)n3;
  out[6] = tot[6];
  out[7] = creal(c->state[F_RHO][0]);
  for (int d = 0; d < 3; ++d) {
    out[8 + d] = creal(c->state[F_MX + d][0]);
    out[11 + d] = creal(c->state[F_BX + d][0]);
  }
  /* Parseval: <g^2> = sum_k |ghat(k)|^2 for g = div B, ghat = i k . B_hat */
  double dsum = 0.0;
  for (int z = 0; z < n; ++z) {
    for (int y = 0; y < n; ++y) {
      for (int x = 0; x < n; ++x) {
        const size_t i = ((size_t)z * n + y) * n + x;
        const cplx g = I * (wavenumber(x, n) * c->state[F_BX][i] + wavenumber(y, n) * c->state[F_BY][i] +
                            wavenumber(z, n) * c->state[F_BZ][i]);
        dsum += creal(g) * creal(g) + cimag(g) * cimag(g);
      }
    }
  }
  out[14] = sqrt(dsum);
  out[15] = c->t;
  out[16] = c->dt_last;
  out[17] = (double)c->step;
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Spectra and velocity-derivative statistics                                                 */
/* ------------------------------------------------------------------------------------------ */

/* Number of spectral shells of an n^3 grid: shells 0 .. round(sqrt(3) k_max). */
int or_num_shells(int n) {
  const int k = or_kmax(n);
  return (int)floor(sqrt(3.0 * k * k) + 0.5) + 1;
}

/*
 * Shell-summed spectra and the velocity-derivative statistics of the hydrodynamic-flow section
 * (theta' and the skewness S_3 of du_1/dx_1).  Readings: the velocity is u = m / rho on the grid,
 * transformed and cut to the dealiased modes (the spectra and derivatives of the truncated
 * field); a mode k belongs to shell s = round(|k|); the shell sums run over the whole spectrum,
 * so that sum_s ek[s] = <|u_D|^2>/2 and sum_s em[s] = <|B|^2>/2 (Parseval, with this oracle's
 * forward normalisation).
 *   ek[s], em[s]  sum over the dealiased k with round(|k|) = s of |u_hat(k)|^2/2, |B_hat(k)|^2/2
 *   stats[0]      theta' = sqrt(<(div u_D)^2>), div u_D formed on the grid
 *   stats[1]      S_3 = <d^3> / <d^2>^{3/2},  d = du_x/dx of u_D, on the grid
 *   stats[2..3]   <d^2>, <d^3>
 *   stats[4]      kinetic helicity <u_D . w>, w = curl u_D, both formed on the grid
 *   stats[5]      magnetic helicity <A . B> with the periodic, mean-free vector potential of the
 *                 Coulomb gauge (curl A = B for solenoidal B, div A = 0): A_hat = i k x B_hat / |k|^2
 *                 for k != 0, A_hat(0) = 0; A and B formed on the grid
 *   stats[6]      max over the grid of |div B| (div B formed on the grid)
 * `nshell` must equal or_num_shells(n).
 */
int or_spectra(or_ctx *c, int nshell, double *ek, double *em, double *stats) {
  const int n = c->p.n;
  const size_t n3 = c->n3;
  if (nshell != or_num_shells(n)) return -1;
  cplx *uh[3];
  double *g = (double *)malloc(sizeof(double) * n3);
  int ok = g != NULL;
  for (int a = 0; a < 3; ++a) ok &= (uh[a] = (cplx *)malloc(sizeof(cplx) * n3)) != NULL;
  if (!ok) {
    free(g);
    for (int a = 0; a < 3; ++a) free(uh[a]);
    return -2;
  }
  /* u = m / rho on the grid, then its dealiased spectrum */
  or_inverse_tmp(c->state[F_RHO], c->real[F_RHO], n, c->tmp);
  for (int a = 0; a < 3; ++a) {
    or_inverse_tmp(c->state[F_MX + a], c->real[F_MX + a], n, c->tmp);
    for (size_t i = 0; i < n3; ++i) g[i] = c->real[F_MX + a][i] / c->real[F_RHO][i];
    or_forward(g, uh[a], n);
    apply_mask(uh[a], n);
  }
  for (int s = 0; s < nshell; ++s) ek[s] = em[s] = 0.0;
  for (int z = 0; z < n; ++z) {
    for (int y = 0; y < n; ++y) {
      for (int x = 0; x < n; ++x) {
        if (!mask23(x, y, z, n)) continue;
        const double kx = wavenumber(x, n), ky = wavenumber(y, n), kz = wavenumber(z, n);
        const int sh = (int)floor(sqrt(kx * kx + ky * ky + kz * kz) + 0.5);
        const size_t i = ((size_t)z * n + y) * n + x;
        for (int a = 0; a < 3; ++a) {
          const cplx v = uh[a][i], b = c->state[F_BX + a][i];
          ek[sh] += 0.5 * (creal(v) * creal(v) + cimag(v) * cimag(v));
          em[sh] += 0.5 * (creal(b) * creal(b) + cimag(b) * cimag(b));
        }
      }
    }
  }
  /* div u_D on the grid */
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        const size_t i = ((size_t)z * n + y) * n + x;
        c->tmp[i] = I * (wavenumber(x, n) * uh[0][i] + wavenumber(y, n) * uh[1][i] + wavenumber(z, n) * uh[2][i]);
      }
  or_fft3d(c->tmp, n, +1);
  double th = 0.0;
  for (size_t i = 0; i < n3; ++i) th += creal(c->tmp[i]) * creal(c->tmp[i]);
  /* d = du_x/dx on the grid */
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        const size_t i = ((size_t)z * n + y) * n + x;
        c->tmp[i] = I * wavenumber(x, n) * uh[0][i];
      }
  or_fft3d(c->tmp, n, +1);
  double m2 = 0.0, m3 = 0.0;
  for (size_t i = 0; i < n3; ++i) {
    const double d = creal(c->tmp[i]);
    m2 += d * d;
    m3 += d * d * d;
  }
  m2 /= (double)n3;
  m3 /= (double)n3;
  stats[0] = sqrt(th / (double)n3);
  stats[1] = m3 / pow(m2, 1.5);
  stats[2] = m2;
  stats[3] = m3;
  /* helicities: per component a, the field on the grid (into g) and the curl or potential
   * component on the grid (in tmp), multiplied point by point */
  double hk = 0.0, hm = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int b1 = (a + 1) % 3, b2 = (a + 2) % 3; /* (curl f)_a = d_b1 f_b2 - d_b2 f_b1 */
    for (int pass = 0; pass < 2; ++pass) {
      /* pass 0: u_D and w = curl u_D; pass 1: B and A */
      for (size_t i = 0; i < n3; ++i) c->tmp[i] = pass == 0 ? uh[a][i] : c->state[F_BX + a][i];
      or_fft3d(c->tmp, n, +1);
      for (size_t i = 0; i < n3; ++i) g[i] = creal(c->tmp[i]);
      for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
          for (int x = 0; x < n; ++x) {
            const size_t i = ((size_t)z * n + y) * n + x;
            const double k[3] = {wavenumber(x, n), wavenumber(y, n), wavenumber(z, n)};
            const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            const cplx f1 = pass == 0 ? uh[b1][i] : c->state[F_BX + b1][i];
            const cplx f2 = pass == 0 ? uh[b2][i] : c->state[F_BX + b2][i];
            cplx v = I * (k[b1] * f2 - k[b2] * f1);
            if (pass == 1) v = k2 > 0.0 ? v / k2 : 0.0;
            c->tmp[i] = v;
          }
      or_fft3d(c->tmp, n, +1);
      double acc = 0.0;
      for (size_t i = 0; i < n3; ++i) acc += g[i] * creal(c->tmp[i]);
      if (pass == 0) hk += acc;
      else hm += acc;
    }
  }
  stats[4] = hk / (double)n3;
  stats[5] = hm / (double)n3;
  /* div B on the grid */
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y)
      for (int x = 0; x < n; ++x) {
        const size_t i = ((size_t)z * n + y) * n + x;
        c->tmp[i] = I * (wavenumber(x, n) * c->state[F_BX][i] + wavenumber(y, n) * c->state[F_BY][i] +
                         wavenumber(z, n) * c->state[F_BZ][i]);
      }
  or_fft3d(c->tmp, n, +1);
  double dmax = 0.0;
  for (size_t i = 0; i < n3; ++i) {
    const double v = fabs(creal(c->tmp[i]));
    if (!(v <= dmax)) dmax = v;
  }
  stats[6] = dmax;
  free(g);
  for (int a = 0; a < 3; ++a) free(uh[a]);
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
