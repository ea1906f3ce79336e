// kernels_spectral.cu -- pointwise work in Fourier space: RHS assembly and the Adams-Bashforth
// update, the step size, and the spectral side of the diagnostics.
//
// RHS of the 3D system (paper, section "Three dimensional numerical tests", Eqs. density,
// velocity, Bfield) at a kept wavevector k, with T_ij, E = u x B and u the forward-transformed
// products (scaled here by N^-3) and rho, m, B the state:
//   rho_t = -i k . m
//   m_t,i = -i sum_j k_j T_ij - i k_i Cs^2 rho - nu |k|^2 u_i
//   B_t   =  i k x E - eta |k|^2 B
// Every stored mode lies inside the 2/3-rule set, so the dealiasing mask is 1 on all of them.
#include <math.h>

#include "fft_device.cuh"
#include "launch_util.cuh"
#include "tma_util.cuh"

namespace mhd {

// rho_hat at wavevector (kx, ky, kz) of one instance's truncated density spectrum (zero outside
// the kept set; kx < 0 through Hermitian symmetry).
template <typename CT>
__device__ __forceinline__ CT rho_at(const CT *rho, int kx, int ky, int kz, int K) {
  if (kx < -K || kx > K || ky < -K || ky > K || kz < -K || kz > K) return CT{0, 0};
  const int NX = K + 1, NK = 2 * K + 1;
  const bool cj = kx < 0;
  if (cj) {
    kx = -kx;
    ky = -ky;
    kz = -kz;
  }
  const CT v = rho[((size_t)(kz >= 0 ? kz : kz + NK) * NK + (ky >= 0 ? ky : ky + NK)) * NX + kx];
  return cj ? CT{v.re, -v.im} : v;
}

// Spectrum of rho f_ABC at (kx, ky, kz): the product with sin(kf s) and cos(kf s) shifts the
// density spectrum by +-kf along s, (rho sin)^(k) = [rho(k - kf s) - rho(k + kf s)] / 2i and
// (rho cos)^(k) = [rho(k - kf s) + rho(k + kf s)] / 2.  The product is band-limited (no aliasing),
// so this equals the transform of the product on the grid.
// `rho(kx, ky, kz)` returns the density spectrum at a wavevector (as rho_at does).
template <typename CT, typename RhoAt>
__device__ __forceinline__ void abc_force(RhoAt rho, int kx, int ky, int kz, const PhysDev &ph, CT f[3]) {
  using R = typename CT::value_type;
  const int q = ph.fkf;
  const R a = (R)ph.fa, b = (R)ph.fb, c = (R)ph.fc, amp = (R)ph.famp, h = (R)0.5;
  CT S[3], Co[3];  // (rho sin(q s)), (rho cos(q s)) for s = x, y, z
  const int d[3][3] = {{q, 0, 0}, {0, q, 0}, {0, 0, q}};
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const CT m = rho(kx - d[s][0], ky - d[s][1], kz - d[s][2]);
    const CT p = rho(kx + d[s][0], ky + d[s][1], kz + d[s][2]);
    S[s] = CT{h * (m.im - p.im), -h * (m.re - p.re)};  // (m - p) / 2i
    Co[s] = CT{h * (m.re + p.re), h * (m.im + p.im)};
  }
  f[0] = CT{amp * (a * S[2].re + c * Co[1].re), amp * (a * S[2].im + c * Co[1].im)};
  f[1] = CT{amp * (b * S[0].re + a * Co[2].re), amp * (b * S[0].im + a * Co[2].im)};
  f[2] = CT{amp * (c * S[1].re + b * Co[0].re), amp * (c * S[1].im + b * Co[0].im)};
}

// FC: element type of the product spectra (FP64, or FP32 in the mixed mode); everything else,
// the state, the history and the arithmetic, is FP64.
template <typename FC>
__device__ __forceinline__ void assemble_mode_fp64(const FC *__restrict__ flux, const cplx64 *y_in, cplx64 *state,
                                cplx64 *__restrict__ hist, cplx64 *ystage, cplx64 *__restrict__ rhs_out,
                                const PhysDev *__restrict__ phys, const StepCoef *__restrict__ coef,
                                const cplx64 *__restrict__ force, int op, int stage, int K, double inv_n3,
                                int inst, size_t m, cplx64 *ynew, int ystride) {
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const int kxi = (int)(m % NX);
  const size_t t = m / NX;
  const int jy = (int)(t % NK), jz = (int)(t / NK);
  const double kx = kxi, ky = kept_wave(jy, K), kz = kept_wave(jz, K);
  const double k2 = kx * kx + ky * ky + kz * kz;
  const double nu = phys[inst].nu, eta = phys[inst].eta, cs2 = phys[inst].cs * phys[inst].cs;

  // the product spectra arrive unnormalised: their factor inv_n3 rides on the wavenumbers and
  // dissipation coefficients they meet (fewer FP64 multiplies than scaling 12 spectra)
  const double skx = kx * inv_n3, sky = ky * inv_n3, skz = kz * inv_n3, nuk2s = nu * k2 * inv_n3;
  const cplx64 *S = y_in + (size_t)inst * 7 * spec + m;
  const FC *F = flux + (size_t)inst * 12 * spec + m;
  cplx64 y[7], f[12];
#pragma unroll
  for (int q = 0; q < 7; ++q) y[q] = S[q * spec];
#pragma unroll
  for (int q = 0; q < 12; ++q) f[q] = c_cvt<cplx64>(F[q * spec]);
  const cplx64 Txx = f[0], Tyy = f[1], Tzz = f[2], Txy = f[3], Txz = f[4], Tyz = f[5];
  const cplx64 Ex = f[6], Ey = f[7], Ez = f[8];

  cplx64 r[7];
  // continuity: -i k . m
  {
    const cplx64 s = {kx * y[1].re + ky * y[2].re + kz * y[3].re, kx * y[1].im + ky * y[2].im + kz * y[3].im};
    r[0] = cplx64{s.im, -s.re};
  }
  // momentum
  {
    const double kk[3] = {kx, ky, kz};
    const cplx64 T[3][3] = {{Txx, Txy, Txz}, {Txy, Tyy, Tyz}, {Txz, Tyz, Tzz}};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cplx64 divT = {skx * T[a][0].re + sky * T[a][1].re + skz * T[a][2].re,
                           skx * T[a][0].im + sky * T[a][1].im + skz * T[a][2].im};
      const cplx64 g = {divT.re + kk[a] * cs2 * y[0].re, divT.im + kk[a] * cs2 * y[0].im};
      const cplx64 u = f[9 + a];
      r[1 + a] = cplx64{g.im - nuk2s * u.re, -g.re - nuk2s * u.im};
    }
    if (force != nullptr && phys[inst].famp != 0.0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const cplx64 fo = force[((size_t)inst * 3 + a) * spec + m];
        r[1 + a] = cplx64{r[1 + a].re + fo.re, r[1 + a].im + fo.im};
      }
    }
  }
  // induction: i k x E - eta k^2 B
  {
    const cplx64 c[3] = {{sky * Ez.re - skz * Ey.re, sky * Ez.im - skz * Ey.im},
                         {skz * Ex.re - skx * Ez.re, skz * Ex.im - skx * Ez.im},
                         {skx * Ey.re - sky * Ex.re, skx * Ey.im - sky * Ex.im}};
    const double etak2 = eta * k2;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      r[4 + a] = cplx64{-c[a].im - etak2 * y[4 + a].re, c[a].re - etak2 * y[4 + a].im};
  }

  const size_t o7 = (size_t)inst * 7 * spec + m;
  if (op == ASM_RHS) {
#pragma unroll
    for (int q = 0; q < 7; ++q) rhs_out[o7 + q * spec] = r[q];
    return;
  }
  const double dt = coef[inst].dt, a1 = coef[inst].a1, a0 = coef[inst].a0;
  const double dta1 = dt * a1, dta0 = dt * a0;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const size_t i = o7 + q * spec;
    const cplx64 rq = r[q];
    if (op == ASM_AB2 || op == ASM_PC_PRED) {
      // y + dt (a1 f^n + a0 f^{n-1}), as dt a1 f^n + (dt a0 f^{n-1} + y)
      cplx64 y0 = state[i];
      if (a0 != 0.0) {
        const cplx64 h = hist[i];
        y0 = cplx64{fma(dta0, h.re, y0.re), fma(dta0, h.im, y0.im)};
      }
      const cplx64 yn = {fma(dta1, rq.re, y0.re), fma(dta1, rq.im, y0.im)};
      if (op == ASM_AB2) {
        state[i] = yn;
        if (ynew) ynew[q * ystride] = yn;
      } else {
        ystage[i] = yn;
      }
      hist[i] = rq;
    } else if (op == ASM_RK_STAGE) {
      const cplx64 acc = stage == 1 ? rq : cplx64{hist[i].re + 2.0 * rq.re, hist[i].im + 2.0 * rq.im};
      hist[i] = acc;
      const double w = (stage < 3 ? 0.5 : 1.0) * dt;
      const cplx64 y0 = state[i];
      ystage[i] = cplx64{y0.re + w * rq.re, y0.im + w * rq.im};
    } else {  // ASM_RK_FINAL, ASM_PC_CORR
      const double w = op == ASM_RK_FINAL ? dt / 6.0 : 0.5 * dt;
      const cplx64 h = hist[i], y0 = state[i];
      const cplx64 acc = {h.re + rq.re, h.im + rq.im};
      state[i] = cplx64{y0.re + w * acc.re, y0.im + w * acc.im};
    }
  }
}

template <typename FC>
__global__ void assemble_kernel(const FC *__restrict__ flux, const cplx64 *y_in, cplx64 *state,
                                cplx64 *__restrict__ hist, cplx64 *ystage, cplx64 *__restrict__ rhs_out,
                                const PhysDev *__restrict__ phys, const StepCoef *__restrict__ coef,
                                const cplx64 *__restrict__ force, int op, int stage, int K, int batch,
                                double inv_n3) {
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const size_t total = spec * batch;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int inst = (int)(idx / spec);
    const size_t m = idx - (size_t)inst * spec;
    if (op != ASM_RHS && coef[inst].skip) continue;
    assemble_mode_fp64<FC>(flux, y_in, state, hist, ystage, rhs_out, phys, coef, force, op, stage, K, inv_n3, inst, m,
                           nullptr, 0);
  }
}

// Mixed precision: RHS in FP32 from the FP32 products and the high parts of the state, update of
// the double-float state (hi, lo) by an error-free two-sum (Knuth), no FP64 arithmetic.
__device__ __forceinline__ void df_add(float &hi, float &lo, float d) {
  const float s = hi + d;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (d - bb) + lo;  // exact rounding error of hi + d, plus lo
  hi = s + e;
  lo = e - (hi - s);
}

__device__ __forceinline__ void assemble_mode_mixed(const cplx32 *__restrict__ flux, const cplx32 *y_in, cplx32 *s_hi,
                                   cplx32 *__restrict__ s_lo, cplx32 *__restrict__ hist, cplx32 *ystage,
                                   cplx64 *__restrict__ rhs_out, const PhysDev *__restrict__ phys,
                                   const StepCoef *__restrict__ coef, const cplx32 *__restrict__ force, int op,
                                   int stage, int K, float inv_n3, int inst, size_t m, cplx32 *ynew, int ystride) {
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const int kxi = (int)(m % NX);
  const size_t t = m / NX;
  const float kx = (float)kxi, ky = (float)kept_wave((int)(t % NK), K), kz = (float)kept_wave((int)(t / NK), K);
  const float k2 = kx * kx + ky * ky + kz * kz;
  const PhysDev ph = phys[inst];
  const float nuk2 = (float)ph.nu * k2, etak2 = (float)ph.eta * k2, cs2 = (float)(ph.cs * ph.cs);

  const size_t base7 = (size_t)inst * 7 * spec + m;
  const cplx32 *F = flux + (size_t)inst * 12 * spec + m;
  cplx32 y[7], f[12];
#pragma unroll
  for (int q = 0; q < 7; ++q) y[q] = y_in[base7 + q * spec];
#pragma unroll
  for (int q = 0; q < 12; ++q) f[q] = c_scale(F[q * spec], inv_n3);
  const cplx32 Txx = f[0], Tyy = f[1], Tzz = f[2], Txy = f[3], Txz = f[4], Tyz = f[5];
  const cplx32 Ex = f[6], Ey = f[7], Ez = f[8];
  cplx32 r[7];
  {
    const cplx32 sm = {kx * y[1].re + ky * y[2].re + kz * y[3].re, kx * y[1].im + ky * y[2].im + kz * y[3].im};
    r[0] = cplx32{sm.im, -sm.re};
  }
  {
    const float kk[3] = {kx, ky, kz};
    const cplx32 T[3][3] = {{Txx, Txy, Txz}, {Txy, Tyy, Tyz}, {Txz, Tyz, Tzz}};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cplx32 g = {kx * T[a][0].re + ky * T[a][1].re + kz * T[a][2].re + kk[a] * cs2 * y[0].re,
                        kx * T[a][0].im + ky * T[a][1].im + kz * T[a][2].im + kk[a] * cs2 * y[0].im};
      const cplx32 u = f[9 + a];
      r[1 + a] = cplx32{g.im - nuk2 * u.re, -g.re - nuk2 * u.im};
    }
    if (force != nullptr && ph.famp != 0.0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const cplx32 fo = force[((size_t)inst * 3 + a) * spec + m];
        r[1 + a] = cplx32{r[1 + a].re + fo.re, r[1 + a].im + fo.im};
      }
    }
  }
  {
    const cplx32 c[3] = {{ky * Ez.re - kz * Ey.re, ky * Ez.im - kz * Ey.im},
                         {kz * Ex.re - kx * Ez.re, kz * Ex.im - kx * Ez.im},
                         {kx * Ey.re - ky * Ex.re, kx * Ey.im - ky * Ex.im}};
#pragma unroll
    for (int a = 0; a < 3; ++a)
      r[4 + a] = cplx32{-c[a].im - etak2 * y[4 + a].re, c[a].re - etak2 * y[4 + a].im};
  }
  if (op == ASM_RHS) {
#pragma unroll
    for (int q = 0; q < 7; ++q) rhs_out[base7 + q * spec] = c_cvt<cplx64>(r[q]);
    return;
  }
  const StepCoef cf = coef[inst];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const size_t i = base7 + q * spec;
    const cplx32 rq = r[q];
    if (op == ASM_AB2 || op == ASM_PC_PRED) {
      cplx32 inc = {cf.fa1 * rq.re, cf.fa1 * rq.im};
      if (cf.fa0 != 0.f) {
        const cplx32 h = hist[i];
        inc.re += cf.fa0 * h.re;
        inc.im += cf.fa0 * h.im;
      }
      if (op == ASM_AB2) {
        cplx32 hi = s_hi[i], lo = s_lo[i];
        df_add(hi.re, lo.re, cf.fdt * inc.re);
        df_add(hi.im, lo.im, cf.fdt * inc.im);
        s_hi[i] = hi;
        s_lo[i] = lo;
        if (ynew) ynew[q * ystride] = hi;
      } else {
        const cplx32 hi = s_hi[i], lo = s_lo[i];
        ystage[i] = cplx32{hi.re + (lo.re + cf.fdt * inc.re), hi.im + (lo.im + cf.fdt * inc.im)};
      }
      hist[i] = rq;
    } else if (op == ASM_RK_STAGE) {
      const cplx32 acc = stage == 1 ? rq : cplx32{hist[i].re + 2.f * rq.re, hist[i].im + 2.f * rq.im};
      hist[i] = acc;
      const float w = (stage < 3 ? 0.5f : 1.f) * cf.fdt;
      const cplx32 hi = s_hi[i], lo = s_lo[i];
      ystage[i] = cplx32{hi.re + (lo.re + w * rq.re), hi.im + (lo.im + w * rq.im)};
    } else {  // ASM_RK_FINAL, ASM_PC_CORR
      const float w = op == ASM_RK_FINAL ? cf.fdt / 6.f : 0.5f * cf.fdt;
      const cplx32 h = hist[i];
      cplx32 hi = s_hi[i], lo = s_lo[i];
      df_add(hi.re, lo.re, w * (h.re + rq.re));
      df_add(hi.im, lo.im, w * (h.im + rq.im));
      s_hi[i] = hi;
      s_lo[i] = lo;
    }
  }
}

__global__ void assemble_df_kernel(const cplx32 *__restrict__ flux, const cplx32 *y_in, cplx32 *s_hi,
                                   cplx32 *__restrict__ s_lo, cplx32 *__restrict__ hist, cplx32 *ystage,
                                   cplx64 *__restrict__ rhs_out, const PhysDev *__restrict__ phys,
                                   const StepCoef *__restrict__ coef, const cplx32 *__restrict__ force, int op,
                                   int stage, int K, int batch, float inv_n3) {
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const size_t total = spec * batch;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int inst = (int)(idx / spec);
    const size_t m = idx - (size_t)inst * spec;
    if (op != ASM_RHS && coef[inst].skip) continue;
    assemble_mode_mixed(flux, y_in, s_hi, s_lo, hist, ystage, rhs_out, phys, coef, force, op, stage, K, inv_n3, inst, m,
                        nullptr, 0);
  }
}

// rho f_ABC of every kept mode into force[inst][3][spec], from the density spectrum of `y_in`.
// A pass of its own: the assembly updates the state in place, so it must not read neighbouring
// modes of it.
template <typename CT>
__global__ void force_kernel(const CT *__restrict__ y_in, CT *__restrict__ force, const PhysDev *__restrict__ phys,
                             int K, int batch) {
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const size_t total = spec * batch;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int inst = (int)(idx / spec);
    const size_t m = idx - (size_t)inst * spec;
    const PhysDev ph = phys[inst];
    if (ph.famp == 0.0) continue;
    const int kxi = (int)(m % NX);
    const size_t t = m / NX;
    CT fo[3];
    const CT *rho = y_in + (size_t)inst * 7 * spec;
    abc_force<CT>([&](int x, int y, int z) { return rho_at(rho, x, y, z, K); }, kxi, kept_wave((int)(t % NK), K),
                  kept_wave((int)(t / NK), K), ph, fo);
#pragma unroll
    for (int a = 0; a < 3; ++a) force[((size_t)inst * 3 + a) * spec + m] = fo[a];
  }
}

// The same force in the double-float mode: formed in FP64 from the double-float density spectrum
// (a pass of its own, only for instances with the force on), stored as double-float values.
__global__ void force_dfloat_kernel(const cdf *__restrict__ y_in, cdf *__restrict__ force,
                                    const PhysDev *__restrict__ phys, int K, int batch) {
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const size_t total = spec * batch;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int inst = (int)(idx / spec);
    const size_t m = idx - (size_t)inst * spec;
    const PhysDev ph = phys[inst];
    if (ph.famp == 0.0) continue;
    const int kxi = (int)(m % NX);
    const size_t t = m / NX;
    cplx64 fo[3];
    const cdf *rho = y_in + (size_t)inst * 7 * spec;
    abc_force<cplx64>(
        [&](int x, int y, int z) {
          const cdf v = rho_at(rho, x, y, z, K);
          return cplx64{dfr_to_double(v.re), dfr_to_double(v.im)};
        },
        kxi, kept_wave((int)(t % NK), K), kept_wave((int)(t / NK), K), ph, fo);
#pragma unroll
    for (int a = 0; a < 3; ++a) force[((size_t)inst * 3 + a) * spec + m] = cdf_from_c64(fo[a].re, fo[a].im);
  }
}

__global__ void split_state_kernel(const cplx64 *__restrict__ in, cplx32 *__restrict__ hi, cplx32 *__restrict__ lo,
                                   size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const cplx64 v = in[i];
    const float hr = (float)v.re, hm = (float)v.im;
    hi[i] = cplx32{hr, hm};
    lo[i] = cplx32{(float)(v.re - (double)hr), (float)(v.im - (double)hm)};
  }
}

__global__ void combine_state_kernel(const cplx32 *__restrict__ hi, const cplx32 *__restrict__ lo,
                                     cplx64 *__restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const cplx32 a = hi[i], b = lo[i];
    out[i] = cplx64{(double)a.re + (double)b.re, (double)a.im + (double)b.im};
  }
}

__global__ void split_cdf_kernel(const cplx64 *__restrict__ in, cdf *__restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const cplx64 v = in[i];
    out[i] = cdf_from_c64(v.re, v.im);
  }
}

__global__ void combine_cdf_kernel(const cdf *__restrict__ in, cplx64 *__restrict__ out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const cdf v = in[i];
    out[i] = cplx64{dfr_to_double(v.re), dfr_to_double(v.im)};
  }
}

// Double-float mode: the RHS of the FP64 assembly above, term by term in the same order, and the
// update of the double-float state, in double-float arithmetic (no FP64 operation per mode).  The
// wavenumbers, k^2 and the product spectra's factor 1/(2 N^3) are exact FP32 numbers.
__device__ __forceinline__ void assemble_mode_dfloat(const cdf *__restrict__ flux, const cdf *y_in, cdf *state,
                                       cdf *__restrict__ hist, cdf *ystage, cplx64 *__restrict__ rhs_out,
                                       const PhysDev *__restrict__ phys, const StepCoef *__restrict__ coef,
                                       const cdf *__restrict__ force, int op, int stage, int K, float inv_n3,
                                       int inst, size_t m, cdf *ynew, int ystride) {
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const int kxi = (int)(m % NX);
  const size_t t = m / NX;
  const int jy = (int)(t % NK), jz = (int)(t / NK);
  const float kx = (float)kxi, ky = (float)kept_wave(jy, K), kz = (float)kept_wave(jz, K);
  const float k2 = __fadd_rn(__fadd_rn(__fmul_rn(kx, kx), __fmul_rn(ky, ky)), __fmul_rn(kz, kz));  // exact
  const dfr nu = phys[inst].nu_df, eta = phys[inst].eta_df, cs2 = phys[inst].cs2_df;
  const float skx = __fmul_rn(kx, inv_n3), sky = __fmul_rn(ky, inv_n3), skz = __fmul_rn(kz, inv_n3);
  const dfr nuk2s = dfr_scale2(k2 * nu, inv_n3);

  const cdf *S = y_in + (size_t)inst * 7 * spec + m;
  const cdf *F = flux + (size_t)inst * 12 * spec + m;
  cdf y[7], f[12];
#pragma unroll
  for (int q = 0; q < 7; ++q) y[q] = S[q * spec];
#pragma unroll
  for (int q = 0; q < 12; ++q) f[q] = F[q * spec];
  const cdf Txx = f[0], Tyy = f[1], Tzz = f[2], Txy = f[3], Txz = f[4], Tyz = f[5];
  const cdf Ex = f[6], Ey = f[7], Ez = f[8];

  cdf r[7];
  {  // continuity: -i k . m
    const cdf s = {kx * y[1].re + ky * y[2].re + kz * y[3].re, kx * y[1].im + ky * y[2].im + kz * y[3].im};
    r[0] = cdf{s.im, -s.re};
  }
  {  // momentum
    const float kk[3] = {kx, ky, kz};
    const cdf T[3][3] = {{Txx, Txy, Txz}, {Txy, Tyy, Tyz}, {Txz, Tyz, Tzz}};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cdf divT = {skx * T[a][0].re + sky * T[a][1].re + skz * T[a][2].re,
                        skx * T[a][0].im + sky * T[a][1].im + skz * T[a][2].im};
      const dfr kc = kk[a] * cs2;
      const cdf g = {divT.re + kc * y[0].re, divT.im + kc * y[0].im};
      const cdf u = f[9 + a];
      r[1 + a] = cdf{g.im - nuk2s * u.re, -g.re - nuk2s * u.im};
    }
    if (force != nullptr && phys[inst].famp != 0.0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const cdf fo = force[((size_t)inst * 3 + a) * spec + m];
        r[1 + a] = cdf{r[1 + a].re + fo.re, r[1 + a].im + fo.im};
      }
    }
  }
  {  // induction: i k x E - eta k^2 B
    const cdf c[3] = {{sky * Ez.re - skz * Ey.re, sky * Ez.im - skz * Ey.im},
                      {skz * Ex.re - skx * Ez.re, skz * Ex.im - skx * Ez.im},
                      {skx * Ey.re - sky * Ex.re, skx * Ey.im - sky * Ex.im}};
    const dfr etak2 = k2 * eta;
#pragma unroll
    for (int a = 0; a < 3; ++a) r[4 + a] = cdf{-c[a].im - etak2 * y[4 + a].re, c[a].re - etak2 * y[4 + a].im};
  }

  const size_t o7 = (size_t)inst * 7 * spec + m;
  if (op == ASM_RHS) {
#pragma unroll
    for (int q = 0; q < 7; ++q) rhs_out[o7 + q * spec] = cplx64{dfr_to_double(r[q].re), dfr_to_double(r[q].im)};
    return;
  }
  const StepCoef cf = coef[inst];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const size_t i = o7 + q * spec;
    const cdf rq = r[q];
    if (op == ASM_AB2 || op == ASM_PC_PRED) {
      // y + dt (a1 f^n + a0 f^{n-1}), as dt a1 f^n + (dt a0 f^{n-1} + y)
      cdf y0 = state[i];
      if (cf.a0 != 0.0) {
        const cdf h = hist[i];
        y0 = cdf{y0.re + cf.dta0_df * h.re, y0.im + cf.dta0_df * h.im};
      }
      const cdf yn = cdf_norm(cdf{y0.re + cf.dta1_df * rq.re, y0.im + cf.dta1_df * rq.im});
      if (op == ASM_AB2) {
        state[i] = yn;
        if (ynew) ynew[q * ystride] = yn;
      } else {
        ystage[i] = yn;
      }
      hist[i] = cdf_norm(rq);
    } else if (op == ASM_RK_STAGE) {
      const cdf acc = cdf_norm(stage == 1 ? rq : cdf{hist[i].re + dfr_scale2(rq.re, 2.f), hist[i].im + dfr_scale2(rq.im, 2.f)});
      hist[i] = acc;
      const dfr w = stage < 3 ? dfr_scale2(cf.dt_df, 0.5f) : cf.dt_df;
      const cdf y0 = state[i];
      ystage[i] = cdf_norm(cdf{y0.re + w * rq.re, y0.im + w * rq.im});
    } else {  // ASM_RK_FINAL, ASM_PC_CORR
      const dfr w = op == ASM_RK_FINAL ? cf.dt6_df : dfr_scale2(cf.dt_df, 0.5f);
      const cdf h = hist[i], y0 = state[i];
      const cdf acc = {h.re + rq.re, h.im + rq.im};
      state[i] = cdf_norm(cdf{y0.re + w * acc.re, y0.im + w * acc.im});
    }
  }
}

__global__ void assemble_dfloat_kernel(const cdf *__restrict__ flux, const cdf *y_in, cdf *state,
                                       cdf *__restrict__ hist, cdf *ystage, cplx64 *__restrict__ rhs_out,
                                       const PhysDev *__restrict__ phys, const StepCoef *__restrict__ coef,
                                       const cdf *__restrict__ force, int op, int stage, int K, int batch,
                                       float inv_n3) {
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const size_t total = spec * batch;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int inst = (int)(idx / spec);
    const size_t m = idx - (size_t)inst * spec;
    if (op != ASM_RHS && coef[inst].skip) continue;
    assemble_mode_dfloat(flux, y_in, state, hist, ystage, rhs_out, phys, coef, force, op, stage, K, inv_n3, inst, m,
                         nullptr, 0);
  }
}

// One thread per instance: the CFL maximum of the flux pass, the step size, the Adams-Bashforth
// coefficients of this step, and the advance of the time state.
__global__ void step_dt_kernel(unsigned long long *__restrict__ smax_bits, const PhysDev *__restrict__ phys,
                               TimeState *__restrict__ ts, StepCoef *__restrict__ coef, int batch, int n, int K,
                               double dt_fixed, double cfl_adv, double cfl_visc) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= batch) return;
  const double m = __longlong_as_double((long long)smax_bits[inst]);
  smax_bits[inst] = 0ull;
  TimeState s = ts[inst];
  StepCoef c = {0.0, 0.0, 0.0, 0.f, 0.f, 0.f, 1};
  if (s.status == 0 && (s.step_limit == 0 || s.step < s.step_limit)) {
    double dt;
    if (dt_fixed > 0.0) {
      dt = dt_fixed;
    } else {
      const double dx = 2.0 * M_PI / (double)n;
      dt = cfl_adv * dx / m;
      const double diff = phys[inst].nu > phys[inst].eta ? phys[inst].nu : phys[inst].eta;
      if (diff > 0.0 && K > 0) {
        const double dtv = cfl_visc / (diff * (double)K * (double)K);
        if (dtv < dt) dt = dtv;
      }
    }
    if (!isfinite(m) || !isfinite(dt) || dt <= 0.0) {
      s.status = 5;  // MHD_ENONFINITE
    } else {
      c.dt = dt;
      c.skip = 0;
      if (s.step > 0) {
        const double r = dt / s.dt_prev;
        c.a1 = 1.0 + 0.5 * r;
        c.a0 = -0.5 * r;
      } else {
        c.a1 = 1.0;
        c.a0 = 0.0;
      }
      c.fdt = (float)c.dt;
      c.fa1 = (float)c.a1;
      c.fa0 = (float)c.a0;
      c.dt_df = dfr_from_double(c.dt);
      c.dta1_df = dfr_from_double(c.dt * c.a1);
      c.dta0_df = dfr_from_double(c.dt * c.a0);
      c.dt6_df = dfr_from_double(c.dt / 6.0);
      s.t += dt;
      s.dt_prev = dt;
      s.dt_last = dt;
      s.step += 1;
    }
  }
  ts[inst] = s;
  coef[inst] = c;
}

// One block: reduce the diagnostic partials of one instance in a fixed order and add the
// spectral terms.  out: [0] ke [1] me [2] eint [3] cross_hel [4] mean_speed [5] mean_bmag
// [6] smax [7] mean_rho [8..10] mean_m [11..13] mean_b [14] divb_rms [15] t [16] dt_last
// [17] step [18] status.
__global__ void diag_finish_kernel(const double *__restrict__ part, int nparts, const double *__restrict__ dpart,
                                   int ndparts, const cplx64 *__restrict__ state, const PhysDev *__restrict__ phys,
                                   const TimeState *__restrict__ ts, double *__restrict__ out, int n, int K) {
  __shared__ double red[32];
  const double inv_n3 = 1.0 / ((double)n * n * n);
  for (int q = 0; q < 7; ++q) {
    double v = 0.0;
    if (q < 6) {
      for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[(size_t)i * 8 + q];
      v = block_sum(v, red);
    } else {
      for (int i = threadIdx.x; i < nparts; i += blockDim.x) v = nan_max(v, part[(size_t)i * 8 + q]);
      v = block_nan_max(v, red);
    }
    if (threadIdx.x == 0) out[q] = q < 6 ? v * inv_n3 : v;
  }
  double d = 0.0;
  for (int i = threadIdx.x; i < ndparts; i += blockDim.x) d += dpart[i];
  d = block_sum(d, red);
  if (threadIdx.x == 0) {
    const int NX = K + 1, NK = 2 * K + 1;
    const size_t spec = (size_t)NK * NK * NX;
    out[7] = state[0].re;
    for (int a = 0; a < 3; ++a) {
      out[8 + a] = state[(1 + a) * spec].re;
      out[11 + a] = state[(4 + a) * spec].re;
    }
    out[14] = sqrt(d);
    out[15] = ts->t;
    out[16] = ts->dt_last;
    out[17] = (double)ts->step;
    out[18] = (double)ts->status;
  }
}

// Partial sums of |k . B_hat|^2 over the full spectrum (k_x > 0 counted twice for the mirrored
// half), one per block over a fixed grid-stride share of the kept modes.
__global__ void __launch_bounds__(256) divb_partials_kernel(const cplx64 *__restrict__ state,
                                                            double *__restrict__ dpart, int K) {
  __shared__ double red[32];
  const int NX = K + 1, NK = 2 * K + 1;
  const int spec = NK * NK * NX;  // < 2^31 for every supported N
  double d = 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < spec; m += gridDim.x * blockDim.x) {
    const int kxi = m % NX;
    const int t = m / NX;
    const double kx = kxi, ky = kept_wave(t % NK, K), kz = kept_wave(t / NK, K);
    const cplx64 bx = state[4 * (size_t)spec + m], by = state[5 * (size_t)spec + m], bz = state[6 * (size_t)spec + m];
    const double re = kx * bx.re + ky * by.re + kz * bz.re;
    const double im = kx * bx.im + ky * by.im + kz * bz.im;
    d += (kxi > 0 ? 2.0 : 1.0) * (re * re + im * im);
  }
  d = block_sum(d, red);
  if (threadIdx.x == 0) dpart[blockIdx.x] = d;
}

// Truncated spectrum -> full half-complex layout [N][N][N/2+1], zeros outside the kept set.
__global__ void expand_kernel(const cplx64 *__restrict__ in, cplx64 *__restrict__ out, int n, int K) {
  const int H = n / 2 + 1, NX = K + 1;
  const size_t total = (size_t)n * n * H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % H);
    const size_t t = i / H;
    const int fy = (int)(t % n), fz = (int)(t / n);
    // FFT index -> kept index (or -1)
    const int jy = fy <= K ? fy : (fy >= n - K ? fy - n + 2 * K + 1 : -1);
    const int jz = fz <= K ? fz : (fz >= n - K ? fz - n + 2 * K + 1 : -1);
    cplx64 v = {0.0, 0.0};
    if (kx <= K && jy >= 0 && jz >= 0) v = in[((size_t)jz * (2 * K + 1) + jy) * NX + kx];
    out[i] = v;
  }
}

__global__ void status_any_kernel(const TimeState *__restrict__ ts, int batch, int32_t *flag) {
  int any = 0;
  for (int i = threadIdx.x; i < batch; i += blockDim.x) any |= ts[i].status != 0;
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) *flag = any;
}

// ------------------------------------------------------------------------------------------

static unsigned grid_for(size_t total, int threads) {
  size_t b = (total + threads - 1) / threads;
  const size_t cap = 152 * 16;  // enough blocks to fill every SM several times; grid-stride beyond
  if (b > cap) b = cap;
  return (unsigned)(b == 0 ? 1 : b);
}

cudaError_t launch_assemble(const cplx64 *flux, const cplx64 *y_in, cplx64 *state, cplx64 *hist, cplx64 *ystage,
                            cplx64 *rhs_out, const PhysDev *phys, const StepCoef *coef, int op, int stage,
                            const Dims &d, cudaStream_t s, const cplx64 *force) {
  const size_t total = d.spec * d.batch;
  // the flux passes leave their spectra doubled (the split's 1/2 is taken here)
  const double inv_n3 = 0.5 / ((double)d.n * d.n * d.n);
  assemble_kernel<cplx64><<<grid_for(total, 256), 256, 0, s>>>(flux, y_in, state, hist, ystage, rhs_out, phys, coef,
                                                               force, op, stage, d.k, d.batch, inv_n3);
  return cudaGetLastError();
}

cudaError_t launch_force(const cplx64 *y_in, cplx64 *force, const PhysDev *phys, const Dims &d, cudaStream_t s) {
  force_kernel<cplx64><<<grid_for(d.spec * d.batch, 256), 256, 0, s>>>(y_in, force, phys, d.k, d.batch);
  return cudaGetLastError();
}

cudaError_t launch_force(const cplx32 *y_in, cplx32 *force, const PhysDev *phys, const Dims &d, cudaStream_t s) {
  force_kernel<cplx32><<<grid_for(d.spec * d.batch, 256), 256, 0, s>>>(y_in, force, phys, d.k, d.batch);
  return cudaGetLastError();
}

cudaError_t launch_assemble_df(const cplx32 *flux, const cplx32 *y_in, cplx32 *s_hi, cplx32 *s_lo, cplx32 *hist,
                               cplx32 *ystage, cplx64 *rhs_out, const PhysDev *phys, const StepCoef *coef, int op,
                               int stage, const Dims &d, cudaStream_t s, const cplx32 *force) {
  const size_t total = d.spec * d.batch;
  const float inv_n3 = (float)(0.5 / ((double)d.n * d.n * d.n));  // with the split's 1/2
  assemble_df_kernel<<<grid_for(total, 256), 256, 0, s>>>(flux, y_in, s_hi, s_lo, hist, ystage, rhs_out, phys, coef,
                                                          force, op, stage, d.k, d.batch, inv_n3);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const cdf *flux, const cdf *y_in, cdf *state, cdf *hist, cdf *ystage, cplx64 *rhs_out,
                            const PhysDev *phys, const StepCoef *coef, int op, int stage, const Dims &d,
                            cudaStream_t s, const cdf *force) {
  const size_t total = d.spec * d.batch;
  const float inv_n3 = (float)(0.5 / ((double)d.n * d.n * d.n));  // a power of two, with the split's 1/2
  assemble_dfloat_kernel<<<grid_for(total, 256), 256, 0, s>>>(flux, y_in, state, hist, ystage, rhs_out, phys, coef,
                                                              force, op, stage, d.k, d.batch, inv_n3);
  return cudaGetLastError();
}

cudaError_t launch_force(const cdf *y_in, cdf *force, const PhysDev *phys, const Dims &d, cudaStream_t s) {
  force_dfloat_kernel<<<grid_for(d.spec * d.batch, 256), 256, 0, s>>>(y_in, force, phys, d.k, d.batch);
  return cudaGetLastError();
}

cudaError_t launch_split_state(const cplx64 *in, cdf *out, size_t count, cudaStream_t s) {
  split_cdf_kernel<<<grid_for(count, 256), 256, 0, s>>>(in, out, count);
  return cudaGetLastError();
}

cudaError_t launch_combine_state(const cdf *in, cplx64 *out, size_t count, cudaStream_t s) {
  combine_cdf_kernel<<<grid_for(count, 256), 256, 0, s>>>(in, out, count);
  return cudaGetLastError();
}

cudaError_t launch_split_state(const cplx64 *in, cplx32 *hi, cplx32 *lo, size_t count, cudaStream_t s) {
  split_state_kernel<<<grid_for(count, 256), 256, 0, s>>>(in, hi, lo, count);
  return cudaGetLastError();
}

cudaError_t launch_combine_state(const cplx32 *hi, const cplx32 *lo, cplx64 *out, size_t count, cudaStream_t s) {
  combine_state_kernel<<<grid_for(count, 256), 256, 0, s>>>(hi, lo, out, count);
  return cudaGetLastError();
}

cudaError_t launch_step_dt(unsigned long long *smax_bits, const PhysDev *phys, TimeState *ts, StepCoef *coef,
                           const Dims &d, double dt_fixed, double cfl_adv, double cfl_visc, cudaStream_t s) {
  step_dt_kernel<<<(d.batch + 127) / 128, 128, 0, s>>>(smax_bits, phys, ts, coef, d.batch, d.n, d.k, dt_fixed, cfl_adv,
                                                       cfl_visc);
  return cudaGetLastError();
}

cudaError_t launch_diag_finish(const double *part, int nparts, const cplx64 *state, const PhysDev *phys,
                               const TimeState *ts, double *out, const Dims &d, cudaStream_t s, double *dpart) {
  divb_partials_kernel<<<kDivbBlocks, 256, 0, s>>>(state, dpart, d.k);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_finish_kernel<<<1, 1024, 0, s>>>(part, nparts, dpart, kDivbBlocks, state, phys, ts, out, d.n, d.k);
  return cudaGetLastError();
}

cudaError_t launch_expand_spectrum(const cplx64 *in, cplx64 *out, const Dims &d, cudaStream_t s) {
  const size_t total = (size_t)d.n * d.n * (d.n / 2 + 1);
  expand_kernel<<<grid_for(total, 256), 256, 0, s>>>(in, out, d.n, d.k);
  return cudaGetLastError();
}

cudaError_t launch_status_any(const TimeState *ts, int batch, int32_t *flag, cudaStream_t s) {
  status_any_kernel<<<1, 256, 0, s>>>(ts, batch, flag);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Assembly and Adams-Bashforth update fused with the next step's inverse z pass
// ------------------------------------------------------------------------------------------
// The update of a kept mode needs only that mode, and the inverse z transform of the new state
// needs only the modes of one (ky', kx) column, so one block can do both for a tile of columns:
// instance blockIdx.y, TC = 2^tsh consecutive columns q of the (ky', kx) plane (cols = NK NX).
//   1. every kept kz row l of those columns: the RHS, the update of state and history (the
//      assembly kernel's arithmetic at that mode, term for term), and the 7 new state values
//      dropped into 7 TC pencils of length N in shared memory at FFT index kept_to_fft(l);
//   2. the pencils' inverse transform, zero-padded by the 2/3 rule (the column pass's transform);
//   3. the z-pass output z_out [b][7][N][cols] that the next step's inverse y pass reads.
// The 12 product spectra and the new state never make the round trip through HBM that the
// separate forward-z -> assembly -> inverse-z kernels cost.  An instance that takes no step
// (coef.skip) keeps its state and still gets its transform.
__device__ __forceinline__ void fused_mode(const cplx64 *flux, cplx64 *state, cplx64 *, cplx64 *hist,
                                           const PhysDev *phys, const StepCoef *coef, const cplx64 *force, int K,
                                           double inv_n3, int inst, size_t m, cplx64 *yn, int ys) {
  assemble_mode_fp64<cplx64>(flux, state, state, hist, nullptr, nullptr, phys, coef, force, ASM_AB2, 0, K, inv_n3,
                             inst, m, yn, ys);
}
__device__ __forceinline__ void fused_mode(const cdf *flux, cdf *state, cdf *, cdf *hist, const PhysDev *phys,
                                           const StepCoef *coef, const cdf *force, int K, float inv_n3, int inst,
                                           size_t m, cdf *yn, int ys) {
  assemble_mode_dfloat(flux, state, state, hist, nullptr, nullptr, phys, coef, force, ASM_AB2, 0, K, inv_n3, inst, m,
                       yn, ys);
}
// mixed: `state` holds the high parts, `lo` the low parts; the transform takes the new high part
__device__ __forceinline__ void fused_mode(const cplx32 *flux, cplx32 *state, cplx32 *lo, cplx32 *hist,
                                           const PhysDev *phys, const StepCoef *coef, const cplx32 *force, int K,
                                           float inv_n3, int inst, size_t m, cplx32 *yn, int ys) {
  assemble_mode_mixed(flux, state, state, lo, hist, nullptr, nullptr, phys, coef, force, ASM_AB2, 0, K, inv_n3, inst,
                      m, yn, ys);
}

// Threads of a block: 7 TC pencils x TPP; the most any (N, VPT) launches.
template <int N, int VPT>
__host__ __device__ constexpr int fused_max_threads() {
  return 7 * (tpp_for<N, VPT>() >= 64 ? tpp_for<N, VPT>() : 64);
}

template <int N, int VPT, typename C>
__global__ void __launch_bounds__(fused_max_threads<N, VPT>(), (fused_max_threads<N, VPT>() <= 448 ? 2 : 1))
    assemble_iz_kernel(const C *__restrict__ flux, C *state, C *lo, C *__restrict__ hist,
                       const PhysDev *__restrict__ phys, const StepCoef *__restrict__ coef,
                       const C *__restrict__ force, C *__restrict__ z_out, int tsh,
                       typename scale_of<C>::type inv_n3, const C *__restrict__ tw) {
  constexpr int TPP = tpp_for<N, VPT>();
  constexpr int P = pencil_pitch<C>(N);
  constexpr int K = (N - 1) / 3;
  constexpr int NK = 2 * K + 1, NX = K + 1;
  constexpr int COLS = NK * NX;
  constexpr size_t SPEC = (size_t)NK * COLS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sm = reinterpret_cast<C *>(smem_raw);
  const int tc = 1 << tsh;
  const int nthr = blockDim.x;
  const int inst = blockIdx.y;
  const int q0 = blockIdx.x * tc;
  const bool skip = coef[inst].skip != 0;

  // 1. update every kept mode of the tile; the new state goes into the pencils
  for (int it = threadIdx.x; it < tc * NK; it += nthr) {
    const int c = it & (tc - 1), l = it >> tsh;
    const int q = q0 + c;
    C *yn = sm + c * P + sm_idx<C>(kept_to_fft(l, K, N));  // field f at yn[f * tc * P]
    if (q < COLS) {
      const size_t m = (size_t)l * COLS + q;
      if (skip) {
#pragma unroll
        for (int f = 0; f < 7; ++f) yn[f * tc * P] = state[((size_t)inst * 7 + f) * SPEC + m];
      } else {
        fused_mode(flux, state, lo, hist, phys, coef, force, K, inv_n3, inst, m, yn, tc * P);
      }
    } else {
#pragma unroll
      for (int f = 0; f < 7; ++f) yn[f * tc * P] = C{0, 0};
    }
  }
  // FFT indices K+1 .. N-K-1 are outside the kept set
  for (int it = threadIdx.x; it < 7 * tc * (N - NK); it += nthr) {
    const int p = it / (N - NK), r = it - p * (N - NK);
    sm[p * P + sm_idx<C>(K + 1 + r)] = C{0, 0};
  }
  __syncthreads();

  // 2. inverse z transforms of the 7 TC pencils
  const int pencil = threadIdx.x / TPP;
  const int t = threadIdx.x - pencil * TPP;
  const bool active = q0 + (pencil & (tc - 1)) < COLS;
  pencil_fft<N, +1, C, VPT, true>(sm + (active ? pencil : 0) * P, t, active, tw);
  __syncthreads();

  // 3. rows z of the next inverse y pass's input, TC consecutive columns per row
  for (int it = threadIdx.x; it < 7 * tc * N; it += nthr) {
    const int c = it & (tc - 1), r = it >> tsh;  // r = f N + z
    const int f = r / N, z = r - f * N;
    const int q = q0 + c;
    if (q < COLS) z_out[((size_t)inst * 7 * N + r) * COLS + q] = c_store(sm[(f * tc + c) * P + sm_idx<C>(z)]);
  }
}

namespace {

template <int N, int VPT, typename C>
cudaError_t assemble_iz_n(const C *flux, C *state, C *lo, C *hist, const PhysDev *phys, const StepCoef *coef,
                          const C *force, C *z_out, const C *tw, int nb, int tile, cudaStream_t s) {
  constexpr int TPP = tpp_for<N, VPT>();
  constexpr int K = (N - 1) / 3;
  constexpr int COLS = (2 * K + 1) * (K + 1);
  constexpr int MAXT = fused_max_threads<N, VPT>();
  if (nb <= 0) return cudaSuccess;
  if (nb > 65535) return cudaErrorInvalidValue;
  int tc = tile > 0 ? tile : (TPP >= 64 ? 1 : 64 / TPP);
  while (tc > 1 && 7 * tc * TPP > MAXT) tc /= 2;
  int tsh = 0;
  while ((2 << tsh) <= tc) ++tsh;
  tc = 1 << tsh;
  const size_t smem = (size_t)7 * tc * pencil_pitch<C>(N) * sizeof(C);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  constexpr auto kfn = assemble_iz_kernel<N, VPT, C>;
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem<kfn>((int)smem);
    if (e != cudaSuccess) return e;
  }
  // the product spectra arrive unnormalised and doubled (the split's 1/2 is taken here)
  const auto inv_n3 = (typename scale_of<C>::type)(0.5 / ((double)N * N * N));
  kfn<<<dim3((COLS + tc - 1) / tc, nb), 7 * tc * TPP, smem, s>>>(flux, state, lo, hist, phys, coef, force, z_out, tsh,
                                                                inv_n3, tw);
  return cudaGetLastError();
}

template <int VPT, typename C>
cudaError_t assemble_iz_v(const C *flux, C *state, C *lo, C *hist, const PhysDev *phys, const StepCoef *coef,
                          const C *force, C *z_out, const C *tw, const Dims &d, int tile, cudaStream_t s) {
  switch (d.n) {
    case 16: return assemble_iz_n<16, VPT>(flux, state, lo, hist, phys, coef, force, z_out, tw, d.batch, tile, s);
    case 32: return assemble_iz_n<32, VPT>(flux, state, lo, hist, phys, coef, force, z_out, tw, d.batch, tile, s);
    case 64: return assemble_iz_n<64, VPT>(flux, state, lo, hist, phys, coef, force, z_out, tw, d.batch, tile, s);
    case 128: return assemble_iz_n<128, VPT>(flux, state, lo, hist, phys, coef, force, z_out, tw, d.batch, tile, s);
    case 256: return assemble_iz_n<256, VPT>(flux, state, lo, hist, phys, coef, force, z_out, tw, d.batch, tile, s);
    case 512: return assemble_iz_n<512, VPT>(flux, state, lo, hist, phys, coef, force, z_out, tw, d.batch, tile, s);
    case 1024: return assemble_iz_n<1024, VPT>(flux, state, lo, hist, phys, coef, force, z_out, tw, d.batch, tile, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_assemble_iz(const cplx64 *flux, cplx64 *state, cplx64 *hist, const PhysDev *phys,
                               const StepCoef *coef, const cplx64 *force, cplx64 *z_out, const cplx64 *tw,
                               const Dims &d, int tile, cudaStream_t s) {
  return assemble_iz_v<8>(flux, state, (cplx64 *)nullptr, hist, phys, coef, force, z_out, tw, d, tile, s);
}

cudaError_t launch_assemble_iz(const cdf *flux, cdf *state, cdf *hist, const PhysDev *phys, const StepCoef *coef,
                               const cdf *force, cdf *z_out, const cdf *tw, const Dims &d, int tile, cudaStream_t s) {
  return assemble_iz_v<8>(flux, state, (cdf *)nullptr, hist, phys, coef, force, z_out, tw, d, tile, s);
}

// `vpt` as the inverse z column pass takes it (0: radix 16 at N >= 512, else 8), so that the
// transform is that pass's to the bit.
cudaError_t launch_assemble_iz(const cplx32 *flux, cplx32 *s_hi, cplx32 *s_lo, cplx32 *hist, const PhysDev *phys,
                               const StepCoef *coef, const cplx32 *force, cplx32 *z_out, const cplx32 *tw,
                               const Dims &d, int tile, int vpt, cudaStream_t s) {
  if (vpt == 16 || (vpt == 0 && d.n >= 512))
    return assemble_iz_v<16>(flux, s_hi, s_lo, hist, phys, coef, force, z_out, tw, d, tile, s);
  return assemble_iz_v<8>(flux, s_hi, s_lo, hist, phys, coef, force, z_out, tw, d, tile, s);
}

}  // namespace mhd
