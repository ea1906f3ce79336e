// fft_device.cuh -- device building blocks: complex arithmetic, small DFTs in registers, and the
// Stockham pencil FFT executed by a group of N/VPT threads (VPT = 8, or 16 in FP32) on a pencil
// held in shared memory.
//
// Transform convention (both directions unscaled):  X[k] = sum_j x[j] exp(DIR * 2 pi i j k / N)
// with DIR = -1 for the forward and +1 for the inverse transform.
#pragma once

#include "dfloat.cuh"
#include "mhd_internal.h"

#include <type_traits>

namespace mhd {

template <typename C>
__device__ __forceinline__ C c_add(C a, C b) { return {a.re + b.re, a.im + b.im}; }
template <typename C>
__device__ __forceinline__ C c_sub(C a, C b) { return {a.re - b.re, a.im - b.im}; }
template <typename C>
__device__ __forceinline__ C c_scale(C a, typename C::value_type s) { return {a.re * s, a.im * s}; }
// a * w
template <typename C>
__device__ __forceinline__ C c_mul(C a, C w) {
  return {a.re * w.re - a.im * w.im, a.re * w.im + a.im * w.re};
}
// a * conj(w)
template <typename C>
__device__ __forceinline__ C c_mulc(C a, C w) {
  return {a.re * w.re + a.im * w.im, a.im * w.re - a.re * w.im};
}
// a * (DIR i)
template <int DIR, typename C>
__device__ __forceinline__ C c_mul_i(C a) {
  return DIR > 0 ? C{-a.im, a.re} : C{a.im, -a.re};
}
// precision conversion
template <typename CT, typename CF>
__device__ __forceinline__ CT c_cvt(CF a) {
  using R = typename CT::value_type;
  return CT{(R)a.re, (R)a.im};
}

// Double-float complex values use the generic forms above through the dfr operators (lazy sums
// and products).  A pass scales its output by a power of two only, given as an FP32 number.
__device__ __forceinline__ cdf c_scale(cdf a, float s) { return cdf{s * a.re, s * a.im}; }

// What a pass stores to global memory: double-float values renormalised, others as they are.
template <typename C>
__device__ __forceinline__ C c_store(C a) { return a; }
__device__ __forceinline__ cdf c_store(cdf a) { return cdf_norm(a); }

// NaN-propagating maximum (a non-finite CFL speed must reach the step-size kernel).
__device__ __forceinline__ double nan_max(double a, double b) {
  if (a != a) return a;
  if (b != b) return b;
  return a > b ? a : b;
}

// ---- DFTs of length 2, 4, 8 on registers, natural order in and out ----

template <int DIR, typename C>
__device__ __forceinline__ void dft2(C *v) {
  const C a = v[0], b = v[1];
  v[0] = c_add(a, b);
  v[1] = c_sub(a, b);
}

template <int DIR, typename C>
__device__ __forceinline__ void dft4(C *v) {
  const C s0 = c_add(v[0], v[2]), d0 = c_sub(v[0], v[2]);
  const C s1 = c_add(v[1], v[3]), d1 = c_mul_i<DIR>(c_sub(v[1], v[3]));
  v[0] = c_add(s0, s1);
  v[2] = c_sub(s0, s1);
  v[1] = c_add(d0, d1);
  v[3] = c_sub(d0, d1);
}

// Length 8 by one decimation-in-frequency split: b_j = a_j + a_{j+4} feeds the even outputs,
// c_j = (a_j - a_{j+4}) W8^j the odd ones, each through a length-4 DFT.
template <int DIR, typename C>
__device__ __forceinline__ void dft8(C *v) {
  using R = typename C::value_type;
  constexpr R h = (R)0.70710678118654752440;  // sqrt(2) / 2
  C b[4], c[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    b[j] = c_add(v[j], v[j + 4]);
    c[j] = c_sub(v[j], v[j + 4]);
  }
  // W8^1 = h (1 + DIR i), W8^2 = DIR i, W8^3 = h (-1 + DIR i)
  c[1] = C{h * (c[1].re - DIR * c[1].im), h * (c[1].im + DIR * c[1].re)};
  c[2] = c_mul_i<DIR>(c[2]);
  c[3] = C{h * (-c[3].re - DIR * c[3].im), h * (-c[3].im + DIR * c[3].re)};
  dft4<DIR>(b);
  dft4<DIR>(c);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    v[2 * m] = b[m];
    v[2 * m + 1] = c[m];
  }
}

// Length 16 as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.  Length-4 DFTs over n1 for each n2, the
// twiddles W16^(n2 k1), then length-4 DFTs over n2 for each k1 (W16 = exp(DIR 2 pi i / 16)).
// ZP: inputs 6..9 are zeros (zero-padded first stage; see pencil_fft): each first-layer length-4
// DFT then has one zero input and loses a butterfly.
template <int DIR, typename C, bool ZP = false>
__device__ __forceinline__ void dft16(C *v) {
  using R = typename C::value_type;
  constexpr R c1 = (R)0.92387953251128675613;  // cos(pi/8)
  constexpr R s1 = (R)0.38268343236508977173;  // sin(pi/8)
  constexpr R h = (R)0.70710678118654752440;   // cos(pi/4)
  C a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C t[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
    if constexpr (ZP) {
      if (n2 < 2) {  // t[2] = v8 or v9 = 0: (t0 + t2, t0 - t2) = (t0, t0)
        const C s1 = c_add(t[1], t[3]), d1 = c_mul_i<DIR>(c_sub(t[1], t[3]));
        t[2] = c_sub(t[0], s1);
        t[1] = c_add(t[0], d1);
        t[3] = c_sub(t[0], d1);
        t[0] = c_add(t[0], s1);
      } else {  // t[1] = v6 or v7 = 0: (t1 + t3, t1 - t3) = (t3, -t3)
        const C s0 = c_add(t[0], t[2]), d0 = c_sub(t[0], t[2]);
        const C d1 = c_mul_i<DIR>(C{-t[3].re, -t[3].im});
        t[0] = c_add(s0, t[3]);
        t[2] = c_sub(s0, t[3]);
        t[1] = c_add(d0, d1);
        t[3] = c_sub(d0, d1);
      }
    } else {
      dft4<DIR>(t);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = t[k1];
  }
  const C w1 = {c1, DIR * s1}, w2 = {h, DIR * h}, w3 = {s1, DIR * c1};
  const C w6 = {-h, DIR * h}, w9 = {-c1, -DIR * s1};
  a[1][1] = c_mul(a[1][1], w1);
  a[1][2] = c_mul(a[1][2], w2);
  a[1][3] = c_mul(a[1][3], w3);
  a[2][1] = c_mul(a[2][1], w2);
  a[2][2] = c_mul_i<DIR>(a[2][2]);  // W16^4 = DIR i
  a[2][3] = c_mul(a[2][3], w6);
  a[3][1] = c_mul(a[3][1], w3);
  a[3][2] = c_mul(a[3][2], w6);
  a[3][3] = c_mul(a[3][3], w9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4<DIR>(t);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
  }
}

// Length 8 in double-float: the same split as above; W8 = h (1 + DIR i) with h = sqrt(2)/2 in
// double-float.
template <int DIR>
__device__ __forceinline__ void dft8(cdf *v) {
  constexpr dfr h = dfr_const(0.70710678118654752440);
  cdf b[4], c[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    b[j] = c_add(v[j], v[j + 4]);
    c[j] = c_sub(v[j], v[j + 4]);
  }
  if constexpr (DIR > 0) {
    c[1] = cdf{h * (c[1].re - c[1].im), h * (c[1].im + c[1].re)};
    c[3] = cdf{h * (-c[3].re - c[3].im), h * (c[3].re - c[3].im)};
  } else {
    c[1] = cdf{h * (c[1].re + c[1].im), h * (c[1].im - c[1].re)};
    c[3] = cdf{h * (c[3].im - c[3].re), h * (-c[3].im - c[3].re)};
  }
  c[2] = c_mul_i<DIR>(c[2]);
  dft4<DIR>(b);
  dft4<DIR>(c);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    v[2 * m] = b[m];
    v[2 * m + 1] = c[m];
  }
}

// The same with inputs 3 and 4 known zeros (the zero-padded first stage): the first layer's
// pairs (v0, v4) and (v3, v7) need no arithmetic, (v0, v0) and (v7, -v7).  The other inputs
// take the operations of dft8, so the results are dft8's.
template <int DIR>
__device__ __forceinline__ void dft8_zp(cdf *v) {
  constexpr dfr h = dfr_const(0.70710678118654752440);
  cdf b[4], c[4];
  b[0] = v[0];
  c[0] = v[0];
  b[3] = v[7];
  c[3] = cdf{-v[7].re, -v[7].im};
#pragma unroll
  for (int j = 1; j < 3; ++j) {
    b[j] = c_add(v[j], v[j + 4]);
    c[j] = c_sub(v[j], v[j + 4]);
  }
  if constexpr (DIR > 0) {
    c[1] = cdf{h * (c[1].re - c[1].im), h * (c[1].im + c[1].re)};
    c[3] = cdf{h * (-c[3].re - c[3].im), h * (c[3].re - c[3].im)};
  } else {
    c[1] = cdf{h * (c[1].re + c[1].im), h * (c[1].im - c[1].re)};
    c[3] = cdf{h * (c[3].im - c[3].re), h * (-c[3].im - c[3].re)};
  }
  c[2] = c_mul_i<DIR>(c[2]);
  dft4<DIR>(b);
  dft4<DIR>(c);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    v[2 * m] = b[m];
    v[2 * m + 1] = c[m];
  }
}

template <int R, int DIR, typename C>
__device__ __forceinline__ void dft_small(C *v) {
  if constexpr (R == 16) dft16<DIR>(v);
  else if constexpr (R == 8) dft8<DIR>(v);
  else if constexpr (R == 4) dft4<DIR>(v);
  else dft2<DIR>(v);
}

// Twiddle load that the compiler may not hoist out of loops: kernels that transform many pencils
// in a loop would otherwise keep every stage's twiddles live in registers across the loop.
__device__ __forceinline__ cdf tw_load(const cdf *p) {
  cdf v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.re.hi), "=f"(v.re.lo), "=f"(v.im.hi), "=f"(v.im.lo)
               : "l"(p));
  return v;
}
// The same from a generic address (a twiddle table a block has staged in shared memory).
__device__ __forceinline__ cdf tw_load_generic(const cdf *p) {
  cdf v;
  asm volatile("ld.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.re.hi), "=f"(v.re.lo), "=f"(v.im.hi), "=f"(v.im.lo)
               : "l"(p));
  return v;
}
__device__ __forceinline__ cplx64 tw_load(const cplx64 *p) {
  cplx64 v;
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.re), "=d"(v.im) : "l"(p));
  return v;
}
__device__ __forceinline__ cplx32 tw_load(const cplx32 *p) {
  cplx32 v;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.re), "=f"(v.im) : "l"(p));
  return v;
}

// The value of x, opaque to the optimiser: index arithmetic derived from it cannot be hoisted out
// of a persistent loop and kept live (in registers or spilled) across iterations.
__device__ __forceinline__ int launder(int x) {
  int y;
  asm volatile("mov.b32 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}

// ---- shared-memory pencil layout ----
// A pencil element e lives at sm_idx<C>(e) = e + e / (128 / sizeof(C)): one pad element per 128
// bytes.  The first Stockham stage writes with a stride of 8 elements; without the pad every lane
// of a wavefront would hit the same banks.  Pencils are `pencil_pitch` apart, an odd number of
// elements, so that lanes walking across pencils (the column loads) also spread over the banks.
template <typename C>
__host__ __device__ constexpr int sm_idx(int e) { return e + e / (int)(128 / sizeof(C)); }
template <typename C>
__host__ __device__ constexpr int pencil_pitch(int n) { return sm_idx<C>(n) | 1; }

// ---- barrier of one pencil's thread group ----
// A pencil is transformed by the TPP = N/VPT consecutive threads of its group and nobody else
// touches it meanwhile, so the stages only need that group to synchronise: within a warp
// (TPP <= 32) a warp barrier over the lanes that exist, otherwise a named barrier per group
// (ids 1..15; id 0 is __syncthreads), falling back to the block barrier when there are more groups.
__device__ __forceinline__ unsigned existing_lanes() {
  const int left = (int)blockDim.x - (int)(threadIdx.x & ~31u);
  return left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
}

template <int TPP>
__device__ __forceinline__ void group_sync() {
  if constexpr (TPP <= 32) {
    __syncwarp(existing_lanes());
  } else {
    if (blockDim.x / TPP <= 15) {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / TPP)), "r"(TPP) : "memory");
    } else {
      __syncthreads();
    }
  }
}

// ---- FP64 twiddles in FMA form ----
// On GB300 the FP64 pipe bounds the FP64 transforms, so their twiddled stages use fewer FP64
// instructions: every twiddle is kept as W = i^q c (1 + i t) with |t| <= 1, and a radix-2
// butterfly (a + W x, a - W x) costs six fused multiply-adds: z = x + i t x (two), z' = i^q z (an
// exact swap and sign change done with integer operations), a +- c z' (four).  The table follows
// the classic one in the same allocation: tw[0..N) classic W_N^m, then N pairs (c, t), then N
// bytes q (fp64_twiddle_bytes).
struct TwF {
  double c, t;
  int q;
};

template <int N, int DIR>
__device__ __forceinline__ TwF twf_load(const cplx64 *__restrict__ tw, int m) {
  const double *ct = reinterpret_cast<const double *>(tw + N) + 2 * m;
  const unsigned char *qt = reinterpret_cast<const unsigned char *>(tw + 2 * N) + m;
  TwF w;
  unsigned short qq;
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(w.c), "=d"(w.t) : "l"(ct));
  asm volatile("ld.global.nc.u8 %0, [%1];" : "=h"(qq) : "l"(qt));
  w.q = qq;
  if (DIR > 0) {  // the inverse uses conj(W) = i^-q c (1 - i t)
    w.t = -w.t;
    w.q = (4 - w.q) & 3;
  }
  return w;
}

// The same twiddle turned by a quarter DIR i (the factor omega_4 of the DIF split).
template <int DIR>
__device__ __forceinline__ TwF twf_quarter(TwF w) {
  w.q = (w.q + (DIR < 0 ? 3 : 1)) & 3;
  return w;
}

__device__ __forceinline__ double flip_sign(double x, unsigned s) {
  return __hiloint2double(__double2hiint(x) ^ (int)s, __double2loint(x));
}

// i^q z, exactly, with integer selects and sign flips.
__device__ __forceinline__ cplx64 rot_quarter(cplx64 z, int q) {
  const bool sw = q & 1;
  const double a = sw ? z.im : z.re, b = sw ? z.re : z.im;
  const unsigned s_re = (unsigned)((q ^ (q >> 1)) & 1) << 31, s_im = (unsigned)((q >> 1) & 1) << 31;
  return cplx64{flip_sign(a, s_re), flip_sign(b, s_im)};
}

// (x0, x1) <- (x0 + W x1, x0 - W x1)
__device__ __forceinline__ void bfly_fma(cplx64 &x0, cplx64 &x1, const TwF &w) {
  const cplx64 z = rot_quarter(cplx64{fma(-w.t, x1.im, x1.re), fma(w.t, x1.re, x1.im)}, w.q);
  const cplx64 a = x0;
  x0 = cplx64{fma(w.c, z.re, a.re), fma(w.c, z.im, a.im)};
  x1 = cplx64{fma(-w.c, z.re, a.re), fma(-w.c, z.im, a.im)};
}

// Length-R DFT of (W^r x_r)_r, r < R, for R = 8, 4, 2, W = W_N^m in DIR's sense, as radix-2
// layers of the decimation-in-frequency split with every twiddle carried into the butterflies:
//   R = 8: layer 1 W^4 (x4); layer 2 W^2 (x2) and (W w8)^2 = W^2 w4 (x2); layer 3 W, W w4, W w8,
//          W w8 w4, with w8 = W_N^(N/8) and w4 = w8^2 a quarter turn.
// Results in natural order in v.
template <int N, int R, int DIR>
__device__ __forceinline__ void dft_twiddled_fma(cplx64 *v, int m, const cplx64 *__restrict__ tw) {
  if constexpr (R == 8) {
    const TwF w1 = twf_load<N, DIR>(tw, m), w2 = twf_load<N, DIR>(tw, 2 * m), w4 = twf_load<N, DIR>(tw, 4 * m);
    const TwF w18 = twf_load<N, DIR>(tw, m + N / 8);  // W w8
#pragma unroll
    for (int j = 0; j < 4; ++j) bfly_fma(v[j], v[j + 4], w4);  // P'_j = v_j, Q'_j = v_j+4
    const TwF w2q = twf_quarter<DIR>(w2);
    bfly_fma(v[0], v[2], w2);   // PP'_0, PQ'_0
    bfly_fma(v[1], v[3], w2);   // PP'_1, PQ'_1
    bfly_fma(v[4], v[6], w2q);  // QP'_0, QQ'_0
    bfly_fma(v[5], v[7], w2q);  // QP'_1, QQ'_1
    bfly_fma(v[0], v[1], w1);                     // X0, X4
    bfly_fma(v[2], v[3], twf_quarter<DIR>(w1));   // X2, X6
    bfly_fma(v[4], v[5], w18);                    // X1, X5
    bfly_fma(v[6], v[7], twf_quarter<DIR>(w18));  // X3, X7
    const cplx64 x0 = v[0], x4 = v[1], x2 = v[2], x6 = v[3], x1 = v[4], x5 = v[5], x3 = v[6], x7 = v[7];
    v[0] = x0; v[1] = x1; v[2] = x2; v[3] = x3; v[4] = x4; v[5] = x5; v[6] = x6; v[7] = x7;
  } else if constexpr (R == 4) {
    const TwF w1 = twf_load<N, DIR>(tw, m), w2 = twf_load<N, DIR>(tw, 2 * m);
    bfly_fma(v[0], v[2], w2);  // P'_0, Q'_0
    bfly_fma(v[1], v[3], w2);  // P'_1, Q'_1
    bfly_fma(v[0], v[1], w1);                    // X0, X2
    bfly_fma(v[2], v[3], twf_quarter<DIR>(w1));  // X1, X3
    const cplx64 x0 = v[0], x2 = v[1], x1 = v[2], x3 = v[3];
    v[0] = x0; v[1] = x1; v[2] = x2; v[3] = x3;
  } else {
    bfly_fma(v[0], v[1], twf_load<N, DIR>(tw, m));
  }
}

// The first (untwiddled) radix-8 stage in the same radix-2 layer form: twiddle 1 everywhere
// except the quarter turns (free) and w8 = c (1 + i DIR), c = sqrt(2)/2, on two butterflies of
// layer 3 (two additions and four FMAs each): 52 FP64 instructions instead of 56.  With ZP the
// inputs 3 and 4 are known zeros (zero-padded inverse transforms: the 2/3-rule gap K+1 .. N-K-1
// always covers them, see pencil_fft) and layer 1 loses two butterflies: 44.
template <int DIR, bool ZP, typename C>
__device__ __forceinline__ void dft8_first_fma(C *v) {
  using R = typename C::value_type;
  constexpr R c = (R)0.70710678118654752440;  // cos(pi/4)
  // layer 1 (twiddle 1): (v_j, v_j+4) <- (v_j + v_j+4, v_j - v_j+4)
  if constexpr (ZP) {  // j = 0 with v4 = 0, j = 3 with v3 = 0
    v[4] = v[0];
    v[3] = v[7];
    v[7] = C{-v[7].re, -v[7].im};
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (ZP && (j == 0 || j == 3)) continue;
    const C a = v[j], b = v[j + 4];
    v[j] = c_add(a, b);
    v[j + 4] = c_sub(a, b);
  }
  // layer 2: twiddle 1 on (0,2), (1,3); w4 on (4,6), (5,7)
  {
    const C a0 = v[0], a2 = v[2], a1 = v[1], a3 = v[3];
    v[0] = c_add(a0, a2);
    v[2] = c_sub(a0, a2);
    v[1] = c_add(a1, a3);
    v[3] = c_sub(a1, a3);
    const C q6 = c_mul_i<DIR>(v[6]), q7 = c_mul_i<DIR>(v[7]);
    const C a4 = v[4], a5 = v[5];
    v[4] = c_add(a4, q6);
    v[6] = c_sub(a4, q6);
    v[5] = c_add(a5, q7);
    v[7] = c_sub(a5, q7);
  }
  // layer 3: 1 on (0,1), w4 on (2,3), w8 on (4,5), w8 w4 on (6,7)
  {
    const C a0 = v[0], a1 = v[1];
    v[0] = c_add(a0, a1);
    v[1] = c_sub(a0, a1);
    const C a2 = v[2], r3 = c_mul_i<DIR>(v[3]);
    v[2] = c_add(a2, r3);
    v[3] = c_sub(a2, r3);
    const C z5 = {v[5].re - DIR * v[5].im, v[5].im + DIR * v[5].re};  // (1 + i DIR) v5
    const C a4 = v[4];
    v[4] = C{fma(c, z5.re, a4.re), fma(c, z5.im, a4.im)};
    v[5] = C{fma(-c, z5.re, a4.re), fma(-c, z5.im, a4.im)};
    const C z7 = c_mul_i<DIR>(C{v[7].re - DIR * v[7].im, v[7].im + DIR * v[7].re});
    const C a6 = v[6];
    v[6] = C{fma(c, z7.re, a6.re), fma(c, z7.im, a6.im)};
    v[7] = C{fma(-c, z7.re, a6.re), fma(-c, z7.im, a6.im)};
  }
  // (X0, X4, X2, X6, X1, X5, X3, X7) -> natural order
  const C x0 = v[0], x4 = v[1], x2 = v[2], x6 = v[3], x1 = v[4], x5 = v[5], x3 = v[6], x7 = v[7];
  v[0] = x0; v[1] = x1; v[2] = x2; v[3] = x3; v[4] = x4; v[5] = x5; v[6] = x6; v[7] = x7;
}

// The first radix-8 stage in double-float: the plain length-8 DFT, or with the zero-padded
// pencil's inputs 3 and 4 (not loaded) left out of the arithmetic.
template <int DIR, bool ZP>
__device__ __forceinline__ void dft8_first_fma(cdf *v) {
  if constexpr (ZP) dft8_zp<DIR>(v);
  else dft8<DIR>(v);
}

// ---- values per thread ----
// FP32 pencils: 16 values per thread (radix 16: two shared-memory stages at N = 256 where radix 8
// needs three; the FP32 passes are bound by instruction issue).  FP64: 8 (their cost is FP64
// instructions, which radix 16 does not reduce).  A pencil is transformed by N / VPT threads.
// Kernels may choose 8 or 16 for FP32 (the radix that suits a pass depends on N and on the pass;
// the column passes let the autotuner pick); FP64 always uses 8.
template <typename C>
__host__ __device__ constexpr int fft_vpt() { return sizeof(C) == 8 ? 16 : 8; }
template <int N, int VPT>
__host__ __device__ constexpr int tpp_for() { return N / VPT > 0 ? N / VPT : 1; }
template <int N, typename C>
__host__ __device__ constexpr int fft_tpp() { return tpp_for<N, fft_vpt<C>()>(); }

// ---- Stockham pencil FFT ----
//
// The transform of length N = product of radices (VPT = 16 or 8 while that many points remain,
// then the rest) runs as a sequence of stages.  Before a stage, sub-transforms of length NS are complete;
// butterfly j (0 <= j < N/R) gathers x[j + r N/R] (r < R), multiplies element r by the twiddle
// W_{NS R}^{r (j mod NS)}, applies a length-R DFT and scatters the results to
// (j div NS) NS R + (j mod NS) + r NS.  After the last stage the pencil holds X in natural order
// (the auto-sorting formulation of Cooley-Tukey by Stockham).  Each of the N/VPT threads of a
// group owns VPT / R butterflies per stage, so it always holds VPT values.  `tw[m]` = W_N^m =
// exp(-2 pi i m / N); the inverse uses its conjugate.
//
// Every thread of the block must call this (it contains group barriers); threads with
// `active == false` only take part in the barriers.  The caller separates the transform from the
// preceding writes and the following reads of the pencil with a block barrier.
// TWG: `tw` may point to shared memory (generic twiddle loads; double-float only).
template <int N, int DIR, int NS, typename C, int VPT, bool ZP, bool TWG = false>
__device__ __forceinline__ void stockham_stages(C *buf, int t, bool active, const C *__restrict__ tw) {
  if constexpr (NS < N) {
    static_assert(VPT == 8 || (VPT == 16 && sizeof(C) == 8), "radix 16 is an FP32 option");
    constexpr int R = (N / NS >= VPT) ? VPT : N / NS;
    constexpr int NB = VPT / R;
    constexpr int TPP = tpp_for<N, VPT>();
    constexpr int TWSTEP = N / (NS * R);
    // FP64 stages with twiddles take them inside the butterflies (FMA form, fewer FP64
    // instructions); the others multiply on load.
    constexpr bool kFma = std::is_same<C, cplx64>::value && NS > 1;
    // The first radix-8 stage: FMA layers, and with ZP the zero inputs 3 and 4 skipped; the first
    // radix-16 stage with ZP skips its zero inputs 6..9.
    constexpr bool kFirst = NS == 1 && R == 8;
    constexpr bool kFirst16 = NS == 1 && R == 16 && ZP;
    constexpr int K = (N - 1) / 3;
    static_assert(!(ZP && kFirst) || (3 * (N / 8) > K && 5 * (N / 8) - 1 < N - K),
                  "inputs 3 and 4 of the first radix-8 stage must lie in the 2/3-rule gap");
    static_assert(!kFirst16 || (6 * (N / 16) > K && 10 * (N / 16) - 1 < N - K),
                  "inputs 6..9 of the first radix-16 stage must lie in the 2/3-rule gap");
    C v[VPT];
    if (active) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int j = t + b * TPP;
        const int k = j % NS;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (kFirst && ZP && (r == 3 || r == 4)) continue;  // zeros, never read
          if (kFirst16 && r >= 6 && r <= 9) continue;
          C x = buf[sm_idx<C>(j + r * (N / R))];
          if (!kFma && NS > 1 && r > 0) {
            C w;
            if constexpr (TWG) w = tw_load_generic(tw + r * k * TWSTEP);
            else w = tw_load(tw + r * k * TWSTEP);
            x = DIR < 0 ? c_mul(x, w) : c_mulc(x, w);
          }
          v[b * R + r] = x;
        }
      }
    }
    group_sync<TPP>();
    if (active) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if constexpr (kFma) {
          dft_twiddled_fma<N, R, DIR>(reinterpret_cast<cplx64 *>(v) + b * R, ((t + b * TPP) % NS) * TWSTEP,
                                      reinterpret_cast<const cplx64 *>(tw));
        } else if constexpr (kFirst) {
          dft8_first_fma<DIR, ZP>(v + b * R);
        } else if constexpr (kFirst16) {
          dft16<DIR, C, true>(v + b * R);
        } else {
          dft_small<R, DIR, C>(v + b * R);
        }
        const int j = t + b * TPP;
        const int k = j % NS;
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[sm_idx<C>(base + r * NS)] = v[b * R + r];
      }
    }
    group_sync<TPP>();
    stockham_stages<N, DIR, NS * R, C, VPT, false, TWG>(buf, t, active, tw);
  }
}

// `t` in [0, N / VPT): the thread's index within its pencil's group.  ZP: the pencil is
// zero-padded by the 2/3 rule (elements K+1 .. N-K-1 are zero, K = (N-1)/3), as every inverse
// transform of a truncated spectrum is; the FP64 first stage then skips the inputs it knows are
// zero (they need not even be written).
template <int N, int DIR, typename C, int VPT = fft_vpt<C>(), bool ZP = false, bool TWG = false>
__device__ __forceinline__ void pencil_fft(C *buf, int t, bool active, const C *__restrict__ tw) {
  stockham_stages<N, DIR, 1, C, VPT, ZP, TWG>(buf, t, active, tw);
}

// FFT index of kept index j (0..2K) along a truncated axis: j for j <= K, else j - (2K+1) + N.
__device__ __forceinline__ int kept_to_fft(int j, int K, int n) { return j <= K ? j : j - (2 * K + 1) + n; }
// Signed wavenumber of kept index j.
__device__ __forceinline__ int kept_wave(int j, int K) { return j <= K ? j : j - (2 * K + 1); }

// Block-wide reductions with a fixed combination order (deterministic for a fixed block size).
// `red` must hold blockDim.x / 32 doubles; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
  }
  return s;
}

// The same in the data's precision: FP32 kernels keep the reduction off the FP64 pipe, which on
// GB300 runs at 1/64 of the FP32 rate (widening the result is exact and monotonic, so the maximum
// is the one an FP64 reduction of the widened values would give).
__device__ __forceinline__ float nan_max(float a, float b) {
  if (a != a) return a;
  if (b != b) return b;
  return a > b ? a : b;
}

__device__ __forceinline__ float block_nan_max(float v, float *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = 0.0f;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    s = red[0];
    for (int i = 1; i < nw; ++i) s = nan_max(s, red[i]);
  }
  return s;
}

__device__ __forceinline__ double block_nan_max(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    s = red[0];
    for (int i = 1; i < nw; ++i) s = nan_max(s, red[i]);
  }
  return s;
}

}  // namespace mhd
