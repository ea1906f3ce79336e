// fft_device.cuh -- device building blocks: complex arithmetic, small DFTs in registers, and the
// Stockham pencil FFT executed by a group of N/8 threads on a pencil held in shared memory.
//
// Transform convention (both directions unscaled):  X[k] = sum_j x[j] exp(DIR * 2 pi i j k / N)
// with DIR = -1 for the forward and +1 for the inverse transform.
#pragma once

#include "mhd_internal.h"

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

template <int R, int DIR, typename C>
__device__ __forceinline__ void dft_small(C *v) {
  if constexpr (R == 8) dft8<DIR>(v);
  else if constexpr (R == 4) dft4<DIR>(v);
  else dft2<DIR>(v);
}

// Twiddle load that the compiler may not hoist out of loops: kernels that transform many pencils
// in a loop would otherwise keep every stage's twiddles live in registers across the loop.
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
// A pencil is transformed by the TPP = N/8 consecutive threads of its group and nobody else
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

// ---- Stockham pencil FFT ----
//
// The transform of length N = product of radices (8 while at least 8 points remain, then 4 or
// 2) runs as a sequence of stages.  Before a stage, sub-transforms of length NS are complete;
// butterfly j (0 <= j < N/R) gathers x[j + r N/R] (r < R), multiplies element r by the twiddle
// W_{NS R}^{r (j mod NS)}, applies a length-R DFT and scatters the results to
// (j div NS) NS R + (j mod NS) + r NS.  After the last stage the pencil holds X in natural order
// (the auto-sorting formulation of Cooley-Tukey by Stockham).  Each of the N/8 threads of a
// group owns 8 / R butterflies per stage, so it always holds 8 values.  `tw[m]` = W_N^m =
// exp(-2 pi i m / N); the inverse uses its conjugate.
//
// Every thread of the block must call this (it contains group barriers); threads with
// `active == false` only take part in the barriers.  The caller separates the transform from the
// preceding writes and the following reads of the pencil with a block barrier.
template <int N, int DIR, int NS, typename C>
__device__ __forceinline__ void stockham_stages(C *buf, int t, bool active, const C *__restrict__ tw) {
  if constexpr (NS < N) {
    constexpr int R = (N / NS >= 8) ? 8 : N / NS;
    constexpr int NB = 8 / R;
    constexpr int TPP = N / 8;
    constexpr int TWSTEP = N / (NS * R);
    C v[8];
    if (active) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int j = t + b * TPP;
        const int k = j % NS;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          C x = buf[sm_idx<C>(j + r * (N / R))];
          if (NS > 1 && r > 0) {
            const C w = tw_load(tw + r * k * TWSTEP);
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
        dft_small<R, DIR, C>(v + b * R);
        const int j = t + b * TPP;
        const int k = j % NS;
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[sm_idx<C>(base + r * NS)] = v[b * R + r];
      }
    }
    group_sync<TPP>();
    stockham_stages<N, DIR, NS * R, C>(buf, t, active, tw);
  }
}

template <int N, int DIR, typename C>
__device__ __forceinline__ void pencil_fft(C *buf, int t, bool active, const C *__restrict__ tw) {
  stockham_stages<N, DIR, 1, C>(buf, t, active, tw);
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
