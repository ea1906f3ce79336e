// kernels_tracers.cu -- passive tracer particles (paper, section "Tracer Particles").
//
// One thread per particle.  Each step a particle takes the magnetic field of the step's start
// state at its position by cloud-in-cell interpolation (Eq. tracer_eq: the 8 corners of its grid
// cell, each weighted by the volume of the sub-cell opposite to it, divided by the cell volume),
// turns its velocity by the Boris rotation with q = M = 1 and no electric field (Eq. boris), and
// moves with the new velocity (Eq. euler), wrapped into the periodic box [0, 2 pi)^3.  The grid
// field comes from the fused flux pass of the same step, which writes it while it holds the field
// on the grid anyway; the gathers are scattered 8-byte loads served mostly by L2.
#include "mhd_internal.h"

namespace mhd {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ double wrap_2pi(double x) {
  double w = x - kTwoPi * floor(x / kTwoPi);
  if (w >= kTwoPi) w -= kTwoPi;
  return w;
}

// Cell corner indexes and weights of the point (x, y, z) on an n^3 periodic grid of spacing h.
struct Cic {
  size_t idx[8];
  double w[8];
};

__device__ __forceinline__ Cic cic_setup(double x, double y, double z, int n) {
  const double h = kTwoPi / (double)n;
  const double gx = x / h, gy = y / h, gz = z / h;
  const int i = (int)floor(gx), j = (int)floor(gy), k = (int)floor(gz);
  const double lx = gx - i, ly = gy - j, lz = gz - k;  // from the lower faces, in cells
  const double ux = 1.0 - lx, uy = 1.0 - ly, uz = 1.0 - lz;
  const int i0 = ((i % n) + n) % n, j0 = ((j % n) + n) % n, k0 = ((k % n) + n) % n;
  const int i1 = i0 + 1 == n ? 0 : i0 + 1, j1 = j0 + 1 == n ? 0 : j0 + 1, k1 = k0 + 1 == n ? 0 : k0 + 1;
  const size_t nn = (size_t)n;
  Cic c;
  const size_t r00 = (k0 * nn + j0) * nn, r10 = (k0 * nn + j1) * nn, r01 = (k1 * nn + j0) * nn,
               r11 = (k1 * nn + j1) * nn;
  c.idx[0] = r00 + i0; c.w[0] = ux * uy * uz;
  c.idx[1] = r00 + i1; c.w[1] = lx * uy * uz;
  c.idx[2] = r10 + i0; c.w[2] = ux * ly * uz;
  c.idx[3] = r10 + i1; c.w[3] = lx * ly * uz;
  c.idx[4] = r01 + i0; c.w[4] = ux * uy * lz;
  c.idx[5] = r01 + i1; c.w[5] = lx * uy * lz;
  c.idx[6] = r11 + i0; c.w[6] = ux * ly * lz;
  c.idx[7] = r11 + i1; c.w[7] = lx * ly * lz;
  return c;
}

template <typename R>
__device__ __forceinline__ double cic_apply(const Cic &c, const R *__restrict__ g) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += (double)g[c.idx[q]] * c.w[q];
  return s;
}

}  // namespace

__global__ void tracer_init_kernel(const double *__restrict__ real, double *__restrict__ tr, long long count, int n) {
  const size_t n3 = (size_t)n * n * n;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < count;
       m += (long long)gridDim.x * blockDim.x) {
    const Cic c = cic_setup(tr[m], tr[count + m], tr[2 * count + m], n);
    // u = m / rho at each corner, then the weighted sum
    double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double rho = real[c.idx[q]];
#pragma unroll
      for (int a = 0; a < 3; ++a) v[a] += real[(1 + a) * n3 + c.idx[q]] / rho * c.w[q];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) tr[(3 + a) * count + m] = v[a];
  }
}

template <typename R>
__global__ void tracer_push_kernel(const R *__restrict__ bg, double *__restrict__ tr, long long count,
                                   const StepCoef *__restrict__ coef, int n) {
  if (coef->skip) return;
  const double dt = coef->dt;
  const size_t n3 = (size_t)n * n * n;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < count;
       m += (long long)gridDim.x * blockDim.x) {
    double p[3], v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p[a] = tr[a * count + m];
      v[a] = tr[(3 + a) * count + m];
    }
    const Cic c = cic_setup(p[0], p[1], p[2], n);
    double t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) t[a] = cic_apply(c, bg + a * n3) * dt / 2.0;
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s[a] = 2.0 * t[a] / (1.0 + t2);
    const double vd[3] = {v[0] + (v[1] * t[2] - v[2] * t[1]), v[1] + (v[2] * t[0] - v[0] * t[2]),
                          v[2] + (v[0] * t[1] - v[1] * t[0])};
    const double vn[3] = {v[0] + (vd[1] * s[2] - vd[2] * s[1]), v[1] + (vd[2] * s[0] - vd[0] * s[2]),
                          v[2] + (vd[0] * s[1] - vd[1] * s[0])};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      tr[a * count + m] = wrap_2pi(p[a] + vn[a] * dt);
      tr[(3 + a) * count + m] = vn[a];
    }
  }
}

static unsigned tracer_blocks(long long count) {
  long long b = (count + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_tracer_init(const double *real, double *tr, long long count, int n, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  tracer_init_kernel<<<tracer_blocks(count), 256, 0, s>>>(real, tr, count, n);
  return cudaGetLastError();
}

cudaError_t launch_tracer_push(const double *bgrid, double *tr, long long count, const StepCoef *coef, int n,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  tracer_push_kernel<double><<<tracer_blocks(count), 256, 0, s>>>(bgrid, tr, count, coef, n);
  return cudaGetLastError();
}

cudaError_t launch_tracer_push(const float *bgrid, double *tr, long long count, const StepCoef *coef, int n,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  tracer_push_kernel<float><<<tracer_blocks(count), 256, 0, s>>>(bgrid, tr, count, coef, n);
  return cudaGetLastError();
}

}  // namespace mhd
