// kernels_spectra.cu -- shell spectra and velocity-derivative statistics of one instance (paper,
// section "for hydrodynamic flow": theta' = <(du_i/dx_i)^2>^(1/2) and the skewness
// S_3 = <(du_1/dx_1)^3> / <(du_1/dx_1)^2>^(3/2); kinetic and magnetic energy spectra), with the
// kinetic and magnetic helicities and the largest |div B| on the grid.
//
// The velocity u = m / rho exists only on the grid, so one fused x pass brings rho and m to real
// rows (inverse x), divides, and sends u back (forward x); the y and z column passes then give the
// truncated spectrum u_hat.  A mode k belongs to shell s = round(|k|), decided exactly in integer
// arithmetic: (2s - 1)^2 <= 4|k|^2 < (2s + 1)^2 (|k|^2 is an integer, so no mode lies on a shell
// boundary).  One block per shell walks every (k_z, k_y) row of the truncated half spectrum, finds
// the k_x run of its shell, and sums in a fixed order, so the spectra are bitwise reproducible.
#include "fft_device.cuh"
#include "launch_util.cuh"

namespace mhd {

namespace {

constexpr int kMaxThreads = 384;

constexpr int pairs_for(int n) { return (n / 8) >= 16 ? 1 : 16 / (n / 8); }

constexpr int threads_for(int tpp, int pencils) {
  int g = kMaxThreads / tpp;
  if (g > pencils) g = pencils;
  int t = g * tpp;
  return (t + 31) / 32 * 32;
}

template <int N, int DIR, typename Ptr>
__device__ __forceinline__ void fft_pencils(int np, Ptr ptr, const cplx64 *__restrict__ tw) {
  constexpr int TPP = tpp_for<N, 8>();
  const int G = blockDim.x / TPP;
  const int g = threadIdx.x / TPP, t = threadIdx.x - g * TPP;
  for (int base = 0; base < np; base += G) {
    const int id = base + g;
    const bool active = g < G && id < np;
    pencil_fft<N, DIR, cplx64, 8, (DIR > 0)>(ptr(active ? id : 0), t, active, tw);  // inverse: zero-padded
  }
  __syncthreads();
}

}  // namespace

// rho, m (fields 0..3 of `in`, [f][z][y][kx <= K] after the inverse y pass) -> u = m / rho on the
// grid -> forward x -> out [3][z][y][kx <= K].  Two real rows per complex pencil, as in the flux
// pass; a block owns PAIRS row pairs.
template <int N>
__global__ void __launch_bounds__(kMaxThreads) velocity_x_kernel(const cplx64 *__restrict__ in,
                                                                  cplx64 *__restrict__ out, int K,
                                                                  const cplx64 *__restrict__ tw) {
  constexpr int KT = (N - 1) / 3;  // the 2/3-rule cut-off, fixed by N
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx64 *sm = reinterpret_cast<cplx64 *>(smem_raw);
  constexpr int P = pencil_pitch<cplx64>(N);
  constexpr int PAIRS = pairs_for(N);
  constexpr size_t NN = (size_t)N * N;
  constexpr int NX = KT + 1;
  const size_t row0 = (size_t)blockIdx.x * PAIRS * 2;
  const int nthr = blockDim.x;

  for (int q = threadIdx.x; q < 4 * PAIRS * NX; q += nthr) {
    const int k = q % NX;
    const int r = q / NX;
    const int f = r % 4, p = r / 4;
    const cplx64 *src = in + ((size_t)f * NN + row0 + 2 * p) * NX;
    cplx64 *pen = sm + (p * 4 + f) * P;
    const cplx64 x0 = src[k], x1 = src[NX + k];
    if (k == 0) {
      pen[0] = cplx64{x0.re, x1.re};
    } else {
      pen[sm_idx<cplx64>(k)] = cplx64{x0.re - x1.im, x0.im + x1.re};
      pen[sm_idx<cplx64>(N - k)] = cplx64{x0.re + x1.im, x1.re - x0.im};
    }
  }
  for (int q = threadIdx.x; q < 4 * PAIRS * (N - 2 * KT - 1); q += nthr) {
    const int z = q % (N - 2 * KT - 1);
    const int r = q / (N - 2 * KT - 1);
    sm[r * P + sm_idx<cplx64>(KT + 1 + z)] = cplx64{0.0, 0.0};
  }
  __syncthreads();
  fft_pencils<N, +1>(4 * PAIRS, [&](int id) { return sm + id * P; }, tw);

  for (int q = threadIdx.x; q < PAIRS * N; q += nthr) {
    const int p = q / N, j = q - p * N;
    cplx64 *b = sm + p * 4 * P + sm_idx<cplx64>(j);
    const cplx64 rho = b[0];
#pragma unroll
    for (int f = 1; f < 4; ++f) {
      const cplx64 m = b[f * P];
      b[f * P] = cplx64{m.re / rho.re, m.im / rho.im};
    }
  }
  __syncthreads();
  fft_pencils<N, -1>(3 * PAIRS, [&](int id) { return sm + ((id / 3) * 4 + 1 + id % 3) * P; }, tw);

  for (int q = threadIdx.x; q < 3 * PAIRS * NX; q += nthr) {
    const int k = q % NX;
    const int r = q / NX;
    const int f = r % 3, p = r / 3;
    const cplx64 *pen = sm + (p * 4 + 1 + f) * P;
    const cplx64 z = pen[sm_idx<cplx64>(k)], zc = pen[sm_idx<cplx64>((N - k) & (N - 1))];
    cplx64 *dst = out + ((size_t)f * NN + row0 + 2 * p) * NX;
    dst[k] = cplx64{0.5 * (z.re + zc.re), 0.5 * (z.im - zc.im)};
    dst[NX + k] = cplx64{0.5 * (z.im + zc.im), 0.5 * (zc.re - z.re)};
  }
}

// Re(conj(f) . (i k x f)) of one mode: with t = k x f, (i t)_a = (-Im t_a, Re t_a).
__device__ __forceinline__ double curl_dot(double kx, double ky, double kz, cplx64 fx, cplx64 fy, cplx64 fz) {
  const cplx64 tx{ky * fz.re - kz * fy.re, ky * fz.im - kz * fy.im};
  const cplx64 ty{kz * fx.re - kx * fz.re, kz * fx.im - kx * fz.im};
  const cplx64 tz{kx * fy.re - ky * fx.re, kx * fy.im - ky * fx.im};
  return (fx.im * tx.re - fx.re * tx.im) + (fy.im * ty.re - fy.re * ty.im) + (fz.im * tz.re - fz.re * tz.im);
}

// One block per shell s.  uh, bh: 3 truncated spectra each (stride `spec`); out[s][5] =
// (sum w |u_hat|^2 / 2, sum w |B_hat|^2 / 2, sum w |k . u_hat|^2, sum w Re(conj(u_hat) . i k x u_hat),
// sum w Re(conj(B_hat) . i k x B_hat) / |k|^2) over the shell, with w = 1 on the k_x = 0 plane and 2
// elsewhere (the half spectrum stands for k and -k).  By Parseval the last two are the shell's
// shares of the kinetic helicity <u . curl u> and of the magnetic helicity <A . B>, A_hat =
// i k x B_hat / |k|^2 (Coulomb gauge, A_hat(0) = 0).  dh = i k_x u_hat_x and gh = i k . B_hat on
// every mode (each mode is visited by exactly one shell's block).
__global__ void __launch_bounds__(256) shell_kernel(const cplx64 *__restrict__ uh, const cplx64 *__restrict__ bh,
                                                    cplx64 *__restrict__ dh, cplx64 *__restrict__ gh,
                                                    double *__restrict__ out, int K) {
  __shared__ double red[32];
  const int NX = K + 1, NK = 2 * K + 1;
  const size_t spec = (size_t)NK * NK * NX;
  const int s = blockIdx.x;
  const long long lo_b = s == 0 ? 0 : (long long)(2 * s - 1) * (2 * s - 1);
  const long long hi_b = (long long)(2 * s + 1) * (2 * s + 1);
  double ek = 0.0, em = 0.0, th = 0.0, hk = 0.0, hm = 0.0;
  for (int r = threadIdx.x; r < NK * NK; r += blockDim.x) {
    const int kz = kept_wave(r / NK, K), ky = kept_wave(r % NK, K);
    const long long q4 = 4LL * (ky * ky + kz * kz);
    if (q4 >= hi_b) continue;
    int kx = 0;
    if (q4 < lo_b) {
      kx = (int)sqrt((double)(lo_b - q4) / 4.0);
      while (kx > 0 && q4 + 4LL * (kx - 1) * (kx - 1) >= lo_b) --kx;
      while (q4 + 4LL * kx * kx < lo_b) ++kx;
    }
    for (; kx <= K && q4 + 4LL * kx * kx < hi_b; ++kx) {
      const size_t m = (size_t)r * NX + kx;
      const double w = kx == 0 ? 1.0 : 2.0;
      const cplx64 ux = uh[m], uy = uh[spec + m], uz = uh[2 * spec + m];
      const cplx64 bx = bh[m], by = bh[spec + m], bz = bh[2 * spec + m];
      ek += w * 0.5 * (ux.re * ux.re + ux.im * ux.im + uy.re * uy.re + uy.im * uy.im + uz.re * uz.re + uz.im * uz.im);
      em += w * 0.5 * (bx.re * bx.re + bx.im * bx.im + by.re * by.re + by.im * by.im + bz.re * bz.re + bz.im * bz.im);
      const double dr = kx * ux.re + ky * uy.re + kz * uz.re, di = kx * ux.im + ky * uy.im + kz * uz.im;
      th += w * (dr * dr + di * di);
      dh[m] = cplx64{-kx * ux.im, kx * ux.re};
      hk += w * curl_dot(kx, ky, kz, ux, uy, uz);
      const long long k2 = (long long)kx * kx + (long long)ky * ky + (long long)kz * kz;
      if (k2 > 0) hm += w * curl_dot(kx, ky, kz, bx, by, bz) / (double)k2;
      const double gr = kx * bx.re + ky * by.re + kz * bz.re, gi = kx * bx.im + ky * by.im + kz * bz.im;
      gh[m] = cplx64{-gi, gr};
    }
  }
  const double a = block_sum(ek, red);
  const double b = block_sum(em, red);
  const double c = block_sum(th, red);
  const double e = block_sum(hk, red);
  const double f = block_sum(hm, red);
  if (threadIdx.x == 0) {
    out[5 * s + 0] = a;
    out[5 * s + 1] = b;
    out[5 * s + 2] = c;
    out[5 * s + 3] = e;
    out[5 * s + 4] = f;
  }
}

// part[block][2] = (sum d^2, sum d^3) over a fixed grid-stride share of the n values of d.
__global__ void __launch_bounds__(256) moments_kernel(const double *__restrict__ d, size_t n, double *__restrict__ part) {
  __shared__ double red[32];
  double s2 = 0.0, s3 = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = d[i];
    s2 += v * v;
    s3 += v * v * v;
  }
  const double a = block_sum(s2, red);
  const double b = block_sum(s3, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// part[block] = max |v| over a fixed grid-stride share of the n values of v (a NaN is kept).
__global__ void __launch_bounds__(256) absmax_kernel(const double *__restrict__ v, size_t n, double *__restrict__ part) {
  __shared__ double red[32];
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = nan_max(m, fabs(v[i]));
  const double r = block_nan_max(m, red);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

namespace {

template <int N>
cudaError_t velocity_n(const cplx64 *in, cplx64 *out, const Dims &d, const cplx64 *tw, cudaStream_t s) {
  constexpr int PAIRS = pairs_for(N);
  const int blocks = N * N / (2 * PAIRS);
  const int threads = threads_for(tpp_for<N, 8>(), 4 * PAIRS);
  const size_t smem = (size_t)4 * PAIRS * pencil_pitch<cplx64>(N) * sizeof(cplx64);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem<velocity_x_kernel<N>>((int)smem);
    if (e != cudaSuccess) return e;
  }
  velocity_x_kernel<N><<<blocks, threads, smem, s>>>(in, out, d.k, tw);
  return cudaGetLastError();
}

}  // namespace

int num_shells(int k) {
  // round(sqrt(3) k): the largest s with (2s - 1)^2 <= 12 k^2
  int s = 0;
  while ((long long)(2 * s + 1) * (2 * s + 1) <= 12LL * k * k) ++s;
  return s + 1;
}

cudaError_t launch_velocity_x(const cplx64 *in, cplx64 *out, const Dims &d, const cplx64 *tw, cudaStream_t s) {
  switch (d.n) {
    case 16: return velocity_n<16>(in, out, d, tw, s);
    case 32: return velocity_n<32>(in, out, d, tw, s);
    case 64: return velocity_n<64>(in, out, d, tw, s);
    case 128: return velocity_n<128>(in, out, d, tw, s);
    case 256: return velocity_n<256>(in, out, d, tw, s);
    case 512: return velocity_n<512>(in, out, d, tw, s);
    case 1024: return velocity_n<1024>(in, out, d, tw, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_shells(const cplx64 *uh, const cplx64 *bh, cplx64 *dh, cplx64 *gh, double *out, const Dims &d,
                          cudaStream_t s) {
  shell_kernel<<<num_shells(d.k), 256, 0, s>>>(uh, bh, dh, gh, out, d.k);
  return cudaGetLastError();
}

cudaError_t launch_absmax(const double *v, size_t n, double *part, int blocks, cudaStream_t s) {
  absmax_kernel<<<blocks, 256, 0, s>>>(v, n, part);
  return cudaGetLastError();
}

cudaError_t launch_moments(const double *v, size_t n, double *part, int blocks, cudaStream_t s) {
  moments_kernel<<<blocks, 256, 0, s>>>(v, n, part);
  return cudaGetLastError();
}

}  // namespace mhd
