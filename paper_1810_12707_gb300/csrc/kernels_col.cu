// kernels_col.cu -- FFT passes along a strided axis (y or z) of the truncated spectral layout.
//
// The data of one pass is viewed as [nslab][L][C]: the transform runs along L for each of the
// nslab * C columns; the C columns of a slab are contiguous in memory.  A block takes TC
// consecutive columns of one slab, so every row of the tile is one coalesced segment of TC complex
// values.  The tile is transposed into shared memory as TC pencils of length N (pitch N + 1, which
// spreads consecutive pencils over the banks), transformed by TC groups of N/8 threads, and
// written back.
//   inverse (DIR = +1): L = 2K + 1 kept rows in, scattered to their FFT indices with the rest of
//                       the pencil zero (the 2/3-rule truncation), all N rows out;
//   forward (DIR = -1): N rows in, only the 2K + 1 kept rows out, times `scale`.
// Used for: inverse z (state -> z), inverse y, forward y, forward z (-> truncated spectra).
#include "fft_device.cuh"
#include "launch_util.cuh"

namespace mhd {

// CI, CO: element types in and out; CC: type of the transform arithmetic (= the output's).
template <int N, int DIR, typename CI, typename CO, typename CC>
__global__ void col_fft_kernel(const CI *__restrict__ in, CO *__restrict__ out, int ntiles, int tc,
                               int cols, int K, double scale, const CC *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CC *sm = reinterpret_cast<CC *>(smem_raw);
  constexpr int TPP = N / 8;
  constexpr int P = pencil_pitch<CC>(N);
  const int NK = 2 * K + 1;
  const int lin = DIR > 0 ? NK : N;
  const int lout = DIR > 0 ? N : NK;
  const int tile = blockIdx.x % ntiles;
  const size_t slab = blockIdx.x / ntiles;
  const int c0 = tile * tc;
  const int nthr = blockDim.x;

  const CI *src = in + slab * (size_t)lin * cols;
  for (int q = threadIdx.x; q < lin * tc; q += nthr) {
    const int l = q / tc, c = q - l * tc;
    const int col = c0 + c;
    CC v = {0, 0};
    if (col < cols) v = c_cvt<CC>(src[(size_t)l * cols + col]);
    const int f = DIR > 0 ? kept_to_fft(l, K, N) : l;
    sm[c * P + sm_idx<CC>(f)] = v;
  }
  if (DIR > 0) {
    const int nz = N - NK;  // FFT indices K+1 .. N-K-1 are outside the kept set
    for (int q = threadIdx.x; q < nz * tc; q += nthr) {
      const int l = q / tc, c = q - l * tc;
      sm[c * P + sm_idx<CC>(K + 1 + l)] = CC{0, 0};
    }
  }
  __syncthreads();

  const int pencil = threadIdx.x / TPP;
  const int t = threadIdx.x - pencil * TPP;
  const bool active = pencil < tc && c0 + pencil < cols;
  pencil_fft<N, DIR, CC>(sm + (active ? pencil : 0) * P, t, active, tw);
  __syncthreads();  // the store loop reads every pencil

  CO *dst = out + slab * (size_t)lout * cols;
  for (int q = threadIdx.x; q < lout * tc; q += nthr) {
    const int l = q / tc, c = q - l * tc;
    const int col = c0 + c;
    if (col < cols) {
      const int f = DIR > 0 ? l : kept_to_fft(l, K, N);
      CC v = sm[c * P + sm_idx<CC>(f)];
      if (DIR < 0) v = c_scale(v, (typename CC::value_type)scale);
      dst[(size_t)l * cols + col] = c_cvt<CO>(v);
    }
  }
}

namespace {

// Columns per block: enough that a tile row is at least 128 bytes and a block at least 128
// threads, but not more than the columns there are.
int pick_tc(int n, int cols) {
  const int tpp = n / 8;
  int tc = 8;
  while (tc * tpp < 128 && tc < 64) tc *= 2;
  while (tc * tpp > 1024) tc /= 2;
  if (tc > cols) tc = cols;
  return tc < 1 ? 1 : tc;
}

template <int N, int DIR, typename CI, typename CO>
cudaError_t launch_col_n(const CI *in, CO *out, int nslab, int cols, double scale, const CO *tw,
                         cudaStream_t s, int tile) {
  const int K = (N - 1) / 3;
  int tc = tile > 0 ? tile : pick_tc(N, cols);
  while (tc * (N / 8) > 1024) tc /= 2;
  if (tc > cols) tc = cols;
  if (tc < 1) tc = 1;
  const int ntiles = (cols + tc - 1) / tc;
  const size_t smem = (size_t)tc * pencil_pitch<CO>(N) * sizeof(CO);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem<col_fft_kernel<N, DIR, CI, CO, CO>>((int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (long long)nslab * ntiles;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  col_fft_kernel<N, DIR, CI, CO, CO><<<(unsigned)blocks, tc * (N / 8), smem, s>>>(in, out, ntiles, tc, cols, K,
                                                                                 scale, tw);
  return cudaGetLastError();
}

template <int DIR, typename CI, typename CO>
cudaError_t launch_col(const CI *in, CO *out, int n, int nslab, int cols, double scale, const CO *tw,
                       cudaStream_t s, int tile) {
  switch (n) {
    case 16: return launch_col_n<16, DIR>(in, out, nslab, cols, scale, tw, s, tile);
    case 32: return launch_col_n<32, DIR>(in, out, nslab, cols, scale, tw, s, tile);
    case 64: return launch_col_n<64, DIR>(in, out, nslab, cols, scale, tw, s, tile);
    case 128: return launch_col_n<128, DIR>(in, out, nslab, cols, scale, tw, s, tile);
    case 256: return launch_col_n<256, DIR>(in, out, nslab, cols, scale, tw, s, tile);
    case 512: return launch_col_n<512, DIR>(in, out, nslab, cols, scale, tw, s, tile);
    case 1024: return launch_col_n<1024, DIR>(in, out, nslab, cols, scale, tw, s, tile);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_col_inverse(const cplx64 *in, cplx64 *out, int n, int nslab, int cols,
                               const cplx64 *tw, cudaStream_t s, int tile) {
  return launch_col<+1>(in, out, n, nslab, cols, 1.0, tw, s, tile);
}
cudaError_t launch_col_inverse(const cplx64 *in, cplx32 *out, int n, int nslab, int cols,
                               const cplx32 *tw, cudaStream_t s, int tile) {
  return launch_col<+1>(in, out, n, nslab, cols, 1.0, tw, s, tile);
}
cudaError_t launch_col_inverse(const cplx32 *in, cplx32 *out, int n, int nslab, int cols,
                               const cplx32 *tw, cudaStream_t s, int tile) {
  return launch_col<+1>(in, out, n, nslab, cols, 1.0, tw, s, tile);
}
cudaError_t launch_col_forward(const cplx64 *in, cplx64 *out, int n, int nslab, int cols,
                               double scale, const cplx64 *tw, cudaStream_t s, int tile) {
  return launch_col<-1>(in, out, n, nslab, cols, scale, tw, s, tile);
}
cudaError_t launch_col_forward(const cplx32 *in, cplx32 *out, int n, int nslab, int cols,
                               double scale, const cplx32 *tw, cudaStream_t s, int tile) {
  return launch_col<-1>(in, out, n, nslab, cols, scale, tw, s, tile);
}

}  // namespace mhd
