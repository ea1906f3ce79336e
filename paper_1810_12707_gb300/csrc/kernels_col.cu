// kernels_col.cu -- FFT passes along a strided axis (y or z) of the truncated spectral layout.
//
// The data of one pass is viewed as [nslab][L][C]: the transform runs along L for each of the
// nslab * C columns; the C columns of a slab are contiguous in memory.  A block takes TC
// consecutive columns of one slab, so every row of the tile is one coalesced segment of TC complex
// values.  The tile is transposed into shared memory as TC pencils of length N (pitch N + 1, which
// spreads consecutive pencils over the banks), transformed by TC groups of N/VPT threads, and
// written back.
//   inverse (DIR = +1): L = 2K + 1 kept rows in, scattered to their FFT indices with the rest of
//                       the pencil zero (the 2/3-rule truncation), all N rows out;
//   forward (DIR = -1): N rows in, only the 2K + 1 kept rows out, times `scale`.
// Used for: inverse z (state -> z), inverse y, forward y, forward z (-> truncated spectra).
#include "fft_device.cuh"
#include "launch_util.cuh"

#include <type_traits>

namespace mhd {

// Double-float passes at N >= 512 stage the twiddle table (N values, 8 KB at 512) in shared
// memory behind the tile: 4-6 % faster per pass at 512^3 than 16-byte L1 loads per butterfly
// element; at 256^3 the copy per block cost more than it saved.
template <typename CC, int N>
constexpr bool tws_staged() { return std::is_same<CC, cdf>::value && N >= 512; }
template <typename CC, int N>
constexpr size_t tws_bytes() { return tws_staged<CC, N>() ? (size_t)N * sizeof(CC) : 0; }

// CI, CO: element types in and out; CC: type of the transform arithmetic (= the output's).
// A block has TC = 2^tsh columns and TC * N/VPT threads: thread (l0, c) = (tid >> tsh, tid & (TC-1))
// moves rows l0, l0 + N/VPT, ... of column c, so consecutive threads touch consecutive columns of a
// row (coalesced) and no index needs a division.
// VPT: values per thread of the transform (8, or 16 for FP32), so N / VPT threads per column.
// One tile (TC columns of one slab): work item w = slab * ntiles + tile.
template <int N, int DIR, typename CI, typename CO, typename CC, int VPT>
__device__ __forceinline__ void col_fft_tile(const CI *__restrict__ in, CO *__restrict__ out, unsigned w, int ntiles,
                                             int tsh, int cols, typename scale_of<CC>::type scale,
                                             const CC *__restrict__ tw, CC *sm) {
  constexpr int TPP = tpp_for<N, VPT>();
  constexpr int P = pencil_pitch<CC>(N);
  constexpr int K = (N - 1) / 3;  // the 2/3-rule cut-off, fixed by N
  constexpr int NK = 2 * K + 1;
  constexpr int LIN = DIR > 0 ? NK : N;
  constexpr int LOUT = DIR > 0 ? N : NK;
  const int tc = 1 << tsh;
  const int tile = (int)(w % (unsigned)ntiles);
  const size_t slab = w / (unsigned)ntiles;
  const int c = threadIdx.x & (tc - 1);
  const int l0 = threadIdx.x >> tsh;  // 0 .. TPP-1
  const int col = tile * tc + c;
  const bool col_ok = col < cols;

  const CI *src = in + slab * (size_t)LIN * cols + col;
  CC *pen = sm + c * P;
  // fully unrolled (the trip count is a constant), so all of a thread's loads are in flight at once
  constexpr int NLD = (LIN + TPP - 1) / TPP;
  CC v[NLD];
#pragma unroll
  for (int i = 0; i < NLD; ++i) {
    const int l = l0 + i * TPP;
    v[i] = CC{0, 0};
    if (col_ok && l < LIN) v[i] = c_cvt<CC>(src[(size_t)l * cols]);
  }
#pragma unroll
  for (int i = 0; i < NLD; ++i) {
    const int l = l0 + i * TPP;
    if (l < LIN) pen[sm_idx<CC>(DIR > 0 ? kept_to_fft(l, K, N) : l)] = v[i];
  }
  if (DIR > 0) {
    // FFT indices K+1 .. N-K-1 are outside the kept set
    for (int l = l0; l < N - NK; l += TPP) pen[sm_idx<CC>(K + 1 + l)] = CC{0, 0};
  }
  // double-float at N >= 512: the twiddle table staged in shared memory behind the pencils
  constexpr bool kTws = tws_staged<CC, N>();
  const CC *twp = tw;
  if constexpr (kTws) {
    CC *tws = sm + tc * P;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = tw[i];
    twp = tws;
  }
  __syncthreads();

  const int pencil = threadIdx.x / TPP;
  const int t = threadIdx.x - pencil * TPP;
  const bool active = pencil < tc && tile * tc + pencil < cols;
  pencil_fft<N, DIR, CC, VPT, (DIR > 0), kTws>(sm + (active ? pencil : 0) * P, t, active, twp);  // inverse: zero-padded
  __syncthreads();  // the store loop reads every pencil

  if (col_ok) {
    CO *dst = out + slab * (size_t)LOUT * cols + col;
    for (int l = l0; l < LOUT; l += TPP) {
      CC v = pen[sm_idx<CC>(DIR > 0 ? l : kept_to_fft(l, K, N))];
      if (DIR < 0 && scale != (typename scale_of<CC>::type)1) v = c_scale(v, scale);
      dst[(size_t)l * cols] = c_store(c_cvt<CO>(v));
    }
  }
}

template <int N, int DIR, typename CI, typename CO, typename CC, int VPT>
__global__ void col_fft_kernel(const CI *__restrict__ in, CO *__restrict__ out, int ntiles, int tsh,
                               int cols, typename scale_of<CC>::type scale, const CC *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  col_fft_tile<N, DIR, CI, CO, CC, VPT>(in, out, blockIdx.x, ntiles, tsh, cols, scale, tw,
                                        reinterpret_cast<CC *>(smem_raw));
}

// Double-float forward passes: the same tile with 4 blocks of 256 threads per SM (64 registers a
// thread), which measured 8 % faster at 512^3 than the 3 blocks that 72 registers allow (the
// inverse passes measured slower so and keep col_fft_kernel).
template <int N, int DIR, typename CI, typename CO, typename CC, int VPT>
__global__ void __launch_bounds__(256, 4) col_fft_kernel_b4(const CI *__restrict__ in, CO *__restrict__ out,
                                                           int ntiles, int tsh, int cols,
                                                           typename scale_of<CC>::type scale,
                                                           const CC *__restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  col_fft_tile<N, DIR, CI, CO, CC, VPT>(in, out, blockIdx.x, ntiles, tsh, cols, scale, tw,
                                        reinterpret_cast<CC *>(smem_raw));
}

// The kernel a pass launches.
template <int N, int DIR, typename CI, typename CO, int VPT>
constexpr auto col_kernel() {
  if constexpr (std::is_same<CO, cdf>::value && DIR < 0) return col_fft_kernel_b4<N, DIR, CI, CO, CO, VPT>;
  else return col_fft_kernel<N, DIR, CI, CO, CO, VPT>;
}

// The same pass as a persistent kernel: a grid of (SMs x resident blocks) takes tiles from the
// work counter ctr[0] until all `total` are done; ctr[1] counts the blocks that have finished, and
// the last one resets both for the next launch (every block has taken its last tile by then; no
// block waits on another).  Each tile's arithmetic is the one col_fft_kernel does.
template <int N, int DIR, typename CI, typename CO, typename CC, int VPT>
__global__ void col_fft_persistent_kernel(const CI *__restrict__ in, CO *__restrict__ out, int ntiles, int tsh,
                                          int cols, typename scale_of<CC>::type scale, const CC *__restrict__ tw,
                                          unsigned total, unsigned *ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(ctr, 1u);
    __syncthreads();
    const unsigned w = next;
    if (w >= total) break;
    col_fft_tile<N, DIR, CI, CO, CC, VPT>(in, out, w, ntiles, tsh, cols, scale, tw, reinterpret_cast<CC *>(smem_raw));
    __syncthreads();  // the tile's shared memory and `next` are free again
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1u) == gridDim.x - 1) {
      ctr[0] = 0u;
      ctr[1] = 0u;
    }
  }
}

namespace {

// Columns per block: enough that a tile row is at least 128 bytes and a block at least 128
// threads, but not more than the columns there are; 16-byte values (FP64 and double-float) at most
// 256 threads a block (the width the autotuner picks for them at N >= 512 on GB300).
int pick_tc(int tpp, int cols, size_t elem) {
  int tc = 8;
  while (tc * tpp < 128 && tc < 64) tc *= 2;
  while (tc * tpp > 1024) tc /= 2;
  while (elem >= 16 && tc > 1 && tc * tpp > 256) tc /= 2;
  while (tc > 1 && tc / 2 >= cols) tc /= 2;  // no more than one power of two above `cols`
  return tc;
}

// log2 of the largest power of two <= v (v >= 1)
int floor_log2(int v) {
  int s = 0;
  while ((2 << s) <= v) ++s;
  return s;
}

// Largest thread count a launch of this instantiation may use (its registers bound it below 1024).
template <int N, int DIR, typename CI, typename CO, int VPT>
int col_max_threads() {
  static int cached = 0;
  if (cached == 0) {
    cudaFuncAttributes a;
    cached = cudaFuncGetAttributes(&a, col_kernel<N, DIR, CI, CO, VPT>()) == cudaSuccess ? a.maxThreadsPerBlock
                                                                                               : 256;
  }
  return cached;
}

// Resident blocks per SM of a persistent launch (per instantiation and block shape).
template <auto Fn>
int resident_blocks(int threads, size_t smem) {
  static int cached_threads = -1, cached = 1;
  static size_t cached_smem = 0;
  if (threads != cached_threads || smem != cached_smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Fn, threads, smem) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    cached = per_sm > 0 ? per_sm : 1;
    cached_threads = threads;
    cached_smem = smem;
  }
  return cached;
}

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    sms = (cudaGetDevice(&dev) == cudaSuccess &&
           cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) ? v : 1;
  }
  return sms;
}

template <int N, int DIR, typename CI, typename CO, int VPT>
cudaError_t launch_col_v(const CI *in, CO *out, int nslab, int cols, double scale, const CO *tw,
                         cudaStream_t s, int tile, unsigned *ctr) {
  constexpr int TPP = tpp_for<N, VPT>();
  int tc = tile > 0 ? tile : pick_tc(TPP, cols, sizeof(CO));
  const int max_threads = col_max_threads<N, DIR, CI, CO, VPT>();
  while (tc > 1 && tc * TPP > max_threads) tc /= 2;
  if (tc < 1) tc = 1;
  const int tsh = floor_log2(tc);  // a requested width that is not a power of two is rounded down
  tc = 1 << tsh;
  const int ntiles = (cols + tc - 1) / tc;
  const size_t smem = (size_t)tc * pencil_pitch<CO>(N) * sizeof(CO) + tws_bytes<CO, N>();
  const long long blocks = (long long)nslab * ntiles;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (ctr != nullptr) {
    constexpr auto kfn = col_fft_persistent_kernel<N, DIR, CI, CO, CO, VPT>;
    if (smem > 48 * 1024) {
      cudaError_t e = ensure_smem<kfn>((int)smem);
      if (e != cudaSuccess) return e;
    }
    long long grid = (long long)sm_count() * resident_blocks<kfn>(tc * TPP, smem);
    if (grid > blocks) grid = blocks;
    kfn<<<(unsigned)grid, tc * TPP, smem, s>>>(in, out, ntiles, tsh, cols, (typename scale_of<CO>::type)scale, tw,
                                               (unsigned)blocks, ctr);
    return cudaGetLastError();
  }
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem<col_kernel<N, DIR, CI, CO, VPT>()>((int)smem);
    if (e != cudaSuccess) return e;
  }
  col_kernel<N, DIR, CI, CO, VPT>()<<<(unsigned)blocks, tc * TPP, smem, s>>>(
      in, out, ntiles, tsh, cols, (typename scale_of<CO>::type)scale, tw);
  return cudaGetLastError();
}

// Radix of a column pass: `vpt` 8 or 16 (FP32 only); 0 picks the library default (radix 8, and
// radix 16 for FP32 at N >= 512, where it measured faster).
template <int N, int DIR, typename CI, typename CO>
cudaError_t launch_col_n(const CI *in, CO *out, int nslab, int cols, double scale, const CO *tw,
                         cudaStream_t s, int tile, int vpt, unsigned *ctr) {
  if constexpr (sizeof(CO) == 8) {
    if (vpt == 16 || (vpt == 0 && N >= 512))
      return launch_col_v<N, DIR, CI, CO, 16>(in, out, nslab, cols, scale, tw, s, tile, ctr);
  }
  return launch_col_v<N, DIR, CI, CO, 8>(in, out, nslab, cols, scale, tw, s, tile, ctr);
}

template <int DIR, typename CI, typename CO>
cudaError_t launch_col(const CI *in, CO *out, int n, int nslab, int cols, double scale, const CO *tw,
                       cudaStream_t s, int tile, int vpt, unsigned *ctr = nullptr) {
  switch (n) {
    case 16: return launch_col_n<16, DIR>(in, out, nslab, cols, scale, tw, s, tile, vpt, ctr);
    case 32: return launch_col_n<32, DIR>(in, out, nslab, cols, scale, tw, s, tile, vpt, ctr);
    case 64: return launch_col_n<64, DIR>(in, out, nslab, cols, scale, tw, s, tile, vpt, ctr);
    case 128: return launch_col_n<128, DIR>(in, out, nslab, cols, scale, tw, s, tile, vpt, ctr);
    case 256: return launch_col_n<256, DIR>(in, out, nslab, cols, scale, tw, s, tile, vpt, ctr);
    case 512: return launch_col_n<512, DIR>(in, out, nslab, cols, scale, tw, s, tile, vpt, ctr);
    case 1024: return launch_col_n<1024, DIR>(in, out, nslab, cols, scale, tw, s, tile, vpt, ctr);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int col_max_tile_df(int n, int dir) {
  auto pick = [&](auto tag_n) -> int {
    constexpr int N = decltype(tag_n)::value;
    const int t = dir > 0 ? col_max_threads<N, +1, cdf, cdf, 8>() : col_max_threads<N, -1, cdf, cdf, 8>();
    int tc = 1;
    while (tc * 2 * tpp_for<N, 8>() <= t && tc < 64) tc *= 2;
    return tc;
  };
  switch (n) {
    case 16: return pick(std::integral_constant<int, 16>());
    case 32: return pick(std::integral_constant<int, 32>());
    case 64: return pick(std::integral_constant<int, 64>());
    case 128: return pick(std::integral_constant<int, 128>());
    case 256: return pick(std::integral_constant<int, 256>());
    case 512: return pick(std::integral_constant<int, 512>());
    case 1024: return pick(std::integral_constant<int, 1024>());
    default: return 1;
  }
}

int col_max_tile(int n, int dir, bool fp64, bool mixed_in, int vpt) {
  const bool r16 = !fp64 && vpt == 16;
  auto pick = [&](auto tag_n) -> int {
    constexpr int N = decltype(tag_n)::value;
    int t;
    if (fp64) t = dir > 0 ? col_max_threads<N, +1, cplx64, cplx64, 8>() : col_max_threads<N, -1, cplx64, cplx64, 8>();
    else if (dir > 0 && mixed_in) t = col_max_threads<N, +1, cplx64, cplx32, 8>();
    else if (dir > 0) t = r16 ? col_max_threads<N, +1, cplx32, cplx32, 16>() : col_max_threads<N, +1, cplx32, cplx32, 8>();
    else t = r16 ? col_max_threads<N, -1, cplx32, cplx32, 16>() : col_max_threads<N, -1, cplx32, cplx32, 8>();
    const int tpp = r16 ? tpp_for<N, 16>() : tpp_for<N, 8>();
    int tc = 1;
    while (tc * 2 * tpp <= t && tc < 64) tc *= 2;
    return tc;
  };
  switch (n) {
    case 16: return pick(std::integral_constant<int, 16>());
    case 32: return pick(std::integral_constant<int, 32>());
    case 64: return pick(std::integral_constant<int, 64>());
    case 128: return pick(std::integral_constant<int, 128>());
    case 256: return pick(std::integral_constant<int, 256>());
    case 512: return pick(std::integral_constant<int, 512>());
    case 1024: return pick(std::integral_constant<int, 1024>());
    default: return 1;
  }
}

cudaError_t launch_col_inverse(const cplx64 *in, cplx64 *out, int n, int nslab, int cols,
                               const cplx64 *tw, cudaStream_t s, int tile, int, unsigned *ctr) {
  return launch_col<+1>(in, out, n, nslab, cols, 1.0, tw, s, tile, 8, ctr);
}
cudaError_t launch_col_inverse(const cplx64 *in, cplx32 *out, int n, int nslab, int cols,
                               const cplx32 *tw, cudaStream_t s, int tile) {
  return launch_col<+1>(in, out, n, nslab, cols, 1.0, tw, s, tile, 8);
}
cudaError_t launch_col_inverse(const cplx32 *in, cplx32 *out, int n, int nslab, int cols,
                               const cplx32 *tw, cudaStream_t s, int tile, int vpt, unsigned *ctr) {
  return launch_col<+1>(in, out, n, nslab, cols, 1.0, tw, s, tile, vpt, ctr);
}
cudaError_t launch_col_forward(const cplx64 *in, cplx64 *out, int n, int nslab, int cols,
                               double scale, const cplx64 *tw, cudaStream_t s, int tile, int, unsigned *ctr) {
  return launch_col<-1>(in, out, n, nslab, cols, scale, tw, s, tile, 8, ctr);
}
cudaError_t launch_col_forward(const cplx32 *in, cplx32 *out, int n, int nslab, int cols,
                               double scale, const cplx32 *tw, cudaStream_t s, int tile, int vpt, unsigned *ctr) {
  return launch_col<-1>(in, out, n, nslab, cols, scale, tw, s, tile, vpt, ctr);
}
cudaError_t launch_col_inverse(const cdf *in, cdf *out, int n, int nslab, int cols, const cdf *tw, cudaStream_t s,
                               int tile, int, unsigned *ctr) {
  return launch_col<+1>(in, out, n, nslab, cols, 1.0, tw, s, tile, 8, ctr);
}
cudaError_t launch_col_forward(const cdf *in, cdf *out, int n, int nslab, int cols, double scale, const cdf *tw,
                               cudaStream_t s, int tile, int, unsigned *ctr) {
  return launch_col<-1>(in, out, n, nslab, cols, scale, tw, s, tile, 8, ctr);
}

}  // namespace mhd
