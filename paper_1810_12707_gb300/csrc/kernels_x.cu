// kernels_x.cu -- passes along the contiguous x axis, where real-space data exists.
//
// Two real rows of the same field are transformed together as one complex pencil
// z = f_row0 + i f_row1.  Inverse (half spectrum -> real rows): with the truncated half spectra
// X0, X1 (kx = 0..K), Z[k] = X0[k] + i X1[k] and Z[N-k] = conj(X0[k]) + i conj(X1[k]) for
// 1 <= k <= K, Z[0] = Re X0[0] + i Re X1[0] (the Hermitian part), zero elsewhere; the real parts
// of the inverse FFT are row 0 and the imaginary parts row 1.  Forward (real rows -> half
// spectra): Z = FFT(row0 + i row1), X0[k] = (Z[k] + conj Z[N-k]) / 2 and
// X1[k] = -i (Z[k] - conj Z[N-k]) / 2, kept for k = 0..K only.
//
// The flux passes store 2 X0 and 2 X1 (the factor 1/2 of the split is left to the assembly, which
// scales the product spectra by 1/(2 N^3): a power of two, so the results are the same bits).
// The flux kernel is the fused pass of the method: the 7 state fields of a block's rows are
// brought to the grid, the 12 products of the RHS are formed pointwise in shared memory (no
// real-space array ever reaches HBM), and their forward transforms leave as truncated half
// spectra.  Rows are indexed r = z*N + y; a block owns PAIRS consecutive row pairs.
#include "fft_device.cuh"
#include "launch_util.cuh"
#include "tma_util.cuh"

namespace mhd {

namespace {

constexpr int kMaxThreads = 384;

constexpr int pairs_for(int n) { return (n / 8) >= 16 ? 1 : 16 / (n / 8); }

constexpr int threads_for(int tpp, int pencils, int max_threads = kMaxThreads) {
  // groups of tpp threads (one pencil each), at most max_threads threads, a multiple of 32
  int g = max_threads / tpp;
  if (g < 1) g = 1;
  if (g > pencils) g = pencils;
  int t = g * tpp;
  return (t + 31) / 32 * 32;
}

// Block size of the flux pass.  At N = 256 and 512 several smaller blocks per SM let one block
// transform while another waits at a barrier (measured on GB300 over 96..384 threads: 128 best at
// 256^3 in both precisions, 192 at 512^3); below, the pencil count caps the block at 192 threads.
// The double-float pass at 512^3 takes 256 (two blocks of 128 registers a thread per SM): 4 %
// faster than 192.
constexpr int flux_max_threads(int n, bool df = false) {
  return n == 256 ? 128 : n == 512 ? (df ? 256 : 192) : kMaxThreads;
}
// Values per thread of the flux pass's transforms: FP32 at N <= 256 uses radix 16 (measured
// faster at 64^3 and 256^3); larger FP32 grids and FP64 use radix 8.
template <int N, typename C>
constexpr int flux_vpt() { return sizeof(C) == 8 && N <= 256 ? 16 : 8; }
template <int N, typename C>
constexpr int flux_threads() {
  return threads_for(tpp_for<N, flux_vpt<N, C>()>(), 12 * pairs_for(N),
                     flux_max_threads(N, std::is_same<C, cdf>::value));
}
// Blocks per SM the register allocation is sized for: about 170 registers a thread in FP64, 85 in
// FP32 with radix 8 and 128 with radix 16 (its 16 values per thread).
template <int N, typename C>
constexpr int flux_min_blocks() {
  const int budget = sizeof(C) == 8 ? (flux_vpt<N, C>() == 16 ? 512 : 768)
                                    : (N == 512 && std::is_same<C, cdf>::value ? 512 : 384);
  const int b = budget / flux_threads<N, C>();
  return b < 1 ? 1 : b;
}

// Run the FFT of `np` pencils (pencil id -> shared-memory pointer `ptr(id)`) with every group of
// N/VPT threads of the block taking one pencil at a time.  Each pencil is touched by its group only,
// so the stages synchronise per group; one block barrier closes the whole transform.
// Every inverse (DIR = +1) transform here starts from a truncated half spectrum, so its pencil is
// zero-padded by the 2/3 rule (see pencil_fft).
template <int N, int DIR, int VPT, typename Ptr, typename C>
__device__ __forceinline__ void fft_pencils(int np, Ptr ptr, const C *__restrict__ tw) {
  constexpr int TPP = tpp_for<N, VPT>();
  const int G = blockDim.x / TPP;
  const int g = threadIdx.x / TPP, t = threadIdx.x - g * TPP;
  for (int base = 0; base < np; base += G) {
    const int id = base + g;
    const bool active = g < G && id < np;
    pencil_fft<N, DIR, C, VPT, (DIR > 0)>(ptr(active ? id : 0), t, active, tw);
  }
  __syncthreads();  // the callers' next phase reads every pencil
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Fused flux pass
// ------------------------------------------------------------------------------------------
// C: complex type of the data and of all arithmetic (cplx64 or cplx32); the CFL maxima are
// combined in FP64.
// bgrid (nullable): the grid magnetic field is also written out, [inst][3][N^3] in the data's
// precision, for the tracer push.
// One work item w = (instance, block of PAIRS row pairs); `sm` the block's dynamic shared memory,
// `red` 32 doubles of shared scratch for the block maximum.
template <int N, typename C>
__device__ __forceinline__ void flux_x_item(const C *__restrict__ in, C *__restrict__ out,
                                            const PhysDev *__restrict__ phys,
                                            unsigned long long *__restrict__ smax_bits, int K, int blocks_per_inst,
                                            const C *__restrict__ tw, typename grid_of<C>::type *__restrict__ bgrid,
                                            unsigned w, C *sm, double *red) {
  constexpr int KT = (N - 1) / 3;  // the 2/3-rule cut-off, fixed by N
  using R = typename C::value_type;
  constexpr int P = pencil_pitch<C>(N);
  constexpr int PAIRS = pairs_for(N);
  constexpr size_t NN = (size_t)N * N;
  constexpr int NX = KT + 1;
  const int inst = (int)(w / (unsigned)blocks_per_inst);
  const int bl = (int)(w - (unsigned)inst * (unsigned)blocks_per_inst);
  const size_t row0 = (size_t)bl * PAIRS * 2;
  // the launch uses exactly this many threads, so every loop below has a constant trip count
  constexpr int nthr = flux_threads<N, C>();

  // 1. load and pack the 7 state fields: pencil (p, f) at sm + (p * 12 + f) * P.  Unrolled: all
  // of a thread's loads are issued before the first shared-memory store.
  constexpr int NLD = 7 * PAIRS * NX;
#pragma unroll
  for (int q0 = 0; q0 < NLD; q0 += nthr) {
    const int q = q0 + (int)threadIdx.x;
    if (q < NLD) {
      const int k = q % NX;
      const int r = q / NX;
      const int f = r % 7, p = r / 7;
      const C *src = in + ((size_t)(inst * 7 + f) * NN + row0 + 2 * p) * NX;
      C *pen = sm + (p * 12 + f) * P;
      const C x0 = src[k], x1 = src[NX + k];
      if (k == 0) {
        pen[0] = C{x0.re, x1.re};
      } else {
        pen[sm_idx<C>(k)] = C{x0.re - x1.im, x0.im + x1.re};
        pen[sm_idx<C>(N - k)] = C{x0.re + x1.im, x1.re - x0.im};
      }
    }
  }
  for (int q = threadIdx.x; q < 7 * PAIRS * (N - 2 * KT - 1); q += nthr) {
    const int z = q % (N - 2 * KT - 1);
    const int r = q / (N - 2 * KT - 1);
    const int f = r % 7, p = r / 7;
    sm[(p * 12 + f) * P + sm_idx<C>(KT + 1 + z)] = C{0, 0};
  }
  __syncthreads();

  // 2. inverse transforms of the 7 fields
  fft_pencils<N, +1, (flux_vpt<N, C>())>(7 * PAIRS, [&](int id) { return sm + ((id / 7) * 12 + id % 7) * P; }, tw);

  // 3. products on the grid (real part: row 0, imaginary part: row 1)
  constexpr bool kDF = std::is_same<C, cdf>::value;
  using SM = typename std::conditional<kDF, double, R>::type;  // type of the CFL maximum
  SM smax = 0;
  // FP64 and double-float: the maximum that blocks of this pass have already published is a
  // lower bound of the pass's maximum.  A point whose FP32 estimate of |u| + c_f lies below
  // `screen` (that bound less 1e-6 relative and 1e-18 absolute, above the estimate's worst error
  // of about 3e-7 relative) cannot raise it, so its exact speed (two FP64 square roots) is not
  // formed.  The pass still yields the exact maximum, whichever blocks ran first; a NaN or an
  // infinite estimate always takes the exact path.
  float screen = 0.f;
  if constexpr (sizeof(SM) == 8) {
    const double lb = __longlong_as_double((long long)*reinterpret_cast<volatile unsigned long long *>(smax_bits + inst));
    screen = (float)(lb * (1.0 - 1e-6) - 1e-18);
  }
  if constexpr (kDF) {
    // double-float products.  The grid values leave the inverse transforms unnormalised; near a
    // zero of a field (a stagnation point) their low part can exceed the high part, and the
    // square of such a pair, which drops lo^2, can come out negative.  So they are renormalised
    // first (then |lo| <= ulp(hi) / 2 and every square is >= 0), as are the velocity components
    // before the speed is formed; the speed's squares are renormalised too, so their high parts
    // are the FP32 roundings the screening estimate assumes, and the exact speed is taken in FP64
    // from the double-float squares.
    const double csd = phys[inst].cs;
    const dfr cs2 = dfr_from_double(csd * csd);
    for (int q = threadIdx.x; q < PAIRS * N; q += nthr) {
      const int p = q / N, j = q - p * N;
      C *b = sm + p * 12 * P + sm_idx<C>(j);
      dfr v[2][7];
#pragma unroll
      for (int f = 0; f < 7; ++f) {
        const C c = b[f * P];
        v[0][f] = dfr_norm(c.re);
        v[1][f] = dfr_norm(c.im);
      }
      if (bgrid != nullptr) {
        constexpr size_t N3 = NN * N;
        double *g = bgrid + (size_t)inst * 3 * N3 + (row0 + 2 * p) * N + j;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          g[c * N3] = dfr_to_double(v[0][4 + c]);
          g[c * N3 + N] = dfr_to_double(v[1][4 + c]);
        }
      }
      dfr *bd = reinterpret_cast<dfr *>(b);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const dfr rho = v[h][0];
        const dfr mx = v[h][1], my = v[h][2], mz = v[h][3];
        const dfr bx = v[h][4], by = v[h][5], bz = v[h][6];
        const dfr ir = dfr_rcp(rho);
        const dfr ux = mx * ir, uy = my * ir, uz = mz * ir;
        const dfr bxx = bx * bx, byy = by * by, bzz = bz * bz;
        const dfr b2 = bxx + byy + bzz;
        const dfr hb = dfr_scale2(b2, 0.5f);
        bd[2 * 0 * P + h] = mx * ux + hb - bxx;   // T_xx
        bd[2 * 1 * P + h] = my * uy + hb - byy;   // T_yy
        bd[2 * 2 * P + h] = mz * uz + hb - bzz;   // T_zz
        bd[2 * 3 * P + h] = mx * uy - bx * by;    // T_xy
        bd[2 * 4 * P + h] = mx * uz - bx * bz;    // T_xz
        bd[2 * 5 * P + h] = my * uz - by * bz;    // T_yz
        bd[2 * 6 * P + h] = uy * bz - uz * by;    // E_x
        bd[2 * 7 * P + h] = uz * bx - ux * bz;    // E_y
        bd[2 * 8 * P + h] = ux * by - uy * bx;    // E_z
        bd[2 * 9 * P + h] = ux;
        bd[2 * 10 * P + h] = uy;
        bd[2 * 11 * P + h] = uz;
        const dfr nx = dfr_norm(ux), ny = dfr_norm(uy), nz = dfr_norm(uz);
        const dfr u2 = dfr_norm(nx * nx + ny * ny + nz * nz), c2 = dfr_norm(cs2 + b2 * ir);
        if (!(sqrtf(u2.hi) + sqrtf(c2.hi) < screen)) {
          const double s = sqrt(dfr_to_double(u2)) + sqrt(dfr_to_double(c2));
          smax = (s != s || s > smax) ? s : smax;  // keeps a NaN once seen
        }
      }
    }
  } else {
  const R cs2 = (R)(phys[inst].cs * phys[inst].cs);
  for (int q = threadIdx.x; q < PAIRS * N; q += nthr) {
    const int p = q / N, j = q - p * N;
    C *b = sm + p * 12 * P + sm_idx<C>(j);
    R v[2][7];
#pragma unroll
    for (int f = 0; f < 7; ++f) {
      const C c = b[f * P];
      v[0][f] = c.re;
      v[1][f] = c.im;
    }
    if (bgrid != nullptr) {
      constexpr size_t N3 = NN * N;
      R *g = bgrid + (size_t)inst * 3 * N3 + (row0 + 2 * p) * N + j;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        g[c * N3] = v[0][4 + c];
        g[c * N3 + N] = v[1][4 + c];
      }
    }
    R *bd = reinterpret_cast<R *>(b);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const R rho = v[h][0];
      const R mx = v[h][1], my = v[h][2], mz = v[h][3];
      const R bx = v[h][4], by = v[h][5], bz = v[h][6];
      const R ir = (R)1 / rho;
      const R ux = mx * ir, uy = my * ir, uz = mz * ir;
      const R b2 = bx * bx + by * by + bz * bz;
      const R hb = (R)0.5 * b2;
      // component h of pencil f at this point is bd[2 * f * P + h]
      bd[2 * 0 * P + h] = mx * ux + hb - bx * bx;   // T_xx
      bd[2 * 1 * P + h] = my * uy + hb - by * by;   // T_yy
      bd[2 * 2 * P + h] = mz * uz + hb - bz * bz;   // T_zz
      bd[2 * 3 * P + h] = mx * uy - bx * by;        // T_xy
      bd[2 * 4 * P + h] = mx * uz - bx * bz;        // T_xz
      bd[2 * 5 * P + h] = my * uz - by * bz;        // T_yz
      bd[2 * 6 * P + h] = uy * bz - uz * by;        // E_x
      bd[2 * 7 * P + h] = uz * bx - ux * bz;        // E_y
      bd[2 * 8 * P + h] = ux * by - uy * bx;        // E_z
      bd[2 * 9 * P + h] = ux;
      bd[2 * 10 * P + h] = uy;
      bd[2 * 11 * P + h] = uz;
      const R u2 = ux * ux + uy * uy + uz * uz, c2 = cs2 + b2 * ir;
      if constexpr (sizeof(R) == 8) {
        if (!(sqrtf((float)u2) + sqrtf((float)c2) < screen)) {
          const R s = sqrt(u2) + sqrt(c2);
          smax = (s != s || s > smax) ? s : smax;  // keeps a NaN once seen
        }
      } else {
        const R s = sqrt(u2) + sqrt(c2);
        smax = (s != s || s > smax) ? s : smax;
      }
    }
  }
  }
  __syncthreads();

  // 4. forward transforms of the 12 products
  fft_pencils<N, -1, (flux_vpt<N, C>())>(12 * PAIRS, [&](int id) { return sm + id * P; }, tw);

  // 5. unpack and store the kept half spectra
  for (int q = threadIdx.x; q < 12 * PAIRS * NX; q += nthr) {
    const int k = q % NX;
    const int r = q / NX;
    const int f = r % 12, p = r / 12;
    const C *pen = sm + (p * 12 + f) * P;
    const C z = pen[sm_idx<C>(k)], zc = pen[sm_idx<C>((N - k) & (N - 1))];
    C *dst = out + ((size_t)(inst * 12 + f) * NN + row0 + 2 * p) * NX;
    dst[k] = c_store(C{z.re + zc.re, z.im - zc.im});
    dst[NX + k] = c_store(C{z.im + zc.im, zc.re - z.re});
  }

  const SM m = block_nan_max(smax, reinterpret_cast<SM *>(red));
  if (threadIdx.x == 0) atomicMax(smax_bits + inst, max_bits((double)m));
}

template <int N, typename C>
__global__ void __launch_bounds__((flux_threads<N, C>()), (flux_min_blocks<N, C>()))
    flux_x_kernel(const C *__restrict__ in, C *__restrict__ out, const PhysDev *__restrict__ phys,
                  unsigned long long *__restrict__ smax_bits, int K, int blocks_per_inst, const C *__restrict__ tw,
                  typename grid_of<C>::type *__restrict__ bgrid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  flux_x_item<N, C>(in, out, phys, smax_bits, K, blocks_per_inst, tw, bgrid, blockIdx.x,
                    reinterpret_cast<C *>(smem_raw), red);
}

// The same pass as a persistent kernel (batched small grids): a grid of resident blocks takes
// work items from ctr[0] until all `total` are done; ctr[1] counts finished blocks and the last
// one resets both (no block waits on another).  Each item computes what flux_x_kernel computes.
template <int N, typename C>
__global__ void __launch_bounds__((flux_threads<N, C>()), (flux_min_blocks<N, C>()))
    flux_x_persistent_kernel(const C *__restrict__ in, C *__restrict__ out, const PhysDev *__restrict__ phys,
                             unsigned long long *__restrict__ smax_bits, int K, int blocks_per_inst,
                             const C *__restrict__ tw, typename grid_of<C>::type *__restrict__ bgrid, unsigned total,
                             unsigned *ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ unsigned next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(ctr, 1u);
    __syncthreads();
    const unsigned w = next;
    if (w >= total) break;
    flux_x_item<N, C>(in, out, phys, smax_bits, K, blocks_per_inst, tw, bgrid, w, reinterpret_cast<C *>(smem_raw),
                      red);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1u) == gridDim.x - 1) {
      ctr[0] = 0u;
      ctr[1] = 0u;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Fused flux pass, persistent and pipelined (one row pair per iteration, N >= 128, FP32)
// ------------------------------------------------------------------------------------------
// Each block walks over row pairs (pair = blockIdx.x, + gridDim.x, ...).  The 7 state rows of
// the next pair (one contiguous chunk of 2 * NX complex values per field) are fetched with bulk
// asynchronous copies into the other of two staging buffers while the current pair is
// transformed, so the copy engine keeps HBM busy during the FFT work.  The arithmetic, its order
// and the results are those of flux_x_kernel.  A wait for a copy that does not complete within
// `wait_polls` polls (kWaitPolls unless a caller lowers it; 0 gives up at once) sets *err = 1.
// Before the block returns, thread 0 then waits, with the full limit kWaitPolls each, for BOTH
// copies the block may still have in flight -- the one it gave up on and the prefetch of the
// next row pair -- so that no bulk copy lands in shared memory after the block has released it;
// if one of those waits also runs out, *err = 2.

template <int N, typename C>
__global__ void __launch_bounds__(kMaxThreads, 1)
    flux_x_pipe_kernel(const C *__restrict__ in, C *__restrict__ out, const PhysDev *__restrict__ phys,
                       unsigned long long *__restrict__ smax_bits, int K, long long total_pairs,
                       const C *__restrict__ tw, int *err, uint32_t wait_polls) {
  constexpr int KT = (N - 1) / 3;  // the 2/3-rule cut-off, fixed by N
  using R = typename C::value_type;
  extern __shared__ __align__(128) unsigned char smem_pipe[];
  __shared__ __align__(8) uint64_t mbar[2];
  constexpr int P = pencil_pitch<C>(N);
  constexpr long long PPI = (long long)N * N / 2;  // row pairs per instance
  constexpr size_t NN = (size_t)N * N;
  constexpr int NX = KT + 1;
  const int chunk = 2 * NX;  // complex values of one field's row pair
  const uint32_t chunk_bytes = (uint32_t)(chunk * sizeof(C));
  C *stage = reinterpret_cast<C *>(smem_pipe);
  C *sm = stage + ((2 * 7 * chunk * sizeof(C) + 127) / 128 * 128) / sizeof(C);
  const int nthr = blockDim.x;

  auto issue = [&](long long pr, int b) {
    const int inst = (int)(pr / PPI);
    const size_t row0 = (size_t)(pr - (long long)inst * PPI) * 2;
    mbar_arrive_expect_tx(&mbar[b], 7 * chunk_bytes);
    for (int f = 0; f < 7; ++f)
      bulk_g2s(stage + (size_t)(b * 7 + f) * chunk, in + ((size_t)(inst * 7 + f) * NN + row0) * NX, chunk_bytes,
               &mbar[b]);
  };

  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  long long pair = blockIdx.x;
  if (threadIdx.x == 0 && pair < total_pairs) issue(pair, 0);
  int issued_next = 0;
  for (int iter = 0; pair < total_pairs; pair += gridDim.x, ++iter) {
    const int buf = iter & 1;
    const long long nxt = pair + gridDim.x;
    if (threadIdx.x == 0) {
      issued_next = nxt < total_pairs;
      if (issued_next) {
        fence_proxy_async();
        issue(nxt, buf ^ 1);
      }
    }
    const bool ok = mbar_wait(&mbar[buf], (iter >> 1) & 1, wait_polls);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        // drain: the copy into stage[buf] that the wait gave up on, and the prefetch into
        // stage[buf ^ 1] issued above; the block's shared memory stays allocated while thread 0
        // is still running
        bool drained = mbar_wait(&mbar[buf], (iter >> 1) & 1, kWaitPolls);
        if (issued_next) drained = mbar_wait(&mbar[buf ^ 1], ((iter + 1) >> 1) & 1, kWaitPolls) && drained;
        if (!drained) atomicExch(err, 2);
      }
      return;
    }
    const int inst = (int)(pair / PPI);
    const size_t row0 = (size_t)(pair - (long long)inst * PPI) * 2;
    const int tx = launder(threadIdx.x);

    // 1. pack the 7 fields of this row pair from the staging buffer
    const C *st = stage + (size_t)buf * 7 * chunk;
    for (int q = tx; q < 7 * NX; q += nthr) {
      const int k = q % NX, f = q / NX;
      const C x0 = st[f * chunk + k], x1 = st[f * chunk + NX + k];
      C *pen = sm + f * P;
      if (k == 0) {
        pen[0] = C{x0.re, x1.re};
      } else {
        pen[sm_idx<C>(k)] = C{x0.re - x1.im, x0.im + x1.re};
        pen[sm_idx<C>(N - k)] = C{x0.re + x1.im, x1.re - x0.im};
      }
    }
    for (int q = tx; q < 7 * (N - 2 * KT - 1); q += nthr) {
      const int z = q % (N - 2 * KT - 1), f = q / (N - 2 * KT - 1);
      sm[f * P + sm_idx<C>(KT + 1 + z)] = C{0, 0};
    }
    __syncthreads();

    // 2. inverse transforms of the 7 fields
    fft_pencils<N, +1, (flux_vpt<N, C>())>(7, [&](int id) { return sm + id * P; }, tw);

    // 3. products on the grid
    const R cs2 = (R)(phys[inst].cs * phys[inst].cs);
    R smax = 0;
    for (int j = tx; j < N; j += nthr) {
      C *b = sm + sm_idx<C>(j);
      R v[2][7];
#pragma unroll
      for (int f = 0; f < 7; ++f) {
        const C c = b[f * P];
        v[0][f] = c.re;
        v[1][f] = c.im;
      }
      R *bd = reinterpret_cast<R *>(b);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const R rho = v[h][0];
        const R mx = v[h][1], my = v[h][2], mz = v[h][3];
        const R bx = v[h][4], by = v[h][5], bz = v[h][6];
        const R ir = (R)1 / rho;
        const R ux = mx * ir, uy = my * ir, uz = mz * ir;
        const R b2 = bx * bx + by * by + bz * bz;
        const R hb = (R)0.5 * b2;
        bd[2 * 0 * P + h] = mx * ux + hb - bx * bx;
        bd[2 * 1 * P + h] = my * uy + hb - by * by;
        bd[2 * 2 * P + h] = mz * uz + hb - bz * bz;
        bd[2 * 3 * P + h] = mx * uy - bx * by;
        bd[2 * 4 * P + h] = mx * uz - bx * bz;
        bd[2 * 5 * P + h] = my * uz - by * bz;
        bd[2 * 6 * P + h] = uy * bz - uz * by;
        bd[2 * 7 * P + h] = uz * bx - ux * bz;
        bd[2 * 8 * P + h] = ux * by - uy * bx;
        bd[2 * 9 * P + h] = ux;
        bd[2 * 10 * P + h] = uy;
        bd[2 * 11 * P + h] = uz;
        const R s = sqrt(ux * ux + uy * uy + uz * uz) + sqrt(cs2 + b2 * ir);
        smax = (s != s || s > smax) ? s : smax;
      }
    }
    __syncthreads();

    // 4. forward transforms of the 12 products
    fft_pencils<N, -1, (flux_vpt<N, C>())>(12, [&](int id) { return sm + id * P; }, tw);

    // 5. unpack and store
      for (int q = tx; q < 12 * NX; q += nthr) {
      const int k = q % NX, f = q / NX;
      const C *pen = sm + f * P;
      const C z = pen[sm_idx<C>(k)], zc = pen[sm_idx<C>((N - k) & (N - 1))];
      C *dst = out + ((size_t)(inst * 12 + f) * NN + row0) * NX;
      dst[k] = C{z.re + zc.re, z.im - zc.im};
      dst[NX + k] = C{z.im + zc.im, zc.re - z.re};
    }

    // CFL maximum of this pair: warp maximum, one atomic per warp
    R m = smax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = nan_max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(smax_bits + inst, max_bits((double)m));
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// Forward x transform of an initial state (m = rho u formed first)
// ------------------------------------------------------------------------------------------
// The real fields are FP64; C = cplx64 transforms in FP64, C = cdf splits each value (and the FP64
// product rho u) into double-float pairs and transforms in double-float.
__device__ __forceinline__ void x_load(double v, double &r) { r = v; }
__device__ __forceinline__ void x_load(double v, dfr &r) { r = dfr_from_double(v); }
__device__ __forceinline__ double x_store(double v) { return v; }
__device__ __forceinline__ double x_store(dfr v) { return dfr_to_double(v); }

template <int N, typename C>
// Rows from `row_begin` on (a multiple of 2 PAIRS); the real arrays hold rows from `row_begin`
// with field stride `fstride` (N^3 for whole fields, less for a slab of z-planes).
__global__ void __launch_bounds__(kMaxThreads) set_x_kernel(const double *__restrict__ rho, const double *__restrict__ u,
                             const double *__restrict__ b, C *__restrict__ out, int K,
                             const C *__restrict__ tw, size_t row_begin, size_t fstride) {
  using R = typename C::value_type;
  constexpr int KT = (N - 1) / 3;  // the 2/3-rule cut-off, fixed by N
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sm = reinterpret_cast<C *>(smem_raw);
  constexpr int P = pencil_pitch<C>(N);
  constexpr int PAIRS = pairs_for(N);
  constexpr size_t NN = (size_t)N * N;
  constexpr int NX = KT + 1;
  const size_t row0 = row_begin + (size_t)blockIdx.x * PAIRS * 2;
  const int nthr = blockDim.x;

  for (int q = threadIdx.x; q < PAIRS * N; q += nthr) {
    const int p = q / N, j = q - p * N;
    const size_t i0 = (row0 - row_begin + 2 * p) * N + j, i1 = i0 + N;
    const double r0 = rho[i0], r1 = rho[i1];
    C *pen = sm + p * 7 * P + sm_idx<C>(j);
    R a, c;
    x_load(r0, a);
    x_load(r1, c);
    pen[0] = C{a, c};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      x_load(r0 * u[d * fstride + i0], a);
      x_load(r1 * u[d * fstride + i1], c);
      pen[(1 + d) * P] = C{a, c};
      x_load(b[d * fstride + i0], a);
      x_load(b[d * fstride + i1], c);
      pen[(4 + d) * P] = C{a, c};
    }
  }
  __syncthreads();
  fft_pencils<N, -1, 8>(7 * PAIRS, [&](int id) { return sm + id * P; }, tw);
  for (int q = threadIdx.x; q < 7 * PAIRS * NX; q += nthr) {
    const int k = q % NX;
    const int r = q / NX;
    const int f = r % 7, p = r / 7;
    const C *pen = sm + (p * 7 + f) * P;
    const C z = pen[sm_idx<C>(k)], zc = pen[sm_idx<C>((N - k) & (N - 1))];
    C *dst = out + ((size_t)f * NN + row0 + 2 * p) * NX;
    dst[k] = c_store(c_scale(C{z.re + zc.re, z.im - zc.im}, (typename scale_of<C>::type)0.5));
    dst[NX + k] = c_store(c_scale(C{z.im + zc.im, zc.re - z.re}, (typename scale_of<C>::type)0.5));
  }
}

// ------------------------------------------------------------------------------------------
// Inverse x transform to real rows
// ------------------------------------------------------------------------------------------
template <int N, typename C>
// Rows from `row_begin` on; `out` holds rows from `row_begin` with field stride `fstride`.
__global__ void __launch_bounds__(kMaxThreads) get_x_kernel(const C *__restrict__ in, double *__restrict__ out, int nf, int K,
                             const C *__restrict__ tw, size_t row_begin, size_t fstride) {
  constexpr int KT = (N - 1) / 3;  // the 2/3-rule cut-off, fixed by N
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sm = reinterpret_cast<C *>(smem_raw);
  constexpr int P = pencil_pitch<C>(N);
  constexpr int PAIRS = pairs_for(N);
  constexpr size_t NN = (size_t)N * N;
  constexpr int NX = KT + 1;
  const size_t row0 = row_begin + (size_t)blockIdx.x * PAIRS * 2;
  const int nthr = blockDim.x;

  for (int q = threadIdx.x; q < nf * PAIRS * NX; q += nthr) {
    const int k = q % NX;
    const int r = q / NX;
    const int f = r % nf, p = r / nf;
    const C *src = in + ((size_t)f * NN + row0 + 2 * p) * NX;
    C *pen = sm + (p * nf + f) * P;
    const C x0 = src[k], x1 = src[NX + k];
    if (k == 0) {
      pen[0] = C{x0.re, x1.re};
    } else {
      pen[sm_idx<C>(k)] = C{x0.re - x1.im, x0.im + x1.re};
      pen[sm_idx<C>(N - k)] = C{x0.re + x1.im, x1.re - x0.im};
    }
  }
  for (int q = threadIdx.x; q < nf * PAIRS * (N - 2 * KT - 1); q += nthr) {
    const int z = q % (N - 2 * KT - 1);
    const int r = q / (N - 2 * KT - 1);
    sm[r * P + sm_idx<C>(KT + 1 + z)] = C{0, 0};
  }
  __syncthreads();
  fft_pencils<N, +1, 8>(nf * PAIRS, [&](int id) { return sm + id * P; }, tw);
  for (int q = threadIdx.x; q < nf * PAIRS * N; q += nthr) {
    const int j = q % N;
    const int r = q / N;
    const int f = r % nf, p = r / nf;
    const C z = sm[(p * nf + f) * P + sm_idx<C>(j)];
    const size_t i0 = f * fstride + (row0 - row_begin + 2 * p) * N + j;
    out[i0] = x_store(z.re);
    out[i0 + N] = x_store(z.im);
  }
}

// ------------------------------------------------------------------------------------------
// Inverse x transform of the state with grid diagnostics
// ------------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kMaxThreads) diag_x_kernel(const cplx64 *__restrict__ in, const PhysDev *__restrict__ phys,
                              double *__restrict__ part, int K, const cplx64 *__restrict__ tw) {
  constexpr int KT = (N - 1) / 3;  // the 2/3-rule cut-off, fixed by N
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx64 *sm = reinterpret_cast<cplx64 *>(smem_raw);
  __shared__ double red[32];
  constexpr int P = pencil_pitch<cplx64>(N);
  constexpr int PAIRS = pairs_for(N);
  constexpr size_t NN = (size_t)N * N;
  constexpr int NX = KT + 1;
  const size_t row0 = (size_t)blockIdx.x * PAIRS * 2;
  const int nthr = blockDim.x;

  for (int q = threadIdx.x; q < 7 * PAIRS * NX; q += nthr) {
    const int k = q % NX;
    const int r = q / NX;
    const int f = r % 7, p = r / 7;
    const cplx64 *src = in + ((size_t)f * NN + row0 + 2 * p) * NX;
    cplx64 *pen = sm + (p * 7 + f) * P;
    const cplx64 x0 = src[k], x1 = src[NX + k];
    if (k == 0) {
      pen[0] = cplx64{x0.re, x1.re};
    } else {
      pen[sm_idx<cplx64>(k)] = cplx64{x0.re - x1.im, x0.im + x1.re};
      pen[sm_idx<cplx64>(N - k)] = cplx64{x0.re + x1.im, x1.re - x0.im};
    }
  }
  for (int q = threadIdx.x; q < 7 * PAIRS * (N - 2 * KT - 1); q += nthr) {
    const int z = q % (N - 2 * KT - 1);
    const int r = q / (N - 2 * KT - 1);
    sm[r * P + sm_idx<cplx64>(KT + 1 + z)] = cplx64{0.0, 0.0};
  }
  __syncthreads();
  fft_pencils<N, +1, 8>(7 * PAIRS, [&](int id) { return sm + id * P; }, tw);

  const double cs2 = phys[0].cs * phys[0].cs;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  double smax = 0.0;
  for (int q = threadIdx.x; q < PAIRS * N; q += nthr) {
    const int p = q / N, j = q - p * N;
    const cplx64 *b = sm + p * 7 * P + sm_idx<cplx64>(j);
    double v[2][7];
#pragma unroll
    for (int f = 0; f < 7; ++f) {
      const cplx64 c = b[f * P];
      v[0][f] = c.re;
      v[1][f] = c.im;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double rho = v[h][0];
      const double ux = v[h][1] / rho, uy = v[h][2] / rho, uz = v[h][3] / rho;
      const double bx = v[h][4], by = v[h][5], bz = v[h][6];
      const double u2 = ux * ux + uy * uy + uz * uz;
      const double b2 = bx * bx + by * by + bz * bz;
      acc[0] += 0.5 * rho * u2;
      acc[1] += 0.5 * b2;
      acc[2] += cs2 * rho * log(rho);
      acc[3] += ux * bx + uy * by + uz * bz;
      acc[4] += sqrt(u2);
      acc[5] += sqrt(b2);
      smax = nan_max(smax, sqrt(u2) + sqrt(cs2 + b2 / rho));
    }
  }
  for (int i = 0; i < 6; ++i) {
    const double s = block_sum(acc[i], red);
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * 8 + i] = s;
  }
  const double m = block_nan_max(smax, red);
  if (threadIdx.x == 0) {
    part[(size_t)blockIdx.x * 8 + 6] = m;
    part[(size_t)blockIdx.x * 8 + 7] = 0.0;
  }
}

// ------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------
namespace {

template <int N, typename C>
cudaError_t flux_n(const C *in, C *out, const PhysDev *phys, unsigned long long *part, const Dims &d, const C *tw,
                   cudaStream_t s, int *err, typename grid_of<C>::type *bgrid, uint32_t wait_polls, unsigned *ctr) {
  constexpr int PAIRS = pairs_for(N);
  if constexpr (PAIRS == 1 && sizeof(C) == 8) {
    if (bgrid != nullptr) err = nullptr;  // the pipelined variant does not write the grid field
    const int chunk = 2 * (d.k + 1);
    const size_t stage_bytes = (2 * 7 * chunk * sizeof(C) + 127) / 128 * 128;
    const size_t smem = stage_bytes + (size_t)12 * pencil_pitch<C>(N) * sizeof(C);
    if (err != nullptr && smem <= 200 * 1024) {
      cudaError_t e = ensure_smem<flux_x_pipe_kernel<N, C>>((int)smem);
      if (e != cudaSuccess) return e;
      const int threads = threads_for(tpp_for<N, flux_vpt<N, C>()>(), 12);
      int per_sm = 0, dev = 0, sms = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flux_x_pipe_kernel<N, C>, threads, smem);
      if (e != cudaSuccess) return e;
      if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
      if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      const long long total = (long long)d.batch * N * N / 2;
      long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
      if (blocks > total) blocks = total;
      flux_x_pipe_kernel<N, C><<<(unsigned)blocks, threads, smem, s>>>(in, out, phys, part, d.k, total, tw, err,
                                                                          wait_polls);
      return cudaGetLastError();
    }
  }
  const int bpi = N * N / (2 * PAIRS);
  const int threads = flux_threads<N, C>();
  const size_t smem = (size_t)12 * PAIRS * pencil_pitch<C>(N) * sizeof(C);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem<flux_x_kernel<N, C>>((int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (long long)bpi * d.batch;
  if (ctr != nullptr) {
    constexpr auto kfn = flux_x_persistent_kernel<N, C>;
    if (smem > 48 * 1024) {
      cudaError_t e = ensure_smem<kfn>((int)smem);
      if (e != cudaSuccess) return e;
    }
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > blocks) grid = blocks;
    kfn<<<(unsigned)grid, threads, smem, s>>>(in, out, phys, part, d.k, bpi, tw, bgrid, (unsigned)blocks, ctr);
    return cudaGetLastError();
  }
  flux_x_kernel<N, C><<<(unsigned)blocks, threads, smem, s>>>(in, out, phys, part, d.k, bpi, tw, bgrid);
  return cudaGetLastError();
}

template <int N, typename C>
cudaError_t set_n(const double *rho, const double *u, const double *b, C *out, const Dims &d,
                  const C *tw, cudaStream_t s, size_t row_begin, size_t nrows, size_t fstride) {
  constexpr int PAIRS = pairs_for(N);
  if (row_begin % (2 * PAIRS) || nrows % (2 * PAIRS)) return cudaErrorInvalidValue;
  const int blocks = (int)(nrows / (2 * PAIRS));
  if (blocks == 0) return cudaSuccess;
  const int threads = threads_for(tpp_for<N, 8>(), 7 * PAIRS);
  const size_t smem = (size_t)7 * PAIRS * pencil_pitch<C>(N) * sizeof(C);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem<set_x_kernel<N, C>>((int)smem);
    if (e != cudaSuccess) return e;
  }
  set_x_kernel<N, C><<<blocks, threads, smem, s>>>(rho, u, b, out, d.k, tw, row_begin, fstride);
  return cudaGetLastError();
}

template <int N, typename C>
cudaError_t get_n(const C *in, double *out, int nf, const Dims &d, const C *tw, cudaStream_t s,
                  size_t row_begin, size_t nrows, size_t fstride) {
  constexpr int PAIRS = pairs_for(N);
  if (row_begin % (2 * PAIRS) || nrows % (2 * PAIRS)) return cudaErrorInvalidValue;
  const int blocks = (int)(nrows / (2 * PAIRS));
  if (blocks == 0) return cudaSuccess;
  const int threads = threads_for(tpp_for<N, 8>(), nf * PAIRS);
  const size_t smem = (size_t)nf * PAIRS * pencil_pitch<C>(N) * sizeof(C);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem<get_x_kernel<N, C>>((int)smem);
    if (e != cudaSuccess) return e;
  }
  get_x_kernel<N, C><<<blocks, threads, smem, s>>>(in, out, nf, d.k, tw, row_begin, fstride);
  return cudaGetLastError();
}

template <int N>
cudaError_t diag_n(const cplx64 *in, const PhysDev *phys, double *part, const Dims &d,
                   const cplx64 *tw, cudaStream_t s) {
  constexpr int PAIRS = pairs_for(N);
  const int blocks = N * N / (2 * PAIRS);
  const int threads = threads_for(tpp_for<N, 8>(), 7 * PAIRS);
  const size_t smem = (size_t)7 * PAIRS * pencil_pitch<cplx64>(N) * sizeof(cplx64);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem<diag_x_kernel<N>>((int)smem);
    if (e != cudaSuccess) return e;
  }
  diag_x_kernel<N><<<blocks, threads, smem, s>>>(in, phys, part, d.k, tw);
  return cudaGetLastError();
}

}  // namespace

#define MHD_DISPATCH_N(n, call)     \
  switch (n) {                      \
    case 16: { constexpr int N = 16; return call; }     \
    case 32: { constexpr int N = 32; return call; }     \
    case 64: { constexpr int N = 64; return call; }     \
    case 128: { constexpr int N = 128; return call; }   \
    case 256: { constexpr int N = 256; return call; }   \
    case 512: { constexpr int N = 512; return call; }   \
    case 1024: { constexpr int N = 1024; return call; } \
    default: return cudaErrorInvalidValue;              \
  }

int flux_x_blocks_per_instance(int n) { return n * n / (2 * pairs_for(n)); }
int diag_x_blocks(int n) { return n * n / (2 * pairs_for(n)); }

cudaError_t launch_flux_x(const cplx64 *in, cplx64 *out, const PhysDev *phys, unsigned long long *smax_bits,
                          const Dims &d, const cplx64 *tw, cudaStream_t s, int *err, double *bgrid,
                          uint32_t wait_polls, unsigned *ctr) {
  MHD_DISPATCH_N(d.n, (flux_n<N>(in, out, phys, smax_bits, d, tw, s, err, bgrid, wait_polls, ctr)));
}

cudaError_t launch_flux_x(const cplx32 *in, cplx32 *out, const PhysDev *phys, unsigned long long *smax_bits,
                          const Dims &d, const cplx32 *tw, cudaStream_t s, int *err, float *bgrid,
                          uint32_t wait_polls, unsigned *ctr) {
  MHD_DISPATCH_N(d.n, (flux_n<N>(in, out, phys, smax_bits, d, tw, s, err, bgrid, wait_polls, ctr)));
}

cudaError_t launch_flux_x(const cdf *in, cdf *out, const PhysDev *phys, unsigned long long *smax_bits, const Dims &d,
                          const cdf *tw, cudaStream_t s, int *, double *bgrid, uint32_t, unsigned *ctr) {
  MHD_DISPATCH_N(d.n, (flux_n<N>(in, out, phys, smax_bits, d, tw, s, nullptr, bgrid, kWaitPolls, ctr)));
}

cudaError_t launch_set_x(const double *rho, const double *u, const double *b, cplx64 *out,
                         const Dims &d, const cplx64 *tw, cudaStream_t s) {
  const size_t nn = (size_t)d.n * d.n;
  MHD_DISPATCH_N(d.n, (set_n<N>(rho, u, b, out, d, tw, s, 0, nn, nn * d.n)));
}

cudaError_t launch_set_x_rows(const double *rho, const double *u, const double *b, cplx64 *out, const Dims &d,
                              const cplx64 *tw, cudaStream_t s, size_t row_begin, size_t nrows, size_t fstride) {
  MHD_DISPATCH_N(d.n, (set_n<N>(rho, u, b, out, d, tw, s, row_begin, nrows, fstride)));
}

cudaError_t launch_get_x(const cplx64 *in, double *out, int nfields, const Dims &d,
                         const cplx64 *tw, cudaStream_t s) {
  const size_t nn = (size_t)d.n * d.n;
  MHD_DISPATCH_N(d.n, (get_n<N>(in, out, nfields, d, tw, s, 0, nn, nn * d.n)));
}

cudaError_t launch_get_x_rows(const cplx64 *in, double *out, int nfields, const Dims &d, const cplx64 *tw,
                              cudaStream_t s, size_t row_begin, size_t nrows, size_t fstride) {
  MHD_DISPATCH_N(d.n, (get_n<N>(in, out, nfields, d, tw, s, row_begin, nrows, fstride)));
}

cudaError_t launch_set_x_rows(const double *rho, const double *u, const double *b, cdf *out, const Dims &d,
                              const cdf *tw, cudaStream_t s, size_t row_begin, size_t nrows, size_t fstride) {
  MHD_DISPATCH_N(d.n, (set_n<N>(rho, u, b, out, d, tw, s, row_begin, nrows, fstride)));
}

cudaError_t launch_get_x_rows(const cdf *in, double *out, int nfields, const Dims &d, const cdf *tw, cudaStream_t s,
                              size_t row_begin, size_t nrows, size_t fstride) {
  MHD_DISPATCH_N(d.n, (get_n<N>(in, out, nfields, d, tw, s, row_begin, nrows, fstride)));
}

cudaError_t launch_diag_x(const cplx64 *in, const PhysDev *phys, double *part, const Dims &d,
                          const cplx64 *tw, cudaStream_t s) {
  MHD_DISPATCH_N(d.n, (diag_n<N>(in, phys, part, d, tw, s)));
}

}  // namespace mhd
