// mhd_noalloc.cu -- mhd_rhs_noalloc: the right-hand side of one small state, computed without
// allocating any memory.
//
// Who this is for: callers that must not call cudaMalloc at the moment they need an RHS, e.g. a
// host framework that has already claimed the device memory for its own pool, or a latency-bound
// loop that cannot afford the implicit device synchronisation an allocation may cause.  The
// caller passes device pointers for the inputs and outputs; every intermediate spectrum lives in
// one file-scope device array (below), which each GPU that loads this library holds until the
// process exits.  The paper has no counterpart of this entry point.
//
// Properties callers rely on:
//   * no cudaMalloc / cudaFree / allocating library routine is called, ever;
//   * n is limited to kNoallocMaxN (32): larger grids return MHD_EINVAL before any GPU work;
//   * the first call on a device looks up the device address of the array (cudaGetSymbolAddress),
//     uploads the twiddle tables into it and waits for the device (cudaDeviceSynchronize) so that
//     the tables are in place whatever stream the work is queued on; make that first call before
//     any stream capture;
//   * every call on a device shares the one array and it keeps the last call's contents: calls
//     that overlap on the GPU (different streams, or different host threads without ordering)
//     race.  The one region that must start at zero, the word the flux pass takes its atomic
//     CFL maximum on, is cleared by each call; every other pass overwrites what it later reads;
//   * work is queued on `stream` (NULL = legacy default stream), the physical parameters
//     included (a one-thread kernel takes them by value, so no host buffer is read after the
//     call returns); outputs are valid once the stream reaches the end of the call's work.
//     After the first call on a device the call does not synchronise the stream.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <vector>

#include "mhd.h"
#include "mhd_internal.h"

using mhd::cplx64;

namespace {

constexpr int kNoallocMaxN = 32;

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// Complex-value counts of the buffers for a grid of n points per axis (one instance).
struct Layout {
  size_t spec, s, r, w1, w2, part_doubles;
};
constexpr Layout layout_for(size_t n) {
  const size_t k = (n - 1) / 3, nx = k + 1, nk = 2 * k + 1;
  const size_t spec = nk * nk * nx;
  const size_t pairs = (n / 8) >= 16 ? 1 : 16 / (n / 8);
  Layout l{spec, 7 * spec, 7 * spec, 0, 0, 0};
  l.w1 = cmax(cmax(cmax(7 * n * nk * nx, 12 * n * n * nx), cmax(12 * spec, (7 * n * n * n + 1) / 2)),
              n * n * (n / 2 + 1));
  l.w2 = cmax(cmax(7 * n * n * nx, 12 * n * nk * nx), 7 * spec);
  l.part_doubles = cmax(n * n / (2 * pairs), n * n / (2 * pairs) * 8);
  return l;
}

constexpr Layout kL = layout_for(kNoallocMaxN);
constexpr size_t kOffS = 0;
constexpr size_t kOffR = kOffS + round256(kL.s * sizeof(cplx64));
constexpr size_t kOffW1 = kOffR + round256(kL.r * sizeof(cplx64));
constexpr size_t kOffW2 = kOffW1 + round256(kL.w1 * sizeof(cplx64));
constexpr size_t kOffPart = kOffW2 + round256(kL.w2 * sizeof(cplx64));
constexpr size_t kOffTw16 = kOffPart + round256(kL.part_doubles * sizeof(double));
constexpr size_t kOffTw32 = kOffTw16 + round256(mhd::fp64_twiddle_size(16));
constexpr size_t kOffPhys = kOffTw32 + round256(mhd::fp64_twiddle_size(32));
constexpr size_t kScratchBytes = kOffPhys + round256(sizeof(mhd::PhysDev));  // about 4.7 MB

}  // namespace

// The scratch array.  In host code its name is only a stand-in: the device address comes from
// cudaGetSymbolAddress in setup_device().
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
unsigned char *g_base[64] = {nullptr};


// Once per device, with that device current: resolve the array's device address and upload the
// twiddle tables (plain copies into the array; nothing is allocated).  A copy from pageable host
// memory may return before the data has reached the device, and the caller's stream need not be
// ordered after the legacy stream the copies use, so the device is synchronised before the
// address is published.
cudaError_t setup_device(unsigned char **base) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    unsigned char *b = static_cast<unsigned char *>(p);
    const std::vector<unsigned char> t16 = mhd::fp64_twiddle_bytes(16), t32 = mhd::fp64_twiddle_bytes(32);
    e = cudaMemcpy(b + kOffTw16, t16.data(), t16.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + kOffTw32, t32.data(), t32.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    g_base[dev] = b;
  }
  *base = g_base[dev];
  return cudaSuccess;
}

// The instance's parameters, written on the caller's stream from kernel arguments.
__global__ void set_phys_kernel(mhd::PhysDev *pd, double nu, double eta, double cs) {
  *pd = mhd::make_phys(nu, eta, cs);
}

}  // namespace

#define NA_CK(call)                                \
  do {                                             \
    if ((call) != cudaSuccess) return MHD_ECUDA;   \
  } while (0)

extern "C" MHD_API mhd_status mhd_rhs_noalloc(int32_t n, const mhd_phys *phys, const double *rho, const double *u,
                                              const double *b, double *drho, double *dm, double *db,
                                              void *stream) {
  if (n != 16 && n != kNoallocMaxN) return MHD_EINVAL;
  if (!phys || !rho || !u || !b || !drho || !dm || !db) return MHD_EINVAL;
  if (!(phys->nu >= 0.0) || !(phys->eta >= 0.0) || !(phys->cs > 0.0) || !isfinite(phys->nu) ||
      !isfinite(phys->eta) || !isfinite(phys->cs))
    return MHD_EINVAL;
  unsigned char *base = nullptr;
  NA_CK(setup_device(&base));
  cudaStream_t s = (cudaStream_t)stream;
  const mhd::Dims d = mhd::make_dims(n, 1);
  cplx64 *S = reinterpret_cast<cplx64 *>(base + kOffS);
  cplx64 *R = reinterpret_cast<cplx64 *>(base + kOffR);
  cplx64 *W1 = reinterpret_cast<cplx64 *>(base + kOffW1);
  cplx64 *W2 = reinterpret_cast<cplx64 *>(base + kOffW2);
  double *part = reinterpret_cast<double *>(base + kOffPart);
  const cplx64 *tw = reinterpret_cast<const cplx64 *>(base + (n == 16 ? kOffTw16 : kOffTw32));
  mhd::PhysDev *pd = reinterpret_cast<mhd::PhysDev *>(base + kOffPhys);
  set_phys_kernel<<<1, 1, 0, s>>>(pd, phys->nu, phys->eta, phys->cs);
  NA_CK(cudaGetLastError());
  // the flux pass takes an atomic maximum here (and screens against it): start from zero
  NA_CK(cudaMemsetAsync(part, 0, sizeof(unsigned long long), s));

  // state spectra from the real-space fields (m = rho u), truncated and normalised
  const size_t n3 = (size_t)n * n * n;
  NA_CK(mhd::launch_set_x(rho, u, b, W2, d, tw, s));
  NA_CK(mhd::launch_col_forward(W2, W1, n, 7 * n, d.nx, 1.0, tw, s));
  NA_CK(mhd::launch_col_forward(W1, S, n, 7, d.nk * d.nx, 1.0 / (double)n3, tw, s));
  // products on the grid and their truncated spectra
  NA_CK(mhd::launch_col_inverse(S, W1, n, 7, d.nk * d.nx, tw, s));
  NA_CK(mhd::launch_col_inverse(W1, W2, n, 7 * n, d.nx, tw, s));
  // the CFL maximum is not needed here; the partials region takes the atomic maxima
  NA_CK(mhd::launch_flux_x(W2, W1, pd, reinterpret_cast<unsigned long long *>(part), d, tw, s));
  NA_CK(mhd::launch_col_forward(W1, W2, n, 12 * n, d.nx, 1.0, tw, s));
  NA_CK(mhd::launch_col_forward(W2, W1, n, 12, d.nk * d.nx, 1.0, tw, s));
  // RHS spectra, then back to the grid
  NA_CK(mhd::launch_assemble(W1, S, S, nullptr, nullptr, R, pd, nullptr, mhd::ASM_RHS, 0, d, s));
  NA_CK(mhd::launch_col_inverse(R, W1, n, 7, d.nk * d.nx, tw, s));
  NA_CK(mhd::launch_col_inverse(W1, W2, n, 7 * n, d.nx, tw, s));
  double *real = reinterpret_cast<double *>(W1);
  NA_CK(mhd::launch_get_x(W2, real, 7, d, tw, s));
  NA_CK(cudaMemcpyAsync(drho, real, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  NA_CK(cudaMemcpyAsync(dm, real + n3, 3 * n3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  NA_CK(cudaMemcpyAsync(db, real + 4 * n3, 3 * n3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return MHD_OK;
}
