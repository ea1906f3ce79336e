// mhd_api.cu -- the C ABI (include/mhd.h): context, device memory, and the order of the passes.
//
// One time step of every instance (paper: pseudo-spectral RHS of section "Three dimensional
// numerical tests" and the Adams-Bashforth step of section "Code G-MHD3D") is six kernels:
//   1. inverse z   state S [b][7][kz'][ky'][kx]  -> W1 [b][7][z][ky'][kx]
//   2. inverse y   W1                            -> W2 [b][7][z][y][kx]
//   3. flux x      W2 (inverse x, 12 products, forward x; CFL partials) -> W1 [b][12][z][y][kx]
//   4. step size   CFL partials -> dt, AB2 coefficients, time advance (per instance)
//   5. forward y   W1 -> W2 [b][12][z][ky'][kx]
//   6. forward z   W2 -> W1 [b][12][kz'][ky'][kx]
//   7. assemble    W1 + S + H -> S (AB2 update), H (this step's RHS)
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "mhd.h"
#include "mhd_internal.h"

using mhd::cdf;
using mhd::cplx32;
using mhd::cplx64;

struct mhd_ctx {
  mhd_params p;
  mhd::Dims d;
  int device = 0;
  cudaStream_t stream = nullptr;
  double dt_fixed = 0.0, cfl_adv = 0.2, cfl_visc = 0.5;
  std::vector<mhd_phys> phys_host;
  std::vector<char> is_set;
  mhd::PhysDev *phys = nullptr;
  int precision = MHD_FP64;
  cplx64 *S = nullptr, *H = nullptr, *W1 = nullptr, *W2 = nullptr, *tw = nullptr;
  cplx32 *tw32 = nullptr;
  cdf *twdf = nullptr;    // double-float mode: W_N^m as double-float values
  cplx64 *S64 = nullptr;  // mixed and double-float modes: FP64 copy of one instance's state for set/get/diagnostics
  int integrator = MHD_AB2;
  void *Y = nullptr;      // stage state of RK4 / predictor-corrector ([b][7][spec], working precision)
  size_t w1_len = 0, w2_len = 0;  // bytes / 16
  double *part = nullptr;
  size_t part_len = 0;
  // CFL maxima as bits for atomic maxima: [0, batch) feed the step size, [batch, 2 batch) take the
  // maxima of evaluations whose step size is not needed (RK stages, mhd_rhs)
  unsigned long long *smax_bits = nullptr;
  int *d_err = nullptr;  // set by a device-side wait that gave up
  mhd::TimeState *ts = nullptr;
  mhd::StepCoef *coef = nullptr;
  double *diag_out = nullptr;
  int32_t *flag = nullptr;
  std::vector<void *> allocs;
  std::string err;
  // options and the captured step
  bool use_graph = true;
  bool flux_pipeline = false;
  uint32_t wait_polls = mhd::kWaitPolls;  // poll limit of the pipelined flux pass's copy waits
  bool persistent = false;    // column and flux passes as persistent work-queue kernels
  bool fuse = false;          // AB2 steps: assembly fused with the next step's inverse z pass
  int fuse_tile = 0;          // columns per block of the fused pass (0: default)
  // the fused steps' z buffer holds the inverse z pass of the state of the first z_nb instances
  // while no entry point has run since the step call numbered z_at
  uint64_t api_calls = 0;
  uint64_t z_at = 0;
  int z_nb = 0;
  unsigned *work_ctr = nullptr;  // two zeroed words per pass of the step (persistent kernels)
  bool forced = false;  // some instance has the ABC body force on
  // tracer particles: per instance a count and device data tr[6][count]; the grid magnetic field
  // the step's flux pass writes for them ([batch][3][N^3], working precision)
  std::vector<int64_t> ntr;
  std::vector<double *> tr;
  void *bgrid = nullptr;
  int tile[4] = {0, 0, 0, 0};
  int radix[4] = {0, 0, 0, 0};  // values per thread of the FP32 column passes (0: default)
  cudaStream_t cap_stream = nullptr;
  // host-pointer set/get: a copy stream and the events that hand staging slots between streams
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_full[8] = {}, ev_free[8] = {};
  // mhd_get_state_async: its own staging (allocated on first use, `ons` slots of `odz`
  // z-planes), copy stream and events, so that its device-to-host copies overlap whatever the
  // context queues next
  cudaStream_t out_stream = nullptr;
  cudaEvent_t ev_ofull[8] = {}, ev_ofree[8] = {}, ev_out_done = nullptr;
  double *oslots = nullptr;
  int odz = 0, ons = 0;
  // recorded on the stream at the end of every entry point but mhd_get_state_async (which leaves
  // W1 behind the y-pass output alone): a host set_state's copies into its W1 slots wait for it
  // only, not for a transfer out queued after it
  cudaEvent_t ev_slots = nullptr;
  bool slots_untouched = false;  // set by mhd_get_state_async for the guard's destructor
  cudaGraphExec_t graph_exec = nullptr;
  // serving pools: only the first `live` instances are stepped (-1: all), one graph per count
  int live = -1;
  std::vector<cudaGraphExec_t> pool_graphs;
  // profiling: events bracketing each launch of mhd_step, resolved at read time
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_marks;  // (kernel kind, index of the start event)
  double prof_ms[9] = {0};
  int64_t prof_count[9] = {0};
};

namespace {
const char *const kKernelNames[9] = {"inverse_z", "inverse_y", "flux_x", "step_dt", "forward_y", "forward_z",
                                     "assemble_ab2", "tracer_push", "assemble_iz"};
}

namespace {

mhd_status fail(mhd_ctx *c, mhd_status st, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return st;
}

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail(c, MHD_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                     \
  } while (0)

// Makes the context's device current for the duration of a call and restores the caller's.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  // every entry point that may touch a context's buffers counts itself here, and marks on its
  // stream where its use of the staging slots in W1 ends
  explicit DeviceGuard(mhd_ctx *c) : DeviceGuard(c->device) {
    ctx = c;
    ++c->api_calls;
  }
  ~DeviceGuard() {
    if (ctx) {
      // (the stream may be 0, the legacy default stream)
      if (!ctx->slots_untouched && ctx->ev_slots) cudaEventRecord(ctx->ev_slots, ctx->stream);
      ctx->slots_untouched = false;
    }
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  mhd_ctx *ctx = nullptr;
};

bool valid_n(int n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; }

// Buffer sizes in 16-byte units (one FP64 complex).  The step of all instances runs in the
// context's precision (8-byte complex values in the mixed mode); set/get/diagnostics and the
// inverse transform of an RHS run one instance at a time in FP64.
struct Sizes {
  size_t S, W1, W2, part;
};

Sizes sizes_for(const mhd::Dims &d, int precision) {
  const size_t n = d.n, nx = d.nx, nk = d.nk, b = d.batch;
  const size_t elem = precision == MHD_FP32_MIXED ? 8 : 16;
  Sizes s;
  s.S = b * 7 * d.spec;
  // step (all instances, working precision)
  size_t w1 = std::max(std::max(7 * n * nk * nx, 12 * n * n * nx), 12 * d.spec) * b * elem;
  // fused AB2 steps keep the inverse z output of the new state behind the 12 product spectra
  w1 = std::max(w1, (12 * d.spec + 7 * n * nk * nx) * b * elem);
  size_t w2 = std::max(7 * n * n * nx, 12 * n * nk * nx) * b * elem;
  // one instance in FP64
  w1 = std::max(w1, std::max(7 * n * nk * nx, 12 * n * n * nx) * 16);
  w1 = std::max(w1, 7 * n * n * n * 8);         // real 7 N^3 staging (set/get/rhs)
  w1 = std::max(w1, n * n * (n / 2 + 1) * 16);  // expanded spectrum
  w2 = std::max(w2, std::max(7 * n * n * nx, 12 * n * nk * nx) * 16);
  w2 = std::max(w2, 7 * d.spec * 16);            // RHS spectra of one instance
  s.W1 = (w1 + 15) / 16;
  s.W2 = (w2 + 15) / 16;
  s.part = std::max((size_t)b * mhd::flux_x_blocks_per_instance(d.n), (size_t)mhd::diag_x_blocks(d.n) * 8);
  return s;
}

size_t footprint(const mhd::Dims &d, int precision) {
  const Sizes s = sizes_for(d, precision);
  return (2 * s.S + s.W1 + s.W2) * sizeof(cplx64) + mhd::fp64_twiddle_size(d.n) + d.n * sizeof(cplx32) +
         (precision == MHD_FP64_DF ? d.n * sizeof(cdf) : 0) +
         s.part * sizeof(double) +
         (precision == MHD_FP64 ? 0 : 7 * d.spec * sizeof(cplx64)) +
         d.batch * (sizeof(mhd::TimeState) + sizeof(mhd::StepCoef) + sizeof(mhd::PhysDev)) +
         (64 + mhd::kDivbBlocks) * sizeof(double);
}

void *dalloc(mhd_ctx *c, size_t bytes) {
  void *p = nullptr;
  if (c->p.dev_alloc) {
    p = c->p.dev_alloc(bytes, c->p.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->allocs.push_back(p);
  return p;
}

void dfree(mhd_ctx *c, void *p) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i] == p) {
      c->allocs.erase(c->allocs.begin() + i);
      break;
    }
  if (c->p.dev_free) c->p.dev_free(p, c->p.alloc_user);
  else cudaFree(p);
}

void free_all(mhd_ctx *c) {
  for (void *p : c->allocs) {
    if (c->p.dev_free) c->p.dev_free(p, c->p.alloc_user);
    else cudaFree(p);
  }
  c->allocs.clear();
}

mhd_status check_inst(mhd_ctx *c, int inst) {
  if (!c) return MHD_EINVAL;
  if (inst < 0 || inst >= c->d.batch) return fail(c, MHD_EINVAL, "instance %d out of range [0, %d)", inst, c->d.batch);
  return MHD_OK;
}

mhd::Dims one(const mhd_ctx *c) {
  mhd::Dims d = c->d;
  d.batch = 1;
  return d;
}

// State of instance `inst`.  FP64: S is [b][7][spec] complex doubles.  Mixed: the same bytes hold
// S_hi [b][7][spec] then S_lo [b][7][spec] (FP32 complex), and H holds [b][7][spec] FP32 complex.
cplx64 *state64(mhd_ctx *c, int inst) { return c->S + (size_t)inst * 7 * c->d.spec; }
cplx32 *state_hi(mhd_ctx *c, int inst) { return reinterpret_cast<cplx32 *>(c->S) + (size_t)inst * 7 * c->d.spec; }
cplx32 *state_lo(mhd_ctx *c, int inst) {
  return reinterpret_cast<cplx32 *>(c->S) + ((size_t)c->d.batch + inst) * 7 * c->d.spec;
}
cplx32 *hist32(mhd_ctx *c, int inst) { return reinterpret_cast<cplx32 *>(c->H) + (size_t)inst * 7 * c->d.spec; }
// Double-float mode: S, H (and the stage state) hold [b][7][spec] double-float complex values, the
// same bytes per value as FP64.
cdf *statedf(mhd_ctx *c, int inst) { return reinterpret_cast<cdf *>(c->S) + (size_t)inst * 7 * c->d.spec; }
cdf *histdf(mhd_ctx *c, int inst) { return reinterpret_cast<cdf *>(c->H) + (size_t)inst * 7 * c->d.spec; }

bool valid_precision(int p) { return p == MHD_FP64 || p == MHD_FP32_MIXED || p == MHD_FP64_DF; }

void drop_graphs(mhd_ctx *c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  for (auto &g : c->pool_graphs) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

// FP64 spectra of instance `inst` for the FP64 utility chains (the mixed state is combined first).
mhd_status state_fp64(mhd_ctx *c, int inst, const cplx64 **out) {
  if (c->precision == MHD_FP64) {
    *out = state64(c, inst);
    return MHD_OK;
  }
  if (c->precision == MHD_FP64_DF)
    CK(mhd::launch_combine_state(statedf(c, inst), c->S64, 7 * c->d.spec, c->stream));
  else
    CK(mhd::launch_combine_state(state_hi(c, inst), state_lo(c, inst), c->S64, 7 * c->d.spec, c->stream));
  *out = c->S64;
  return MHD_OK;
}

// inverse z then inverse y of 7 fields of one instance: S-layout `src` -> W2 [7][z][y][kx]
mhd_status inverse_zy(mhd_ctx *c, const cplx64 *src) {
  const mhd::Dims &d = c->d;
  CK(mhd::launch_col_inverse(src, c->W1, d.n, 7, d.nk * d.nx, c->tw, c->stream));
  CK(mhd::launch_col_inverse(c->W1, c->W2, d.n, 7 * d.n, d.nx, c->tw, c->stream));
  return MHD_OK;
}

mhd_status copy_out(mhd_ctx *c, void *dst, const void *src, size_t bytes, int on_device) {
  CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return MHD_OK;
}

// Inverse-transform 7 truncated spectra (S layout) of one instance into real rho/m/B outputs.
mhd_status spectra_to_real(mhd_ctx *c, const cplx64 *src, double *a, double *b3, double *c3, int on_device) {
  const size_t n3 = (size_t)c->d.n * c->d.n * c->d.n;
  mhd_status st = inverse_zy(c, src);
  if (st) return st;
  double *real = reinterpret_cast<double *>(c->W1);
  CK(mhd::launch_get_x(c->W2, real, 7, one(c), c->tw, c->stream));
  if ((st = copy_out(c, a, real, n3 * sizeof(double), on_device))) return st;
  if ((st = copy_out(c, b3, real + n3, 3 * n3 * sizeof(double), on_device))) return st;
  if ((st = copy_out(c, c3, real + 4 * n3, 3 * n3 * sizeof(double), on_device))) return st;
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

}  // namespace

extern "C" {

size_t mhd_footprint_bytes(int32_t n, int32_t precision, int32_t batch) {
  if (!valid_n(n) || batch < 1 || !valid_precision(precision)) return 0;
  return footprint(mhd::make_dims(n, batch), precision);
}

const char *mhd_last_error(const mhd_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void mhd_destroy(mhd_ctx *ctx) {
  if (!ctx) return;
  {
    DeviceGuard g(ctx);
    g.ctx = nullptr;  // no mark: the context goes
    cudaStreamSynchronize(ctx->stream);  // 0 is the legacy default stream
    if (ctx->out_stream) cudaStreamSynchronize(ctx->out_stream);  // copies into the caller's buffers
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    drop_graphs(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->out_stream) cudaStreamDestroy(ctx->out_stream);
    for (cudaEvent_t e : {ctx->ev_out_done, ctx->ev_slots})
      if (e) cudaEventDestroy(e);
    for (int i = 0; i < 8; ++i) {
      if (ctx->ev_full[i]) cudaEventDestroy(ctx->ev_full[i]);
      if (ctx->ev_free[i]) cudaEventDestroy(ctx->ev_free[i]);
      if (ctx->ev_ofull[i]) cudaEventDestroy(ctx->ev_ofull[i]);
      if (ctx->ev_ofree[i]) cudaEventDestroy(ctx->ev_ofree[i]);
    }
    free_all(ctx);
  }
  delete ctx;
}

mhd_status mhd_init(const mhd_params *p, const mhd_phys *phys, mhd_ctx **out) {
  if (!out) return MHD_EINVAL;
  *out = nullptr;
  if (!p || !phys) return MHD_EINVAL;
  if (!valid_n(p->n) || p->batch < 1) return MHD_EINVAL;
  if (p->integrator < MHD_AB2 || p->integrator > MHD_PC) return MHD_EINVAL;
  if (!valid_precision(p->precision)) return MHD_EINVAL;
  if ((p->dev_alloc == nullptr) != (p->dev_free == nullptr)) return MHD_EINVAL;
  for (int i = 0; i < p->batch; ++i) {
    if (!(phys[i].nu >= 0.0) || !(phys[i].eta >= 0.0) || !(phys[i].cs > 0.0) || !isfinite(phys[i].nu) ||
        !isfinite(phys[i].eta) || !isfinite(phys[i].cs))
      return MHD_EINVAL;
  }
  if (!(isfinite(p->dt))) return MHD_EINVAL;
  mhd_ctx *c = new (std::nothrow) mhd_ctx;
  if (!c) return MHD_ENOMEM;
  c->p = *p;
  c->d = mhd::make_dims(p->n, p->batch);
  c->precision = p->precision;
  c->integrator = p->integrator;
  c->stream = (cudaStream_t)p->stream;
  c->dt_fixed = p->dt > 0.0 ? p->dt : 0.0;
  c->cfl_adv = p->cfl_adv > 0.0 ? p->cfl_adv : 0.2;
  c->cfl_visc = p->cfl_visc > 0.0 ? p->cfl_visc : 0.5;
  c->phys_host.assign(phys, phys + p->batch);
  c->is_set.assign(p->batch, 0);
  c->ntr.assign(p->batch, 0);
  c->tr.assign(p->batch, nullptr);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return MHD_ECUDA;
  }
  const Sizes s = sizes_for(c->d, c->precision);
  c->w1_len = s.W1;
  c->w2_len = s.W2;
  c->part_len = s.part;
  bool ok = (c->S = (cplx64 *)dalloc(c, s.S * sizeof(cplx64))) != nullptr;
  ok = ok && (c->H = (cplx64 *)dalloc(c, s.S * sizeof(cplx64))) != nullptr;
  ok = ok && (c->W1 = (cplx64 *)dalloc(c, s.W1 * sizeof(cplx64))) != nullptr;
  ok = ok && (c->W2 = (cplx64 *)dalloc(c, s.W2 * sizeof(cplx64))) != nullptr;
  ok = ok && (c->tw = (cplx64 *)dalloc(c, mhd::fp64_twiddle_size(c->d.n))) != nullptr;
  ok = ok && (c->tw32 = (cplx32 *)dalloc(c, (size_t)c->d.n * sizeof(cplx32))) != nullptr;
  if (c->precision != MHD_FP64) ok = ok && (c->S64 = (cplx64 *)dalloc(c, 7 * c->d.spec * sizeof(cplx64))) != nullptr;
  if (c->precision == MHD_FP64_DF) ok = ok && (c->twdf = (cdf *)dalloc(c, (size_t)c->d.n * sizeof(cdf))) != nullptr;
  if (c->integrator != MHD_AB2)
    ok = ok && (c->Y = dalloc(c, s.S * (c->precision == MHD_FP32_MIXED ? sizeof(cplx32) : sizeof(cplx64)))) != nullptr;
  ok = ok && (c->part = (double *)dalloc(c, s.part * sizeof(double))) != nullptr;
  ok = ok && (c->smax_bits = (unsigned long long *)dalloc(c, 2 * p->batch * sizeof(unsigned long long))) != nullptr;
  ok = ok && (c->d_err = (int *)dalloc(c, 4 * sizeof(int))) != nullptr;
  ok = ok && (c->work_ctr = (unsigned *)dalloc(c, 16 * sizeof(unsigned))) != nullptr;
  ok = ok && (c->ts = (mhd::TimeState *)dalloc(c, p->batch * sizeof(mhd::TimeState))) != nullptr;
  ok = ok && (c->coef = (mhd::StepCoef *)dalloc(c, p->batch * sizeof(mhd::StepCoef))) != nullptr;
  ok = ok && (c->phys = (mhd::PhysDev *)dalloc(c, p->batch * sizeof(mhd::PhysDev))) != nullptr;
  ok = ok && (c->diag_out = (double *)dalloc(c, (32 + mhd::kDivbBlocks) * sizeof(double))) != nullptr;
  ok = ok && (c->flag = (int32_t *)dalloc(c, 4 * sizeof(int32_t))) != nullptr;
  if (!ok) {
    free_all(c);
    delete c;
    return MHD_ENOMEM;
  }
  std::vector<mhd::PhysDev> pd(p->batch);
  for (int i = 0; i < p->batch; ++i) pd[i] = mhd::make_phys(phys[i].nu, phys[i].eta, phys[i].cs);
  const std::vector<cplx64> w = mhd::twiddle_table(c->d.n);
  const std::vector<unsigned char> w64 = mhd::fp64_twiddle_bytes(c->d.n);
  std::vector<cplx32> w32(w.size());
  for (size_t i = 0; i < w.size(); ++i) w32[i] = cplx32{(float)w[i].re, (float)w[i].im};
  std::vector<cdf> wdf(w.size());
  for (size_t i = 0; i < w.size(); ++i) wdf[i] = cdf{mhd::dfr_const(w[i].re), mhd::dfr_const(w[i].im)};
  cudaError_t e = cudaMemcpyAsync(c->phys, pd.data(), pd.size() * sizeof(mhd::PhysDev), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->tw, w64.data(), w64.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->tw32, w32.data(), w32.size() * sizeof(cplx32), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && c->twdf)
    e = cudaMemcpyAsync(c->twdf, wdf.data(), wdf.size() * sizeof(cdf), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->S, 0, s.S * sizeof(cplx64), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->H, 0, s.S * sizeof(cplx64), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ts, 0, p->batch * sizeof(mhd::TimeState), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->smax_bits, 0, 2 * p->batch * sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, 4 * sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->work_ctr, 0, 16 * sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_slots, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_slots, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    if (c->ev_slots) cudaEventDestroy(c->ev_slots);
    free_all(c);
    delete c;
    return MHD_ECUDA;
  }
  *out = c;
  return MHD_OK;
}

}  // extern "C"

// ---- host-pointer transfers, pipelined over slabs of z-planes ----
// The 7 real fields of one instance cross the host link slab by slab on a second stream while the
// context's stream transforms the slab before (x and y passes); the staging slots (2 to 8) live
// in W1 behind the y-pass output, so nothing is allocated.
namespace {

struct SlabPlan {
  int dz;           // z-planes per slab
  int ns;           // slots, 2..8, used in turn
  double *slot[8];  // 7 fields x dz N^2 doubles each
};

// As many slots of N/8 z-planes as W1 holds behind the y-pass output, up to one per slab (so
// that a transfer in can run ahead of the transforms); thinner slabs when not even two fit.
bool slab_plan(mhd_ctx *c, SlabPlan *pl) {
  const mhd::Dims &d = c->d;
  const size_t n = d.n, nn = n * n;
  const size_t head = (7 * n * d.nk * d.nx + 15) / 16 * 16;  // y-pass output, complex values
  if (head >= c->w1_len) return false;
  const size_t avail = (c->w1_len - head) * 2;  // doubles
  int dz = (int)(n / 8);
  while (dz > 1 && (size_t)14 * dz * nn > avail) dz /= 2;
  if ((size_t)14 * dz * nn > avail) return false;
  int ns = (int)std::min<size_t>(avail / ((size_t)7 * dz * nn), (size_t)8);
  ns = std::min(ns, (int)((n + dz - 1) / dz));
  if (ns < 2) ns = 2;
  pl->dz = dz;
  pl->ns = ns;
  for (int k = 0; k < ns; ++k)
    pl->slot[k] = reinterpret_cast<double *>(c->W1 + head) + (size_t)7 * k * dz * nn;
  return true;
}

mhd_status ensure_copy_stream(mhd_ctx *c) {
  if (c->copy_stream) return MHD_OK;
  CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  for (int i = 0; i < 8; ++i) {
    CK(cudaEventCreateWithFlags(&c->ev_full[i], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_free[i], cudaEventDisableTiming));
  }
  return MHD_OK;
}

// Host rho, u, B -> truncated spectra `Si` (FP64) of one instance.  Returns MHD_EINVAL without
// queueing anything when no staging plan fits (the caller then takes the unpipelined path).
// C = cplx64: FP64 transforms into FP64 spectra; C = cdf: double-float transforms into the
// double-float state (the values are split at the x pass).
template <typename C>
mhd_status set_state_host(mhd_ctx *c, const double *rho, const double *u, const double *b, C *Si, const C *tw) {
  SlabPlan pl;
  if (!slab_plan(c, &pl)) return MHD_EINVAL;
  mhd_status st = ensure_copy_stream(c);
  if (st) return st;
  const mhd::Dims &d = c->d;
  const mhd::Dims d1 = one(c);
  const int n = d.n;
  const size_t nn = (size_t)n * n, n3 = nn * n;
  // the staging slots are free once the last entry point that used W1 there has finished; a
  // transfer out queued since (mhd_get_state_async) does not hold the copies in
  cudaError_t e = cudaStreamWaitEvent(c->copy_stream, c->ev_slots, 0);
  int i = 0;
  for (int z0 = 0; z0 < n && e == cudaSuccess; z0 += pl.dz, ++i) {
    const int dzc = std::min(pl.dz, n - z0), k = i % pl.ns;
    double *slot = pl.slot[k];
    const size_t off = (size_t)z0 * nn, cnt = (size_t)dzc * nn;
    if (i >= pl.ns) e = cudaStreamWaitEvent(c->copy_stream, c->ev_free[k], 0);
    for (int f = 0; f < 7 && e == cudaSuccess; ++f) {
      const double *src = f == 0 ? rho + off : f < 4 ? u + (f - 1) * n3 + off : b + (f - 4) * n3 + off;
      e = cudaMemcpyAsync(slot + f * cnt, src, cnt * sizeof(double), cudaMemcpyHostToDevice, c->copy_stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_full[k], c->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_full[k], 0);
    C *w1 = reinterpret_cast<C *>(c->W1), *w2 = reinterpret_cast<C *>(c->W2);
    if (e == cudaSuccess)
      e = mhd::launch_set_x_rows(slot, slot + cnt, slot + 4 * cnt, w2, d1, tw, c->stream, (size_t)z0 * n,
                                 (size_t)dzc * n, cnt);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_free[k], c->stream);
    for (int f = 0; f < 7 && e == cudaSuccess; ++f) {
      const size_t slab0 = (size_t)f * n + z0;  // y pass of these z-planes
      e = mhd::launch_col_forward(w2 + slab0 * n * d.nx, w1 + slab0 * d.nk * d.nx, n, dzc, d.nx, 1.0, tw,
                                  c->stream);
    }
  }
  if (e == cudaSuccess)
    e = mhd::launch_col_forward(reinterpret_cast<C *>(c->W1), Si, n, 7, d.nk * d.nx, 1.0 / (double)n3, tw, c->stream);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(c->copy_stream);  // the host buffers must outlive the copies in flight
    return fail(c, MHD_ECUDA, "set_state: %s", cudaGetErrorString(e));
  }
  return MHD_OK;
}

// Staging of a device-to-host transfer: two slots of 7 x dz N^2 doubles, the stream that copies
// out of them and the events that hand them between that stream and the context's stream.
struct Staging {
  int dz;
  int ns;  // slots, 2..8, used in turn
  double *slot[8];
  cudaStream_t cs;
  cudaEvent_t *full, *free;
};

// The staging of mhd_get_state_async, allocated on first use: slots of N/8 z-planes, as many as
// there are slabs (8: the whole state, so that the transforms never wait for the copies out) when
// that takes at most half the context's footprint (it takes about 36 % at every N), else fewer (at
// least 2, then thinner slabs).
mhd_status async_staging(mhd_ctx *c, Staging *sg) {
  const size_t n = c->d.n, nn = n * n;
  if (!c->out_stream) {
    CK(cudaStreamCreateWithFlags(&c->out_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 8; ++i) {
      CK(cudaEventCreateWithFlags(&c->ev_ofull[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&c->ev_ofree[i], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&c->ev_out_done, cudaEventDisableTiming));
  }
  if (!c->oslots) {
    const size_t cap = footprint(c->d, c->precision) / 2;
    int dz = (int)(n / 8), ns = 8;
    while (ns > 2 && (size_t)7 * ns * dz * nn * sizeof(double) > cap) --ns;
    while (dz > 1 && (size_t)7 * ns * dz * nn * sizeof(double) > cap) dz /= 2;
    const size_t bytes = (size_t)7 * ns * dz * nn * sizeof(double);
    c->oslots = static_cast<double *>(dalloc(c, bytes));
    if (!c->oslots) return fail(c, MHD_ENOMEM, "get_state_async: staging of %zu bytes", bytes);
    c->odz = dz;
    c->ons = ns;
  }
  sg->dz = c->odz;
  sg->ns = c->ons;
  for (int k = 0; k < c->ons; ++k) sg->slot[k] = c->oslots + (size_t)7 * k * c->odz * nn;
  sg->cs = c->out_stream;
  sg->full = c->ev_ofull;
  sg->free = c->ev_ofree;
  return MHD_OK;
}

// Truncated spectra `src` of one instance -> host rho, m, B through the staging `sg`.  `wait`:
// return once the copies have landed; otherwise the copies are still in flight on sg.cs when it
// returns (ev_out_done marks their end).
template <typename C>
mhd_status get_state_staged(mhd_ctx *c, const C *src, const C *tw, double *rho, double *m, double *b,
                            const Staging &sg, bool wait) {
  const mhd::Dims &d = c->d;
  const mhd::Dims d1 = one(c);
  const int n = d.n;
  const size_t nn = (size_t)n * n, n3 = nn * n;
  C *w1 = reinterpret_cast<C *>(c->W1), *w2 = reinterpret_cast<C *>(c->W2);
  cudaError_t e = cudaSuccess;
  // the slots' previous copies (an earlier asynchronous get) end before they are written again
  if (!wait && c->ev_out_done) e = cudaStreamWaitEvent(c->stream, c->ev_out_done, 0);
  if (e == cudaSuccess) e = mhd::launch_col_inverse(src, w1, n, 7, d.nk * d.nx, tw, c->stream);  // z pass
  int i = 0;
  for (int z0 = 0; z0 < n && e == cudaSuccess; z0 += sg.dz, ++i) {
    const int dzc = std::min(sg.dz, n - z0), k = i % sg.ns;
    double *slot = sg.slot[k];
    const size_t off = (size_t)z0 * nn, cnt = (size_t)dzc * nn;
    if (i >= sg.ns) e = cudaStreamWaitEvent(c->stream, sg.free[k], 0);  // slot copied out
    for (int f = 0; f < 7 && e == cudaSuccess; ++f) {
      const size_t slab0 = (size_t)f * n + z0;  // y pass of these z-planes
      e = mhd::launch_col_inverse(w1 + slab0 * d.nk * d.nx, w2 + slab0 * n * d.nx, n, dzc, d.nx, tw, c->stream);
    }
    if (e == cudaSuccess)
      e = mhd::launch_get_x_rows(w2, slot, 7, d1, tw, c->stream, (size_t)z0 * n, (size_t)dzc * n, cnt);
    if (e == cudaSuccess) e = cudaEventRecord(sg.full[k], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sg.cs, sg.full[k], 0);
    for (int f = 0; f < 7 && e == cudaSuccess; ++f) {
      double *dst = f == 0 ? rho + off : f < 4 ? m + (f - 1) * n3 + off : b + (f - 4) * n3 + off;
      e = cudaMemcpyAsync(dst, slot + f * cnt, cnt * sizeof(double), cudaMemcpyDeviceToHost, sg.cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sg.free[k], sg.cs);
  }
  if (!wait) {
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_out_done, sg.cs);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(sg.cs);
      return fail(c, MHD_ECUDA, "get_state_async: %s", cudaGetErrorString(e));
    }
    return MHD_OK;
  }
  const cudaError_t e2 = cudaStreamSynchronize(sg.cs);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, MHD_ECUDA, "get_state: %s", cudaGetErrorString(e));
  return MHD_OK;
}

// Truncated spectra `src` of one instance -> host rho, m, B through the staging slots in W1.
// MHD_EINVAL (nothing queued) when no staging plan fits.
template <typename C>
mhd_status get_state_host(mhd_ctx *c, const C *src, const C *tw, double *rho, double *m, double *b) {
  SlabPlan pl;
  if (!slab_plan(c, &pl)) return MHD_EINVAL;
  mhd_status st = ensure_copy_stream(c);
  if (st) return st;
  if (c->out_stream) CK(cudaStreamSynchronize(c->out_stream));  // an earlier asynchronous get
  // two slots: more measured slower for the synchronous transfer out
  const Staging sg = {pl.dz, 2, {pl.slot[0], pl.slot[1]}, c->copy_stream, c->ev_full, c->ev_free};
  return get_state_staged(c, src, tw, rho, m, b, sg, true);
}

}  // namespace

extern "C" {

mhd_status mhd_set_state(mhd_ctx *c, int32_t inst, const double *rho, const double *u, const double *b,
                         int32_t on_device) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (!rho || !u || !b) return fail(c, MHD_EINVAL, "null input");
  DeviceGuard g(c);
  const mhd::Dims &d = c->d;
  const size_t n3 = (size_t)d.n * d.n * d.n;
  const bool fp64 = c->precision == MHD_FP64;
  const bool dfl = c->precision == MHD_FP64_DF;
  cplx64 *Si = fp64 ? state64(c, inst) : c->S64;
  if (dfl) {
    // double-float transforms straight into the double-float state; device inputs go through the
    // same row kernels over all rows
    cdf *Sd = statedf(c, inst);
    if (on_device || (st = set_state_host(c, rho, u, b, Sd, c->twdf)) == MHD_EINVAL) {
      const double *r = rho, *uu = u, *bb = b;
      if (!on_device) {
        double *real = reinterpret_cast<double *>(c->W1);
        CK(cudaMemcpyAsync(real, rho, n3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(real + n3, u, 3 * n3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(real + 4 * n3, b, 3 * n3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        r = real;
        uu = real + n3;
        bb = real + 4 * n3;
      }
      cdf *w1 = reinterpret_cast<cdf *>(c->W1), *w2 = reinterpret_cast<cdf *>(c->W2);
      CK(mhd::launch_set_x_rows(r, uu, bb, w2, one(c), c->twdf, c->stream, 0, (size_t)d.n * d.n, n3));
      CK(mhd::launch_col_forward(w2, w1, d.n, 7 * d.n, d.nx, 1.0, c->twdf, c->stream));
      CK(mhd::launch_col_forward(w1, Sd, d.n, 7, d.nk * d.nx, 1.0 / ((double)n3), c->twdf, c->stream));
    } else if (st) {
      return st;
    }
  } else if (!on_device && (st = set_state_host(c, rho, u, b, Si, c->tw)) != MHD_EINVAL) {
    if (st) return st;
  } else {
    const double *r = rho, *uu = u, *bb = b;
    if (!on_device) {
      double *real = reinterpret_cast<double *>(c->W1);
      CK(cudaMemcpyAsync(real, rho, n3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      CK(cudaMemcpyAsync(real + n3, u, 3 * n3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      CK(cudaMemcpyAsync(real + 4 * n3, b, 3 * n3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      r = real;
      uu = real + n3;
      bb = real + 4 * n3;
    }
    CK(mhd::launch_set_x(r, uu, bb, c->W2, one(c), c->tw, c->stream));
    CK(mhd::launch_col_forward(c->W2, c->W1, d.n, 7 * d.n, d.nx, 1.0, c->tw, c->stream));
    CK(mhd::launch_col_forward(c->W1, Si, d.n, 7, d.nk * d.nx, 1.0 / ((double)n3), c->tw, c->stream));
  }
  if (fp64) {
    CK(cudaMemsetAsync(c->H + (size_t)inst * 7 * d.spec, 0, 7 * d.spec * sizeof(cplx64), c->stream));
  } else if (dfl) {
    CK(cudaMemsetAsync(histdf(c, inst), 0, 7 * d.spec * sizeof(cdf), c->stream));
  } else {
    CK(mhd::launch_split_state(c->S64, state_hi(c, inst), state_lo(c, inst), 7 * d.spec, c->stream));
    CK(cudaMemsetAsync(hist32(c, inst), 0, 7 * d.spec * sizeof(cplx32), c->stream));
  }
  CK(cudaMemsetAsync(c->ts + inst, 0, sizeof(mhd::TimeState), c->stream));
  CK(cudaMemsetAsync(c->smax_bits + inst, 0, sizeof(unsigned long long), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->is_set[inst] = 1;
  return MHD_OK;
}

mhd_status mhd_get_state(mhd_ctx *c, int32_t inst, double *rho, double *m, double *b, int32_t on_device) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (!rho || !m || !b) return fail(c, MHD_EINVAL, "null output");
  DeviceGuard g(c);
  if (c->precision == MHD_FP64_DF) {
    // double-float transforms straight from the double-float state
    const cdf *Sd = statedf(c, inst);
    if (!on_device && (st = get_state_host(c, Sd, c->twdf, rho, m, b)) != MHD_EINVAL) return st;
    const mhd::Dims &d = c->d;
    const size_t n3 = (size_t)d.n * d.n * d.n;
    cdf *w1 = reinterpret_cast<cdf *>(c->W1), *w2 = reinterpret_cast<cdf *>(c->W2);
    CK(mhd::launch_col_inverse(Sd, w1, d.n, 7, d.nk * d.nx, c->twdf, c->stream));
    CK(mhd::launch_col_inverse(w1, w2, d.n, 7 * d.n, d.nx, c->twdf, c->stream));
    double *real = reinterpret_cast<double *>(c->W1);
    CK(mhd::launch_get_x_rows(w2, real, 7, one(c), c->twdf, c->stream, 0, (size_t)d.n * d.n, n3));
    if ((st = copy_out(c, rho, real, n3 * sizeof(double), on_device))) return st;
    if ((st = copy_out(c, m, real + n3, 3 * n3 * sizeof(double), on_device))) return st;
    if ((st = copy_out(c, b, real + 4 * n3, 3 * n3 * sizeof(double), on_device))) return st;
    CK(cudaStreamSynchronize(c->stream));
    return MHD_OK;
  }
  const cplx64 *src = nullptr;
  if ((st = state_fp64(c, inst, &src))) return st;
  if (!on_device && (st = get_state_host(c, src, c->tw, rho, m, b)) != MHD_EINVAL) return st;
  return spectra_to_real(c, src, rho, m, b, on_device);
}

mhd_status mhd_get_state_async(mhd_ctx *c, int32_t inst, double *rho, double *m, double *b) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (!rho || !m || !b) return fail(c, MHD_EINVAL, "null output");
  DeviceGuard g(c);
  c->slots_untouched = true;  // this transfer leaves W1 behind the y-pass output alone
  Staging sg;
  if ((st = async_staging(c, &sg))) return st;
  if (c->precision == MHD_FP64_DF) return get_state_staged(c, statedf(c, inst), c->twdf, rho, m, b, sg, false);
  const cplx64 *src = nullptr;
  if ((st = state_fp64(c, inst, &src))) return st;
  return get_state_staged(c, src, c->tw, rho, m, b, sg, false);
}

mhd_status mhd_get_spectrum(mhd_ctx *c, int32_t inst, int32_t field, double *out, int32_t on_device) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (field < 0 || field >= 7 || !out) return fail(c, MHD_EINVAL, "bad field or null output");
  DeviceGuard g(c);
  const mhd::Dims &d = c->d;
  const size_t full = (size_t)d.n * d.n * (d.n / 2 + 1);
  const cplx64 *src = nullptr;
  if ((st = state_fp64(c, inst, &src))) return st;
  CK(mhd::launch_expand_spectrum(src + (size_t)field * d.spec, c->W1, d, c->stream));
  if ((st = copy_out(c, out, c->W1, full * sizeof(cplx64), on_device))) return st;
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

}  // extern "C"

// Event marks around the launches of mhd_step while profiling is on.
static cudaError_t prof_begin(mhd_ctx *c, int kind, bool on) {
  if (!on) return cudaSuccess;
  if (c->ev_used + 2 > c->ev_pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      c->ev_pool.push_back(e);
    }
  }
  c->ev_marks.push_back({kind, c->ev_used});
  cudaError_t err = cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
  c->ev_used += 2;
  return err;
}

static cudaError_t prof_end(mhd_ctx *c, bool on) {
  if (!on) return cudaSuccess;
  return cudaEventRecord(c->ev_pool[c->ev_marks.back().second + 1], c->stream);
}

#define LAUNCH(kind, call)                     \
  do {                                         \
    CK(prof_begin(c, kind, prof));             \
    CK(call);                                  \
    CK(prof_end(c, prof));                     \
  } while (0)

// Steps 1-6 of the pass order for the instances in `d` starting at state `S`; leaves the 12
// product spectra in W1.
// CF: complex type of the passes (cplx64 or cplx32); `tw` the matching twiddle table.  `advance`
// runs the step-size kernel after the flux pass.
// `bgrid` (nullable) receives the grid magnetic field for the tracers.
// `z_in` (nullable): the inverse z pass of S is already there (a fused step wrote it); step 1 is
// skipped and the inverse y pass reads it.
template <typename CF, typename CS>
static mhd_status flux_spectra_t(mhd_ctx *c, const mhd::Dims &d, int inst0, const CS *S, const mhd::PhysDev *phys,
                                 mhd::TimeState *ts, mhd::StepCoef *coef, bool advance, const CF *tw,
                                 typename mhd::grid_of<CF>::type *bgrid, const CF *z_in = nullptr) {
  const int b = d.batch;
  const bool prof = advance && c->profiling;
  CF *w1 = reinterpret_cast<CF *>(c->W1);
  CF *w2 = reinterpret_cast<CF *>(c->W2);
  unsigned *ctr = c->persistent ? c->work_ctr : nullptr;  // two words per pass: 0, 2, 4, 6, 8
  auto wc = [&](int pass) { return ctr ? ctr + 2 * pass : nullptr; };
  if (!z_in)
    LAUNCH(0, mhd::launch_col_inverse(S, w1, d.n, b * 7, d.nk * d.nx, tw, c->stream, c->tile[0], c->radix[0], wc(0)));
  LAUNCH(1, mhd::launch_col_inverse(z_in ? z_in : w1, w2, d.n, b * 7 * d.n, d.nx, tw, c->stream, c->tile[1],
                                    c->radix[1], wc(1)));
  // The CFL maximum of an advancing pass goes to the first slot (zero at the pass's start: the
  // dt kernel resets it after reading).  Evaluations that take no step (later RK stages, the
  // corrector, mhd_rhs) write to a second slot that nothing reads; its maxima are not exact
  // (the flux pass screens against the slot's earlier content), which changes no result.
  unsigned long long *bits = c->smax_bits + (advance ? 0 : c->d.batch) + inst0;
  LAUNCH(2, mhd::launch_flux_x(w2, w1, phys, bits, d, tw, c->stream, c->flux_pipeline ? c->d_err : nullptr, bgrid,
                               c->wait_polls, wc(2)));
  if (advance) {
    LAUNCH(3, mhd::launch_step_dt(bits, phys, ts, coef, d, c->dt_fixed, c->cfl_adv, c->cfl_visc, c->stream));
  }
  LAUNCH(4, mhd::launch_col_forward(w1, w2, d.n, b * 12 * d.n, d.nx, 1.0, tw, c->stream, c->tile[2], c->radix[2],
                                    wc(3)));
  LAUNCH(5, mhd::launch_col_forward(w2, w1, d.n, b * 12, d.nk * d.nx, 1.0, tw, c->stream, c->tile[3], c->radix[3],
                                    wc(4)));
  return MHD_OK;
}

// Fused AB2 steps: the assembly kernel also runs the next step's inverse z pass of the new state;
// its output (z layout [b][7][N][nk nx]) lives in W1 behind the 12 product spectra, which the step
// overwrites only after the inverse y pass has read it.  A step sequence starts with a plain
// inverse z pass into the same place (fused_prologue).
static bool fused_ab2(const mhd_ctx *c) { return c->fuse && c->integrator == MHD_AB2; }

template <typename C>
static C *zbuf(mhd_ctx *c, const mhd::Dims &d) {
  return reinterpret_cast<C *>(c->W1) + 12 * d.spec * (size_t)d.batch;
}

static mhd_status fused_prologue(mhd_ctx *c, const mhd::Dims &d) {
  const bool prof = c->profiling;
  const int b = d.batch;
  if (c->precision == MHD_FP64)
    LAUNCH(0, mhd::launch_col_inverse(state64(c, 0), zbuf<cplx64>(c, d), d.n, b * 7, d.nk * d.nx, c->tw, c->stream,
                                      c->tile[0], c->radix[0]));
  else if (c->precision == MHD_FP64_DF)
    LAUNCH(0, mhd::launch_col_inverse(statedf(c, 0), zbuf<cdf>(c, d), d.n, b * 7, d.nk * d.nx, c->twdf, c->stream,
                                      c->tile[0], c->radix[0]));
  else
    LAUNCH(0, mhd::launch_col_inverse(state_hi(c, 0), zbuf<cplx32>(c, d), d.n, b * 7, d.nk * d.nx, c->tw32,
                                      c->stream, c->tile[0], c->radix[0]));
  return MHD_OK;
}

// One RHS evaluation (steps 1-6 of the pass order at the state `y_in`, dt on the first
// evaluation of a step) and the assembly operation `op` for the `d.batch` instances from `inst0`.
static mhd_status eval_and_assemble(mhd_ctx *c, const mhd::Dims &d, int inst0, const void *y_in, cplx64 *rhs_out,
                                    const mhd::PhysDev *phys, mhd::TimeState *ts, mhd::StepCoef *coef, bool first,
                                    int op, int stage, void *bgrid = nullptr) {
  const bool prof = op != mhd::ASM_RHS && c->profiling;
  mhd_status st;
  const size_t off = (size_t)inst0 * 7 * d.spec;
  // a fused AB2 step of the whole step sequence (inst0 = 0): it reads and writes the z buffer
  const bool fz = op == mhd::ASM_AB2 && inst0 == 0 && fused_ab2(c);
  if (c->precision == MHD_FP64) {
    const cplx64 *yi = static_cast<const cplx64 *>(y_in);
    cplx64 *Z = fz ? zbuf<cplx64>(c, d) : nullptr;
    if ((st = flux_spectra_t<cplx64>(c, d, inst0, yi, phys, ts, coef, first && op != mhd::ASM_RHS, c->tw,
                                     static_cast<double *>(bgrid), Z)))
      return st;
    cplx64 *Y = c->Y ? static_cast<cplx64 *>(c->Y) + off : nullptr;
    cplx64 *force = c->forced ? c->W2 : nullptr;  // W2 is free after the forward z pass
    if (force) LAUNCH(6, mhd::launch_force(yi, force, phys, d, c->stream));
    if (fz)
      LAUNCH(8, mhd::launch_assemble_iz(c->W1, state64(c, 0), c->H, phys, coef, force, Z, c->tw, d, c->fuse_tile,
                                        c->stream));
    else
      LAUNCH(6, mhd::launch_assemble(c->W1, yi, state64(c, inst0), c->H + off, Y, rhs_out, phys, coef, op, stage, d,
                                     c->stream, force));
  } else if (c->precision == MHD_FP64_DF) {
    const cdf *yi = static_cast<const cdf *>(y_in);
    cdf *Z = fz ? zbuf<cdf>(c, d) : nullptr;
    if ((st = flux_spectra_t<cdf>(c, d, inst0, yi, phys, ts, coef, first && op != mhd::ASM_RHS, c->twdf,
                                  static_cast<double *>(bgrid), Z)))
      return st;
    cdf *Y = c->Y ? static_cast<cdf *>(c->Y) + off : nullptr;
    cdf *force = c->forced ? reinterpret_cast<cdf *>(c->W2) : nullptr;  // W2 is free after the forward z pass
    if (force) LAUNCH(6, mhd::launch_force(yi, force, phys, d, c->stream));
    if (fz)
      LAUNCH(8, mhd::launch_assemble_iz(reinterpret_cast<const cdf *>(c->W1), statedf(c, 0), histdf(c, 0), phys,
                                        coef, force, Z, c->twdf, d, c->fuse_tile, c->stream));
    else
      LAUNCH(6, mhd::launch_assemble(reinterpret_cast<const cdf *>(c->W1), yi, statedf(c, inst0), histdf(c, inst0),
                                     Y, rhs_out, phys, coef, op, stage, d, c->stream, force));
  } else {
    const cplx32 *yi = static_cast<const cplx32 *>(y_in);
    cplx32 *Z = fz ? zbuf<cplx32>(c, d) : nullptr;
    if ((st = flux_spectra_t<cplx32>(c, d, inst0, yi, phys, ts, coef, first && op != mhd::ASM_RHS, c->tw32,
                                     static_cast<float *>(bgrid), Z)))
      return st;
    cplx32 *Y = c->Y ? static_cast<cplx32 *>(c->Y) + off : nullptr;
    cplx32 *force = c->forced ? reinterpret_cast<cplx32 *>(c->W2) : nullptr;  // free after forward z
    if (force) LAUNCH(6, mhd::launch_force(yi, force, phys, d, c->stream));
    if (fz)
      LAUNCH(8, mhd::launch_assemble_iz(reinterpret_cast<const cplx32 *>(c->W1), state_hi(c, 0), state_lo(c, 0),
                                        hist32(c, 0), phys, coef, force, Z, c->tw32, d, c->fuse_tile, c->radix[0],
                                        c->stream));
    else
      LAUNCH(6, mhd::launch_assemble_df(reinterpret_cast<const cplx32 *>(c->W1), yi, state_hi(c, inst0),
                                        state_lo(c, inst0), hist32(c, inst0), Y, rhs_out, phys, coef, op, stage, d,
                                        c->stream, force));
  }
  return MHD_OK;
}

// The RHS of instances [inst0, inst0 + d.batch) into `rhs_out` (mode 0), or one time step of the
// context's solver (mode 1).
static mhd_status rhs_or_step(mhd_ctx *c, const mhd::Dims &d, int inst0, cplx64 *rhs_out,
                              const mhd::PhysDev *phys, mhd::TimeState *ts, mhd::StepCoef *coef, int mode) {
  const size_t off = (size_t)inst0 * 7 * d.spec;
  const void *y = c->precision == MHD_FP64      ? (const void *)state64(c, inst0)
                  : c->precision == MHD_FP64_DF ? (const void *)statedf(c, inst0)
                                                : (const void *)state_hi(c, inst0);
  const void *Y = nullptr;
  if (c->Y) Y = c->precision == MHD_FP32_MIXED ? (const void *)(static_cast<cplx32 *>(c->Y) + off)
                                               : (const void *)(static_cast<cplx64 *>(c->Y) + off);
  if (mode == 0) return eval_and_assemble(c, d, inst0, y, rhs_out, phys, ts, coef, true, mhd::ASM_RHS, 0);
  // tracers: the first evaluation (at y^n) also writes the grid field; the push follows the step
  void *bg = nullptr;
  for (int i = inst0; i < inst0 + d.batch && !bg; ++i)
    if (c->ntr[i] > 0) bg = c->bgrid;
  mhd_status st;
  switch (c->integrator) {
    case MHD_RK4:
      if ((st = eval_and_assemble(c, d, inst0, y, nullptr, phys, ts, coef, true, mhd::ASM_RK_STAGE, 1, bg))) return st;
      for (int sg = 2; sg <= 3; ++sg)
        if ((st = eval_and_assemble(c, d, inst0, Y, nullptr, phys, ts, coef, false, mhd::ASM_RK_STAGE, sg))) return st;
      st = eval_and_assemble(c, d, inst0, Y, nullptr, phys, ts, coef, false, mhd::ASM_RK_FINAL, 0);
      break;
    case MHD_PC:
      if ((st = eval_and_assemble(c, d, inst0, y, nullptr, phys, ts, coef, true, mhd::ASM_PC_PRED, 0, bg))) return st;
      st = eval_and_assemble(c, d, inst0, Y, nullptr, phys, ts, coef, false, mhd::ASM_PC_CORR, 0);
      break;
    default:
      st = eval_and_assemble(c, d, inst0, y, nullptr, phys, ts, coef, true, mhd::ASM_AB2, 0, bg);
  }
  if (st || !bg) return st;
  const bool prof = c->profiling;
  const size_t n3 = (size_t)d.n * d.n * d.n;
  for (int i = inst0; i < inst0 + d.batch; ++i) {
    if (c->ntr[i] == 0) continue;
    const size_t goff = (size_t)(i - inst0) * 3 * n3;
    if (c->precision != MHD_FP32_MIXED)
      LAUNCH(7, mhd::launch_tracer_push(static_cast<const double *>(c->bgrid) + goff, c->tr[i], c->ntr[i], coef + i,
                                        d.n, c->stream));
    else
      LAUNCH(7, mhd::launch_tracer_push(static_cast<const float *>(c->bgrid) + goff, c->tr[i], c->ntr[i], coef + i,
                                        d.n, c->stream));
  }
  return MHD_OK;
}

extern "C" {

mhd_status mhd_rhs(mhd_ctx *c, int32_t inst, double *drho, double *dm, double *db, int32_t on_device) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (!drho || !dm || !db) return fail(c, MHD_EINVAL, "null output");
  if (!c->is_set[inst]) return fail(c, MHD_ESTATE, "instance %d has no state", inst);
  DeviceGuard g(c);
  const mhd::Dims d = one(c);
  if ((st = rhs_or_step(c, d, inst, c->W2, c->phys + inst, nullptr, nullptr, 0))) return st;
  // W2 holds the RHS spectra; inverse_zy reads its source before overwriting W2
  CK(mhd::launch_col_inverse(c->W2, c->W1, d.n, 7, d.nk * d.nx, c->tw, c->stream));
  CK(mhd::launch_col_inverse(c->W1, c->W2, d.n, 7 * d.n, d.nx, c->tw, c->stream));
  const size_t n3 = (size_t)d.n * d.n * d.n;
  double *real = reinterpret_cast<double *>(c->W1);
  CK(mhd::launch_get_x(c->W2, real, 7, d, c->tw, c->stream));
  if ((st = copy_out(c, drho, real, n3 * sizeof(double), on_device))) return st;
  if ((st = copy_out(c, dm, real + n3, 3 * n3 * sizeof(double), on_device))) return st;
  if ((st = copy_out(c, db, real + 4 * n3, 3 * n3 * sizeof(double), on_device))) return st;
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

}  // extern "C"

// Advance the first `nb` instances `nsteps` steps, replaying the CUDA graph kept in *graph (captured
// on first use after one direct step) unless graphs are off or profiling is on.
static mhd_status step_prefix(mhd_ctx *c, int nb, int32_t nsteps, cudaGraphExec_t *graph) {
  if (nb <= 0 || nsteps <= 0) return MHD_OK;
  mhd::Dims d = c->d;
  d.batch = nb;
  int s = 0;
  const bool fused = fused_ab2(c);
  if (fused) {
    // the z buffer is current when the previous entry point was a step call over the same
    // instances; otherwise a plain inverse z pass refills it, and the steps' fused assembly keeps
    // it current from there
    const bool current = c->z_nb == nb && c->z_at + 1 == c->api_calls;
    c->z_nb = 0;
    if (!current) {
      mhd_status st = fused_prologue(c, d);
      if (st) return st;
    }
  }
  if (c->use_graph && !c->profiling) {
    if (!*graph) {
      // one direct step first (it also raises the kernels' shared-memory limits, which is not a
      // stream operation), then capture one step on a private stream and instantiate it
      mhd_status st = rhs_or_step(c, d, 0, nullptr, c->phys, c->ts, c->coef, 1);
      if (st) return st;
      ++s;
      if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      cudaStream_t user = c->stream;
      c->stream = c->cap_stream;
      CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      st = rhs_or_step(c, d, 0, nullptr, c->phys, c->ts, c->coef, 1);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
      c->stream = user;
      if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      CK(e);
      e = cudaGraphInstantiateWithFlags(graph, g, 0);
      cudaGraphDestroy(g);
      CK(e);
    }
    for (; s < nsteps; ++s) CK(cudaGraphLaunch(*graph, c->stream));
  } else {
    for (; s < nsteps; ++s) {
      mhd_status st = rhs_or_step(c, d, 0, nullptr, c->phys, c->ts, c->coef, 1);
      if (st) return st;
    }
  }
  if (fused) {
    c->z_at = c->api_calls;
    c->z_nb = nb;
  }
  return MHD_OK;
}

extern "C" {

mhd_status mhd_step(mhd_ctx *c, int32_t nsteps) {
  if (!c) return MHD_EINVAL;
  if (nsteps < 0) return fail(c, MHD_EINVAL, "negative step count");
  if (c->live >= 0) return fail(c, MHD_ESTATE, "context belongs to a pool: use mhd_pool_step");
  for (int i = 0; i < c->d.batch; ++i)
    if (!c->is_set[i]) return fail(c, MHD_ESTATE, "instance %d has no state", i);
  DeviceGuard g(c);
  return step_prefix(c, c->d.batch, nsteps, &c->graph_exec);
}

static mhd_status prof_resolve(mhd_ctx *c) {
  if (c->ev_marks.empty()) return MHD_OK;
  CK(cudaStreamSynchronize(c->stream));
  for (const auto &m : c->ev_marks) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev_pool[m.second], c->ev_pool[m.second + 1]));
    c->prof_ms[m.first] += ms;
    c->prof_count[m.first] += 1;
  }
  c->ev_marks.clear();
  c->ev_used = 0;
  return MHD_OK;
}

mhd_status mhd_profile(mhd_ctx *c, int32_t enable) {
  if (!c) return MHD_EINVAL;
  DeviceGuard g(c);
  mhd_status st = prof_resolve(c);
  if (st) return st;
  if (enable) {
    for (int i = 0; i < 9; ++i) {
      c->prof_ms[i] = 0.0;
      c->prof_count[i] = 0;
    }
  }
  c->profiling = enable != 0;
  return MHD_OK;
}

mhd_status mhd_profile_read(mhd_ctx *c, mhd_kernel_time *out, int32_t max, int32_t *count) {
  if (!c || (!out && max > 0) || !count) return MHD_EINVAL;
  DeviceGuard g(c);
  mhd_status st = prof_resolve(c);
  if (st) return st;
  int k = 0;
  for (int i = 0; i < 9 && k < max; ++i, ++k) out[k] = mhd_kernel_time{kKernelNames[i], c->prof_ms[i], c->prof_count[i]};
  *count = k;
  return MHD_OK;
}

mhd_status mhd_autotune(mhd_ctx *c, int32_t reps, int32_t *tiles, int32_t *radix, double *ms) {
  if (!c) return MHD_EINVAL;
  if (reps < 1 || reps > 100) return fail(c, MHD_EINVAL, "reps must be 1..100");
  DeviceGuard g(c);
  const mhd::Dims &d = c->d;
  const int b = d.batch;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, MHD_ECUDA, "event creation failed");
  }
  // one launch of column pass `kind` with tile width `tile` and radix `vpt`, on the step's
  // buffers and shapes
  auto run = [&](int kind, int tile, int vpt) -> cudaError_t {
    if (c->precision == MHD_FP64_DF) {
      cdf *w1 = reinterpret_cast<cdf *>(c->W1), *w2 = reinterpret_cast<cdf *>(c->W2);
      switch (kind) {
        case 0: return mhd::launch_col_inverse(statedf(c, 0), w1, d.n, b * 7, d.nk * d.nx, c->twdf, c->stream, tile);
        case 1: return mhd::launch_col_inverse(w1, w2, d.n, b * 7 * d.n, d.nx, c->twdf, c->stream, tile);
        case 2: return mhd::launch_col_forward(w1, w2, d.n, b * 12 * d.n, d.nx, 1.0, c->twdf, c->stream, tile);
        default: return mhd::launch_col_forward(w2, w1, d.n, b * 12, d.nk * d.nx, 1.0, c->twdf, c->stream, tile);
      }
    }
    if (c->precision == MHD_FP64) {
      cplx64 *w1 = c->W1, *w2 = c->W2;
      switch (kind) {
        case 0: return mhd::launch_col_inverse(state64(c, 0), w1, d.n, b * 7, d.nk * d.nx, c->tw, c->stream, tile);
        case 1: return mhd::launch_col_inverse(w1, w2, d.n, b * 7 * d.n, d.nx, c->tw, c->stream, tile);
        case 2: return mhd::launch_col_forward(w1, w2, d.n, b * 12 * d.n, d.nx, 1.0, c->tw, c->stream, tile);
        default: return mhd::launch_col_forward(w2, w1, d.n, b * 12, d.nk * d.nx, 1.0, c->tw, c->stream, tile);
      }
    }
    cplx32 *w1 = reinterpret_cast<cplx32 *>(c->W1), *w2 = reinterpret_cast<cplx32 *>(c->W2);
    switch (kind) {
      case 0: return mhd::launch_col_inverse(state_hi(c, 0), w1, d.n, b * 7, d.nk * d.nx, c->tw32, c->stream, tile, vpt);
      case 1: return mhd::launch_col_inverse(w1, w2, d.n, b * 7 * d.n, d.nx, c->tw32, c->stream, tile, vpt);
      case 2: return mhd::launch_col_forward(w1, w2, d.n, b * 12 * d.n, d.nx, 1.0, c->tw32, c->stream, tile, vpt);
      default: return mhd::launch_col_forward(w2, w1, d.n, b * 12, d.nk * d.nx, 1.0, c->tw32, c->stream, tile, vpt);
    }
  };
  const size_t elem = c->precision == MHD_FP32_MIXED ? sizeof(cplx32) : sizeof(cplx64);
  const size_t pitch = (size_t)(d.n + d.n / (128 / (int)elem)) | 1;  // pencil pitch, as the kernels lay it out
  int best[4], best_vpt[4];
  double best_ms[4];
  cudaError_t err = cudaSuccess;
  const bool fp64 = c->precision != MHD_FP32_MIXED;  // radix 8 only
  for (int kind = 0; kind < 4 && err == cudaSuccess; ++kind) {
    best[kind] = 0;
    best_vpt[kind] = 0;
    best_ms[kind] = 1e300;
    for (int vpt = 8; vpt <= (fp64 ? 8 : 16) && err == cudaSuccess; vpt *= 2) {
      const int max_tc = c->precision == MHD_FP64_DF ? mhd::col_max_tile_df(d.n, kind < 2 ? +1 : -1)
                                                     : mhd::col_max_tile(d.n, kind < 2 ? +1 : -1, fp64, false, vpt);
      for (int tc = 1; tc <= max_tc && err == cudaSuccess; tc *= 2) {
        if (tc * pitch * elem > 227 * 1024) break;
        if ((err = run(kind, tc, vpt)) != cudaSuccess) break;  // warm-up (raises the shared-memory limit)
        if ((err = cudaEventRecord(e0, c->stream)) != cudaSuccess) break;
        for (int r = 0; r < reps && err == cudaSuccess; ++r) err = run(kind, tc, vpt);
        if (err != cudaSuccess || (err = cudaEventRecord(e1, c->stream)) != cudaSuccess) break;
        if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float t = 0.0f;
        if ((err = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
        const double per = (double)t / reps;
        if (per < best_ms[kind]) {
          best_ms[kind] = per;
          best[kind] = tc;
          best_vpt[kind] = fp64 ? 0 : vpt;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(c, MHD_ECUDA, "autotune: %s", cudaGetErrorString(err));
  for (int k = 0; k < 4; ++k) {
    c->tile[k] = best[k];
    c->radix[k] = best_vpt[k];
    if (tiles) tiles[k] = best[k];
    if (radix) radix[k] = fp64 ? 8 : best_vpt[k];
    if (ms) ms[k] = best_ms[k];
  }
  drop_graphs(c);
  return MHD_OK;
}

mhd_status mhd_set_option(mhd_ctx *c, int32_t option, int64_t value) {
  if (!c) return MHD_EINVAL;
  DeviceGuard g(c);
  if (option == MHD_OPT_CUDA_GRAPH) {
    if (value != 0 && value != 1) return fail(c, MHD_EINVAL, "graph option must be 0 or 1");
    c->use_graph = value != 0;
  } else if (option == MHD_OPT_FLUX_PIPELINE) {
    if (value != 0 && value != 1) return fail(c, MHD_EINVAL, "pipeline option must be 0 or 1");
    c->flux_pipeline = value != 0;
  } else if (option == MHD_OPT_PERSISTENT) {
    if (value != 0 && value != 1) return fail(c, MHD_EINVAL, "persistent option must be 0 or 1");
    c->persistent = value != 0;
  } else if (option == MHD_OPT_FUSED_UPDATE) {
    if (value != 0 && value != 1) return fail(c, MHD_EINVAL, "fused update option must be 0 or 1");
    c->fuse = value != 0;
  } else if (option == MHD_OPT_TILE_FUSED) {
    if (value < 0 || value > 64) return fail(c, MHD_EINVAL, "tile must be 0..64");
    c->fuse_tile = (int)value;
  } else if (option == MHD_OPT_WAIT_POLLS) {
    if (value < 0 || value > (int64_t)mhd::kWaitPolls)
      return fail(c, MHD_EINVAL, "wait poll limit must be 0..%u", (unsigned)mhd::kWaitPolls);
    c->wait_polls = (uint32_t)value;
  } else if (option >= MHD_OPT_TILE_INV_Z && option <= MHD_OPT_TILE_FWD_Z) {
    if (value < 0 || value > 64) return fail(c, MHD_EINVAL, "tile must be 0..64");
    c->tile[option - MHD_OPT_TILE_INV_Z] = (int)value;
  } else if (option >= MHD_OPT_RADIX_INV_Z && option <= MHD_OPT_RADIX_FWD_Z) {
    if (value != 0 && value != 8 && value != 16) return fail(c, MHD_EINVAL, "radix must be 0, 8 or 16");
    c->radix[option - MHD_OPT_RADIX_INV_Z] = (int)value;
  } else {
    return fail(c, MHD_EINVAL, "unknown option %d", option);
  }
  CK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);
  return MHD_OK;
}

mhd_status mhd_set_forcing(mhd_ctx *c, int32_t inst, double amp, double a, double b, double cc, int32_t kf) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (!isfinite(amp) || !isfinite(a) || !isfinite(b) || !isfinite(cc)) return fail(c, MHD_EINVAL, "non-finite forcing");
  if (kf < 1 || kf > c->d.k) return fail(c, MHD_EINVAL, "forcing wavenumber %d outside 1..%d", kf, c->d.k);
  DeviceGuard g(c);
  const mhd::PhysDev pd = mhd::make_phys(c->phys_host[inst].nu, c->phys_host[inst].eta, c->phys_host[inst].cs, amp, a,
                                         b, cc, kf);
  CK(cudaMemcpyAsync(c->phys + inst, &pd, sizeof pd, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (amp != 0.0 && !c->forced) {
    c->forced = true;  // the step gains the force pass: recapture
    drop_graphs(c);
  }
  return MHD_OK;
}

mhd_status mhd_synchronize(mhd_ctx *c) {
  if (!c) return MHD_EINVAL;
  DeviceGuard g(c);
  int32_t any = 0, err = 0;
  CK(mhd::launch_status_any(c->ts, c->d.batch, c->flag, c->stream));
  CK(cudaMemcpyAsync(&any, c->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&err, c->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->out_stream) CK(cudaStreamSynchronize(c->out_stream));  // mhd_get_state_async copies
  if (err == 1) return fail(c, MHD_ETIMEOUT, "a device-side wait gave up (its copies were drained)");
  if (err) return fail(c, MHD_ETIMEOUT, "a device-side wait gave up and a copy did not complete in the drain");
  return any ? MHD_ENONFINITE : MHD_OK;
}

mhd_status mhd_tracers_set(mhd_ctx *c, int32_t inst, int64_t count, const double *pos) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (count < 0 || (count > 0 && !pos)) return fail(c, MHD_EINVAL, "bad tracer count or null positions");
  if (c->live >= 0) return fail(c, MHD_ESTATE, "tracers are not available on pool contexts");
  if (count > 0 && !c->is_set[inst]) return fail(c, MHD_ESTATE, "instance %d has no state", inst);
  DeviceGuard g(c);
  CK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);  // the step gains or loses launches
  dfree(c, c->tr[inst]);
  c->tr[inst] = nullptr;
  c->ntr[inst] = 0;
  if (count == 0) return MHD_OK;
  const mhd::Dims d = one(c);
  const size_t n3 = (size_t)d.n * d.n * d.n;
  if (!c->bgrid) {
    const size_t elem = c->precision == MHD_FP32_MIXED ? sizeof(float) : sizeof(double);
    if (!(c->bgrid = dalloc(c, (size_t)c->d.batch * 3 * n3 * elem))) return fail(c, MHD_ENOMEM, "tracer grid buffer");
  }
  double *t = static_cast<double *>(dalloc(c, (size_t)count * 6 * sizeof(double)));
  if (!t) return fail(c, MHD_ENOMEM, "tracer arrays (%lld particles)", (long long)count);
  // positions, wrapped into [0, 2 pi), stored by component
  const double L = 2.0 * M_PI;
  std::vector<double> h((size_t)count * 3);
  for (int64_t m = 0; m < count; ++m)
    for (int a = 0; a < 3; ++a) {
      const double x = pos[3 * m + a];
      if (!std::isfinite(x)) {
        dfree(c, t);
        return fail(c, MHD_EINVAL, "tracer %lld has a non-finite position", (long long)m);
      }
      double w = x - L * floor(x / L);
      if (w >= L) w -= L;
      h[(size_t)a * count + m] = w;
    }
  CK(cudaMemcpyAsync(t, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  // initial velocities: the grid velocity at the particles
  const cplx64 *Si = nullptr;
  if ((st = state_fp64(c, inst, &Si))) return st;
  if ((st = inverse_zy(c, Si))) return st;
  double *real = reinterpret_cast<double *>(c->W1);
  CK(mhd::launch_get_x(c->W2, real, 7, d, c->tw, c->stream));
  CK(mhd::launch_tracer_init(real, t, count, d.n, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->tr[inst] = t;
  c->ntr[inst] = count;
  return MHD_OK;
}

mhd_status mhd_tracers_get(mhd_ctx *c, int32_t inst, double *pos, double *vel) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  const int64_t count = c->ntr[inst];
  if (count == 0) return MHD_OK;
  DeviceGuard g(c);
  std::vector<double> h((size_t)count * 6);
  CK(cudaMemcpyAsync(h.data(), c->tr[inst], h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int64_t m = 0; m < count; ++m)
    for (int a = 0; a < 3; ++a) {
      if (pos) pos[3 * m + a] = h[(size_t)a * count + m];
      if (vel) vel[3 * m + a] = h[(size_t)(3 + a) * count + m];
    }
  return MHD_OK;
}

int64_t mhd_tracers_count(mhd_ctx *c, int32_t inst) {
  if (!c || inst < 0 || inst >= c->d.batch) return -1;
  return c->ntr[inst];
}

int32_t mhd_num_shells(int32_t n) { return valid_n(n) ? mhd::num_shells((n - 1) / 3) : 0; }

mhd_status mhd_spectra(mhd_ctx *c, int32_t inst, double *ek, double *em, int32_t nshells, mhd_flow_stats *stats) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  const mhd::Dims d = one(c);
  const int ns = mhd::num_shells(d.k);
  if ((ek || em) && nshells != ns) return fail(c, MHD_EINVAL, "nshells must equal mhd_num_shells(n)");
  DeviceGuard g(c);
  const size_t n3 = (size_t)d.n * d.n * d.n;
  const size_t part_len = sizes_for(c->d, c->precision).part;
  const int mblocks = (int)std::min<size_t>(2 * 152, part_len / 2);
  if ((size_t)5 * ns > part_len || mblocks < 1) return fail(c, MHD_EINVAL, "scratch too small for the spectra");
  const cplx64 *Si = nullptr;
  if ((st = state_fp64(c, inst, &Si))) return st;
  // u_hat: inverse z, y of the state; u = m / rho with the x passes; forward y, z
  if ((st = inverse_zy(c, Si))) return st;
  CK(mhd::launch_velocity_x(c->W2, c->W1, d, c->tw, c->stream));
  CK(mhd::launch_col_forward(c->W1, c->W2, d.n, 3 * d.n, d.nx, 1.0, c->tw, c->stream));
  CK(mhd::launch_col_forward(c->W2, c->W1, d.n, 3, d.nk * d.nx, 1.0 / (double)n3, c->tw, c->stream));
  // shells; the spectrum of du_x/dx into W2 and that of div B into W1 past n^3 complex values
  // (clear of u_hat, 3 spec values, and of all that the du_x/dx chain below writes into W1: its
  // z-pass output and n^3 real values; W1 holds at least 7 n^3 doubles)
  cplx64 *gh = c->W1 + n3;
  CK(mhd::launch_shells(c->W1, Si + 4 * d.spec, c->W2, gh, c->part, d, c->stream));
  std::vector<double> sh((size_t)5 * ns);
  CK(cudaMemcpyAsync(sh.data(), c->part, sh.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // du_x/dx on the grid, then its moments
  CK(mhd::launch_col_inverse(c->W2, c->W1, d.n, 1, d.nk * d.nx, c->tw, c->stream));
  CK(mhd::launch_col_inverse(c->W1, c->W2, d.n, d.n, d.nx, c->tw, c->stream));
  double *real = reinterpret_cast<double *>(c->W1);
  CK(mhd::launch_get_x(c->W2, real, 1, d, c->tw, c->stream));
  CK(mhd::launch_moments(real, n3, c->part, mblocks, c->stream));
  std::vector<double> mp((size_t)2 * mblocks);
  CK(cudaMemcpyAsync(mp.data(), c->part, mp.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  // div B on the grid (into W2), then its largest magnitude
  CK(mhd::launch_col_inverse(gh, c->W2, d.n, 1, d.nk * d.nx, c->tw, c->stream));
  CK(mhd::launch_col_inverse(c->W2, c->W1, d.n, d.n, d.nx, c->tw, c->stream));
  double *dreal = reinterpret_cast<double *>(c->W2);
  CK(mhd::launch_get_x(c->W1, dreal, 1, d, c->tw, c->stream));
  CK(mhd::launch_absmax(dreal, n3, c->part, mblocks, c->stream));  // after the copy of mp (stream order)
  std::vector<double> ap((size_t)mblocks);
  CK(cudaMemcpyAsync(ap.data(), c->part, ap.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  double th = 0.0, m2 = 0.0, m3 = 0.0, hk = 0.0, hm = 0.0, dmax = 0.0;
  for (int s = 0; s < ns; ++s) {
    if (ek) ek[s] = sh[5 * s];
    if (em) em[s] = sh[5 * s + 1];
    th += sh[5 * s + 2];
    hk += sh[5 * s + 3];
    hm += sh[5 * s + 4];
  }
  for (int b = 0; b < mblocks; ++b) dmax = (ap[b] != ap[b] || ap[b] > dmax) ? ap[b] : dmax;
  for (int b = 0; b < mblocks; ++b) {
    m2 += mp[2 * b];
    m3 += mp[2 * b + 1];
  }
  m2 /= (double)n3;
  m3 /= (double)n3;
  if (stats) {
    stats->theta = sqrt(th);
    stats->d2 = m2;
    stats->d3 = m3;
    stats->s3 = m3 / pow(m2, 1.5);
    stats->kin_hel = hk;
    stats->mag_hel = hm;
    stats->divb_max = dmax;
  }
  return MHD_OK;
}

mhd_status mhd_diagnostics(mhd_ctx *c, int32_t inst, mhd_diag *out) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (!out) return fail(c, MHD_EINVAL, "null output");
  DeviceGuard g(c);
  const mhd::Dims d = one(c);
  const cplx64 *Si = nullptr;
  if ((st = state_fp64(c, inst, &Si))) return st;
  if ((st = inverse_zy(c, Si))) return st;
  CK(mhd::launch_diag_x(c->W2, c->phys + inst, c->part, d, c->tw, c->stream));
  CK(mhd::launch_diag_finish(c->part, mhd::diag_x_blocks(d.n), Si, c->phys + inst, c->ts + inst, c->diag_out, d,
                             c->stream, c->diag_out + 32));
  double h[24];
  CK(cudaMemcpyAsync(h, c->diag_out, 19 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof *out);
  out->ke = h[0];
  out->me = h[1];
  out->eint = h[2];
  out->cross_hel = h[3];
  out->mean_speed = h[4];
  out->mean_bmag = h[5];
  out->smax = h[6];
  out->mean_rho = h[7];
  for (int a = 0; a < 3; ++a) {
    out->mean_m[a] = h[8 + a];
    out->mean_b[a] = h[11 + a];
  }
  out->divb_rms = h[14];
  out->t = h[15];
  out->dt = h[16];
  out->step = (int64_t)h[17];
  out->status = (int32_t)h[18];
  const double cs = c->phys_host[inst].cs;
  out->mach_s = out->mean_speed / cs;
  out->v_a = out->mean_rho > 0.0 ? out->mean_bmag / sqrt(out->mean_rho) : 0.0;
  out->mach_a = out->v_a > 0.0 ? out->mean_speed / out->v_a : 0.0;
  return MHD_OK;
}

size_t mhd_checkpoint_doubles(const mhd_ctx *c) { return c ? 4 * 7 * c->d.spec + 8 : 0; }

mhd_status mhd_checkpoint(mhd_ctx *c, int32_t inst, double *buf, int32_t on_device) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (!buf) return fail(c, MHD_EINVAL, "null buffer");
  DeviceGuard g(c);
  const size_t sp = 7 * c->d.spec;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (c->precision != MHD_FP32_MIXED) {  // FP64, or double-float values in the same bytes
    CK(cudaMemcpyAsync(buf, state64(c, inst), sp * sizeof(cplx64), k, c->stream));
    CK(cudaMemcpyAsync(buf + 2 * sp, c->H + (size_t)inst * sp, sp * sizeof(cplx64), k, c->stream));
  } else {
    CK(cudaMemcpyAsync(buf, state_hi(c, inst), sp * sizeof(cplx32), k, c->stream));
    CK(cudaMemcpyAsync(buf + sp, state_lo(c, inst), sp * sizeof(cplx32), k, c->stream));
    CK(cudaMemcpyAsync(buf + 2 * sp, hist32(c, inst), sp * sizeof(cplx32), k, c->stream));
    // the FP32 history fills half of its slot; the rest is written as zeros
    if (on_device) CK(cudaMemsetAsync(buf + 3 * sp, 0, sp * sizeof(cplx32), c->stream));
    else memset(buf + 3 * sp, 0, sp * sizeof(cplx32));
  }
  static_assert(sizeof(mhd::TimeState) % sizeof(double) == 0 && sizeof(mhd::TimeState) <= 8 * sizeof(double),
                "time state fits the tail");
  CK(cudaMemcpyAsync(buf + 4 * sp, c->ts + inst, sizeof(mhd::TimeState), k, c->stream));
  // the rest of the tail is written as zeros, so equal states give byte-identical checkpoints
  constexpr size_t used = sizeof(mhd::TimeState) / sizeof(double);
  if (used < 8) {
    if (on_device) CK(cudaMemsetAsync(buf + 4 * sp + used, 0, (8 - used) * sizeof(double), c->stream));
    else memset(buf + 4 * sp + used, 0, (8 - used) * sizeof(double));
  }
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

mhd_status mhd_restore(mhd_ctx *c, int32_t inst, const double *buf, int32_t on_device) {
  mhd_status st = check_inst(c, inst);
  if (st) return st;
  if (!buf) return fail(c, MHD_EINVAL, "null buffer");
  DeviceGuard g(c);
  const size_t sp = 7 * c->d.spec;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (c->precision != MHD_FP32_MIXED) {  // FP64, or double-float values in the same bytes
    CK(cudaMemcpyAsync(state64(c, inst), buf, sp * sizeof(cplx64), k, c->stream));
    CK(cudaMemcpyAsync(c->H + (size_t)inst * sp, buf + 2 * sp, sp * sizeof(cplx64), k, c->stream));
  } else {
    CK(cudaMemcpyAsync(state_hi(c, inst), buf, sp * sizeof(cplx32), k, c->stream));
    CK(cudaMemcpyAsync(state_lo(c, inst), buf + sp, sp * sizeof(cplx32), k, c->stream));
    CK(cudaMemcpyAsync(hist32(c, inst), buf + 2 * sp, sp * sizeof(cplx32), k, c->stream));
  }
  CK(cudaMemcpyAsync(c->ts + inst, buf + 4 * sp, sizeof(mhd::TimeState), k, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->is_set[inst] = 1;
  return MHD_OK;
}

// ------------------------------------------------------------------------------------------
// Serving pools
// ------------------------------------------------------------------------------------------
}  // extern "C"

struct mhd_pool {
  mhd_ctx *ctx = nullptr;
  std::vector<int> pos_of;     // slot handle -> instance position (-1: free)
  std::vector<int> handle_at;  // instance position -> slot handle
};

// Copy instance `from` onto position `to` (state, history, time state, parameters).
static mhd_status move_instance(mhd_ctx *c, int from, int to) {
  const size_t sp = 7 * c->d.spec;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  if (c->precision != MHD_FP32_MIXED) {  // FP64, or double-float values in the same bytes
    CK(cudaMemcpyAsync(state64(c, to), state64(c, from), sp * sizeof(cplx64), k, c->stream));
    CK(cudaMemcpyAsync(c->H + (size_t)to * sp, c->H + (size_t)from * sp, sp * sizeof(cplx64), k, c->stream));
  } else {
    CK(cudaMemcpyAsync(state_hi(c, to), state_hi(c, from), sp * sizeof(cplx32), k, c->stream));
    CK(cudaMemcpyAsync(state_lo(c, to), state_lo(c, from), sp * sizeof(cplx32), k, c->stream));
    CK(cudaMemcpyAsync(hist32(c, to), hist32(c, from), sp * sizeof(cplx32), k, c->stream));
  }
  CK(cudaMemcpyAsync(c->ts + to, c->ts + from, sizeof(mhd::TimeState), k, c->stream));
  CK(cudaMemcpyAsync(c->phys + to, c->phys + from, sizeof(mhd::PhysDev), k, c->stream));
  c->phys_host[to] = c->phys_host[from];
  CK(cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

static mhd_status pool_position(mhd_pool *p, int32_t slot, int *pos) {
  if (!p) return MHD_EINVAL;
  if (slot < 0 || slot >= (int)p->pos_of.size() || p->pos_of[slot] < 0)
    return fail(p->ctx, MHD_EINVAL, "slot %d is not in use", slot);
  *pos = p->pos_of[slot];
  return MHD_OK;
}

extern "C" {

mhd_status mhd_pool_create(const mhd_params *params, mhd_pool **out) {
  if (!out) return MHD_EINVAL;
  *out = nullptr;
  if (!params || params->batch < 1) return MHD_EINVAL;
  std::vector<mhd_phys> ph(params->batch, mhd_phys{0.0, 0.0, 1.0});
  mhd_ctx *c = nullptr;
  mhd_status st = mhd_init(params, ph.data(), &c);
  if (st) return st;
  mhd_pool *p = new (std::nothrow) mhd_pool;
  if (!p) {
    mhd_destroy(c);
    return MHD_ENOMEM;
  }
  p->ctx = c;
  c->live = 0;
  c->pool_graphs.assign(params->batch + 1, nullptr);
  p->pos_of.assign(params->batch, -1);
  p->handle_at.assign(params->batch, -1);
  *out = p;
  return MHD_OK;
}

void mhd_pool_destroy(mhd_pool *p) {
  if (!p) return;
  mhd_destroy(p->ctx);
  delete p;
}

const char *mhd_pool_last_error(const mhd_pool *p) { return p ? mhd_last_error(p->ctx) : "null pool"; }

mhd_status mhd_pool_admit(mhd_pool *p, const mhd_phys *phys, const double *rho, const double *u, const double *b,
                          int32_t on_device, int64_t nsteps, int32_t *slot) {
  if (!p || !phys || !slot) return MHD_EINVAL;
  mhd_ctx *c = p->ctx;
  if (nsteps < 1) return fail(c, MHD_EINVAL, "a run needs at least one step");
  if (!(phys->nu >= 0.0) || !(phys->eta >= 0.0) || !(phys->cs > 0.0) || !isfinite(phys->nu) ||
      !isfinite(phys->eta) || !isfinite(phys->cs))
    return fail(c, MHD_EINVAL, "bad physical parameters");
  if (c->live >= c->d.batch) return MHD_EBUSY;
  int handle = -1;
  for (int h = 0; h < (int)p->pos_of.size(); ++h)
    if (p->pos_of[h] < 0) {
      handle = h;
      break;
    }
  if (handle < 0) return MHD_EBUSY;
  DeviceGuard g(c);
  const int pos = c->live;
  const mhd::PhysDev pd = mhd::make_phys(phys->nu, phys->eta, phys->cs);
  CK(cudaMemcpyAsync(c->phys + pos, &pd, sizeof pd, cudaMemcpyHostToDevice, c->stream));
  c->phys_host[pos] = *phys;
  mhd_status st = mhd_set_state(c, pos, rho, u, b, on_device);
  if (st) return st;
  const int64_t lim = nsteps;
  CK(cudaMemcpyAsync(&c->ts[pos].step_limit, &lim, sizeof lim, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  p->pos_of[handle] = pos;
  p->handle_at[pos] = handle;
  c->live = pos + 1;
  *slot = handle;
  return MHD_OK;
}

mhd_status mhd_pool_step(mhd_pool *p, int32_t k) {
  if (!p) return MHD_EINVAL;
  mhd_ctx *c = p->ctx;
  if (k < 0) return fail(c, MHD_EINVAL, "negative step count");
  DeviceGuard g(c);
  return step_prefix(c, c->live, k, &c->pool_graphs[c->live]);
}

mhd_status mhd_pool_progress(mhd_pool *p, int64_t *steps, int32_t *status, int32_t *finished) {
  if (!p || !steps || !status || !finished) return MHD_EINVAL;
  mhd_ctx *c = p->ctx;
  DeviceGuard g(c);
  std::vector<mhd::TimeState> ts(c->live > 0 ? c->live : 1);
  if (c->live > 0) {
    CK(cudaMemcpyAsync(ts.data(), c->ts, c->live * sizeof(mhd::TimeState), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  for (int h = 0; h < (int)p->pos_of.size(); ++h) {
    const int pos = p->pos_of[h];
    if (pos < 0) {
      steps[h] = -1;
      status[h] = 0;
      finished[h] = 0;
    } else {
      steps[h] = ts[pos].step;
      status[h] = ts[pos].status;
      finished[h] = ts[pos].status != 0 || (ts[pos].step_limit > 0 && ts[pos].step >= ts[pos].step_limit);
    }
  }
  return MHD_OK;
}

mhd_status mhd_pool_diagnostics(mhd_pool *p, int32_t slot, mhd_diag *out) {
  int pos = 0;
  mhd_status st = pool_position(p, slot, &pos);
  if (st) return st;
  return mhd_diagnostics(p->ctx, pos, out);
}

mhd_status mhd_pool_retire(mhd_pool *p, int32_t slot, double *rho, double *m, double *b, int32_t on_device) {
  int pos = 0;
  mhd_status st = pool_position(p, slot, &pos);
  if (st) return st;
  mhd_ctx *c = p->ctx;
  DeviceGuard g(c);
  if (rho && m && b) {
    if ((st = mhd_get_state(c, pos, rho, m, b, on_device))) return st;
  }
  const int last = c->live - 1;
  if (pos != last) {
    if ((st = move_instance(c, last, pos))) return st;
    p->handle_at[pos] = p->handle_at[last];
    p->pos_of[p->handle_at[pos]] = pos;
  }
  p->pos_of[slot] = -1;
  p->handle_at[last] = -1;
  c->live = last;
  return MHD_OK;
}

mhd_status mhd_pool_info(const mhd_pool *p, int32_t *live, int32_t *max_slots) {
  if (!p || !live || !max_slots) return MHD_EINVAL;
  *live = p->ctx->live;
  *max_slots = p->ctx->d.batch;
  return MHD_OK;
}

}  // extern "C"
