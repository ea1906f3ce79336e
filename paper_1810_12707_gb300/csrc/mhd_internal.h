// mhd_internal.h -- declarations shared by the host code and the kernel translation units.
//
// Spectral storage keeps only the modes the 2/3 rule retains (|k_x|, |k_y|, |k_z| <= K with
// K = floor((N-1)/3)), so every stored array is already dealiased:
//   state / history / RHS  [inst][field][kz' < NK][ky' < NK][kx < NX]
// with NX = K + 1 (kx = 0..K; the kx < 0 half follows from Hermitian symmetry) and NK = 2K + 1;
// a kept index j maps to the wavenumber j for j <= K and j - NK (= -K..-1) above.  Between the
// FFT passes of one step, fields live in scratch buffers with one more axis expanded to N:
//   after inverse z   [inst][field][z < N][ky' < NK][kx < NX]
//   after inverse y   [inst][field][z < N][y < N][kx < NX]
//   after forward x   [inst][flux][z < N][y < N][kx < NX]   (12 product fields)
//   after forward y   [inst][flux][z < N][ky' < NK][kx < NX]
//   after forward z   [inst][flux][kz' < NK][ky' < NK][kx < NX]
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "dfloat.cuh"

namespace mhd {

constexpr int kStateFields = 7;  // rho, m_x, m_y, m_z, B_x, B_y, B_z
constexpr int kFluxFields = 12;  // T_xx T_yy T_zz T_xy T_xz T_yz, E_x E_y E_z, u_x u_y u_z

template <typename R>
struct alignas(2 * sizeof(R)) cplx {
  using value_type = R;
  R re, im;
};
using cplx64 = cplx<double>;
using cplx32 = cplx<float>;

// Per-instance time-stepping state, device resident.
struct TimeState {
  double t;            // simulated time
  double dt_prev;      // step size of the previous step (0 before the first)
  double dt_last;      // step size of the last completed step, for diagnostics
  int64_t step;        // steps taken
  int32_t status;      // 0, or MHD_ENONFINITE once the instance stopped
  int32_t pad;
  int64_t step_limit;  // 0: no limit; else the instance stops advancing at this step count
};

// Coefficients of the current step, written by the dt kernel and read by the update kernel:
// y^{n+1} = y^n + dt (a1 f^n + a0 f^{n-1}); skip != 0 leaves the instance unchanged.
struct StepCoef {
  double dt, a1, a0;
  float fdt, fa1, fa0;  // the same, rounded once, for the mixed-precision update
  int32_t skip;
  // the double-float update's weights, split from their FP64 values: dt, dt a1, dt a0, dt / 6
  dfr dt_df, dta1_df, dta0_df, dt6_df;
};

// Per-instance physical parameters in device memory; famp != 0 switches on the ABC body force
// rho f, f = famp (fa sin kf z + fc cos kf y, fb sin kf x + fa cos kf z, fc sin kf y + fb cos kf x).
struct PhysDev {
  double nu, eta, cs;
  double famp, fa, fb, fc;
  int fkf, pad;
  dfr nu_df, eta_df, cs2_df;  // nu, eta and cs^2 split into double-float (the double-float assembly)
};

__host__ __device__ inline PhysDev make_phys(double nu, double eta, double cs, double famp = 0.0, double fa = 0.0,
                                             double fb = 0.0, double fc = 0.0, int kf = 1) {
  return PhysDev{nu, eta, cs, famp, fa, fb, fc, kf, 0, dfr_const(nu), dfr_const(eta), dfr_const(cs * cs)};
}

// Element type a pass scales its output by (a power of two in the double-float passes), and of a
// grid field written out for the tracers (FP64 for the double-float passes).
template <typename C>
struct scale_of {
  using type = typename C::value_type;
};
template <>
struct scale_of<cdf> {
  using type = float;
};
template <typename C>
struct grid_of {
  using type = typename C::value_type;
};
template <>
struct grid_of<cdf> {
  using type = double;
};

struct Dims {
  int n;      // grid points per axis
  int k;      // K = floor((n-1)/3)
  int nx;     // K + 1
  int nk;     // 2K + 1
  int batch;  // instances
  size_t spec;  // complex values of one truncated spectrum: nk * nk * nx
};

inline Dims make_dims(int n, int batch) {
  Dims d;
  d.n = n;
  d.k = (n - 1) / 3;
  d.nx = d.k + 1;
  d.nk = 2 * d.k + 1;
  d.batch = batch;
  d.spec = (size_t)d.nk * d.nk * d.nx;
  return d;
}

// ---- launchers (each returns the launch status; all work goes on `s`) ----
// The FFT passes exist in two precisions: FP64 throughout, and FP32 arithmetic and storage
// (the first inverse pass reads the FP64 state and writes FP32).  The transform arithmetic runs
// in the precision of the output; `tw` is the table W_N^m = exp(-2 pi i m / N), m < N, rounded to
// that precision.

// Column FFTs along the middle axis of [nslab][L][C]: inverse (sign +1) expands L from the
// NK kept indices to N; forward (sign -1) keeps only the NK kept outputs and multiplies by
// `scale`.
// `tile` > 0 forces the number of columns per block (else the library's choice).
// Host twiddle tables (twiddles.cu).  twiddle_table: W_N^m = exp(-2 pi i m/N), m < N.
// fp64_twiddle_bytes: the table every FP64 transform reads, fp64_twiddle_size(n) bytes: the
// classic table, then N pairs (c, t), then N bytes q with W_N^m = i^q c (1 + i t), |t| <= 1.
std::vector<cplx64> twiddle_table(int n);
std::vector<unsigned char> fp64_twiddle_bytes(int n);
constexpr size_t fp64_twiddle_size(int n) { return (size_t)n * (2 * sizeof(cplx64) + 1); }

// `ctr` (nullable): two zeroed unsigned words of device memory owned by the caller; when given,
// the pass runs as a persistent kernel (one grid of resident blocks taking tiles from ctr[0]) and
// leaves the words zeroed again.  Results are the same bits either way.
cudaError_t launch_col_inverse(const cplx64 *in, cplx64 *out, int n, int nslab, int cols,
                               const cplx64 *tw, cudaStream_t s, int tile = 0, int vpt = 0, unsigned *ctr = nullptr);
cudaError_t launch_col_inverse(const cplx64 *in, cplx32 *out, int n, int nslab, int cols,
                               const cplx32 *tw, cudaStream_t s, int tile = 0);
// vpt (FP32 passes): values per thread of the transform, 8 (radix 8) or 16 (radix 16); 0 = the
// library's default for the grid size.
cudaError_t launch_col_inverse(const cplx32 *in, cplx32 *out, int n, int nslab, int cols,
                               const cplx32 *tw, cudaStream_t s, int tile = 0, int vpt = 0, unsigned *ctr = nullptr);
// Largest power-of-two tile width (columns per block, <= 64) a column pass can launch with:
// dir +1 inverse, -1 forward; fp64 the transform type; mixed_in an FP64 input to an FP32 inverse.
int col_max_tile(int n, int dir, bool fp64, bool mixed_in = false, int vpt = 8);
cudaError_t launch_col_forward(const cplx64 *in, cplx64 *out, int n, int nslab, int cols,
                               double scale, const cplx64 *tw, cudaStream_t s, int tile = 0, int vpt = 0,
                               unsigned *ctr = nullptr);
cudaError_t launch_col_forward(const cplx32 *in, cplx32 *out, int n, int nslab, int cols,
                               double scale, const cplx32 *tw, cudaStream_t s, int tile = 0, int vpt = 0,
                               unsigned *ctr = nullptr);
// Double-float passes (MHD_FP64_DF): data, twiddles (W_N^m as hi + lo pairs) and arithmetic in
// double-float, radix 8; `scale` must be a power of two.
cudaError_t launch_col_inverse(const cdf *in, cdf *out, int n, int nslab, int cols, const cdf *tw, cudaStream_t s,
                               int tile = 0, int vpt = 0, unsigned *ctr = nullptr);
cudaError_t launch_col_forward(const cdf *in, cdf *out, int n, int nslab, int cols, double scale, const cdf *tw,
                               cudaStream_t s, int tile = 0, int vpt = 0, unsigned *ctr = nullptr);
int col_max_tile_df(int n, int dir);

// Fused x pass: inverse real transforms of the 7 state fields row by row, the products on the
// grid, forward real transforms of the 12 product fields (kx <= K kept), and the maximum of
// |u| + c_f per instance, accumulated as an atomic maximum on the bits into smax_bits[batch]
// (which must start at 0).  With `err` non-null, FP32 and N >= 128 the persistent, bulk-copy
// pipelined variant runs: a wait for a copy that gives up after `wait_polls` polls sets *err = 1
// (and *err = 2 if the copies still in flight do not complete within kWaitPolls polls each).
// With `bgrid` non-null the grid magnetic field is written to bgrid[inst][3][N^3] as well (the
// plain variant runs).
constexpr uint32_t kWaitPolls = 1u << 22;
// `ctr` (nullable, not with the pipelined variant): two zeroed unsigned words; the pass then runs
// as a persistent kernel taking row-pair blocks from ctr[0] (same results).
cudaError_t launch_flux_x(const cplx64 *in, cplx64 *out, const PhysDev *phys, unsigned long long *smax_bits,
                          const Dims &d, const cplx64 *tw, cudaStream_t s, int *err = nullptr,
                          double *bgrid = nullptr, uint32_t wait_polls = kWaitPolls, unsigned *ctr = nullptr);
cudaError_t launch_flux_x(const cplx32 *in, cplx32 *out, const PhysDev *phys, unsigned long long *smax_bits,
                          const Dims &d, const cplx32 *tw, cudaStream_t s, int *err = nullptr,
                          float *bgrid = nullptr, uint32_t wait_polls = kWaitPolls, unsigned *ctr = nullptr);
// Double-float flux pass (MHD_FP64_DF): products in double-float, exact FP64 CFL maximum as in
// the FP64 pass, grid magnetic field for the tracers in FP64.
cudaError_t launch_flux_x(const cdf *in, cdf *out, const PhysDev *phys, unsigned long long *smax_bits, const Dims &d,
                          const cdf *tw, cudaStream_t s, int *err = nullptr, double *bgrid = nullptr,
                          uint32_t wait_polls = kWaitPolls, unsigned *ctr = nullptr);
int flux_x_blocks_per_instance(int n);

// Forward real transform along x of 7 real fields given as rho, u (3), B (3) on the grid, with
// the momentum m = rho u formed first: [7][N^3] real of ONE instance -> [7][z][y][kx <= K].
cudaError_t launch_set_x(const double *rho, const double *u, const double *b, cplx64 *out,
                         const Dims &d, const cplx64 *tw, cudaStream_t s);
// Inverse real transform along x of `nfields` fields of one instance: [f][z][y][kx <= K] ->
// real [f][N^3].
cudaError_t launch_get_x(const cplx64 *in, double *out, int nfields, const Dims &d,
                         const cplx64 *tw, cudaStream_t s);
// The same two x passes over rows [row_begin, row_begin + nrows) only (a slab of z-planes: row =
// z N + y), with the real arrays holding just those rows, field stride `fstride` doubles.
// row_begin and nrows must be multiples of the kernels' row-pair block (N >= 16: a multiple of N
// suffices).
cudaError_t launch_set_x_rows(const double *rho, const double *u, const double *b, cplx64 *out, const Dims &d,
                              const cplx64 *tw, cudaStream_t s, size_t row_begin, size_t nrows, size_t fstride);
cudaError_t launch_get_x_rows(const cplx64 *in, double *out, int nfields, const Dims &d, const cplx64 *tw,
                              cudaStream_t s, size_t row_begin, size_t nrows, size_t fstride);
// The same in double-float: FP64 values (and the FP64 product rho u) split into double-float pairs
// on the way in, double-float values summed into FP64 on the way out; transforms in double-float.
cudaError_t launch_set_x_rows(const double *rho, const double *u, const double *b, cdf *out, const Dims &d,
                              const cdf *tw, cudaStream_t s, size_t row_begin, size_t nrows, size_t fstride);
cudaError_t launch_get_x_rows(const cdf *in, double *out, int nfields, const Dims &d, const cdf *tw, cudaStream_t s,
                              size_t row_begin, size_t nrows, size_t fstride);
// Inverse x pass of the 7 state fields of one instance with per-block partial sums of the grid
// diagnostics: part[block][8] = (sum ke, me, eint, u.B, |u|, |B|, max s, unused).
cudaError_t launch_diag_x(const cplx64 *in, const PhysDev *phys, double *part, const Dims &d,
                          const cplx64 *tw, cudaStream_t s);
int diag_x_blocks(int n);

// dt of every instance from its CFL maximum (or the fixed dt), the AB2 coefficients of this
// step, and the advance of the per-instance time state; resets smax_bits to 0 for the next pass.
cudaError_t launch_step_dt(unsigned long long *smax_bits, const PhysDev *phys, TimeState *ts, StepCoef *coef,
                           const Dims &d, double dt_fixed, double cfl_adv, double cfl_visc, cudaStream_t s);

// What the assembly does with the RHS r it computes (f evaluated at the state `y_in`), with y the
// instance's state, h its history buffer and Y the stage state:
enum AsmOp {
  ASM_RHS = 0,       // rhs_out = r
  ASM_AB2 = 1,       // y += dt (a1 r + a0 h);  h = r
  ASM_RK_STAGE = 2,  // h = r (stage 1) or h + 2 r (stages 2, 3);  Y = y + c dt r, c = 1/2, 1/2, 1
  ASM_RK_FINAL = 3,  // y += dt/6 (h + r)
  ASM_PC_PRED = 4,   // Y = y + dt (a1 r + a0 h);  h = r
  ASM_PC_CORR = 5    // y += dt/2 (h + r)
};

// Spectral assembly of the RHS from the 12 product spectra (scaled by N^-3) and the state y_in,
// followed by `op`; `stage` is the RK4 stage (1..3) for ASM_RK_STAGE.
// `force` (nullable): rho f spectra [inst][3][spec] from launch_force, added to the momentum RHS
// of the instances whose famp is non-zero.
cudaError_t launch_assemble(const cplx64 *flux, const cplx64 *y_in, cplx64 *state, cplx64 *hist, cplx64 *ystage,
                            cplx64 *rhs_out, const PhysDev *phys, const StepCoef *coef, int op, int stage,
                            const Dims &d, cudaStream_t s, const cplx64 *force = nullptr);
// Spectra of the ABC body force rho f at the state y_in: force[inst][3][spec] (instances with
// famp == 0 are skipped).  Must run before an assembly that updates y_in in place.
cudaError_t launch_force(const cplx64 *y_in, cplx64 *force, const PhysDev *phys, const Dims &d, cudaStream_t s);
cudaError_t launch_force(const cplx32 *y_in, cplx32 *force, const PhysDev *phys, const Dims &d, cudaStream_t s);

// Mixed precision keeps the state as double-float pairs: S_hi and S_lo ([inst][7][spec] FP32
// complex each, hi + lo carrying a 48-bit significand), the history and the stage state in FP32.
// Updates of y add the FP32 increment to (hi, lo) with an error-free two-sum; ASM_RHS writes the
// RHS in FP64 to `rhs_out`.
cudaError_t launch_assemble_df(const cplx32 *flux, const cplx32 *y_in, cplx32 *s_hi, cplx32 *s_lo, cplx32 *hist,
                               cplx32 *ystage, cplx64 *rhs_out, const PhysDev *phys, const StepCoef *coef, int op,
                               int stage, const Dims &d, cudaStream_t s, const cplx32 *force = nullptr);
// FP64 spectra <-> (hi, lo) pairs of `count` complex values.
cudaError_t launch_split_state(const cplx64 *in, cplx32 *hi, cplx32 *lo, size_t count, cudaStream_t s);
cudaError_t launch_combine_state(const cplx32 *hi, const cplx32 *lo, cplx64 *out, size_t count, cudaStream_t s);

// Double-float mode (MHD_FP64_DF): state, history and stage state as double-float complex values
// [inst][7][spec]; the RHS, the update and the force spectra in double-float arithmetic; ASM_RHS
// writes the RHS in FP64 to `rhs_out`.
cudaError_t launch_assemble(const cdf *flux, const cdf *y_in, cdf *state, cdf *hist, cdf *ystage, cplx64 *rhs_out,
                            const PhysDev *phys, const StepCoef *coef, int op, int stage, const Dims &d,
                            cudaStream_t s, const cdf *force = nullptr);
cudaError_t launch_force(const cdf *y_in, cdf *force, const PhysDev *phys, const Dims &d, cudaStream_t s);
// FP64 spectra <-> double-float complex values.
cudaError_t launch_split_state(const cplx64 *in, cdf *out, size_t count, cudaStream_t s);
cudaError_t launch_combine_state(const cdf *in, cplx64 *out, size_t count, cudaStream_t s);

// The Adams-Bashforth assembly (ASM_AB2) of `d.batch` instances fused with the inverse z pass of
// the new state: reads the 12 product spectra `flux` [b][12][spec], state, history and the force
// spectra (nullable), updates state and history as launch_assemble does, and writes the z-pass
// output z_out [b][7][N][nk nx] (the layout launch_col_inverse gives the inverse z pass).
// `tile`: columns per block (0 picks).  Mixed mode: s_hi / s_lo the state's parts, `vpt` the
// inverse z pass's radix option.
cudaError_t launch_assemble_iz(const cplx64 *flux, cplx64 *state, cplx64 *hist, const PhysDev *phys,
                               const StepCoef *coef, const cplx64 *force, cplx64 *z_out, const cplx64 *tw,
                               const Dims &d, int tile, cudaStream_t s);
cudaError_t launch_assemble_iz(const cdf *flux, cdf *state, cdf *hist, const PhysDev *phys, const StepCoef *coef,
                               const cdf *force, cdf *z_out, const cdf *tw, const Dims &d, int tile, cudaStream_t s);
cudaError_t launch_assemble_iz(const cplx32 *flux, cplx32 *s_hi, cplx32 *s_lo, cplx32 *hist, const PhysDev *phys,
                               const StepCoef *coef, const cplx32 *force, cplx32 *z_out, const cplx32 *tw,
                               const Dims &d, int tile, int vpt, cudaStream_t s);

// Final reduction of the diagnostic partials of one instance plus the spectral terms; writes
// 24 doubles to `out` (see mhd_api.cu for the order).
// Shell spectra (kernels_spectra.cu).  launch_velocity_x: rho, m (fields 0..3 of [7][z][y][kx],
// one instance) -> u = m / rho -> forward x -> [3][z][y][kx].  launch_shells: one block per shell,
// out[s][5] = (E_u, E_B, sum |k.u_hat|^2, kinetic helicity, magnetic helicity) of shell s,
// dh = i k_x u_hat_x and gh = i k . B_hat on every kept mode.  launch_moments: part[b][2] =
// (sum v^2, sum v^3) of a fixed share of v; launch_absmax: part[b] = max |v| of a fixed share.
int num_shells(int k);
cudaError_t launch_velocity_x(const cplx64 *in, cplx64 *out, const Dims &d, const cplx64 *tw, cudaStream_t s);
cudaError_t launch_shells(const cplx64 *uh, const cplx64 *bh, cplx64 *dh, cplx64 *gh, double *out, const Dims &d,
                          cudaStream_t s);
cudaError_t launch_moments(const double *v, size_t n, double *part, int blocks, cudaStream_t s);
cudaError_t launch_absmax(const double *v, size_t n, double *part, int blocks, cudaStream_t s);

// Tracer particles (kernels_tracers.cu).  Particle data: tr[6][count] = x, y, z, vx, vy, vz (FP64,
// positions in [0, 2 pi)).  launch_tracer_init: velocities = CIC of u = m / rho from the real
// state fields real[7][N^3] (rho, m, B) at the stored positions.  launch_tracer_push: one Boris
// push over coef->dt in the grid field bgrid[3][N^3] (skipped when coef->skip is set).
cudaError_t launch_tracer_init(const double *real, double *tr, long long count, int n, cudaStream_t s);
cudaError_t launch_tracer_push(const double *bgrid, double *tr, long long count, const StepCoef *coef, int n,
                               cudaStream_t s);
cudaError_t launch_tracer_push(const float *bgrid, double *tr, long long count, const StepCoef *coef, int n,
                               cudaStream_t s);

// dpart: kDivbBlocks doubles of scratch for the partial sums of the div B norm.
constexpr int kDivbBlocks = 2 * 152;
cudaError_t launch_diag_finish(const double *part, int nparts, const cplx64 *state,
                               const PhysDev *phys, const TimeState *ts, double *out,
                               const Dims &d, cudaStream_t s, double *dpart);

// Expand one truncated spectrum to the full half-complex layout [N][N][N/2+1] (zeros outside).
cudaError_t launch_expand_spectrum(const cplx64 *in, cplx64 *out, const Dims &d, cudaStream_t s);

// Any instance with a non-zero status -> *flag = 1.
cudaError_t launch_status_any(const TimeState *ts, int batch, int32_t *flag, cudaStream_t s);

}  // namespace mhd
