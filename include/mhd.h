/*
 * mhd.h -- C ABI of the GB300 (sm_103a) pseudo-spectral compressible MHD library.
 *
 * The library evolves the isothermal compressible MHD system of the paper's 3D tests (section
 * "Three dimensional numerical tests", Eqs. density, velocity, Bfield):
 *     d(rho)/dt   = -div(rho u)
 *     d(rho u)/dt = -div[ rho u(x)u + (Cs^2 rho + |B|^2/2) I - B(x)B ] + nu lap(u)
 *     dB/dt       = -div( u(x)B - B(x)u ) + eta lap(B)
 * on the periodic box [0, 2 pi)^3 with N^3 points, pseudo-spectrally (section "Code G-MHD3D":
 * derivatives as i k products in Fourier space, products on the grid), with the 2/3-rule
 * truncation (a mode is kept iff 3|k_x| < N, 3|k_y| < N and 3|k_z| < N) applied to every product
 * and to the initial state, and the explicit Adams-Bashforth time step the paper reports its
 * results with, taken here as second order with variable step (forward Euler on the first step)
 * and a CFL-limited dt:
 *     dt = min( cfl_adv * (2 pi / N) / max_x(|u| + sqrt(Cs^2 + |B|^2 / rho)),
 *               cfl_visc / (max(nu, eta) * k_max^2) ),    k_max = floor((N - 1) / 3)
 * unless a fixed dt is given.
 *
 * Conventions shared by every entry point:
 *   - real fields are float64, x fastest: value (x_i, y_j, z_k) at index (k*N + j)*N + i, with
 *     x_i = 2 pi i / N; a vector field is three such arrays stacked (x, y, z components);
 *   - spectra are forward-normalised: fhat(k) = N^-3 sum_x f(x) exp(-i k.x);
 *   - a pointer flagged `on_device` = 1 is a CUDA device pointer of the current device, else a
 *     host pointer (pageable or pinned); input arrays are only read during the call and never
 *     retained; output arrays are written before the call returns;
 *   - every entry point returns an mhd_status; nothing throws across the ABI; mhd_last_error()
 *     explains.  MHD_EINVAL, MHD_ESTATE and MHD_EBUSY are found before any work is issued and
 *     leave the context usable (mhd_tracers_set has dropped the instance's earlier tracers by
 *     the time it rejects a position), as does MHD_ENONFINITE; after MHD_ENOMEM, MHD_ECUDA or
 *     MHD_ETIMEOUT the context may only be destroyed;
 *   - work is issued on the stream given at init; entry points that return host data
 *     synchronise that stream, mhd_step does not.
 */
#ifndef MHD_H_
#define MHD_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MHD_API __attribute__((visibility("default")))
#else
#define MHD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MHD_OK = 0,
  MHD_EINVAL = 1,     /* bad argument (size, index, null pointer, parameter out of range) */
  MHD_ENOMEM = 2,     /* device allocation failed */
  MHD_ECUDA = 3,      /* a CUDA call failed; see mhd_last_error */
  MHD_ESTATE = 4,     /* call not valid in the current state (e.g. step before set_state) */
  MHD_ENONFINITE = 5, /* an instance produced a non-finite speed or step: it stopped advancing */
  MHD_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  MHD_EBUSY = 7       /* no free slot */
} mhd_status;

typedef enum {
  MHD_FP64 = 0,       /* IEEE double everywhere */
  MHD_FP32_MIXED = 1, /* FFT passes, grid products and the RHS assembly in FP32; the state kept
                         as a double-float pair of FP32 arrays (hi + lo, a 48-bit significand)
                         and advanced with an error-free two-sum; history and RK stage states in
                         FP32; dt computed in FP64 (from an FP32 CFL maximum); the k = 0 modes,
                         whose RHS is exactly zero, held exactly; diagnostics, spectra and
                         set/get of the state in FP64 */
  MHD_FP64_DF = 2     /* FP64-tolerance mode without FP64 arithmetic in the step: every value of
                         the step -- state, history, stage state, the intermediate spectra and the
                         grid products -- is a double-float pair (hi + lo FP32, a 48-bit
                         significand), and every transform, product, RHS term and update is done
                         in double-float arithmetic on the FP32 pipe with error-free
                         transformations (Knuth's TwoSum, an FMA-based TwoProd); the CFL maximum
                         is taken exactly in FP64 at the few grid points that can reach it, and dt
                         is computed in FP64 as in MHD_FP64; diagnostics, spectra and set/get of
                         the state in FP64.  Same memory footprint as MHD_FP64. */
} mhd_precision;

/* Explicit time solvers (paper, section "Code G-MHD3D", Table I; its results use
 * Adams-Bashforth).  Each step takes dt from the CFL condition at the step's start state. */
typedef enum {
  MHD_AB2 = 0, /* Adams-Bashforth 2, variable step, forward Euler on the first step; 1 RHS/step */
  MHD_RK4 = 1, /* classical Runge-Kutta 4; 4 RHS/step */
  MHD_PC = 2   /* AB2 predictor + one trapezoidal (Adams-Moulton 2) corrector; 2 RHS/step */
} mhd_integrator;

typedef struct mhd_ctx mhd_ctx;

typedef struct {
  int32_t n;          /* grid points per axis: a power of two, 16 <= n <= 1024 */
  int32_t batch;      /* independent instances sharing n, >= 1 */
  int32_t precision;  /* mhd_precision */
  int32_t integrator; /* mhd_integrator */
  double dt;          /* > 0: fixed step; <= 0: CFL step */
  double cfl_adv;     /* advective Courant number (default 0.2 when <= 0) */
  double cfl_visc;    /* diffusive number (default 0.5 when <= 0) */
  void *stream;       /* cudaStream_t the library issues all work on; NULL = legacy default */
  /* Optional device allocator (e.g. a framework's caching allocator).  NULL = cudaMalloc/Free.
   * dev_alloc returns NULL on failure; blocks must be at least 256-byte aligned. */
  void *(*dev_alloc)(size_t bytes, void *user);
  void (*dev_free)(void *ptr, void *user);
  void *alloc_user;
} mhd_params;

/* Physical parameters of one instance (paper, section "Normalisation of the MHD equations":
 * Cs = u0 / M_s with u0 = 1; Re = 1 / nu and R_m = 1 / eta for unit density and length). */
typedef struct {
  double nu;  /* kinematic viscosity (mu of Eq. velocity), >= 0 */
  double eta; /* magnetic diffusivity, >= 0 */
  double cs;  /* isothermal sound speed, > 0 */
} mhd_phys;

/* Scalar diagnostics of one instance; <.> is the average over the N^3 grid points
 * (paper, section "Governing equations": mean speed, Mach numbers, Alfven speed; energies of
 * section "for magnetohydrodynamic flow"). */
typedef struct {
  double t;          /* simulated time */
  double dt;         /* step size of the last step (0 before the first) */
  double ke;         /* <rho |u|^2 / 2> */
  double me;         /* <|B|^2 / 2> */
  double eint;       /* <Cs^2 rho ln rho>: ke + me + eint is conserved in the ideal limit */
  double cross_hel;  /* <u . B> */
  double mean_speed; /* <|u|> */
  double mean_bmag;  /* <|B|> */
  double smax;       /* max over the grid of |u| + sqrt(Cs^2 + |B|^2 / rho) */
  double mean_rho;   /* <rho>, the k = 0 density mode */
  double mean_m[3];  /* <rho u> */
  double mean_b[3];  /* <B> */
  double divb_rms;   /* sqrt(<(div B)^2>), spectral */
  double mach_s;     /* <|u|> / Cs */
  double v_a;        /* Alfven speed <|B|> / sqrt(<rho>) (Heaviside-Lorentz units) */
  double mach_a;     /* <|u|> / v_a (0 when v_a = 0) */
  int64_t step;      /* steps taken since set_state */
  int32_t status;    /* MHD_OK, or MHD_ENONFINITE once the instance stopped advancing */
  int32_t reserved;
} mhd_diag;

/* Bytes of device memory a context of this size holds (state, history, two scratch buffers). */
MHD_API size_t mhd_footprint_bytes(int32_t n, int32_t precision, int32_t batch);

/* Create a context for `p->batch` instances of size `p->n`; `phys` points to p->batch entries.
 * Allocates all device memory up front.  MHD_EINVAL on bad sizes or parameters, MHD_ENOMEM when
 * the allocation fails (nothing is leaked), MHD_ECUDA on other CUDA failures. */
MHD_API mhd_status mhd_init(const mhd_params *p, const mhd_phys *phys, mhd_ctx **out);

/* Release everything the context holds (NULL is a no-op). */
MHD_API void mhd_destroy(mhd_ctx *ctx);

/* Text of the last error on this context ("" if none); valid until the next call on it. */
MHD_API const char *mhd_last_error(const mhd_ctx *ctx);

/* Set instance `inst` from real-space rho (N^3), u (3 N^3) and B (3 N^3).  The evolved momentum
 * is m = rho u; every field is transformed and projected onto the 2/3-rule modes.  Resets the
 * instance's time, step count, history and status.  Synchronises the stream. */
MHD_API mhd_status mhd_set_state(mhd_ctx *ctx, int32_t inst, const double *rho, const double *u,
                         const double *b, int32_t on_device);

/* Real-space rho (N^3), m = rho u (3 N^3) and B (3 N^3) of instance `inst`.  Synchronises. */
MHD_API mhd_status mhd_get_state(mhd_ctx *ctx, int32_t inst, double *rho, double *m, double *b,
                         int32_t on_device);

/* The same as mhd_get_state into HOST buffers (page-locked ones reach the link's rate), but
 * returning once the transforms and copies are queued: the copies run on a stream of their own,
 * so they overlap whatever the context queues next (a following mhd_set_state's host-to-device
 * copies, for instance).  The buffers must stay valid and unread until mhd_synchronize returns
 * (mhd_get_state and mhd_destroy also wait for them).  The first call allocates its staging,
 * kept until mhd_destroy: the whole state, 7 N^3 doubles (about 36 % of mhd_footprint_bytes of
 * one instance), when that is at most half of mhd_footprint_bytes, else fewer slabs of N/8
 * z-planes (at least two, then thinner ones).  Errors: MHD_EINVAL (bad instance, null buffer),
 * MHD_ENOMEM (staging), MHD_ECUDA. */
MHD_API mhd_status mhd_get_state_async(mhd_ctx *ctx, int32_t inst, double *rho, double *m, double *b);

/* Real-space right-hand side of instance `inst` at its current state (the inverse transform of
 * the dealiased RHS spectra): d rho/dt (N^3), d m/dt (3 N^3), d B/dt (3 N^3).  The state, the
 * history and the time are unchanged.  Synchronises. */
MHD_API mhd_status mhd_rhs(mhd_ctx *ctx, int32_t inst, double *drho, double *dm, double *db,
                   int32_t on_device);

/* Spectrum of state field `field` (0 rho, 1-3 m, 4-6 B) of instance `inst` in the full
 * half-complex layout: complex (re, im) pairs at [kz][ky][kx] for kz, ky in FFT index order
 * 0..N-1 and kx = 0..N/2, i.e. N * N * (N/2 + 1) pairs; modes outside the 2/3 rule are 0.
 * Synchronises. */
MHD_API mhd_status mhd_get_spectrum(mhd_ctx *ctx, int32_t inst, int32_t field, double *out, int32_t on_device);

/* Advance every instance `nsteps` steps.  Asynchronous: returns once the work is queued.  An
 * instance whose CFL speed or step becomes non-finite stops advancing and reports
 * MHD_ENONFINITE in its diagnostics and from mhd_synchronize. */
MHD_API mhd_status mhd_step(mhd_ctx *ctx, int32_t nsteps);

/* ABC body force rho f on instance `inst` (paper, section "for magnetohydrodynamic flow"):
 * f = amp (A sin kf z + C cos kf y, B sin kf x + A cos kf z, C sin kf y + B cos kf x), added to the
 * momentum equation.  amp = 0 switches it off (the default).  1 <= kf <= k_max.  Synchronises. */
MHD_API mhd_status mhd_set_forcing(mhd_ctx *ctx, int32_t inst, double amp, double A, double B, double C, int32_t kf);

/* Wait for queued work; MHD_ENONFINITE if any instance stopped advancing. */
MHD_API mhd_status mhd_synchronize(mhd_ctx *ctx);

/* Diagnostics of instance `inst` at its current state.  Synchronises. */
MHD_API mhd_status mhd_diagnostics(mhd_ctx *ctx, int32_t inst, mhd_diag *out);

/* Tracer particles of instance `inst` (paper, section "Tracer Particles").  `count` particles are
 * placed at pos[m][3] (HOST, x y z of particle m; wrapped into [0, 2 pi)); their initial velocity is
 * the grid velocity u = m / rho interpolated by cloud-in-cell weights (Eq. tracer_eq, weights
 * normalised by the cell volume).  Every later mhd_step moves them once per step: the grid
 * magnetic field of the step's start state is interpolated to each particle the same way, the
 * velocity is turned by the Boris rotation with q = M = 1 and no electric field (Eq. boris), and
 * the position advances by the new velocity times the step's dt (Eq. euler), wrapped into the box.
 * Tracers are passive: they do not change the flow.  count = 0 removes them.  Positions and
 * velocities are kept in FP64 in device memory; the interpolated field has the context's
 * precision.  Not part of checkpoints; not available on pool contexts (MHD_ESTATE).  Needs a state
 * (MHD_ESTATE otherwise); MHD_EINVAL for a negative count or a non-finite position.  Synchronises. */
MHD_API mhd_status mhd_tracers_set(mhd_ctx *ctx, int32_t inst, int64_t count, const double *pos);
/* Current positions and velocities, HOST arrays [count][3] (either may be NULL).  Synchronises. */
MHD_API mhd_status mhd_tracers_get(mhd_ctx *ctx, int32_t inst, double *pos, double *vel);
/* Number of tracers of instance `inst`, or -1 for a bad context or index. */
MHD_API int64_t mhd_tracers_count(mhd_ctx *ctx, int32_t inst);

/* Velocity-derivative statistics of the hydrodynamic-flow section, all of the dealiased velocity
 * u = m / rho (its spectrum cut to the kept modes), and the helicities and div B of the state: */
typedef struct {
  double theta;    /* theta' = <(div u)^2>^(1/2) */
  double s3;       /* S_3 = <d^3> / <d^2>^(3/2), d = du_x/dx */
  double d2;       /* <d^2> */
  double d3;       /* <d^3> */
  double kin_hel;  /* kinetic helicity <u . curl u> */
  double mag_hel;  /* magnetic helicity <A . B>, A the periodic mean-free vector potential of the
                      Coulomb gauge: A_hat = i k x B_hat / |k|^2 (k != 0), so curl A = B for a
                      solenoidal B */
  double divb_max; /* max over the grid of |div B| */
} mhd_flow_stats;

/* Number of spectral shells of an n^3 grid, round(sqrt(3) k_max) + 1 with k_max = floor((n-1)/3);
 * 0 for an unsupported n. */
MHD_API int32_t mhd_num_shells(int32_t n);

/* Shell spectra of instance `inst` (paper, section "for hydrodynamic flow": kinetic and magnetic
 * energy spectra, theta' and S_3; the helicities and max |div B| of the same state).  Mode k belongs to shell round(|k|); per shell s,
 *   ek[s] = sum |u_hat(k)|^2 / 2,   em[s] = sum |B_hat(k)|^2 / 2
 * over the kept modes of the full spectrum (both k and -k), with f_hat(k) = N^-3 sum f e^{-ik.x},
 * so sum_s em[s] = <|B|^2>/2 and, when rho = 1, sum_s ek[s] = <|u|^2>/2.
 * ek, em: HOST arrays of `nshells` doubles (= mhd_num_shells(n)), or NULL to skip; stats: HOST,
 * or NULL.  Computed on the GPU in FP64 (after combining the mixed-precision state), with a fixed
 * summation order: repeated calls give identical bits.  Uses the context's scratch buffers; do
 * not overlap with a step of the same context.  Synchronises.  MHD_EINVAL for a wrong nshells. */
MHD_API mhd_status mhd_spectra(mhd_ctx *ctx, int32_t inst, double *ek, double *em, int32_t nshells,
                               mhd_flow_stats *stats);

/* Checkpoint support.  The restartable state of an instance is its state spectra, its history
 * (the previous step's RHS spectra), and (t, dt_prev, step).  Both calls move
 * mhd_checkpoint_doubles(ctx) doubles through `buf` (host or device), in a layout private to the
 * library that mhd_restore accepts for the same n and precision.  mhd_checkpoint writes every one
 * of those doubles (unused slots as zeros), so equal states give byte-identical checkpoints.  Both
 * synchronise. */
MHD_API size_t mhd_checkpoint_doubles(const mhd_ctx *ctx);
MHD_API mhd_status mhd_checkpoint(mhd_ctx *ctx, int32_t inst, double *buf, int32_t on_device);
MHD_API mhd_status mhd_restore(mhd_ctx *ctx, int32_t inst, const double *buf, int32_t on_device);

/* Execution options of a context (mhd_set_option; the paper has no counterpart: these choose how
 * the library runs a step, never what it computes, except the radix, which changes FP32
 * rounding).  Changing one discards the captured step.  MHD_EINVAL for an unknown option or a
 * value outside the ranges below, before anything changes.
 *   MHD_OPT_CUDA_GRAPH     1 (default): mhd_step captures one step as a CUDA graph on its first
 *                          call (after one direct step) and replays it; 0: direct launches.
 *                          Profiling (mhd_profile) always uses direct launches.
 *   MHD_OPT_TILE_INV_Z ... MHD_OPT_TILE_FWD_Z: columns per block of the four column FFT passes
 *                          (inverse z, inverse y, forward y, forward z); 0 (default) = chosen by
 *                          the library; otherwise 1..64, rounded down to a power of two
 *                          (mhd_autotune sets these).
 *   MHD_OPT_RADIX_INV_Z ... MHD_OPT_RADIX_FWD_Z: transform radix of the same four passes in the
 *                          mixed mode: 8 or 16 values per thread (two shared-memory stages at
 *                          N = 256 with 16, three with 8); 0 (default) = 16 at N >= 512, else 8.
 *                          FP64 contexts accept and ignore them (their passes use radix 8).
 *   MHD_OPT_FLUX_PIPELINE  1: the fused x pass of the mixed mode at N >= 128 runs as a persistent
 *                          kernel that prefetches the next rows with bulk copies (TMA); 0
 *                          (default): one block per row pair, which measured faster on GB300.
 *                          Results are identical.
 *   MHD_OPT_WAIT_POLLS     poll limit, 0..4194304 (default 4194304), of that pipelined kernel's
 *                          wait for each of its copies.  A wait that runs out makes the block
 *                          record the failure, wait (up to 4194304 polls each) for the copies it
 *                          still has in flight, and return; mhd_synchronize then reports
 *                          MHD_ETIMEOUT and the context may only be destroyed.  0 gives up at
 *                          once, so that a caller can exercise that path without a fault.
 *   MHD_OPT_PERSISTENT     1: the four column passes and the flux pass run as persistent
 *                          kernels, one grid of resident blocks per pass taking tiles from a work
 *                          counter (for batches of small grids: no per-block launch cost, no
 *                          tail); 0 (default): one block per tile.  No block waits on another.
 *                          Results are identical.
 *   MHD_OPT_FUSED_UPDATE   1: an Adams-Bashforth step (MHD_AB2) runs the assembly and update in
 *                          one kernel with the next step's inverse z transform of the new state
 *                          (6 launches a step instead of 7; a step call that does not directly
 *                          follow another adds one plain inverse z pass first).  0 (default):
 *                          separate kernels, which measured faster on GB300 at N >= 256 (the
 *                          fused kernel reads the spectra in column tiles, not coalesced rows).
 *                          Results are identical; RK4 and PC steps are never fused.
 *   MHD_OPT_TILE_FUSED     columns per block of that fused kernel: 0 (default) = chosen by the
 *                          library, otherwise 1..64 rounded down to a power of two and capped by
 *                          the kernel's block size. */
enum {
  MHD_OPT_CUDA_GRAPH = 0,
  MHD_OPT_TILE_INV_Z = 1,
  MHD_OPT_TILE_INV_Y = 2,
  MHD_OPT_TILE_FWD_Y = 3,
  MHD_OPT_TILE_FWD_Z = 4,
  MHD_OPT_FLUX_PIPELINE = 5,
  MHD_OPT_RADIX_INV_Z = 6,
  MHD_OPT_RADIX_INV_Y = 7,
  MHD_OPT_RADIX_FWD_Y = 8,
  MHD_OPT_RADIX_FWD_Z = 9,
  MHD_OPT_WAIT_POLLS = 10,
  MHD_OPT_PERSISTENT = 11,
  MHD_OPT_FUSED_UPDATE = 12,
  MHD_OPT_TILE_FUSED = 13
};
MHD_API mhd_status mhd_set_option(mhd_ctx *ctx, int32_t option, int64_t value);

/* Autotuner of the column FFT passes (the paper has no counterpart: its FFTs are library calls).
 * For each of the four passes (inverse z, inverse y, forward y, forward z), every power-of-two
 * tile width from 1 to 64 columns that fits the thread and shared-memory limits, and in the
 * mixed mode each radix (8 and 16 values per thread), is launched `reps` times (1..100) on the
 * context's own buffers, with the step's shapes (all instances, the working precision), and timed
 * with CUDA events on the context's stream; the fastest choice is set with the MHD_OPT_TILE_* and
 * MHD_OPT_RADIX_* options.  The chosen widths go to tiles[4], the radices to radix[4] and the mean
 * milliseconds per launch to ms[4] (HOST arrays, each may be NULL).  Tile width does not change
 * any result (each column's transform is the same); radix changes the rounding of the FP32 passes
 * only.  The scratch buffers are overwritten; the state is only read.  Synchronises. */
MHD_API mhd_status mhd_autotune(mhd_ctx *ctx, int32_t reps, int32_t *tiles, int32_t *radix, double *ms);

/* Per-kernel device time of mhd_step, for measurement (a service of the library, not of the
 * paper).  While profiling is on, every kernel that mhd_step launches is bracketed by CUDA events
 * on the context's stream.  mhd_profile(ctx, 1) clears the totals and starts recording,
 * mhd_profile(ctx, 0) stops.  mhd_profile_read synchronises and fills up to `max` entries (name,
 * summed milliseconds, launch count), one per kernel kind, and stores how many it wrote in
 * *count.  MHD_EINVAL for a NULL context or count, or a NULL `out` with max > 0. */
typedef struct {
  const char *name; /* static string owned by the library */
  double total_ms;
  int64_t launches;
} mhd_kernel_time;
MHD_API mhd_status mhd_profile(mhd_ctx *ctx, int32_t enable);
MHD_API mhd_status mhd_profile_read(mhd_ctx *ctx, mhd_kernel_time *out, int32_t max, int32_t *count);

/* ---- Serving pools (the paper has no counterpart; a service of the library) ----
 * A pool holds up to p->batch instances ("slots") of one grid size and precision, all resident in
 * device memory, and steps the live ones together (continuous batching): runs are admitted while
 * others are in flight and retired as they finish, and every run's result is bitwise the result
 * it would have alone (instances never interact).  Internally the live instances are kept
 * contiguous: retiring one moves the last live instance into its place, so slot handles stay
 * valid while positions change.  Each live count gets its own captured CUDA graph. */
typedef struct mhd_pool mhd_pool;
/* p->batch = number of slots; p->dt, cfl_*, stream, allocator as for mhd_init. */
MHD_API mhd_status mhd_pool_create(const mhd_params *p, mhd_pool **out);
MHD_API void mhd_pool_destroy(mhd_pool *pool);
MHD_API const char *mhd_pool_last_error(const mhd_pool *pool);
/* Admit a run: state from real-space rho, u, B (as mhd_set_state), parameters `phys`, and a budget
 * of `nsteps` >= 1 steps after which it stops advancing.  *slot receives its handle.  MHD_EBUSY
 * when every slot is in use.  Synchronises. */
MHD_API mhd_status mhd_pool_admit(mhd_pool *pool, const mhd_phys *phys, const double *rho, const double *u,
                                  const double *b, int32_t on_device, int64_t nsteps, int32_t *slot);
/* Advance every live run by k steps (runs at their budget or stopped by a non-finite state do not
 * change).  Asynchronous. */
MHD_API mhd_status mhd_pool_step(mhd_pool *pool, int32_t k);
/* Per slot handle (arrays of p->batch entries): steps taken (-1 for a free slot), status, and
 * whether the run is finished (budget reached or stopped).  Synchronises. */
MHD_API mhd_status mhd_pool_progress(mhd_pool *pool, int64_t *steps, int32_t *status, int32_t *finished);
/* Diagnostics of the run in `slot`.  Synchronises. */
MHD_API mhd_status mhd_pool_diagnostics(mhd_pool *pool, int32_t slot, mhd_diag *out);
/* Copy out the run's real-space rho, m, B (skipped if any pointer is NULL) and free its slot.
 * Synchronises. */
MHD_API mhd_status mhd_pool_retire(mhd_pool *pool, int32_t slot, double *rho, double *m, double *b,
                                   int32_t on_device);
MHD_API mhd_status mhd_pool_info(const mhd_pool *pool, int32_t *live, int32_t *max_slots);

/* Right-hand side of one state that allocates no memory.  For callers that must not call
 * cudaMalloc when they need it (a host framework that already owns the device memory pool, or a
 * latency-bound loop that cannot take the device synchronisation an allocation may bring).  The
 * paper has no counterpart; this is a service of the library.
 *   n               16 or 32 (at most 32): anything else returns MHD_EINVAL before any GPU work
 *   phys            host pointer to the instance's nu, eta, cs
 *   rho, u, b       DEVICE pointers: real-space rho (N^3), u (3 N^3), B (3 N^3) as for
 *                   mhd_set_state (m = rho u, projection onto the 2/3-rule modes)
 *   drho, dm, db    DEVICE pointers receiving what mhd_rhs returns for that state
 *   stream          cudaStream_t to queue the work on (NULL = legacy default stream)
 * Intermediate spectra live in one file-scope device array of about 4.7 MB that every GPU which
 * loads the library keeps until the process exits.  The first call on a device resolves that
 * array's address, uploads its twiddle tables and synchronises the device; make it before any
 * stream capture.  All calls on a device share the array and it keeps the last call's contents,
 * so calls that overlap on the GPU race; each call clears the one word that must start at zero.
 * After the first call on a device, the call queues its work (the parameters too, as kernel
 * arguments) and returns without synchronising: the outputs are valid once the stream has reached
 * that point.  MHD_ECUDA if a CUDA call fails. */
MHD_API mhd_status mhd_rhs_noalloc(int32_t n, const mhd_phys *phys, const double *rho, const double *u,
                                   const double *b, double *drho, double *dm, double *db, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MHD_H_ */
