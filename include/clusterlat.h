/*
 * clusterlat.h -- C ABI of the GB300 lattice scalar-field evolution library
 * (libclusterlat.so).
 *
 * The library evolves nf interacting classical scalar fields on a periodic
 * d-dimensional lattice (d = 1, 2, 3) with the staggered leapfrog of
 * arXiv:0712.0813 Sec. III: field values f live at integer times t, their time
 * derivatives v = f' half a step later; each step advances f by dt with v,
 * evaluates f'' from the new f and advances v by dt.  Sec. II fixes the
 * problem statement (a model file with the potential and its derivatives, a
 * parameter set with lattice size, box, time step, couplings and an expansion
 * switch; outputs computed from the evolving fields); the Abstract fixes the
 * scope (1D/2D/3D, with or without expansion of the universe).
 *
 * Equations (program units; the paper gives none, these are the readings the
 * library implements):
 *   lap f(x)   = dx^-2 sum_d [f(x+e_d) + f(x-e_d) - 2 f(x)],  dx = L/N, periodic
 *   V          = phi^4/4 + sum_i (q_i/2) phi^2 chi_i^2   (field 0 = phi, i>=1 = chi_i)
 *   f_i''      = lap f_i - dV/df_i + (a''/a) f_i          (conformally rescaled)
 *   a''        = (-a'^2 + kappa2 (2 G + 3 V)) / a,  kappa2 = (8 pi/3)(phi0/M_pl)^2
 *   G          = <sum_i sum_d 1/2 ((f_i(x+e_d) - f_i(x))/dx)^2>,  V = <V(f)>
 *   a'(t+dt/2) from the implicit midpoint a'_new - a'_old = dt(-a'_mid^2/a + Q).
 *   Start-up: a(0) = 1, a'(0) = kappa sqrt(K + G + V) with K = <sum 1/2 u^2>,
 *   f'(0) = u + a'(0) f, then half steps for v and a'.
 *
 * Memory: every array argument is a HOST pointer owned by the caller; the
 * library copies in and out and never keeps a caller pointer.  Host arrays are
 * float64 in the layout [field][z][y][x] (x fastest; 2D [field][y][x], 1D
 * [field][x]): nf * N^d contiguous doubles.  Device state is owned by the
 * handle and lives in HBM until ce_free.
 *
 * Errors: every int-returning call returns CE_OK (0) or a negative CE_E* code
 * and sets a thread-local message readable with ce_last_error().  Invalid
 * arguments never touch the GPU.  Device-side failures (non-finite energies,
 * a negative discriminant in the a' update) are latched in a device status
 * word and reported by the next synchronising call.
 *
 * Threading: a handle is not thread-safe; separate handles are independent.
 * Work is issued asynchronously on the handle's stream.
 */
#ifndef CLUSTERLAT_H
#define CLUSTERLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define CE_OK          0
#define CE_EINVAL     -1  /* bad argument or configuration                 */
#define CE_ENOMEM     -2  /* device or host allocation failed              */
#define CE_ECUDA      -3  /* a CUDA runtime call failed (no device, ...)   */
#define CE_ETIMEOUT   -4  /* a bounded device wait gave up                 */
#define CE_ENONFINITE -5  /* NaN/Inf in the global sums or a' update       */
#define CE_ESTATE     -6  /* call out of order (e.g. step before set_fields) */

/* ---- precision ------------------------------------------------------- */
#define CE_F64 0          /* fields, velocities and arithmetic in FP64       */
#define CE_F32 1          /* fields and velocities in FP32; global sums and
                             a, a', a'' in FP64                              */

/* ---- velocity conventions for ce_set_fields / ce_get_fields ----------- */
#define CE_VEL_SYNC      0  /* v = u(t) = f'(t) - (a'/a) f(t), synchronised
                               with f (equals f' without expansion)          */
#define CE_VEL_STAGGERED 1  /* v = f'(t + dt/2), the leapfrog's own velocity;
                               with ce_scalars_t this is a complete state    */

/* ---- kernel selection (ce_config.kernel) ------------------------------ */
#define CE_KERNEL_AUTO    0 /* FP32: z-sweep kernel where it applies; else the
                               row kernel for 2D sides >= 512 and 3D sides >= 256
                               it takes; else the column kernel (3D) or the
                               line-sweep kernel (2D sides >= 320); else generic.  FP64: generic (its two-pass
                               form), or the z-sweep kernel when plan hints
                               (tile_rows, stages, zchunks) are given          */
#define CE_KERNEL_GENERIC 1 /* one thread per site, any d and N              */
#define CE_KERNEL_SWEEP   2 /* 3D z-sweep kernel (CE_EINVAL if it does not apply) */
#define CE_KERNEL_ROWS    3 /* the batched row-sweep kernel on this one lattice:
                               any d, N a multiple of 4 (FP32) / 2 (FP64)      */
#define CE_KERNEL_PLANES  4 /* sweep kernel with plain loads and register
                               neighbours, any N: z-sweeps of warp columns in
                               3D, y-sweeps of warp strips in 2D (CE_EINVAL
                               in 1D)                                          */

/* ---- config flags ---------------------------------------------------- */
#define CE_FLAG_ALLOW_UNSTABLE_DT 1  /* skip the dt < 2/omega_max check       */
#define CE_FLAG_TEST_TMA_STALL    2  /* failure-detection tests only: every plane
                                        the z-sweep kernel loads announces 16 bytes
                                        that never arrive, so its bounded waits run
                                        out (~0.5 ms) and each launch latches
                                        CE_ETIMEOUT; no GPU fault is involved     */

/* Device allocator hooks (optional).  alloc returns a device pointer of at
 * least `bytes` (256-byte aligned) usable on `stream`, or NULL; release
 * returns it.  Both NULL: the library uses cudaMalloc/cudaFree. */
typedef void* (*ce_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*ce_release_fn)(void* ptr, size_t bytes, void* stream, void* ctx);

typedef struct {
  int dims;              /* 1, 2 or 3 (Abstract: 1D/2D/3D)                     */
  int64_t N;             /* sites per side, 3 <= N, N^dims <= 2^34            */
  double L;              /* box side (> 0)                                    */
  double dt;             /* time step (> 0); rejected above 2/omega_max unless
                            CE_FLAG_ALLOW_UNSTABLE_DT                          */
  int nfields;           /* 1..4: field 0 = phi, 1.. = chi_i                  */
  double q[3];           /* couplings q_i of chi_i (>= 0)                     */
  int expansion;         /* 0: a == 1; 1: self-consistent a(t) (Abstract)     */
  double phi0_over_mpl;  /* gravity coupling, kappa2 = 8 pi/3 (phi0/M_pl)^2;
                            <= 0 selects the default 0.342                    */
  double phi0;           /* homogeneous phi used only in the dt check (<= 0: 1) */
  int precision;         /* CE_F64 or CE_F32                                  */
  int kernel;            /* CE_KERNEL_*                                       */
  int flags;             /* CE_FLAG_*                                         */
  int tile_rows;         /* z-sweep tile rows (4, 8 or 16); 0 = automatic     */
  int stages;            /* z-sweep TMA pipeline stages (3..5); 0 = automatic */
  int zchunks;           /* z-sweep chunks per tile column; 0 = automatic     */
  void* stream;          /* cudaStream_t to issue work on; NULL = own stream  */
  ce_alloc_fn alloc;     /* optional device allocator                         */
  ce_release_fn release;
  void* alloc_ctx;
} ce_config;

/* Scale-factor state that, with f(t) and f'(t+dt/2), makes a complete
 * leapfrog state (checkpoint / resume, Sec. II grid images). */
typedef struct {
  double a;              /* a(t)                                              */
  double ap_half;        /* a'(t + dt/2)                                      */
  double app;            /* a''(t)                                            */
  double t;              /* program time                                      */
  int64_t step;          /* full steps taken since the start-up               */
} ce_scalars_t;

/* Outputs at integer time t (Sec. II outputs; definitions are readings). */
typedef struct {
  double K[4];           /* <1/2 u_i^2>, u synchronised (CE_VEL_SYNC)          */
  double G[4];           /* gradient energy of field i                        */
  double V;              /* <V(f)>                                            */
  double E;              /* sum K + sum G + V                                 */
  double a;              /* a(t)                                              */
  double ap;             /* a'(t) = a'(t+dt/2) - dt/2 a''(t)                  */
  double t;
  double friedmann_resid;/* |a'^2/kappa2 - E| / E (0 without expansion)       */
  int64_t step;
} ce_energy_t;

typedef struct ce_sim ce_sim;

/* Create a simulation handle and allocate its device state (f twice for the
 * ping-pong of the fused step, the velocity state twice, small scratch).
 * cfg is read, not kept (stream and allocator hooks are kept).  *out receives
 * the handle.  Errors: CE_EINVAL (bad config, NULL pointers), CE_ENOMEM,
 * CE_ECUDA (no device / CUDA failure). */
int ce_create(const ce_config* cfg, ce_sim** out);

/* Load a state (Sec. II: the program starts from initial conditions set on
 * the lattice; Sec. III: f at integer time, v half a step later).  f, v: host
 * float64, nf * N^dims each, layout above.
 *  mode CE_VEL_SYNC:      v = u(0); runs the start-up (a=1, a'(0) from the
 *                         Friedmann equation, half kick); sc must be NULL.
 *  mode CE_VEL_STAGGERED: f = f(t), v = f'(t+dt/2) and *sc the matching scalars;
 *                         restores a state saved by ce_get_fields exactly.
 * In CE_F32 the values are rounded to float32.  Synchronises.
 * Errors: CE_EINVAL, CE_ECUDA, CE_ENONFINITE (no real a'(0)). */
int ce_set_fields(ce_sim* sim, const double* f, const double* v, int mode,
                  const ce_scalars_t* sc);

/* Advance n >= 0 full steps (Sec. III staggered leapfrog).  Asynchronous on the
 * handle's stream; device-side failures surface at the next synchronising
 * call.  Errors: CE_EINVAL (n < 0), CE_ESTATE (no fields set), CE_ECUDA. */
int ce_step(ce_sim* sim, int64_t n);

/* Block until the handle's stream is idle and report any latched device
 * error (CE_ENONFINITE). */
int ce_synchronize(ce_sim* sim);

/* Per-field mean <f_i> and population variance <(f_i - <f_i>)^2> at the
 * current integer time, FP64 sums.  Sec. II leaves the choice of outputs to
 * the run's parameters; per-field means and population variances are the
 * library's reading of the basic field statistics such a run writes out.
 * mean, var: host arrays of nf doubles, owned by the caller.  Synchronises.
 * Errors: CE_EINVAL (NULL argument), CE_ESTATE (no fields set), a latched
 * device error, CE_ECUDA. */
int ce_means_variances(ce_sim* sim, double* mean, double* var);

/* Energies and scale factor at the current integer time (Sec. II outputs;
 * Abstract: evolution with expansion of the universe).  *out: caller-owned.
 * Synchronises.  Errors: CE_EINVAL, CE_ESTATE, a latched device error, CE_ECUDA. */
int ce_energy(ce_sim* sim, ce_energy_t* out);

/* Copy the state out (Sec. II: the program writes field values on the
 * lattice; Sec. III staggering of f and v).  f, v: caller-owned host float64
 * arrays of nf * N^dims, layout above.
 *  mode CE_VEL_SYNC:      v = u(t) (synchronised); sc may be NULL.
 *  mode CE_VEL_STAGGERED: v = f'(t+dt/2); *sc (required) receives the scalars.
 * Synchronises.  Errors: CE_EINVAL (NULL argument, or sc NULL with
 * CE_VEL_STAGGERED), CE_ESTATE (no fields set), CE_ECUDA. */
int ce_get_fields(ce_sim* sim, double* f, double* v, int mode, ce_scalars_t* sc);

/* The staggered state at n chosen sites, without downloading the lattice (for
 * probing lattices of many GB; no counterpart in the paper).  sites: host
 * array of n linear site indices x + N y + N^2 z in [0, N^dims).  f, v: host
 * float64 arrays of nf * n, field-major (f[i * n + k] is field i at sites[k]);
 * v = f'(t+dt/2) formed exactly as ce_get_fields(CE_VEL_STAGGERED) forms it.
 * *sc (required) receives the scalars.  Synchronises.
 * Errors: CE_EINVAL (NULL argument, n < 0, a site out of range), CE_ESTATE (no
 * fields set), a latched device error, CE_ECUDA. */
int ce_sample_fields(ce_sim* sim, const int64_t* sites, int64_t n, double* f, double* v, ce_scalars_t* sc);

/* Release the handle and its device memory (the end of a run, Sec. II).  Waits
 * for the handle's queued work; a member of a batch leaves the batch unusable.
 * NULL-safe; the handle must not be used afterwards. */
void ce_free(ce_sim* sim);

/* Thread-local description of the last error ("" if none); the string is
 * owned by the library and valid until the next call on this thread.  The
 * paper has no counterpart (its program is run from the command line, Sec. II);
 * this is how the library reports a failed call. */
const char* ce_last_error(void);

/* Bytes of device memory the handle holds (state + scratch). */
int64_t ce_device_bytes(const ce_sim* sim);

/* Which kernel ce_step launches: CE_KERNEL_GENERIC, _SWEEP, _ROWS or _PLANES. */
int ce_kernel_in_use(const ce_sim* sim);

/* The z-sweep launch plan in use: tile rows, pipeline stages and z-chunks
 * (all 0 when the generic kernel runs).  Errors: CE_EINVAL (NULL argument). */
int ce_sweep_plan(const ce_sim* sim, int* rows, int* stages, int* zchunks);

/* Switch the z-sweep launch plan of an existing handle (0 = automatic); the
 * state is kept.  Synchronises.  Errors: CE_EINVAL (no z-sweep kernel on this
 * handle, or no compiled variant matches), CE_ESTATE (member of a batch). */
int ce_replan(ce_sim* sim, int rows, int stages, int zchunks);

/* Binned power spectrum of field `field` at the current integer time.
 * With the unnormalised DFT fhat(n) = sum_x f(x) exp(-2 pi i n.x / N) over the
 * integer modes n (components in (-N/2, N/2]), bin b collects the modes with
 * floor(|n| + 1/2) = b: power[b] = mean of |fhat(n)|^2 over the bin, count[b]
 * = number of modes, k[b] = 2 pi b / L.  The mean field lands in bin 0.
 * (Sec. II: spectra are among the program's outputs; the definition is a
 * convention.)  Host arrays of nbins doubles; 1 <= nbins <= ceil(sqrt(dims)
 * N/2) + 2.  The first call allocates a cuFFT plan and work buffers, kept by
 * the handle.  Synchronises.  Errors: CE_EINVAL, CE_ESTATE, CE_ENOMEM, CE_ECUDA. */
int ce_spectrum(ce_sim* sim, int field, int nbins, double* k, double* power, double* count);

/* Grid image (Sec. II: a complete state from which a run can be resumed).
 * ce_save writes a header (lattice, model, a, a'(t+dt/2), a'', t, step) and
 * f(t), f'(t+dt/2) as float64; ce_load restores it into a handle created with
 * the same dims, N, L, dt, fields, couplings and expansion, so that the
 * continuation is bit-identical to an uninterrupted run.  Both synchronise.
 * Errors: CE_EINVAL (I/O failure, not an image, mismatched lattice), CE_ESTATE. */
int ce_save(ce_sim* sim, const char* path);
int ce_load(ce_sim* sim, const char* path);

/* ---- batches: many lattices, one persistent launch per step ------------
 * A batch groups existing handles (any mix of dimensions and sizes, same
 * precision and number of fields, fields already set) and advances all of
 * them together: each step is ONE launch of a persistent kernel whose CTAs
 * pull work items (row segments of one 2D or 3D lattice, swept along its
 * slowest axis) from a queue, followed, when the batch holds 1D lattices, by
 * one launch that steps all of them (blocks of 16-byte site groups); each
 * lattice keeps its own scale factor, computed by the CTA that completes that
 * lattice's last item or block.  Per site the arithmetic is the
 * same fused staggered-leapfrog step as ce_step (Sec. III).  While a handle
 * belongs to a batch, ce_step and ce_set_fields on it return CE_ESTATE; the
 * read-out calls (ce_energy, ce_get_fields, ...) wait for the batch first.
 * A lattice advanced alone in a batch and inside any mix gives bit-identical
 * results (its items and their summation order do not depend on the mix). */
typedef struct ce_batch ce_batch;

/* sims: n handles; sweep_len: sites per item along the sweep axis (0 = 128);
 * ctas_per_sm: cap on the persistent kernel's resident CTAs per SM, 0..8
 * (0 = as many as fit); stream: cudaStream_t for the batch's work (NULL = its
 * own stream).
 * Errors: CE_EINVAL (mixed precision or field count, N not a multiple of 4
 * (FP32) / 2 (FP64), duplicates), CE_ESTATE (a member without fields or
 * already in a batch), CE_ECUDA. */
int ce_batch_create(ce_sim* const* sims, int n, int sweep_len, int ctas_per_sm, void* stream, ce_batch** out);

/* Advance every member by n >= 0 steps (asynchronous, CUDA graphs of 32). */
int ce_batch_step(ce_batch* b, int64_t n);

/* Wait for the batch and report any member's latched device error. */
int ce_batch_synchronize(ce_batch* b);

/* Per-member status after waiting for the batch: status[k] is CE_OK or the
 * error member k latched on the device (CE_ENONFINITE, CE_ETIMEOUT).  Members
 * evolve independently, so a failed member leaves the others' results valid.
 * status: caller-owned host array of n >= members ints.
 * Errors: CE_EINVAL (NULL, n too small), CE_ECUDA. */
int ce_batch_status(ce_batch* b, int* status, int n);

/* Members, work units per step (items of the persistent kernel plus blocks of
 * the 1D launch), persistent CTAs, total sites. */
int ce_batch_info(const ce_batch* b, int* members, int* items, int* blocks, int64_t* sites);

/* Release the batch (members stay valid with their current state).  NULL-safe. */
void ce_batch_free(ce_batch* b);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int ce_version(void);

/* Allocation-free per-field mean and population variance of field arrays the
 * caller already holds in device memory.  The paper has no counterpart: this
 * call exists for callers that cannot let a library allocate device memory --
 * code whose HBM is owned by another allocator (a framework's caching
 * allocator, or a fixed arena reserved at start-up, where an extra cudaMalloc
 * fails or fragments the pool) and latency-critical loops that cannot afford
 * the implicit device synchronisation of cudaMalloc/cudaFree.
 *   f:         DEVICE pointer to nfields * n values, float32 (precision CE_F32)
 *              or float64 (CE_F64); field i starts at element i * n.
 *   mean, var: DEVICE pointers to nfields doubles each, written by the call.
 *   stream:    cudaStream_t to run on (NULL: the legacy default stream).  The
 *              call is asynchronous; read the outputs after that stream is done.
 * Limits: 1 <= nfields <= 4 and 1 <= n <= 2^34; anything else is CE_EINVAL.
 * Scratch: one static 64 KiB device array inside the library, held by every
 * GPU that loads it until the process exits; the call makes no cudaMalloc,
 * cudaFree or other allocating call.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress): make that first call
 * before any stream capture.  The address is cached per process and per device
 * index for the life of the process: do not call this entry point again after
 * cudaDeviceReset (or anything else that destroys the device's primary
 * context) in the same process.  All calls share the array, so calls that overlap
 * on the GPU (other streams, other threads) race and must be serialised by the
 * caller; each call overwrites every scratch value it reads, so nothing needs
 * clearing between calls.
 * Errors: CE_EINVAL (NULL pointer, limits), CE_ECUDA (set-up or launch). */
int ce_moments_noalloc(const void* f, int precision, int64_t n, int nfields, void* stream,
                       double* mean, double* var);

#ifdef __cplusplus
}
#endif
#endif
