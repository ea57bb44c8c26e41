/*
 * micropolar.h - C ABI of the GB300 micropolar elastoplastic FFT solver.
 *
 * The library solves the periodic micropolar elastoplastic cell problem of
 * Francis, Lebensohn, Pourahmadian, Dingreville (2024) by the FFT-based
 * basic scheme with time stepping (their Algorithm 2), applying the
 * closed-form micropolar radial return (their Algorithm 1) at every voxel.
 * All compute runs in hand-written CUDA kernels for sm_103a; there is no CPU
 * fallback: every entry point that computes returns MP_E_CUDA / MP_E_NO_DEVICE
 * when no GPU is usable.
 *
 * Conventions shared by every entry point
 *   - Grid n[0] = N1 (x1, fastest), n[1] = N2 (x2), n[2] = N3 (x3); voxel
 *     index v = x1 + N1 * (x2 + N2 * x3); voxel size h (cell side N_j h).
 *     Each N_j must be 1 or an even number <= 512 whose prime factors are 2
 *     and 3, else MP_E_UNSUPPORTED_SIZE.
 *   - A second-order tensor is 9 numbers V_kl stored row-major (3k + l),
 *     k, l = 0..2 standing for the paper's 1..3.  e_kl, gamma_kl, t_kl, m_kl
 *     follow the paper's index order (eq. strains, eq. elast_constitutive_aniso).
 *   - Field arrays are voxel-major: value (v, kl) at [9 v + 3 k + l].
 *   - precision (MP_PRECISION_*):
 *     0 = plain FP64: fields, FFTs, Green operator, radial return;
 *     1 = FP32 fields, FFTs, Green operator and trial stresses, with the scalar
 *         solve of the radial return (radius, equivalent stress, plastic
 *         multiplier of eq. trial_stresses2, scale factor) in FP64, the
 *         accumulated plastic strains p, q in FP64, the error measure's sums,
 *         means and ratios (eq. err) in FP64 (the per-voxel norms of FP32
 *         field differences are FP32 quantities and their maxima are exact),
 *         and the homogenized averages accumulated in compensated FP32
 *         pairs (per thread) and folded in FP64 (p, q summed in FP64).
 *         Without a prescribed iteration schedule or a manufactured source, an
 *         increment whose error sets no new low (below 0.99 times the last
 *         one) in 64 iterations while above the tolerance (the FP32
 *         rounding floor) continues in the increment form e^{i+1} = e^i -
 *         Gamma0 * (tau^i - tau^{i-1}); one that stalls there for 128
 *         iterations (or, if longer, twice the longest gap between its
 *         earlier lows) finishes in FP64 in the full form restarted from
 *         the current iterate (an FP64 copy of the cell's state, allocated
 *         at the first such increment) and returns to FP32 for
 *         the next increment (once the increment form has stalled in a
 *         solve, later full-form stalls go to FP64 directly); iters_fp64
 *         counts those FP64 iterations;
 *     2 = as 1, but the level return's radius, square root, multiplier
 *         increment and scale factor are formed in FP32 (the trial
 *         equivalent stress is itself an FP32 quantity); p, q and the sums
 *         as in 1.
 *   - Status codes only; nothing throws or aborts across this boundary.  The
 *     message of the last failure is available from mp_last_error().
 *   - Host pointers are read during the call and not retained.  Output host
 *     buffers are caller-allocated; a NULL output pointer skips that output.
 *   - Device memory is obtained through the mp_alloc callbacks given to
 *     mp_create (e.g. a framework's caching allocator), else cudaMalloc.
 */
#ifndef MICROPOLAR_GB300_H
#define MICROPOLAR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MP_ABI_VERSION 2

typedef enum mp_status {
  MP_OK = 0,
  MP_E_INVALID_ARG = 1,      /* malformed input (NULL, non-positive sizes, t_Y <= 0, ...)   */
  MP_E_INADMISSIBLE = 2,     /* moduli violate eq. energetic_bounds (gamma - beta >= 0 read) */
  MP_E_UNSUPPORTED_SIZE = 3, /* a grid size outside {1} U {even 2^a 3^b <= 512}              */
  MP_E_NOT_CONVERGED = 4,    /* max_iter fixed-point iterations without err <= tol          */
  MP_E_DIVERGED = 5,         /* err non-finite or above div_limit                          */
  MP_E_OOM = 6,              /* device allocation failed                                    */
  MP_E_CUDA = 7,             /* a CUDA runtime call failed                                  */
  MP_E_TIMEOUT = 8,          /* a bounded wait expired                                      */
  MP_E_CANCELLED = 9,        /* request cancelled                                           */
  MP_E_NO_DEVICE = 10        /* no usable CUDA device                                       */
} mp_status;

/* Per-phase isotropic micropolar moduli (eq. stiffnesses_iso) and the
 * yield / hardening parameters of eq. yield_function_f ... radius_2
 * (Tables 1-5 list them in this order).  elastic != 0 marks a phase with
 * infinite yield stresses (it never yields; tY..mH ignored). */
typedef struct mp_phase {
  double lambda, mu, kappa, alpha, beta, gamma;
  double tY, tH, mY, mH, a1, b1;
  int32_t elastic;
  int32_t reserved;
} mp_phase;

/* Error measure of eq. err: 0 = local (eq. err_local), 1 = average (eq. err_average). */
#define MP_ERR_LOCAL 0
#define MP_ERR_AVERAGE 1
/* Reference medium: 0 = phase-volume average <A>, <B> (Algorithm 2),
 * 1 = midrange (min + max) / 2 of each modulus over the phases present,
 * 2 = explicit ref_moduli[6] = (lambda0, mu0, kappa0, alpha0, beta0, gamma0). */
#define MP_REF_MEAN 0
#define MP_REF_MIDRANGE 1
#define MP_REF_EXPLICIT 2
/* Arithmetic of a solve (see the conventions above). */
#define MP_PRECISION_FP64 0
#define MP_PRECISION_MIXED 1
#define MP_PRECISION_FP32_RETURN 2

/* The cell problem (Algorithm 2 inputs). */
typedef struct mp_problem {
  int32_t n[3];
  double h;
  const uint16_t* phase;        /* host, N1*N2*N3 phase ids < n_phases                    */
  int32_t n_phases;
  const mp_phase* phases;       /* host, n_phases                                         */
  int32_t n_steps;              /* load increments; the zero initial state is index 0    */
  const double* time;           /* host, n_steps + 1, strictly increasing                 */
  const double* E;              /* host, (n_steps + 1) * 9 prescribed <e> per time        */
  const double* G;              /* host, (n_steps + 1) * 9 prescribed <gamma> per time    */
  double tol;                   /* equilibrium tolerance epsilon (> 0)                    */
  int32_t err_kind;             /* MP_ERR_*                                               */
  int32_t max_iter;             /* per step; <= 0 means 10000                             */
  int32_t ref_kind;             /* MP_REF_*                                               */
  const double* ref_moduli;     /* 6 values when ref_kind == MP_REF_EXPLICIT             */
  int32_t precision;            /* MP_PRECISION_*: 0 FP64, 1 FP32 fields + FP64 scalars, 2 */
  const int32_t* lockstep_iters;/* optional host n_steps: run exactly these iterations    */
  double div_limit;             /* err above this => MP_E_DIVERGED; <= 0 means 1e6        */
  /* Optional source term of a numerically manufactured solution (Appendix
   * D.1, eq. manufactured_polarization_stress): at time index s the
   * polarizations become tau = t - A0 e - t^m(s), mu = m - B0 gamma - m^m(s).
   * Host arrays of (n_steps + 1) * N1*N2*N3 * 9 values, voxel-major per time
   * (index 0, the zero state, is not read); both NULL (no source) or both
   * given.  The library keeps a device copy of n_steps * N1*N2*N3 * 18
   * values of the field type for the solve. */
  const double* tau_m;
  const double* mu_m;
} mp_problem;

/* Results (caller-allocated host buffers; any pointer may be NULL).
 * Per step s = 1..n_steps (stored at index s - 1): homogenized stress
 * T = <t>, couple stress M = <m>, <e>, <gamma> (9 each), P = <p>, Q = <q>,
 * T_eq = <t_eq(t)>, M_eq = <m_eq(m)>, the last error and the number of
 * fixed-point iterations.  Final-step fields: e, g (gamma), t, m as
 * N1*N2*N3*9 and p, q as N1*N2*N3, all FP64. */
typedef struct mp_result {
  double *T, *M, *Eavg, *Gavg;
  double *P, *Q, *Teq, *Meq, *err;
  int32_t* iters;
  int32_t* iters_fp64;          /* per step: iterations run in FP64 (see mp_batch_solve)  */
  double *e, *g, *t, *m, *p, *q;
  int32_t steps_done;           /* out: steps committed                                   */
  int32_t failed_step;          /* out: 1-based step that failed, 0 if none               */
  double ref_moduli_used[6];    /* out: reference medium actually used                    */
} mp_result;

/* Device-memory callbacks (both may be NULL for cudaMalloc / cudaFree). */
typedef struct mp_alloc {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, size_t bytes, void* user);
  void* user;
} mp_alloc;

typedef struct mp_ctx mp_ctx;
typedef struct mp_rve mp_rve;

/* Library / context ---------------------------------------------------- */

int32_t mp_abi_version(void);

/* Create a context bound to CUDA device `device`.  `alloc` may be NULL.
 * Returns MP_E_NO_DEVICE when the device cannot be used. */
mp_status mp_create(mp_ctx** ctx, int32_t device, const mp_alloc* alloc);
void mp_destroy(mp_ctx* ctx);
/* Message describing the last failure on `ctx` (or a global one for NULL). */
const char* mp_last_error(const mp_ctx* ctx);

/* Validation only (no GPU work): checks sizes, eq. energetic_bounds with the
 * gamma - beta >= 0 reading, yield parameters, load path and reference
 * medium.  Usable without a GPU. */
mp_status mp_validate(const mp_problem* problem, char* message, size_t message_len);

/* Whole solve (Algorithm 2) ---------------------------------------------
 * Copies the problem to the device, runs every load increment (predictor,
 * fixed-point iterations to err <= tol, commit) and copies the requested
 * results back to the host.  `stream` is a cudaStream_t (NULL = default). */
mp_status mp_solve(mp_ctx* ctx, const mp_problem* problem, mp_result* result, void* stream);

/* Device-resident solve in stages (the same computation as mp_solve):
 *   mp_rve_create   validate, allocate the cell's device state, upload
 *                   phase map, phase table and load path;
 *   mp_rve_run      advance up to `n_steps` load increments on the device
 *                   (returns after they completed; the error of each
 *                   fixed-point iteration is read back to decide the loop);
 *   mp_rve_results  copy per-step homogenized results (and the fields of the
 *                   last committed step, if requested) to host buffers;
 *   mp_rve_destroy  release the device state.
 * mp_rve_run returns MP_E_NOT_CONVERGED / MP_E_DIVERGED when a step fails;
 * the state then stays at the failed step. */
mp_status mp_rve_create(mp_ctx* ctx, const mp_problem* problem, mp_rve** rve, void* stream);
mp_status mp_rve_run(mp_rve* rve, int32_t n_steps, void* stream);
mp_status mp_rve_results(mp_rve* rve, mp_result* result, void* stream);
/* Reset to the zero initial state (time index 0) without reallocating. */
mp_status mp_rve_reset(mp_rve* rve, void* stream);
int32_t mp_rve_steps_done(const mp_rve* rve);
/* Total fixed-point iterations run so far (sum over committed and current steps). */
int64_t mp_rve_iterations(const mp_rve* rve);
void mp_rve_destroy(mp_rve* rve);

/* Checkpoint / resume of a device-resident cell between load increments.
 * The committed state of Algorithm 2 is the checkpoint: history h_t, h_m,
 * plastic strains p, q, the next increment's predictor and the converged
 * iterate it extrapolates from, the transform constants, the per-increment
 * result rows, errors and iteration counts, and the increment count.
 * mp_checkpoint with host_buf == NULL stores the required size in *bytes;
 * otherwise it writes the image (at most *bytes) and stores its size.
 * mp_resume loads an image into a cell created from the same problem (grid,
 * precision, phases, load path, tolerance and reference medium are checked
 * through a digest; MP_E_INVALID_ARG otherwise); mp_rve_run then continues
 * exactly as the checkpointed cell would have (bit-identical results).
 * The image is host-endian and tied to this library version. */
mp_status mp_checkpoint(mp_rve* rve, void* host_buf, size_t* bytes, void* stream);
mp_status mp_resume(mp_rve* rve, const void* host_buf, size_t bytes, void* stream);

/* Launch-schedule autotuner (on by default for a new context).  When on,
 * mp_rve_create (and so mp_solve) times the candidate schedules of a new
 * cell shape and precision on the cell's first load increment - pass-A rows
 * per work item (the default, half, a quarter), and for cells with the fused
 * spectral pass that pass or the three separate column passes - keeps the
 * fastest, caches it in the context for later cells of the same shape and
 * resets the cell to its zero state.  Schedules only split the work
 * differently: results agree to rounding.  mp_rve_config writes up to n of
 * {rows per pass-A item, fused spectral pass (1/0), pass-A grid, y grid,
 * z grid, schedule timed or cached (1/0)}. */
mp_status mp_set_autotune(mp_ctx* ctx, int32_t enable);
mp_status mp_rve_config(const mp_rve* rve, int32_t* cfg, int32_t n);

/* Kernel classes of the per-increment work, for launch counts and timings. */
#define MP_KC_FFT_Y_FWD 0 /* y-direction forward transform pass                        */
#define MP_KC_GREEN_Z 1   /* z forward + Green operator + z inverse pass                */
#define MP_KC_FFT_Y_INV 2 /* y-direction inverse transform pass                         */
#define MP_KC_PASS_A 3    /* x inverse, Algorithm 1, error partials, polarization, x fwd */
#define MP_KC_REDUCE 4    /* iteration error reduction                                   */
#define MP_KC_START 5     /* increment start: initial state, predictor pass              */
#define MP_KC_COMMIT 6    /* commit of a converged increment and homogenized averages    */
#define MP_KC_SPECTRAL 7  /* fused pass: y fwd, z fwd, Green operator, z inv, y inv       */
#define MP_KC_COUNT 8

/* Cells whose y and z lengths are 256 (FP32 fields) run classes 0-2 as the
 * one fused launch of class 7; other cells run classes 0-2.
 * Enable / disable per-kernel CUDA-event timing of mp_rve_run (events
 * recorded on the run's stream around every launch of every class; the
 * host waits for each increment's commit while enabled).  Launch counts are
 * kept for every class regardless. */
mp_status mp_rve_profile(mp_rve* rve, int32_t enable);
/* Accumulated milliseconds (every class, while enabled) and launch counts
 * per class, MP_KC_COUNT entries each (either pointer may be NULL);
 * reset != 0 zeroes both afterwards. */
mp_status mp_rve_profile_read(const mp_rve* rve, double* ms, int64_t* launches, int32_t reset);

/* Batched solves -----------------------------------------------------------
 * mp_batch_solve solves `count` independent cell problems (each its own
 * grid, phases, load path, tolerance and precision) together: every round
 * runs one fixed-point iteration of Algorithm 2 for every cell still
 * iterating, in launches shared by all of them, and each cell leaves its
 * loop, commits and starts its next increment on its own error (eq. err).
 * Rounds run in windows of 8 launched back to back: each cell's loop test
 * is taken on the device after every round, a cell whose loop ended skips
 * the window's remaining rounds, and the host reads the window's errors
 * once (commits and starts happen between windows).
 * A cell's results are identical (bit for bit) whichever cells it shares the
 * batch with; they agree with mp_solve's to rounding (mp_solve runs
 * separately compiled single-cell forms of the kernels and sums its error
 * and homogenized-average reductions in another order).  results[i] receives problem i's
 * outputs as mp_solve would write them (results may be NULL for none);
 * per_item[i] (may be NULL) its status.  Returns MP_OK when every problem
 * succeeded, else the status of the first that failed (message from
 * mp_last_error(ctx)).  Device memory for each cell is taken from the
 * context's allocator when the cell is admitted and released when it ends;
 * cells that do not fit wait until earlier ones finish.
 * An FP32 cell whose error has not fallen by 1% in 64 iterations while above
 * its tolerance (the floor set by the rounding of its FP32 transforms) continues
 * the increment in the increment form e^{i+1} = e^i - Gamma0 * (tau^i -
 * tau^{i-1}), whose transforms round relative to the change of the
 * polarization; if that sets no new low for 128 iterations (or twice the
 * longest gap between its earlier lows, if longer), it finishes the
 * increment in FP64 (iters_fp64), in the full form restarted from its
 * current iterate; once that has happened in a cell's solve, its later
 * full-form stalls go to FP64 directly.  A prescribed iteration schedule
 * disables both. */
typedef struct mp_batch_stats {
  int64_t rounds;              /* iteration rounds of the FP32 and of the FP64 engine       */
  int64_t rounds_fp64;
  int64_t voxel_iters;         /* voxels x fixed-point iterations, all cells               */
  int64_t voxel_iters_fp64;    /* ... of them run in FP64                                  */
  int64_t escalations;         /* FP32 increments finished in FP64                         */
  int64_t delta_switches;      /* FP32 increments continued in the increment form          */
} mp_batch_stats;
/* stats (may be NULL) receives the work counters of the call. */
mp_status mp_batch_solve(mp_ctx* ctx, const mp_problem* const* problems, int32_t count,
                         mp_result* results, mp_status* per_item, void* stream, mp_batch_stats* stats);

/* Serving (continuous batching) ---------------------------------------------
 * A server owns one block of device memory (its HBM budget), one stream and
 * one worker thread.  mp_server_submit (thread-safe) validates and copies a
 * problem and queues it; the worker admits queued requests in arrival order
 * whenever the request's device footprint fits the free part of the budget
 * (and fewer than max_resident are resident), and runs rounds of the batched
 * engine above over all resident requests, so requests that arrive while
 * others are on the GPU join the running rounds.  A request's state stays in
 * device memory from admission to completion; its results are written to the
 * mp_result given at submission (which must stay valid until mp_server_wait
 * returns for its ticket), and results are identical to those of the same
 * request solved alone through mp_batch_solve.  mp_server_wait blocks until
 * the request ends (timeout_ms < 0: no limit) and returns its status, or
 * MP_E_TIMEOUT if it has not ended within timeout_ms (the ticket stays
 * valid); each ticket is waited for successfully once.  mp_server_destroy
 * cancels queued and resident requests (MP_E_CANCELLED) and frees the
 * server; no other call may be in progress on the server then.  Messages of
 * the server calls are the calling thread's: mp_last_error(NULL). */
typedef struct mp_server mp_server;
typedef struct mp_server_opts {
  size_t hbm_budget_bytes;  /* device bytes for resident requests; 0 = half of the free memory */
  int32_t max_resident;     /* most requests resident at once; <= 0 means 1024              */
  int32_t reserved;
} mp_server_opts;
typedef struct mp_server_stats {
  int64_t submitted, completed, queued, resident, peak_resident;
  int64_t rounds, voxel_iters;
  size_t budget_bytes, resident_bytes;
} mp_server_stats;
mp_status mp_server_create(mp_ctx* ctx, const mp_server_opts* opts, mp_server** server);
mp_status mp_server_submit(mp_server* server, const mp_problem* problem, mp_result* result,
                           uint64_t* ticket);
mp_status mp_server_wait(mp_server* server, uint64_t ticket, int32_t timeout_ms);
mp_status mp_server_query(mp_server* server, mp_server_stats* stats);
void mp_server_destroy(mp_server* server);

/* Convergence trace: while enabled, mp_rve_run records one row of 7 doubles
 * per fixed-point iteration: (increment, iteration, err, err_e, err_t,
 * err_gamma, err_m) - eq. err and its four per-field terms.
 * mp_rve_trace(rve, 0) stops and discards the trace.  mp_rve_trace_read
 * copies up to `capacity` rows to `out` (may be NULL), returns the number of
 * rows recorded (-1 for a NULL rve) and discards them when clear != 0. */
mp_status mp_rve_trace(mp_rve* rve, int32_t enable);
int64_t mp_rve_trace_read(mp_rve* rve, double* out, int64_t capacity, int32_t clear);

/* Hot-path components on device buffers -----------------------------------
 * Real type of tensor buffers: double for precision 0, float for 1 and 2
 * (precision 2 selects the FP32 level return in mp_radial_return).
 *
 * mp_radial_return: Algorithm 1 at `count` material points.  Inputs e, g
 * (gamma), e_n, g_n, t_n, m_n are count*9 tensors, p_n, q_n count doubles,
 * phase count uint16 ids into `phases` (host table).  Outputs t, m
 * (count*9) and p, q (count doubles).  All pointers are device pointers and
 * must not alias outputs with inputs. */
mp_status mp_radial_return(mp_ctx* ctx, int32_t precision, int64_t count, const uint16_t* phase,
                           int32_t n_phases, const mp_phase* phases, const void* e, const void* g,
                           const void* e_n, const void* g_n, const void* t_n, const void* m_n,
                           const double* p_n, const double* q_n, void* t, void* m, double* p,
                           double* q, void* stream);

/* mp_green_apply: one Lippmann-Schwinger update without the mean, i.e. the
 * Fourier transform of the polarizations (tau, mu), the reference medium's
 * Green operator (eq. micropolar_LippmannSchwinger_iteration) and the
 * inverse transform: outputs the strain and curvature fluctuations e~, g~
 * (zero mean; zero at the Nyquist frequencies).  tau, mu, e_out, g_out are
 * N1*N2*N3*9 device tensors of the precision's real type; ref_moduli[6] on
 * the host.  Uses a device work buffer of 18 complex values per half-
 * spectrum point, obtained from the context's allocator. */
mp_status mp_green_apply(mp_ctx* ctx, int32_t precision, const int32_t n[3], double h,
                         const double ref_moduli[6], const void* tau, const void* mu, void* e_out,
                         void* g_out, void* stream);

/* Allocation-free variant ------------------------------------------------
 * The paper has no counterpart: this is a library-side convenience.
 *
 * mp_green_apply_static computes exactly what mp_green_apply computes, for
 * callers that cannot allocate device memory at the point of the call - for
 * example an application that runs this library inside a fixed device-memory
 * budget reserved up front by another runtime, or a latency-critical loop
 * that must not trigger the implicit device synchronisation or the
 * out-of-memory failures that cudaMalloc / cudaFree can bring.  It calls no
 * allocator at all.  Instead it works in one static device array of
 * MP_STATIC_SCRATCH_BYTES that every GPU loading the library keeps until the
 * process exits: 32 KiB for a status word and the twiddle tables, the rest
 * for the 18-component half spectrum, which limits the grid to
 * (N1 / 2) N2 N3 * 18 * (8 bytes FP32 | 16 bytes FP64) <= 8 MiB - 32 KiB
 * (e.g. 48^3 in FP32, 32^3 in FP64); larger grids return
 * MP_E_UNSUPPORTED_SIZE with a message.
 * The first call on a device looks up the array's device address for that
 * device (with the context's device current); make that first call before
 * any stream capture.  Calls share the array: calls whose GPU work overlaps
 * (other streams or host threads) race on it and must be serialised by the
 * caller.  Arguments as for mp_green_apply; ctx must not be NULL
 * (MP_E_INVALID_ARG), its device is made current for the call and the
 * caller's current device is restored before returning. */
#define MP_STATIC_SCRATCH_BYTES (8u * 1024u * 1024u)
mp_status mp_green_apply_static(mp_ctx* ctx, int32_t precision, const int32_t n[3], double h,
                                const double ref_moduli[6], const void* tau, const void* mu,
                                void* e_out, void* g_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MICROPOLAR_GB300_H */
