/*
 * pic_gb300.h -- C ABI of the GB300 (sm_103a) adaptive electron sub-cycling
 * particle integrator of Tangtartharakul, Chen and Arefiev, "Particle
 * integrator for particle-in-cell simulations of ultra-high intensity
 * laser-plasma interactions" (arXiv 2102.10983).
 *
 * Problem statement (Secs. II-IV): normalized units omega = c = m = |e| = 1
 * (time 1/omega, length c/omega, momentum m c, fields m omega c/|e|); a 1D
 * staggered Yee grid carrying E_y and B_z only; per electron, each macro step
 * dt picks k from the rotation-angle criterion |Psi| <= Psi_max (Sec. IV,
 * Algorithm 1), then takes m = 4^k Boris sub-steps h = dt/4^k (Sec. III,
 * Eqs. eq:p - eq:x), the first with the transitional step (h_old + h)/2, each
 * with E_y and B_z interpolated in time by order-p Lagrange polynomials over
 * the stored field levels (Sec. VI, Eqs. eq:lagrange1-2 - eq:lagrange2-3) and
 * in space by the tent shape function (Sec. III, Eqs. eq:Enp, eq:Bnp).
 *
 * Grid convention: E_y lives on nodes x = i dx at times n dt ("level n"); B_z
 * lives on nodes x = (i + 1/2) dx at times (n + 1/2) dt (uploaded together with
 * E level n).  This is the paper's staggering shifted by half a cell.
 *
 * Conventions of every call:
 *  - Return value: PIC_OK (0) or one of the PIC_E* codes below.  No call
 *    throws; pic_last_error() gives a static, human-readable reason.
 *  - Pointers marked "where" are host pointers (PIC_HOST) or device pointers
 *    of the current CUDA device (PIC_DEVICE).  They are borrowed: the caller
 *    owns them and they need only stay valid until the call returns (host) or
 *    until the work queued on the context's stream has finished (device).
 *  - The context owns its particle store, its field ring and its counters; it
 *    allocates them in pic_create and frees them in pic_destroy.
 *  - All work is queued on the context's stream (a cudaStream_t passed as
 *    void*, NULL = legacy default stream).  Calls with host destinations, and
 *    pic_push_step with a non-NULL stats pointer, synchronize that stream.
 *  - A context is not thread-safe; one host thread drives it at a time.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PIC_OK 0
#define PIC_EINVAL 1    /* bad argument (sizes, orders, pointers, missing levels) */
#define PIC_ENOMEM 2    /* device or host allocation failed                        */
#define PIC_ECUDA 3     /* a CUDA runtime call failed                              */
#define PIC_ERANGE 4    /* particles left the field window this step (frozen)      */
#define PIC_EKMAX 5     /* the criterion was capped at k_max for some particle     */
#define PIC_ETIMEOUT 6  /* a bounded device-side wait gave up                      */

/* memory spaces */
#define PIC_HOST 0
#define PIC_DEVICE 1

/* arithmetic forms */
#define PIC_FP64 0   /* all-FP64 push; matches the FP64 oracle bit for bit       */
#define PIC_MIXED 1  /* FP32 interpolation, rotation and criterion; position kept
                        as an exact integer cell plus an FP32 in-cell offset      */

/* schedules of the push (how uneven sub-cycle counts are spread over warps) */
#define PIC_SCHED_PLAIN 0   /* one thread per particle, no binning               */
#define PIC_SCHED_BINNED 1  /* m = 1 particles streamed; k > 0 particles compacted
                               by warp ballot into per-k queues and drained by
                               warps of equal k                                   */
#define PIC_SCHED_PREDICTED 2 /* binned, and before each launch the particles an
                                 attached predictor (pic_attach_predictor) expects
                                 to take a long sub-cycle (k >= 3) are binned by
                                 predicted k and pushed first (shorter ones are
                                 left to the stream's in-warp compaction); a
                                 particle that sees no field is predicted k = 0
                                 without the network; the criterion still
                                 decides every k                               */

/* per-particle status byte: low 7 bits = k of the last macro step; bit 7 set =
   the particle left the field window and is frozen */
#define PIC_STATUS_LOST 0x80

typedef struct {
  double dt;          /* macro step (the field solver's step), > 0; the mixed
                         form also needs 2^-100 <= dt < 2^100 in FP32           */
  double dx;          /* cell size, > 0                                          */
  double psi_max;     /* rotation-angle threshold Psi_max, > 0 (Sec. IV)         */
  double qm;          /* charge/mass in units of |e|/m; -1 for the electron      */
  int32_t order;      /* Lagrange order p, 1..5 (Sec. VI); p+1 levels are used   */
  int32_t k_max;      /* cap on k, 0..7; m <= 4^k_max                            */
  int32_t precision;  /* PIC_FP64 or PIC_MIXED                                   */
  int32_t field_time; /* 0: sub-step fields at the position time t_n + (j-1)h;
                         1: at the middle of the j-th sub-interval of
                            [t_n - dt/2, t_n + dt/2]                              */
  int32_t schedule;   /* PIC_SCHED_*                                             */
  int32_t heavy_budget; /* binned schedules: Boris sub-steps a long (k >= 3)
                           sub-cycle may take per launch; the rest continues in
                           the next launch while the particle runs behind the
                           stream and then catches up (the same bits either
                           way; a call finishes every particle unless carry
                           is set).  0: 256; < 0: no limit                    */
  int32_t diagnostics; /* PIC_FP64 form: PIC_DIAG_WORK accumulates, per particle,
                          the work of the electric field over every Boris push
                          (App. B; read with pic_work_read); 0: none          */
  int32_t carry;      /* binned schedules, for programs that push one step (or
                         a few) per call, each after uploading the next field
                         level.  0: every call ends with a closing launch that
                         finishes the long sub-cycles its last step deferred.
                         c >= 1: they are carried into the next call instead,
                         where they run beside the next step's stream; a
                         particle may then be left up to c - 1 steps behind a
                         call's last step (ring_levels >= order + 1 + c).
                         While sub-cycles are carried the particle store is
                         mid-step: pic_particles_read, pic_features,
                         pic_predict and pic_attach_predictor first finish them
                         (as pic_finish), as does a pic_push_step whose first
                         step does not follow the last one pushed, and
                         pic_fields_upload refuses to replace a level they
                         still need.  Same bits as carry = 0.                 */
} pic_params;

/* pic_params.diagnostics */
#define PIC_DIAG_WORK 1

typedef struct {
  int64_t k_hist[8];      /* macro steps taken with each k                       */
  int64_t substeps;       /* Boris sub-steps taken (sum of m)                     */
  int64_t n_star;         /* sub-steps of macro steps with k > 0 (Sec. VII)       */
  int64_t clamped;        /* macro steps whose k was capped at k_max              */
  int64_t out_of_window;  /* particles frozen because they left the window        */
  int32_t error;          /* device error word (0 = none)                         */
  int32_t reserved;
} pic_step_stats;

typedef struct pic_ctx pic_ctx;

/* Create a context for up to `capacity` particles and a field window of
 * `window_cells` nodes (a power of two, >= 16) held for `ring_levels` time
 * levels (>= order + 1; more levels let several steps run per call).
 * `stream` is a cudaStream_t (or NULL).  On success *out receives the context.
 * Errors: PIC_EINVAL (parameters out of range), PIC_ENOMEM, PIC_ECUDA. */
int pic_create(const pic_params* prm, int64_t capacity, int64_t window_cells,
               int32_t ring_levels, void* stream, pic_ctx** out);

/* Free everything the context owns.  NULL is accepted. */
int pic_destroy(pic_ctx* ctx);

/* Load n particles (n <= capacity): position x at t_n, momentum (px, py, pz)
 * at t_n - h_old/2, and the status byte (k_prev | PIC_STATUS_LOST); status may
 * be NULL (all k_prev = 0, i.e. h_old = dt).  All arrays have n FP64 (status:
 * uint8) entries in `where` memory.  In PIC_MIXED form x is split on the device
 * into an integer cell and an FP32 offset, and p is rounded to FP32.
 * Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_particles_write(pic_ctx* ctx, const double* x, const double* px, const double* py,
                        const double* pz, const uint8_t* status, int64_t n, int32_t where);

/* Copy the first n particles out (FP64; status as above).  Any output pointer
 * may be NULL to skip it.  Synchronizes the stream when where == PIC_HOST.
 * Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_particles_read(pic_ctx* ctx, double* x, double* px, double* py, double* pz,
                       uint8_t* status, int64_t n, int32_t where);

/* Store field level `level`: Ey = E_y at t = level*dt on nodes i0 .. i0+W-1 and
 * Bz = B_z at t = (level + 1/2) dt on nodes i0+1/2 .. i0+W-1/2 (W = the
 * context's window), each W FP64 values in `where` memory.  The level replaces
 * the oldest one in the ring (slot level mod ring_levels).  (Eqs. eq:Ey,
 * eq:Bz give the staggering; Sec. VI the history the interpolation needs.)
 * With pic_params.carry = c the slot must not hold a level that carried
 * sub-cycles still need (PIC_EINVAL, nothing written): after a call whose
 * last step was `last`, levels last - c + 1 - order .. last.
 * Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_fields_upload(pic_ctx* ctx, int64_t level, int64_t i0, const double* Ey,
                      const double* Bz, int32_t where);

/* Advance all loaded particles through macro steps n .. n+n_steps-1 (each one
 * is Algorithm 1 of Sec. IV with the order-p interpolation of Sec. VI).  Step
 * s needs levels s-p .. s in the ring (error PIC_EINVAL otherwise).  If stats
 * is non-NULL the stream is synchronized, the counters of these steps are
 * returned and reset, and PIC_ERANGE / PIC_EKMAX report frozen or capped
 * particles (the step still completes for all others).  With stats == NULL
 * nothing synchronizes and the counters keep accumulating (pic_stats_read).
 * Errors: PIC_EINVAL, PIC_ECUDA, PIC_ERANGE, PIC_EKMAX, PIC_ETIMEOUT. */
int pic_push_step(pic_ctx* ctx, int64_t n, int64_t n_steps, pic_step_stats* stats);

/* Energy-balance diagnostic (App. B, Eqs. EQ_35A, eq:ke_nosub,
 * eq:work_nosub), FP64 form with diagnostics = PIC_DIAG_WORK: the work the
 * electric field has done on each of the first n particles since
 * pic_particles_write (which zeroes it), summed over every Boris push as
 * (q hp / 2) E' . (v_before + v_after), with hp the push's momentum step
 * (the transitional (h_old + h)/2 or h), E' its field and v = p/gamma before
 * and after it; compare with the kinetic energy gamma - 1.  work: n FP64 in
 * `where` memory.  Errors: PIC_EINVAL (not enabled), PIC_ECUDA. */
int pic_work_read(pic_ctx* ctx, double* work, int64_t n, int32_t where);

/* With pic_params.carry: finish every long sub-cycle carried from the last
 * call (one closing launch, queued on the stream) and return the status bytes
 * to their public form.  Needs the levels of the carried steps, which
 * pic_fields_upload keeps.  With carry >= 2 a particle left behind the last
 * step still takes the criterion of the steps it catches up with: those
 * counts (k histogram, sub-steps) go to the counters that the next
 * pic_stats_read, or pic_push_step with stats, returns.  No-op when nothing
 * is carried (any schedule or form).  Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_finish(pic_ctx* ctx);

/* Read (and optionally reset) the accumulated counters.  Synchronizes. */
int pic_stats_read(pic_ctx* ctx, pic_step_stats* stats, int32_t reset);

/* Replace the stream on which the context queues its work (with carried
 * sub-cycles, after waiting for the old stream). */
int pic_set_stream(pic_ctx* ctx, void* stream);

/* Turn CUDA-event timing of the push on (1) or off (0).  When on, two events
 * recorded on the context's stream bracket the push kernel launch of every
 * step of pic_push_step (not the per-step half-step, binning or predictor
 * kernels; the last step's bracket also holds the call's closing launch).
 * Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_timing_enable(pic_ctx* ctx, int32_t on);

/* Sum of the bracketed durations (milliseconds) and the number of timed steps
 * since the last reset; synchronizes the stream.  Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_timing_read(pic_ctx* ctx, double* total_ms, int64_t* steps, int32_t reset);

/* Set the context's device error word to `word` (queued on the stream), as
 * the give-up path of a bounded device wait does, so that a host program (or
 * a test) can check its handling of PIC_ETIMEOUT without making a device wait
 * run out.  The next pic_push_step with stats, or pic_stats_read, reports it.
 * Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_inject_error(pic_ctx* ctx, int32_t word);

/* Number of kernel launches the context has queued since creation. */
int64_t pic_launch_count(const pic_ctx* ctx);

/* Static reason for the last error on this context (or of pic_create and
 * pic_push_mixed_noalloc when ctx is NULL). */
const char* pic_last_error(const pic_ctx* ctx);

/* ---- learned sub-cycle-count predictor (not in the paper) ----------------
 * An MLP 6 -> 64 -> 64 -> 8 (ReLU; softmax cross-entropy over k = 0..7) that
 * predicts the exponent the criterion of Sec. IV will pick at the next macro
 * step, from phi = (asinh|E_y|, asinh|B_z|, asinh p_x, asinh p_y, asinh p_z,
 * log gamma).  BF16 tensor-core operands, FP32 accumulation and FP32 master
 * parameters (packed: W1[64][6] b1[64] W2[64][64] b2[64] W3[8][64] b3[8]).
 * It never changes a trajectory: the criterion decides every sub-step. */

/* Features of every loaded particle after macro step n (mixed form): E_y and B_z
 * at the particle extrapolated to t_{n+1} from step n's levels (which must
 * still be in the ring), and the particle's momentum.  phi: device, n x 6 FP32.
 * Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_features(pic_ctx* ctx, int64_t n, float* phi);

typedef struct pic_mlp pic_mlp;

/* Attach a predictor to a PIC_SCHED_PREDICTED context: every `every` steps of
 * pic_push_step (and at the first step of each call), the features after the
 * previous step go through the network and the particles it predicts to take
 * k >= 3 are binned by that k into a queue that the launches of the next
 * `every` steps push ahead of the stream.  The predictor must outlive its use
 * by the context.  Errors: PIC_EINVAL. */
int pic_attach_predictor(pic_ctx* ctx, pic_mlp* mlp, int32_t every);

/* Number of packed FP32 parameters (5128). */
int pic_mlp_param_count(void);

/* Create a predictor (He-uniform weights from `seed`, zero biases) whose work
 * is queued on `stream`.  Errors: PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA. */
int pic_mlp_create(uint64_t seed, void* stream, pic_mlp** out);

int pic_mlp_destroy(pic_mlp* mlp);

/* Copy the packed parameters out (set = 0) or in (set = 1; also resets the
 * optimizer state).  buf holds pic_mlp_param_count() floats in `where` memory. */
int pic_mlp_params(pic_mlp* mlp, float* buf, int32_t set, int32_t where);

/* Gradient of the mean cross-entropy over n samples (phi: device n x 6 FP32;
 * label: device n uint8 in 0..7) into grad_out (host, packed) and the loss into
 * loss_out (host).  Either output may be NULL.  Synchronizes. */
int pic_mlp_grad(pic_mlp* mlp, const float* phi, const uint8_t* label, int64_t n,
                 float* grad_out, float* loss_out);

/* One Adam step (beta 0.9 / 0.999) with learning rate lr on the batch; the
 * batch loss (before the step) goes to loss_out (host) if non-NULL. */
int pic_mlp_train_step(pic_mlp* mlp, const float* phi, const uint8_t* label, int64_t n,
                       float lr, float* loss_out);

/* Predicted class (argmax of the logits; ties go to the smaller k) of n
 * samples: pred is device n uint8.  Asynchronous. */
int pic_mlp_infer(pic_mlp* mlp, const float* phi, int64_t n, uint8_t* pred);

/* pic_features of every loaded particle after macro step n followed by
 * pic_mlp_infer, fused into one pass (the features never reach memory): the
 * predictor's class for each particle's next step, in pred (device, one uint8
 * per loaded particle).  The same classes as the two calls.  Queued on the
 * context's stream.  Errors: PIC_EINVAL, PIC_ECUDA. */
int pic_predict(pic_ctx* ctx, const pic_mlp* mlp, int64_t n, uint8_t* pred);

/* ---- batched ensembles (not in the paper) -----------------------------------
 * Many independent problems (each its own dt, dx, Psi_max, q/m, k cap, field-
 * time reading, particle count and field window) advanced together: one store,
 * one persistent launch per macro step (mixed form, binned schedule); all share
 * the Lagrange order p and the window size W.  Particles of ensemble e occupy
 * positions [first_e, first_e + n_e) of the concatenated arrays, in ensemble
 * order. */
typedef struct {
  double dt, dx, psi_max, qm;
  int32_t k_max, field_time;
  int64_t n_particles;
} pic_ensemble;

typedef struct pic_batch pic_batch;

/* Create a batch of n_ens (1..65535) ensembles; window_cells a power of two in
 * [16, 2^28]; ring_levels >= order + 2.  Errors: PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA. */
int pic_batch_create(const pic_ensemble* ens, int32_t n_ens, int32_t order,
                     int64_t window_cells, int32_t ring_levels, void* stream, pic_batch** out);
int pic_batch_destroy(pic_batch* b);

/* Stream chunk length (a multiple of 32 in [32, 8192]), resident blocks per SM
 * (1 .. the kernel's occupancy) and whether multi-step pic_batch_push_step
 * calls are captured into one CUDA graph and launched as such (needs a
 * non-NULL stream). */
int pic_batch_config(pic_batch* b, int32_t chunk, int32_t blocks_per_sm, int32_t use_graph);

/* Sub-steps a long (k >= 3) sub-cycle may take per particle and launch (as
 * pic_params.heavy_budget: the rest continues in the next launch while the
 * particle runs behind the stream, with the same bits; a call finishes every
 * particle).  0: 1024; < 0: no limit.  Errors: PIC_EINVAL. */
int pic_batch_heavy_budget(pic_batch* b, int32_t budget);

/* Load / read all particles, concatenated in ensemble order (FP64 in and out,
 * mixed layout inside; status as for pic_particles_write). */
int pic_batch_particles_write(pic_batch* b, const double* x, const double* px, const double* py,
                              const double* pz, const uint8_t* status, int32_t where);
int pic_batch_particles_read(pic_batch* b, double* x, double* px, double* py, double* pz,
                             uint8_t* status, int32_t where);

/* Level `level` of every ensemble: i0 (host, n_ens) the window origins; Ey and
 * Bz n_ens x W FP64 in `where` memory (ensemble-major).  Same grid convention
 * as pic_fields_upload. */
int pic_batch_fields_upload(pic_batch* b, int64_t level, const int64_t* i0, const double* Ey,
                            const double* Bz, int32_t where);

/* Macro steps n .. n+n_steps-1 of every ensemble (stats: totals over the
 * batch; as for pic_push_step). */
int pic_batch_push_step(pic_batch* b, int64_t n, int64_t n_steps, pic_step_stats* stats);

/* Event timing of each pushed step: on/off; with non-NULL outputs, also return
 * (and reset) the summed milliseconds and the number of timed steps. */
int pic_batch_timing(pic_batch* b, int32_t on, double* total_ms, int64_t* steps);

/* Kernel launches queued so far. */
int64_t pic_batch_launch_count(const pic_batch* b);

/* Pick the stream chunk length and blocks per SM: every candidate runs `steps`
 * macro steps from step n, each from the same saved particle state (restored
 * afterwards); the fastest is kept and returned (ms per step in ms_out).  The
 * levels of steps n .. n+steps-1 must be in the ring.  Allocates a temporary
 * copy of the particle state. */
int pic_batch_autotune(pic_batch* b, int64_t n, int32_t steps, int32_t* chunk_out,
                       int32_t* blocks_out, double* ms_out);

const char* pic_batch_last_error(const pic_batch* b);

/* ---- single-electron studies of Secs. IV-VII ------------------------------
 * Electrons from rest through the Gaussian-enveloped plane wave of Eqs.
 * laser5 - laser3, a = a0 exp(-(xi - xi0)^2 / (2 sigma^2)) sin xi,
 * E_y = B_z = -da/dxi, sampled on the grid (E_y at i dx, n dt; B_z at
 * (i + 1/2) dx, (n + 1/2) dt: the "perfectly propagating PIC" of Sec. III) and
 * pushed with the method (FP64, Algorithm 1, order-p Lagrange in time, tent
 * in space).  Each case runs n_electrons electrons with x0 = j lambda /
 * n_electrons (j = 0 .. n_electrons - 1) for n_steps macro steps. */
typedef struct {
  double a0, xi0, sigma;  /* pulse (normalized units, lambda = 2 pi)                */
  double dt, dx;          /* macro step and cell                                    */
  double psi_max;         /* criterion threshold; a huge value turns sub-cycling off */
  double qm;              /* charge / mass, -1                                       */
  int32_t order, k_max, field_time;
  int32_t n_electrons;    /* 1 .. 256                                                */
  int64_t n_steps;
} pic_study_case;

typedef struct {
  /* maxima over the case's electrons and macro steps: eps_dephasing =
   * |R - 1| with R = gamma - p_x (Sec. IV, Eq. R error); eps_energy =
   * |gamma - gamma_th| / gamma_th with gamma_th = 1 + a^2/2 at the momentum's
   * phase (Eq. gamma error); gamma_max */
  double eps_dephasing, eps_energy, gamma_max;
  double eps_dephasing_first, eps_energy_first, gamma_max_first;  /* electron j = 0 */
  double n_star_mean;     /* N* (sub-steps of macro steps with k > 0, Sec. VII), mean */
  int64_t n_steps;        /* N */
  int64_t n_star_first;   /* N* of electron j = 0                                   */
  int64_t substeps;       /* Boris sub-steps, all electrons                          */
  int64_t k_hist[8];      /* macro steps per k, all electrons                        */
} pic_study_result;

/* Run n_cases (1 .. 65535) study cases on the GPU (host arrays; allocates
 * temporary device memory; synchronizes the stream).  Errors: PIC_EINVAL,
 * PIC_ENOMEM, PIC_ECUDA. */
int pic_study_run(const pic_study_case* cases, int32_t n_cases, pic_study_result* out, void* stream);

/* Allocation-free variant of the binned mixed-precision push (no counterpart
 * in the paper: it exists for host programs that may not call cudaMalloc at
 * push time, e.g. because another framework owns and carves up all device
 * memory, or because a real-time loop must avoid the allocator).  The caller
 * owns every input and output; the weight tables, per-k queues, work cursor
 * and counters live in one fixed file-scope __device__ array of ~12.8 MB that
 * every GPU loading the library holds until the process exits.  Nothing is
 * allocated: no cudaMalloc/cudaFree, no allocating library call.
 *
 *  prm:        as for pic_create; precision must be PIC_MIXED, schedule
 *              PIC_SCHED_BINNED, diagnostics and carry 0 (every call
 *              finishes its particles).
 *  n_particles <= 65,536 (the size the static queues hold); larger counts are
 *              rejected with PIC_EINVAL.
 *  cell, frac, px, py, pz, status: device arrays of n_particles entries in the
 *              mixed layout (x = (cell + frac) dx, frac in [0, 1); p FP32;
 *              status byte as in pic_particles_write), updated in place.
 *  Ey_levels, Bz_levels, level_i0: host arrays of order + n_steps entries;
 *              entry r describes level n0 - order + r: device pointers to
 *              window_cells FP32 values of E_y (t = level dt) and B_z
 *              (t = (level + 1/2) dt), node i stored at index
 *              i & (window_cells - 1), the window being nodes
 *              [level_i0[r], level_i0[r] + window_cells).
 *  n0, n_steps: macro steps n0 .. n0 + n_steps - 1 are taken.
 *  stream:     cudaStream_t (or NULL); all work is queued on it.
 *  stats:      optional; if non-NULL the stream is synchronized and the
 *              counters of this call are returned (PIC_ERANGE / PIC_EKMAX as
 *              for pic_push_step).  With stats == NULL nothing synchronizes
 *              (except a first call per key, below).
 * Set-up: the first call on a device looks up the scratch array's device
 * address (cudaGetSymbolAddress); the first call with each (order,
 * field_time) builds that pair's weight table in the array and synchronizes
 * the stream once.  Make those first calls before any stream capture.  Tables
 * are never rewritten, so changing the parameters between calls is safe.
 * Every call shares the array and finds the previous call's contents; the
 * call clears what must start at zero.  Calls that run concurrently on the GPU
 * (other streams, other host threads) race on the array and must be
 * serialized by the caller.
 * A bounded device wait that gives up (PIC_ETIMEOUT) leaves part of the
 * particles unpushed.  It sets an error word in the array that stays set
 * until a call with stats != NULL reports it, so the give-up of an
 * asynchronous call (stats == NULL) is returned by the next call that passes
 * stats.
 * Errors: PIC_EINVAL, PIC_ECUDA, PIC_ERANGE, PIC_EKMAX, PIC_ETIMEOUT. */
int pic_push_mixed_noalloc(const pic_params* prm, int64_t n_particles, int32_t* cell,
                           float* frac, float* px, float* py, float* pz, uint8_t* status,
                           const float* const* Ey_levels, const float* const* Bz_levels,
                           const int64_t* level_i0, int64_t window_cells, int64_t n0,
                           int64_t n_steps, void* stream, pic_step_stats* stats);

/* Set the error word of pic_push_mixed_noalloc's array on the current device
 * to `word` (queued on `stream`), as a bounded device wait that gives up does,
 * so that a host program can check its handling of PIC_ETIMEOUT without making
 * a device wait run out.  Errors: PIC_ECUDA. */
int pic_noalloc_inject_error(int32_t word, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_H */
