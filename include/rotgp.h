/*
 * rotgp.h -- C ABI of the GB300 split-step Crank-Nicolson solver for the
 * rotating Gross-Pitaevskii (GP) equation.
 *
 * The method is the one of Kumar, Loncar, Muruganandam, Adhikari and Balaz,
 * "C and Fortran OpenMP programs for rotating Bose-Einstein condensates",
 * Sec. 2: the rotating-frame GP equation in dimensionless form (Eq. 3d in 3D,
 * Eq. 2d in quasi-2D), split into H1 = V + g|psi|^2 (Eq. eq1),
 * H2 = -(1/2) d^2/dx^2 - i Omega y d/dx (Eq. eq2) and
 * H3 = -(1/2) d^2/dy^2 + i Omega x d/dy (Eq. eq3) [+ -(1/2) d^2/dz^2 in 3D],
 * each propagated over the full time step in that order: H1 exactly, the
 * others by Crank-Nicolson (Eq. eqD.9) with the tridiagonal systems of
 * Eqs. eqD.11/eq5.  Imaginary time substitutes i Delta -> Delta and
 * renormalises psi to unit norm after every step.
 *
 * Conventions shared by every entry point
 *  - Grid: n[a] = number of intervals N along axis a (the paper's NX, NY,
 *    NZ); coordinates x_i = -N_x h_x/2 + i h_x, i = 0..N_x (Sec. 2).  psi is
 *    zero on every edge (Dirichlet).  Wave functions crossing the ABI hold
 *    all (N_x+1)(N_y+1)[(N_z+1)] points, edges included, x fastest, as
 *    interleaved complex numbers (re, im) of float or double.
 *  - Ownership: the library allocates and owns every device buffer of a
 *    context.  Caller buffers (src, dst, phase_R, obs) are only read or
 *    written during the call.  The caller owns the CUDA stream it passes.
 *  - Asynchrony: step, set and init calls only enqueue work on the context's
 *    stream.  rotgp_observables, rotgp_get_psi and rotgp_sync synchronise it
 *    and report errors raised on the device since the last synchronisation
 *    (a non-finite norm, ROTGP_ENONFINITE).
 *  - Errors: every int-returning call returns ROTGP_OK (0) or a negative
 *    code below; rotgp_last_error gives a message.  A context is used by one
 *    host thread at a time.
 */
#ifndef ROTGP_H
#define ROTGP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ROTGP_OK 0
#define ROTGP_EINVAL (-1)       /* bad argument                              */
#define ROTGP_ENOMEM (-2)       /* device or host allocation failed          */
#define ROTGP_ECUDA (-3)        /* a CUDA runtime call or launch failed      */
#define ROTGP_ENONFINITE (-4)   /* NaN/Inf norm seen by the step reduction   */
#define ROTGP_EUNSUPPORTED (-5) /* form or shape not available for this
                                   context (see the call)                    */
#define ROTGP_ETIMEOUT (-6)     /* a bounded device wait (TMA load) ran out  */

#define ROTGP_FP64 0 /* complex double throughout                           */
#define ROTGP_FP32 1 /* complex float bulk; norm, energy, mu, rms in double  */

typedef struct rotgp_ctx rotgp_ctx;

/* dim = 2 or 3; n[a] >= 4 intervals; h[a] > 0.  Entries a >= dim ignored. */
typedef struct {
  int dim;
  int n[3];
  double h[3];
} rotgp_grid;

/* Dimensionless physics of Eqs. 3d / 2d: trap anisotropies gamma, nu,
 * lambda (lambda unused in 2D), nonlinearity g (g_2D in 2D, g_3D in 3D),
 * rotation frequency omega, time step dt > 0. */
typedef struct {
  double gamma, nu, lambda, g, omega, dt;
} rotgp_phys;

/* Observables of the current state (Sec. 2, Eqs. e2dr/e3dr and e2d/e3d):
 *  norm      h_x h_y [h_z] sum |psi|^2
 *  mu, energy      real-part forms (Eqs. e2dr/e3dr, alpha = 1 and 1/2),
 *                  kinetic term read as -(1/2) psi_R lap psi_R; if
 *                  sum psi_R^2 < 1e-3 sum |psi|^2 the global phase is first
 *                  rotated by -i
 *  mu_c, energy_c  complex forms (Eqs. e2d/e3d)
 *  rms_*     sqrt(<x^2>), sqrt(<y^2>), sqrt(<z^2>) (0 in 2D), sqrt(<r^2>)
 *  max_density     max |psi|^2
 *  mu4, energy4    the complex forms with fourth-order central differences
 *                  for the derivatives (points beyond the grid read as
 *                  zero), the accuracy of the energies printed in the
 *                  paper's Table 1; mu_c and energy_c use the three-point
 *                  differences of the CN sweeps themselves
 *  step      number of steps taken by this context
 *  vortices  sum of |winding| over plaquettes of the z = 0 plane inside 0.9
 *            of the ellipse R^2 = 6<x^2>, 6<y^2> of that plane (not in the
 *            paper, which counts vortices by eye)
 *  flags     bit 0: Omega >= min(gamma, nu) (rotating-frame potential not
 *            confining) */
typedef struct {
  double norm, mu, energy, mu_c, energy_c;
  double rms_x, rms_y, rms_z, rms_r, max_density;
  double mu4, energy4;
  long long step;
  int vortices;
  int flags;
} rotgp_obs;

/* Per-kernel timing record (rotgp_profile_read). */
typedef struct {
  char name[32];
  long long launches;
  double total_ms;
  double bytes_per_launch; /* algorithmic bytes one launch moves            */
} rotgp_kstat;

/* Line-solver parameters of a context (rotgp_info). */
typedef struct {
  int precision;
  int halo;               /* H: points over which a truncated line carry
                             (forward or backward) is re-solved           */
  int table_len;          /* coefficient entries stored per line          */
  int chunk[3];           /* C: points per pipeline chunk, per axis       */
  int segments[3];        /* independent segments each line is split into */
  int lines_per_lane[3];  /* lines one GPU thread solves together         */
  int ring[3];            /* chunk slots in flight per warp               */
  int stencil_taps[3];    /* taps of the banded-inverse stencil in use,
                             0 when the axis uses the Thomas solve        */
  int warps_per_block[3];
  int fused_xy;           /* 1: H1 and the x and y sweeps run as one tile
                             pass (ROTGP_SOLVER_FUSED)                    */
  int hybrid_cluster[3];  /* CTAs sharing one line in the exact partition
                             solve (ROTGP_SOLVER_HYBRID), 0 if not used   */
  double decay;           /* largest per-point decay of a truncated carry */
  size_t device_bytes;    /* device memory owned by the context           */
} rotgp_solver_info;

/* Create a context for one condensate on the current CUDA device; stream is
 * a cudaStream_t (NULL = legacy default stream).  The state is zero until
 * rotgp_init_analytic or rotgp_set_psi.  When Delta/h^2 is so large that a
 * truncated line carry decays too slowly (chunk halo above 64 points) every
 * sweep takes the exact partition solve (ROTGP_SOLVER_HYBRID); fails with
 * ROTGP_EUNSUPPORTED if that has no tile shape for the line length, or if the
 * Thomas multipliers do not reach their fixed point within 512 points. */
int rotgp_create(const rotgp_grid* grid, const rotgp_phys* phys, int precision,
                 void* stream, rotgp_ctx** out);
void rotgp_destroy(rotgp_ctx* ctx);

/* Message of the last error on ctx (or of the last failed rotgp_create or
 * rotgp_observables_noalloc on this thread when ctx is NULL).  Valid until
 * the next call on ctx. */
const char* rotgp_last_error(const rotgp_ctx* ctx);

/* Change the physics (all fields); rebuilds the per-line tables on the
 * device.  Same limits as rotgp_create. */
int rotgp_set_phys(rotgp_ctx* ctx, const rotgp_phys* phys);
/* Change only Omega (rotation ramps). */
int rotgp_set_omega(rotgp_ctx* ctx, double omega);

/* Initial state of Eq. fun, normalised to unit norm:
 *   psi = (x + i y)/sqrt(pi d_xy^2) exp(-(x^2+y^2)/(2 d_xy^2) + 2 pi i R)
 *   [* (pi d_z^2)^(-1/4) exp(-z^2/(2 d_z^2)) in 3D]
 * function = 1 (one vortex) or 0 (Gaussian: x + i y -> 1).  With
 * random_phase != 0, R(x_i, y_j) in [0,1) is drawn on the device from the
 * counter-based SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014):
 * number n = j (N_x + 1) + i of the stream seeded with `seed`, i.e. the
 * state seed + (n + 1) 0x9E3779B97F4A7C15 through the generator's output
 * mix, top 53 bits scaled by 2^-53.  The same R depends on (i, j) only and
 * is shared by every z plane.  random_phase = 0 leaves the phase out (R = 0).
 * The state is fully determined by (grid, function, seed, d_xy, d_z), so a
 * C caller reproduces a seeded start without any host-side generator.
 * ROTGP_EINVAL for another function value or a width <= 0. */
int rotgp_init_analytic(rotgp_ctx* ctx, int function, int random_phase, unsigned long long seed,
                        double d_xy, double d_z);

/* The same initial state with the random numbers R supplied by the caller:
 * phase_R = host array of (N_x+1)(N_y+1) doubles in [0,1) (x fastest), read
 * during the call; NULL for no random phase. */
int rotgp_init_analytic_field(rotgp_ctx* ctx, int function, const double* phase_R, double d_xy,
                              double d_z);

/* Load a wave function of (N+1)^d points (see conventions) from host or
 * device memory, complex double (src_is_fp64 = 1) or complex float; edge
 * points are ignored.  normalise = 1 renormalises the loaded state to unit
 * norm (h_x h_y [h_z] sum |psi|^2 = 1, applied as the pending scale, as
 * after an imaginary-time step); normalise = 0 keeps the values as they are
 * (real-time runs from a given state).  Synchronises the stream; with
 * normalise = 1 a zero or non-finite norm gives ROTGP_ENONFINITE. */
int rotgp_set_psi(rotgp_ctx* ctx, const void* src, int src_on_device, int src_is_fp64,
                  int normalise);

/* Store the current wave function into (N+1)^d points of host or device
 * memory, complex double or float; synchronises the stream. */
int rotgp_get_psi(rotgp_ctx* ctx, void* dst, int dst_on_device, int dst_is_fp64);

/* The density integrated along z, h_z sum_k |psi(x_i, y_j, z_k)|^2, on the
 * (N_x+1)(N_y+1) plane (x fastest, edges zero) into host or device doubles:
 * the paper's reduced 2D density of a 3D state (Sec. 3, the z-integrated
 * densities compared with 2D lattices); in 2D the density itself.  Applies
 * the pending renormalisation; synchronises the stream. */
int rotgp_column_density(rotgp_ctx* ctx, double* dst, int dst_on_device);

/* Enqueue n split steps in imaginary time (i Delta -> Delta, then
 * renormalisation) or in real time.  n >= 0.  Eq. split with the substeps
 * of Eqs. eq1-eq3 (and z in 3D), each line solved as in Eqs. eqD.9-eqD.11.
 * Real time in complex float keeps the norm to about 1e-12 to 3e-10 per
 * step (the CN map and the H1 rotation are unitary in exact arithmetic;
 * the kernels order their float arithmetic so that rounding adds no
 * systematic gain); in complex double to 1e-16. */
int rotgp_step_imag(rotgp_ctx* ctx, long long n);
int rotgp_step_real(rotgp_ctx* ctx, long long n);

/* n split steps under a time-dependent rotation frequency: step k (k = 0 ..
 * n-1) propagates with Omega = omega[k], held fixed within the step (host
 * array of n doubles, read during the call; imag = 1 imaginary time, 0 real
 * time).  This serves the paper's real-time runs that change Omega (Sec. 3,
 * dynamics from an imaginary-time state) and linear or any other ramps.
 * The line coefficient tables of the x and y sweeps are rebuilt on the
 * device whenever Omega changes (z lines carry no rotation term); after the
 * call the context's Omega is omega[n-1].  The line solver must already be
 * sized for the largest |Omega| of the schedule: ROTGP_EUNSUPPORTED if it
 * is not (create the context with that Omega and lower it first).  The call
 * enqueues the steps and returns. */
int rotgp_step_schedule(rotgp_ctx* ctx, long long n, int imag, const double* omega);

/* Evaluate the observables of the current state; synchronises the stream. */
int rotgp_observables(rotgp_ctx* ctx, rotgp_obs* out);

/* Synchronise the stream and report pending device-side errors. */
int rotgp_sync(rotgp_ctx* ctx);

/* Line-solver parameters chosen for this context. */
int rotgp_info(const rotgp_ctx* ctx, rotgp_solver_info* out);

/* Launch shape of one sweep (axis 0 = x, 1 = y, 2 = z): lines solved per
 * GPU thread (1, or 2 for complex float), chunk length C (8, 16 or 64;
 * C >= the halo H of rotgp_info; complex float takes 8 or 16 with 2 lines
 * per thread, and 8 or 16 (TMA forms, even N_x) or 16 or 64 with one;
 * double takes 16 or 64), ring slots (3 or 4; 5 or 6 too in the TMA forms
 * with one line per thread and chunk 8), warps per block (1..8; the TMA
 * forms size their own blocks: one wave of persistent warps, up to 16 per
 * block, taking 32-line units round-robin) and
 * segments each line is split into (clamped to the number of chunks).
 * The one-line-per-thread TMA forms (chunk 8 or 16) solve the unfolded
 * system psi' = 2 A^-1 psi - psi and serve imaginary-time steps; real-time
 * steps of an axis so tuned run the default two-lines-per-thread form, whose
 * folded weights keep the CN map's norm to float rounding.  Changes speed only: every shape gives results
 * equal up to the truncation bound of the chunked line solver.  Used by the
 * autotuner.  On an axis in the exact partition solve (ROTGP_SOLVER_HYBRID)
 * only `segments` applies: the number of CTAs (1, 2, 4 or 8, one cluster)
 * that share each line; results are equal up to rounding.
 * ROTGP_EINVAL for a shape that is not built or does not fit. */
int rotgp_tune(rotgp_ctx* ctx, int axis, int lines_per_lane, int chunk, int ring,
               int warps_per_block, int segments);

/* Line solver of one sweep (axis 0 = x, 1 = y, 2 = z).
 * ROTGP_SOLVER_THOMAS: the Thomas algorithm on each line (chunked, with the
 *   truncated-carry halo of rotgp_info); every precision.
 * ROTGP_SOLVER_STENCIL: the same CN substep as psi' = (2 A^{-1} - I) psi
 *   with W = 2 A^{-1} - I applied as a banded stencil (its entries decay
 *   geometrically away from the diagonal; the dropped tail is below 2e-10
 *   of the largest weight and the end rows of each line are exact).
 *   Complex float only, and only where rotgp_info reports stencil taps at
 *   create time (ROTGP_EUNSUPPORTED otherwise).
 * ROTGP_SOLVER_FUSED (axis 0 or 1): H1 and the x and y sweeps, both in
 *   stencil form, as one pass over each z plane in tiles with K-point
 *   halos (the result equals the separate stencil sweeps up to float
 *   rounding).  In 2D it is the whole step.  Selecting THOMAS or STENCIL
 *   on axis 0 or 1 turns it off.
 * The stencil and fused forms apply to imaginary-time steps only: real-time
 * steps always use the Thomas form, whose Crank-Nicolson map stays unitary
 * with rounded coefficients (independently rounded stencil weights would
 * let the norm drift by ~1e-7 per step in float).
 * ROTGP_SOLVER_HYBRID: the same Thomas solution of every whole line with
 *   nothing truncated, by a partition method: each line is cut into
 *   segments that run the Thomas recurrences locally from zero carries, the
 *   true carries follow from composing the segments' affine summaries (the
 *   reduced system), and the segments rerun from them.  A line lives in the
 *   shared memory of one CTA or of a cluster of up to 8 CTAs (distributed
 *   shared memory), so each point is read and written once per sweep;
 *   complex float and double, both propagation modes.  It serves long lines
 *   whose carries decay slowly (a truncation halo of more than 16 points),
 *   and it is the only form when they decay too slowly for any truncation
 *   (halo above 64 points).  ROTGP_EUNSUPPORTED when the line is too long
 *   for a cluster of 8 tiles of about 200 KB.
 * A new context uses ROTGP_SOLVER_THOMAS on every axis, except that complex
 * float axes with a halo above 16 points take ROTGP_SOLVER_HYBRID, and every
 * axis does when the halo exceeds 64 points. 
 * The y and z sweeps in stencil form, and the fused pass, stage their
 * tiles with TMA loads whose waits are bounded: a wait that runs out
 * (about 2 s) makes the next synchronising call return ROTGP_ETIMEOUT. */
#define ROTGP_SOLVER_THOMAS 0
#define ROTGP_SOLVER_STENCIL 1
#define ROTGP_SOLVER_FUSED 2
#define ROTGP_SOLVER_HYBRID 3
int rotgp_set_solver(rotgp_ctx* ctx, int axis, int solver);

/* Pick the fastest line-solver forms for this context by timing them.
 * Candidates: every combination of ROTGP_SOLVER_THOMAS / ROTGP_SOLVER_STENCIL
 * per axis that the context supports, and the fused x-y pass with each form
 * of the z sweep; then, for the chosen forms, the lines per lane, chunk
 * length and segment count of each Thomas sweep together, its ring depth,
 * and the segment count of each stencil y/z sweep (as rotgp_tune).  Each candidate runs one warm-up step
 * and then twice `steps` imaginary-time steps from a copy of the current
 * state, timed with CUDA events on the context's stream (the faster repeat
 * counts); the state, its pending renormalisation and the step counter are
 * restored afterwards, and the fastest candidate stays selected.  *choice (if not NULL) receives it as a bit set: bit a =
 * axis a in stencil form, bit 3 = fused x-y pass, bit 4 + a = axis a in the
 * exact partition solve (candidates include every supported combination
 * with it).  Synchronises the stream.
 * ROTGP_EINVAL if steps < 1. */
int rotgp_autotune(rotgp_ctx* ctx, int steps, int* choice);

/* Check of the bounded device waits of the TMA tile passes: runs one CTA
 * whose wait on a shared-memory barrier can never be satisfied (it is armed
 * for 16 bytes that no copy delivers).  The wait must give up by itself
 * after its bound (about 2 s of device time) and the kernel return
 * normally.  ROTGP_OK when it did (*seconds, if not NULL, receives the
 * device time the wait took), ROTGP_ECUDA otherwise.  Synchronises stream. */
int rotgp_check_bounded_wait(void* stream, double* seconds);

/* Per-kernel CUDA-event timing.  While enabled, every kernel launch of the
 * context is bracketed by events on its stream.  rotgp_profile_read
 * synchronises, fills up to max records (one per kernel name), sets *count
 * and clears the accumulated records. */
int rotgp_profile_enable(rotgp_ctx* ctx, int on);
int rotgp_profile_read(rotgp_ctx* ctx, rotgp_kstat* out, int max, int* count);

/* Observables of a wave function held in the caller's device memory, with
 * no device-memory allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- code whose device
 * memory belongs to another allocator, code under a fixed memory budget
 * reserved up front, and monitoring loops that must not add the device
 * synchronisation cudaMalloc/cudaFree can bring.
 *  grid, phys, precision  as for rotgp_create (dt is not used)
 *  psi_device  device pointer to (N_x+1)(N_y+1)[(N_z+1)] complex points in
 *              the ABI layout (complex double for ROTGP_FP64, complex float
 *              for ROTGP_FP32); edge points are read as zero
 *  stream      cudaStream_t to run on; the call synchronises it
 *  out         host struct filled like rotgp_observables, except that step
 *              is 0 and vortices is -1 (not evaluated)
 * Scratch: a file-scope device array of about 448 KiB inside the library, which
 * every GPU that loads the library holds until exit.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current and keeps it for the life of the process; make that
 * first call before any stream capture.  A cudaDeviceReset reloads the
 * library's device image, so calls after a device reset in the same process
 * are not supported.  All
 * calls share the array: calls whose work overlaps on the GPU race and must
 * be ordered by the caller.  At most 33,554,432 grid points; larger grids
 * are rejected with ROTGP_EINVAL (message via rotgp_last_error(NULL)). */
int rotgp_observables_noalloc(const rotgp_grid* grid, const rotgp_phys* phys, int precision,
                              const void* psi_device, void* stream, rotgp_obs* out);

/* ------------------------------------------------------------------ batch
 * Many independent condensates (each its own grid and physics) advanced
 * together.  The paper has no batched form; this serves workloads of many
 * small instances (parameter sweeps).  Each instance is a context on a
 * stream of the batch's own.  A block of n steps of the active instances
 * runs in one of three modes:
 *  ROTGP_BATCH_PERSISTENT  one cooperative kernel launch for all n steps of
 *    every active instance (2D instances of one precision whose whole lines
 *    fit one CTA's shared memory: up to about 1500 points per line in
 *    complex float, 750 in complex double).  Each split step is the exact
 *    line solve (ROTGP_SOLVER_HYBRID) on tiles of 16 whole lines: the CTAs
 *    take the tiles of all instances in turn and meet at grid barriers
 *    between the x and y phases; each barrier wait is bounded (about 2 s of
 *    device time) and a wait that runs out makes rotgp_batch_sync (and the
 *    calls that synchronise) return ROTGP_ETIMEOUT.  The instances' own
 *    solver forms do not apply in this mode.  Results equal, bit for bit,
 *    those of each instance stepped alone with ROTGP_SOLVER_HYBRID on both
 *    axes and one CTA per line (rotgp_tune segments = 1).
 *  ROTGP_BATCH_GRAPH  the instances' own kernels, captured once as a CUDA
 *    graph (fork from the batch stream into the instance streams, join
 *    back) and replayed; results equal those of single contexts bit for bit.
 *  ROTGP_BATCH_DIRECT  the same kernels launched directly.
 * All calls are ordered after earlier work on the caller's stream and
 * before its later work. */
#define ROTGP_BATCH_DIRECT 0
#define ROTGP_BATCH_GRAPH 1
#define ROTGP_BATCH_PERSISTENT 2
typedef struct rotgp_batch rotgp_batch;

/* count instances; grids[i], phys[i] as for rotgp_create; stream = the
 * caller's cudaStream_t.  Errors as rotgp_create (message: NULL batch). */
int rotgp_batch_create(int count, const rotgp_grid* grids, const rotgp_phys* phys,
                       int precision, void* stream, rotgp_batch** out);
void rotgp_batch_destroy(rotgp_batch* batch);
const char* rotgp_batch_last_error(const rotgp_batch* batch);
int rotgp_batch_count(const rotgp_batch* batch);
/* The context of instance `index` (owned by the batch; valid until
 * rotgp_batch_destroy): initial states, I/O, solver controls. */
int rotgp_batch_context(rotgp_batch* batch, int index, rotgp_ctx** ctx);
/* rotgp_autotune on every instance (invalidates captured graphs). */
int rotgp_batch_autotune(rotgp_batch* batch, int steps);
/* n steps of every instance, imaginary (imag = 1) or real time, in `mode`
 * (ROTGP_BATCH_*).  ROTGP_EUNSUPPORTED if the persistent mode does not fit
 * the instances. */
int rotgp_batch_step(rotgp_batch* batch, long long n, int imag, int mode);
/* Synchronise; reports device-side errors of any instance and a timed-out
 * grid barrier of the persistent mode (ROTGP_ETIMEOUT). */
int rotgp_batch_sync(rotgp_batch* batch);
/* rotgp_observables of every instance into out[0 .. count-1]. */
int rotgp_batch_observables(rotgp_batch* batch, rotgp_obs* out);
/* Imaginary time until each instance converges: every check_every steps
 * the active instances' mu is compared with the previous check; instance i
 * is converged when |mu - mu_prev| <= rel_tol |mu| and its vortex count is
 * unchanged, and is then left out of later steps.  Stops after max_steps.
 * steps_out[i] = the steps instance i took; converged_out[i] (if not NULL)
 * = 1 if it converged.  mode as for rotgp_batch_step. */
int rotgp_batch_converge(rotgp_batch* batch, double rel_tol, long long check_every,
                         long long max_steps, int mode, long long* steps_out,
                         int* converged_out);

/* ------------------------------------------------------------- warm start
 * A learned initial state for fast-rotating imaginary-time runs: a
 * convolutional encoder-decoder (684,642 parameters, bfloat16 weights and
 * activations, float accumulation, float master weights and Adam state)
 * that maps the parameters (Omega, g, nu) of a 2D run on a G x G grid of
 * half-width L (points x_j = -L + j 2L/G) to a proposed wave function.  It
 * stands in for the paper's practice (Sec. 1, Sec. 3) of starting a fast
 * rotating run from a lattice converged beforehand at a lower Omega; the
 * proposal only seeds imaginary-time propagation (load it with
 * rotgp_set_psi(..., normalise = 1)), which decides the converged state.
 * The paper has no network; everything here is this library's own.  Input
 * planes: the Thomas-Fermi amplitude of the rotating trap, x / L, y / L,
 * Omega, g / 1000 and (nu - 1) / 0.1; output: 2 L psi on points 0 .. G-1
 * of each axis.  Layout of the flat float parameter vector: per layer i =
 * 0 .. 11, the weights W_i[ky][kx][ci][co] then the bias b_i[co]; layer
 * channels (ci -> co): 6->32, 32->32, 32->64, 64->64, 64->128, 128->128,
 * 128->128, 128->128, 128->64, 64->32, 32->32, 32->2 (3 x 3 convolutions;
 * 2 x 2 mean pooling after layers 1, 3, 5; nearest upsampling with the
 * outputs of layers 5, 3, 1 added before layers 8, 9, 10; ReLU after every
 * layer but the last).  A context serves one CUDA stream and up to
 * max_batch runs per call. */
typedef struct rotgp_ws rotgp_ws;
long long rotgp_ws_param_count(void);
/* grid = G (a multiple of 16, 16 .. 1024); the parameters start at zero. */
int rotgp_ws_create(int grid, int max_batch, void* stream, rotgp_ws** out);
void rotgp_ws_destroy(rotgp_ws* ws);
const char* rotgp_ws_last_error(const rotgp_ws* ws);
/* Parameters to / from a host float array of rotgp_ws_param_count() values
 * (setting them also resets the optimiser state). */
int rotgp_ws_set_params(rotgp_ws* ws, const float* params);
int rotgp_ws_get_params(rotgp_ws* ws, float* params);
/* Proposals for n runs: prm = host array (Omega, g, nu) x n; psi = n ABI
 * wave functions of (G+1)^2 complex double (host or device), edges zero.
 * random_phase != 0 multiplies each by the random phase exp(2 pi i R) of
 * Eq. fun, R drawn from SplitMix64(seed) exactly as rotgp_init_analytic
 * draws it, which keeps the start's symmetry breaking (a smooth proposal
 * alone has to nucleate its vortices by instability).  Synchronises the
 * stream. */
int rotgp_ws_propose(rotgp_ws* ws, int n, const double* prm, double half_width, int random_phase,
                     unsigned long long seed, void* psi, int psi_on_device);
/* One Adam step (learning rate lr, beta1 0.9, beta2 0.999) on the mean
 * squared error between the outputs for prm and 2 L psi of the n target
 * wave functions psi (ABI layout, complex double, host or device); *loss
 * receives the loss before the step.  Synchronises the stream. */
int rotgp_ws_train_step(rotgp_ws* ws, int n, const double* prm, double half_width,
                        const void* psi, int psi_on_device, float lr, double* loss);
/* Loss and its gradient with respect to the parameters for given input
 * planes (host float, [n][G][G][6]) and targets (host float, [n][G][G][2]);
 * grads (host, param_count floats) may be NULL.  For checks of the
 * network's kernels.  Synchronises the stream. */
int rotgp_ws_gradients(rotgp_ws* ws, int n, const void* inputs, const float* targets,
                       double* loss, float* grads);

#ifdef __cplusplus
}
#endif
#endif /* ROTGP_H */
