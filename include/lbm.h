/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D2Q9 lid-driven cavity library.
 *
 * The method is the lattice Boltzmann scheme of Xiang & Shi, "Flow Simulation of Lid-Driven
 * Rectangular Cavity by Using Lattice Boltzmann Method" (arXiv 2211.05009):
 *   Sec. 2.1  Eq. 1 (BGK collision + streaming), Eq. 2 (equilibrium), Eq. 3 (moments),
 *             Eq. 5 (nu = c_s^2 (tau - 1/2) dt);
 *   Sec. 2.2  (i) initial state, (ii) non-equilibrium-extrapolation walls and moving lid,
 *             (iii) Eq. 6 steady-state criterion;
 *   Sec. 3    c = 1, dx = dt = 1, lid speed U; Table 1 / Table 2 stream-function post-processing;
 *   Sec. 3.3  observing-point time series.
 *
 * Geometry: nx nodes along x (the cavity width L = nx), ny nodes along y (height, ny = nx*Ar).
 * The walls are the outer ring of nodes (x = 0, x = nx-1, y = 0, y = ny-1); the lid is the top
 * row y = ny-1 and moves along +x.  Fields exchanged through this ABI are row-major
 * [ny][nx] FP64 with y = 0 at the bottom; population fields are [9][ny][nx] FP64 in the
 * velocity order 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *
 * Conventions for every call:
 *  - The return value is LBM_OK (0) or one of the LBM_E* codes below; lbm_last_error() gives the
 *    detail.  No call aborts the process, traps on the GPU or prints.
 *  - The context owns its device state (populations, velocity snapshot, reduction scratch).
 *    Output buffers belong to the caller.  A "buffer" argument may be device memory, or host
 *    memory (pageable or pinned); the library finds out which and copies as needed.
 *  - Work is queued on the context's CUDA stream (lbm_set_stream; default: the legacy stream)
 *    and calls return without waiting, except the ones documented as synchronising (those that
 *    return host scalars, and any call given host buffers).
 *  - One host thread at a time per context.  Contexts are independent.
 *  - There is no CPU fallback: without a usable CUDA device lbm_create returns LBM_ECUDA.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes and types */
#define LBM_OK 0
#define LBM_EINVAL 1    /* bad argument: nx or ny < 3, tau <= 1/2, NULL where not allowed ...   */
#define LBM_ENOMEM 2    /* device or host allocation failed (allocator hook included)           */
#define LBM_ECUDA 3     /* a CUDA runtime call failed; the message names it                     */
#define LBM_EDIVERGED 4 /* the mass or the Eq. 6 residual became NaN or Inf                      */
#define LBM_ETIMEOUT 5  /* a bounded device-side wait ran out                                    */
#define LBM_ENOTREADY 6 /* the value does not exist yet (no residual before the first 100 steps) */
#define LBM_EIO 7       /* checkpoint file could not be written, read or did not match          */
#define LBM_ETOOBIG 8   /* grid too large for the fixed scratch of lbm_stream_function_static   */

/* Storage type of the populations.  Arithmetic is FP64 for LBM_F64 and FP32 otherwise.
 * The *S types (and LBM_F64) store the shifted deviation g_j = f_j - w_j instead of f_j.
 * LBM_Q16S (no counterpart in the paper, which fixes no precision) stores, per population, a
 * 16-bit code of h_j = g_j - w_j rho_ref: the deviation from the rest state at a reference
 * density 1 + rho_ref that follows the cavity's mean density (set from the mass at every
 * 100-step checkpoint, so the slow mass change of the Sec. 2.2 (ii) walls does not use up the
 * range).  Code = sign, 2-bit exponent E, 13-bit mantissa M of a = |h_j| / S_j:
 * a = M 2^-15 (E = 0) or (2^13 + M) 2^(E-16) (E = 1..3), rounded to nearest, ties to even.
 * S_j is a power of two fixed at creation from the lid speed: 2 S_j = the power of two at or
 * above K_j w_j max(|U|, 0.01), K = 2 (rest), 5 (axes), 11/2 (diagonals) -- above the largest
 * deviations met in lid-driven cavities from Re 74 to 8000.  A value beyond the largest code (2 - 2^-13) S_j
 * saturates; a checkpoint step (every 100th) that stores a saturated code reports a non-finite
 * residual (LBM_EDIVERGED).  13-bit precision over the range that carries the flow, against
 * binary16's 10: in the 2048^2, Re 8000, U 0.05 cavity the velocity stays within 1e-3 U of the
 * FP64 run where binary16 and bfloat16 do not.  Single cavities only (lbm_batch_create rejects
 * it). */
typedef enum {
    LBM_F64 = 0,   /* g_j = f_j - w_j in FP64                              */
    LBM_F32 = 1,   /* f_j in FP32                                          */
    LBM_F32S = 2,  /* g_j = f_j - w_j in FP32                              */
    LBM_F16S = 3,  /* g_j in IEEE binary16                                 */
    LBM_BF16S = 4, /* g_j in bfloat16                                      */
    LBM_Q16S = 5   /* h_j = g_j - w_j rho_ref in the 16-bit code above    */
} lbm_dtype;

/* lbm_create_ex flags */
#define LBM_FLAG_LID_CORNERS_MOVING 1u /* the two top corner nodes move with the lid (default: at rest) */

#define LBM_MAX_PROBES 4
#define LBM_RESIDUAL_INTERVAL 100 /* Eq. 6 compares velocity fields 100 steps apart */

typedef struct lbm_ctx lbm_ctx;

typedef struct {
    int nx, ny;          /* nodes, walls included                                     */
    long pitch;          /* device row pitch in elements (>= nx)                      */
    double tau;          /* relaxation time of Eq. 1                                  */
    double nu;           /* (tau - 1/2)/3, Eq. 5                                      */
    double U;            /* lid speed                                                 */
    double Re;           /* U nx / nu                                                 */
    int dtype;           /* lbm_dtype                                                 */
    unsigned flags;      /* LBM_FLAG_*                                                */
    long step;           /* time steps taken since the state was initialised/loaded   */
    size_t device_bytes; /* device memory the context holds                           */
    int launch_config;   /* launch shape of the step kernel (lbm_set_launch_config)   */
} lbm_info;

/* ------------------------------------------------------------------ lifetime */

/* Create a cavity of nx x ny nodes for Reynolds number Re = U L / nu with L = nx (Sec. 1) and
 * lid speed U_lid (Sec. 2.2 ii); nu = U nx / Re and tau = 3 nu + 1/2 (Eq. 5, c_s^2 = 1/3).
 * The state is initialised per Sec. 2.2 (i): rho = 1, u = 0 except u_x = U on the lid, f = f^eq.
 * Errors: LBM_EINVAL (nx < 3, ny < 3, Re <= 0, tau <= 1/2, out == NULL, unknown dtype),
 * LBM_ENOMEM, LBM_ECUDA.  On failure *out is NULL and lbm_last_error(NULL) holds the reason. */
int lbm_create(int nx, int ny, double Re, double U_lid, lbm_dtype dtype, lbm_ctx **out);

/* As lbm_create, with LBM_FLAG_* flags.  The library turns Re into tau exactly as lbm_create does
 * (Re = U L / nu with L = nx, Sec. 1; tau = 3 nu + 1/2, Eq. 5), so a caller that wants a flag
 * still never computes tau.  Errors: those of lbm_create, and LBM_EINVAL for an unknown flag. */
int lbm_create_flags(int nx, int ny, double Re, double U_lid, lbm_dtype dtype, unsigned flags,
                     lbm_ctx **out);

/* As lbm_create with tau given directly and LBM_FLAG_* flags. */
int lbm_create_ex(int nx, int ny, double tau, double U_lid, lbm_dtype dtype, unsigned flags,
                  lbm_ctx **out);

/* Release everything the context holds (waits for its queued work).  NULL is a no-op. */
void lbm_destroy(lbm_ctx *ctx);

/* Message of the last failed call on ctx, or of the last failed lbm_create* on this thread when
 * ctx is NULL.  Valid until the next call on the same context/thread. Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Queue all later work of ctx on the given cudaStream_t (e.g. PyTorch's current stream).
 * NULL selects the legacy default stream.  Waits for work already queued on the old stream. */
int lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* Device allocator hook used by every later lbm_create*: alloc(bytes, user) returns device
 * memory or NULL (-> LBM_ENOMEM); release(ptr, user) frees it.  Pass NULLs for cudaMalloc. */
int lbm_set_allocator(void *(*alloc)(size_t bytes, void *user),
                      void (*release)(void *ptr, void *user), void *user);

int lbm_get_info(const lbm_ctx *ctx, lbm_info *info);

/* ------------------------------------------------------------------ the time step */

/* Advance n >= 0 time steps of Eq. 1 with the Sec. 2.2 (ii) walls: for every node pull
 * f_j(x - c_j) (streaming), form rho and u (Eq. 3) and collide towards f^eq (Eq. 2); wall nodes
 * take f^eq(rho_f, u_w) + (1 - 1/tau)[f(x_f) - f^eq(rho_f, u_f)] from their inner neighbour
 * x_f.  One fused kernel per step.  After every step whose global index is a multiple of 100
 * the library also forms, in FP64, the mass sum rho and the Eq. 6 residual against the velocity
 * field of 100 steps earlier, and samples the probes (lbm_probe).  Asynchronous.
 * Errors: LBM_EINVAL (n < 0), LBM_ECUDA. */
int lbm_step(lbm_ctx *ctx, long n);

/* Run until the Eq. 6 residual (checked every 100 steps) drops below tol, or max_steps steps
 * have been taken.  *steps_done (may be NULL) receives the steps taken in this call.  The host
 * reads each checkpoint one 100-step chunk behind the GPU (no stall); it stops once two
 * consecutive checkpoints are below tol, so the returned state itself satisfies the criterion
 * (lbm_residual < tol).  Synchronising.  Returns LBM_OK when converged, LBM_ENOTREADY when
 * max_steps ran out first, LBM_EDIVERGED on NaN/Inf. */
int lbm_run_to_residual(lbm_ctx *ctx, double tol, long max_steps, long *steps_done);

/* ------------------------------------------------------------------ launch shapes */

/* The fused step kernel has several launch shapes (rows per thread, warps per block, register
 * budget).  They compute bitwise-identical populations; only speed differs (the FP64 checkpoint
 * sums may differ in the last bits, since the partial sums are grouped by block). */
int lbm_launch_config_count(void);

/* Select shape cfg in [0, lbm_launch_config_count()).  Synchronising.  LBM_EINVAL if out of range. */
int lbm_set_launch_config(lbm_ctx *ctx, int cfg);

/* Time every shape on a scratch context of the same size (the caller's state is not touched; the
 * scratch needs as much device memory as ctx): three rounds over all shapes of steps_per_trial
 * (>= 2) plain steps and two checkpoint steps each, best time per shape, and select the shape
 * with the lowest cost of a 100-step interval (99 plain + 1 checkpoint).  *best / *best_glups
 * (either may be NULL) receive the choice and its step rate in 1e9 lattice updates per second.
 * Synchronising. */
int lbm_autotune(lbm_ctx *ctx, int steps_per_trial, int *best, double *best_glups);

/* ------------------------------------------------------------------ observables */

/* Macroscopic fields (Eq. 3) of the current state into caller buffers [ny][nx] FP64, any of
 * which may be NULL.  Wall nodes report (rho_f, u_w), the moments their populations carry. */
int lbm_moments(lbm_ctx *ctx, double *rho, double *ux, double *uy);

/* Replace the state by f = f^eq(rho, u) node by node (Sec. 2.2 i generalised to a given field,
 * e.g. a warm start).  Inputs [ny][nx] FP64; resets the step count and the Eq. 6 snapshot. */
int lbm_set_moments(lbm_ctx *ctx, const double *rho, const double *ux, const double *uy);

/* lbm_set_moments with options.  LBM_INIT_NEQ (no counterpart in the paper; a consistent warm
 * start after the first-order Chapman-Enskog expansion of BGK): the post-collision state becomes
 *   f*_j = f^eq_j(rho, u) + (1 - 1/tau) f^neq_j,
 *   f^neq_j = -tau w_j rho / c_s^2 (c_ja c_jb - c_s^2 delta_ab) d_a u_b,   c_s^2 = 1/3,
 * with d_a u_b from central differences inside and three-point one-sided differences on the ring
 * (both exact for quadratic fields), so the start already carries the stress of its velocity field.
 * The moments are still (rho, u).  flags = 0 is lbm_set_moments.  LBM_EINVAL for unknown flags. */
#define LBM_INIT_NEQ 1
int lbm_set_moments_ex(lbm_ctx *ctx, const double *rho, const double *ux, const double *uy, int flags);

/* Current post-collision populations as FP64 f_j (not deviations), [9][ny][nx]. */
int lbm_get_populations(lbm_ctx *ctx, double *f);

/* Replace the populations (FP64 f_j, [9][ny][nx]); rounded to the storage type.  The step count
 * and snapshot are kept.  Non-finite input is accepted and shows up as LBM_EDIVERGED later. */
int lbm_set_populations(lbm_ctx *ctx, const double *f);

/* Eq. 6 residual of the latest 100-step pair (host scalar, synchronising).
 * LBM_ENOTREADY before the first 100 steps; LBM_EDIVERGED (and *r = NaN) if non-finite. */
int lbm_residual(lbm_ctx *ctx, double *r);

/* Total mass sum_x rho(x) of the current state, reduced in FP64 (host scalar, synchronising).
 * LBM_EDIVERGED if non-finite. */
int lbm_mass(lbm_ctx *ctx, double *m);

/* Stream function of the current state with u_x = dPsi/dy, Psi = 0 on the bottom wall and the
 * trapezoid rule in y (dy = 1), integrated in FP64 (the Psi of Table 1 / Table 2, with the sign
 * that makes the primary vortex a minimum; the paper prints -Psi, Table 1 also divided by U nx).
 * psi: optional [ny][nx] FP64 buffer (NULL: not stored).  psi_min (host) receives the minimum,
 * xc / yc its node as x/nx and y/nx (width units, as in Table 1).  Synchronising. */
int lbm_stream_function(lbm_ctx *ctx, double *psi, double *psi_min, double *xc, double *yc);

/* Extrema of Psi restricted to the node window [i0, i1) x [j0, j1) (for secondary vortices,
 * Table 1), with node indices.  Any output pointer may be NULL.  Synchronising. */
int lbm_stream_function_window(lbm_ctx *ctx, int i0, int i1, int j0, int j1, double *psi_min,
                               int *imin, int *jmin, double *psi_max, int *imax, int *jmax);

/* Add an observing point (Sec. 3.3) at (x, y) in width units from the bottom-left corner, i.e.
 * node (floor(x nx + 1/2), floor(y nx + 1/2)) clamped into the grid.  After every step t with
 * t % every == 0 the velocity (u_x, u_y) of that node is written as two FP64 values to
 * dev_series[2 k], dev_series[2 k + 1] with k = (sample number) mod cap; dev_series is a
 * caller-owned DEVICE buffer of 2*cap doubles that must outlive the probe.  Returns the probe
 * index (>= 0) or a negative LBM_E* code (LBM_EINVAL: every < 1, cap < 1, more than
 * LBM_MAX_PROBES probes, dev_series not device memory). */
int lbm_probe(lbm_ctx *ctx, double x, double y, int every, double *dev_series, long cap);

/* Samples written so far by probe p (may exceed cap when the ring wrapped). */
int lbm_probe_count(lbm_ctx *ctx, int p, long *n);

/* Remove all probes. */
int lbm_probe_clear(lbm_ctx *ctx);

/* Allocation-free stream function.  The paper has no counterpart: this is a service for callers
 * that cannot call cudaMalloc -- e.g. a solver embedded in an application that reserves its whole
 * device-memory budget at start-up and forbids allocation afterwards.  It computes what
 * lbm_stream_function computes (Psi = 0 on the bottom wall, u_x = dPsi/dy, trapezoid rule in y,
 * FP64 sums), but from a caller-supplied velocity field and without a context:
 *   ux      DEVICE [ny][nx] FP64 u_x field (e.g. from lbm_moments into device memory), read only;
 *   psi     optional DEVICE [ny][nx] FP64 output (NULL: not written);
 *   result  DEVICE buffer of 3 doubles: psi_min, and its node as x/nx and y/nx (width units);
 *   stream  cudaStream_t to queue on (NULL: legacy stream).  Asynchronous; nothing is copied to
 *           the host and no host synchronisation happens.
 * Scratch: a fixed device array of LBM_STATIC_SCRATCH_DOUBLES doubles (4 MiB), defined in the
 * library and held by every GPU that loads it until the process exits.  A call needs
 * nx*ceil(ny/32) + 2*ceil(ny/32)*ceil(nx/128) doubles of it (a 4096 x 4000 grid fits), and
 * ceil(ny/32) may not exceed 65535 (ny <= 2,097,120; one launch row per 32-row segment); other
 * grids return LBM_ETOOBIG without launching anything.  Every element a call reads it has
 * written first, so nothing needs to be cleared between calls; but all calls share the one
 * array, so calls that can overlap on the GPU (other streams, other host threads) race and
 * must be ordered by the caller.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Errors: LBM_EINVAL (NULL ux/result, nx or ny < 1), LBM_ETOOBIG, LBM_ECUDA.  A CUDA error
 * that an earlier, unrelated call left pending is reported as LBM_ECUDA before anything is
 * launched and is left pending for its owner; an error of this call's own launches is cleared. */
#define LBM_STATIC_SCRATCH_DOUBLES (1 << 19)
int lbm_stream_function_static(const double *ux, int nx, int ny, double *psi, double *result,
                               void *stream);

/* ------------------------------------------------------------------ ALU throughput */

/* Fused multiply-add throughput of the current device, in FLOP/s (2 per FMA), FP64 (fp64 != 0)
 * or FP32 -- the ALU denominator of the step kernels' roofline where memory bandwidth is not the
 * bound (no counterpart in the paper; GB300's FP64 rate is a small fraction of its FP32 rate).
 * A kernel of 8 blocks x 256 threads per SM runs 8 independent FMA chains per thread for
 * trips x 16 chain steps (1 <= trips <= 1e6); 3 warm-up launches, then the best of 5 timed with
 * CUDA events on the legacy stream.  *flops_per_s and *ms (host, may be NULL) receive the rate
 * and that launch's time.  Allocates and frees a small output array.  Synchronising.
 * Errors: LBM_EINVAL (trips), LBM_ENOMEM, LBM_ECUDA. */
int lbm_fma_peak(int fp64, int trips, double *flops_per_s, double *ms);

/* ------------------------------------------------------------------ batched sweep */

/* A set of independent cavities of uneven sizes stepped together in one persistent GPU launch per
 * 100-step interval (the Re x Ar survey of Sec. 3.3, Fig. 17).  Cavity i has nx[i] x ny[i] nodes,
 * Reynolds number Re[i] and lid speed U[i] (tau_i from Re = U nx / nu and Eq. 5, as lbm_create);
 * all share one storage type.  Every cavity starts from the Sec. 2.2 (i) state.  At each
 * checkpoint every active cavity gets its own Eq. 6 residual and mass; lbm_batch_run_to_residual
 * retires cavities whose residual fell below tol and compacts the work list, so converged
 * cavities cost nothing afterwards.  The launch is cooperative; every grid-barrier wait inside it
 * is bounded (default 2 s) and a wait that runs out makes the call return LBM_ETIMEOUT.  A whole
 * 100-step interval (both launches) is captured once in a CUDA graph and replayed.  Work items
 * are (cavity, 32-lane column strip, rows per item) with a tile shape from LBM_BATCH_SHAPES
 * (lbm_batch_autotune picks one).  Device memory comes from cudaMalloc (the allocator hook
 * applies to single cavities only). */
#define LBM_BATCH_MAX 512
typedef struct lbm_batch lbm_batch;

/* Errors: LBM_EINVAL (n outside 1..LBM_BATCH_MAX, a grid < 3, tau <= 1/2), LBM_ENOMEM, LBM_ECUDA;
 * on failure *out is NULL and lbm_batch_last_error(NULL) holds the reason. */
int lbm_batch_create(int n, const int *nx, const int *ny, const double *Re, const double *U,
                     lbm_dtype dtype, lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);
const char *lbm_batch_last_error(const lbm_batch *b);
int lbm_batch_set_stream(lbm_batch *b, void *cuda_stream);

/* Advance every active cavity n >= 0 steps (no retirement).  Synchronising. */
int lbm_batch_step(lbm_batch *b, long n);

/* Run until every cavity's Eq. 6 residual is below tol (> 0) or max_steps more steps were taken;
 * steps_done[n] (host, may be NULL) receives each cavity's steps in this call.  LBM_OK when all
 * converged, LBM_ENOTREADY otherwise, LBM_EDIVERGED if a cavity went non-finite. */
int lbm_batch_run_to_residual(lbm_batch *b, double tol, long max_steps, long *steps_done);

/* Latest per-cavity Eq. 6 residuals (host r[n]) and states (host status[n] or NULL: 0 active,
 * 1 converged, 2 stopped at the step cap, 3 non-finite). */
int lbm_batch_residual(lbm_batch *b, double *r, int *status);

/* Global step of each cavity's current state (host steps[n]). */
int lbm_batch_cavity_steps(lbm_batch *b, long *steps);

/* Cavity i's moments / populations / stream function, as the single-cavity calls, into DEVICE
 * buffers sized for that cavity.  Synchronising. */
int lbm_batch_moments(lbm_batch *b, int i, double *rho, double *ux, double *uy);
int lbm_batch_get_populations(lbm_batch *b, int i, double *f);
int lbm_batch_stream_function(lbm_batch *b, int i, double *psi, double *psi_min, double *xc,
                              double *yc);

/* Replace cavity i's state by f = f^eq(rho, u) from DEVICE [ny_i][nx_i] FP64 fields (a warm
 * start); its Eq. 6 snapshot becomes u.  Only for an active cavity while the batch sits on a
 * checkpoint boundary (step multiple of 100, e.g. right after lbm_batch_create).  Synchronising. */
int lbm_batch_set_moments(lbm_batch *b, int i, const double *rho, const double *ux, const double *uy);
/* The same with the flags of lbm_set_moments_ex (LBM_INIT_NEQ uses cavity i's tau). */
int lbm_batch_set_moments_ex(lbm_batch *b, int i, const double *rho, const double *ux, const double *uy,
                             int flags);

/* One observing point per cavity at (x[i], y[i]) (width units, as lbm_probe); after every step
 * t with t % every == 0 cavity i writes (u_x, u_y) to dev_series[2 (i cap + k)], k = sample
 * number mod cap.  dev_series: caller-owned DEVICE buffer of 2 n cap doubles. */
int lbm_batch_probe(lbm_batch *b, const double *x, const double *y, int every, double *dev_series,
                    long cap);

/* Cavity i's parameters (launch_config holds the batch's tile shape). */
int lbm_batch_info(lbm_batch *b, int i, lbm_info *info);

/* Tile shapes of the batch kernel (no counterpart in the paper): rows per work item x load path x
 * resident 128-thread blocks per SM (register budget 96 for 5, 128 for 4, 64 for 8)
 *   0: 2 rows, L2 loads, 5 (default)  1: 1 row, L2, 5         2: 4 rows, L2, 5
 *   3: 2 rows, L1-cached loads, 5     4: 1 row, L1, 5         5: 4 rows, L1, 5
 *   6: 2 rows, L1, 4                  7: 4 rows, L1, 4        8: 2 rows, L2, 8
 *   9: 4 rows, L1, 8
 * Every shape computes bitwise-identical populations; Eq. 6 partial sums group per item, so
 * residuals agree to rounding.  lbm_batch_set_shape synchronises; LBM_EINVAL outside
 * 0..LBM_BATCH_SHAPES-1. */
#define LBM_BATCH_SHAPES 10
int lbm_batch_set_shape(lbm_batch *b, int shape);

/* Time every tile shape for `steps` (1..10000) plain steps on the batch's current state (probes
 * off), restore the state exactly (a temporary copy of one population pool is allocated: its
 * size in bytes is lbm_info.device_bytes / 2 at most; LBM_ENOMEM if that fails) and keep, among
 * the shapes within 2 % of the fastest trial, the one with the fewest rows per work item (finer
 * items keep more warps busy once cavities retire; ties by time).  chosen (host, may be NULL)
 * receives it, ms (host [LBM_BATCH_SHAPES], may be NULL) the trial times in milliseconds.
 * Synchronising. */
int lbm_batch_autotune(lbm_batch *b, int steps, int *chosen, float *ms);

/* Current tile shape, its rows per item, the persistent grid's block count and the number of
 * captured-interval replays so far (each host pointer may be NULL).  LBM_ECUDA (with the
 * driver's message in lbm_batch_last_error) if graph capture was refused and intervals are
 * launched directly. */
int lbm_batch_launch_info(lbm_batch *b, int *shape, int *rows_per_item, int *blocks,
                          long *graph_launches);

/* Limit of each grid-barrier wait in seconds (default 2).  absent_block >= 0 makes that block of
 * the next launch leave before its first barrier -- a fault-injection hook for testing the
 * timeout path (the other blocks' waits run out and the call returns LBM_ETIMEOUT). */
int lbm_batch_set_barrier_limit(lbm_batch *b, double seconds, int absent_block);

/* ------------------------------------------------------------------ learned warm start */

/* Not in the paper: a convolutional encoder-decoder that predicts an initial fine field for the
 * solver from (Re, Ar, a coarse field), to cut the steps to the Eq. 6 steady state; the plain run
 * from rest remains the fallback and the reference.  Architecture: 5 levels of two 3x3 convolutions
 * (widths w, 2w, 4w, 8w, 8w; leaky ReLU 0.1), 2x2 average pooling down, nearest x2 up with
 * skip concatenation, a 3x3 output head.  Input tensor [7][H][W] FP32 (see lbm_warm_input),
 * output [3][H][W]: corrections to input channels 0..2.  All convolutions run on BF16 tensor
 * cores (tcgen05 by default) with FP32 accumulation; master weights and Adam state are FP32.  H, W: multiples of 16
 * with (H/16)(W/16) a multiple of 8.  Tensor arguments are DEVICE pointers. */
#define LBM_WARM_RHO_SCALE 100.0f /* channel 0 holds (rho - 1) * LBM_WARM_RHO_SCALE */
typedef struct lbm_net lbm_net;

/* He-uniform initial weights from a seeded generator; biases zero. */
int lbm_net_create(int width, unsigned long long seed, lbm_net **out);
void lbm_net_destroy(lbm_net *n);
const char *lbm_net_last_error(const lbm_net *n);
int lbm_net_set_stream(lbm_net *n, void *cuda_stream);
long lbm_net_param_count(const lbm_net *n);
/* Flat FP32 parameter / gradient vectors (host or device buffers of lbm_net_param_count floats).
 * Order: per convolution (the 10 encoder, 8 decoder, 1 head convolutions in graph order) its
 * weights [co][ci][3][3] then its biases [co]. */
int lbm_net_get_params(lbm_net *n, float *p);
int lbm_net_set_params(lbm_net *n, const float *p);
int lbm_net_get_grads(lbm_net *n, float *g);
int lbm_net_zero_grads(lbm_net *n);
/* out[3][H][W] = network(in[7][H][W]).  Asynchronous. */
int lbm_net_forward(lbm_net *n, const float *in, int H, int W, float *out);
/* Forward, loss = mean over masked pixels and 3 channels of e^2, e = base + out - target with the
 * masked mean of e removed in channel 0 (the density channel counts up to a constant), backward:
 * gradients are ADDED to the accumulated gradient (lbm_net_zero_grads clears it).  mask [H][W]
 * is 0/1; base, target [3][H][W].  *loss (host, may be NULL).  Synchronising. */
int lbm_net_backward(lbm_net *n, const float *in, const float *base, const float *target,
                     const float *mask, int H, int W, double *loss);
/* GEMM back end of the convolutions: 1 = tcgen05 (5th-generation tensor cores, TMEM
 * accumulator) on an explicit im2col matrix; 2 = tcgen05 with the forward and data-gradient
 * products as implicit GEMMs (the im2col rows are gathered inside the kernel,
 * lbm_nn_conv3x3_bf16_tc05; bitwise the same results as 1, a fifth of the DRAM traffic, but
 * slower: its gather is bound by instruction issue); 3 = tcgen05 with those products as implicit
 * GEMMs over a channels-last BF16 copy of the input whose A tiles arrive as TMA boxes
 * (lbm_nn_conv3x3_bf16_tma; the default: the same sums as 1 in another order, equal to FP32
 * rounding, and a forward + backward pass 14-22 % faster); the weight gradient always runs on the
 * explicit im2col; 0 =
 * mma.sync.  Shapes a back end does not take run on 1.  With tcgen05, lbm_net_forward
 * synchronises, and a bounded tensor-core wait that runs out makes forward/backward return
 * LBM_ETIMEOUT. */
int lbm_net_set_backend(lbm_net *n, int backend);
/* One Adam step on the accumulated gradient times grad_scale (e.g. 1/batch). */
int lbm_net_adam_step(lbm_net *n, float lr, float beta1, float beta2, float eps, float grad_scale);
int lbm_net_save(lbm_net *n, const char *path);
int lbm_net_load(lbm_net *n, const char *path);

/* Network input for a fine nx x ny cavity (rows padded to H >= ny) from a coarse nxc x nyc
 * solution (DEVICE [nyc][nxc] FP64 rho, ux, uy, e.g. lbm_moments of a coarse run): bilinear image
 * of (rho - 1) * LBM_WARM_RHO_SCALE, ux / U, uy / U on the fine nodes, Re / 4000, Ar / 2, the wall
 * mask and the valid-row mask.  in: DEVICE [7][H][nx] FP32.  Asynchronous. */
int lbm_warm_input(const double *rho_c, const double *ux_c, const double *uy_c, int nxc, int nyc,
                   double Re, double Ar, double U, int nx, int ny, int H, float *in, void *stream);
/* Fine fields (DEVICE [ny][nx] FP64) from the input and the network output: base + correction,
 * unscaled -- ready for lbm_set_moments.  Asynchronous. */
int lbm_warm_output(const float *in, const float *out, int nx, int ny, int H, double U, double *rho,
                    double *ux, double *uy, void *stream);
/* Smooth a network output [3][H][W] (DEVICE) in place by `passes` 3x3 box-filter passes over rows
 * [0, ny) (neighbourhoods clamped to those rows and the W columns; padding rows copied).  The
 * warm start's convergence suffers from small-scale, non-solenoidal noise in the predicted
 * correction more than from its smooth part.  scratch: DEVICE, 3 H W floats.  Asynchronous. */
int lbm_warm_smooth(float *out, int ny, int H, int W, int passes, float *scratch, void *stream);
/* Training target [3][H][nx] FP32 (DEVICE) from a fine steady solution (DEVICE [ny][nx] FP64):
 * (rho - 1) * LBM_WARM_RHO_SCALE, ux / U, uy / U on rows < ny, zero on the padding rows.
 * Asynchronous. */
int lbm_warm_target(const double *rho, const double *ux, const double *uy, int nx, int ny, int H, double U,
                    float *target, void *stream);

/* The network's tensor-core product, exposed for tests and reuse: C[M][N] (op)= sum_k A[M][K]
 * B[N][K] with A, B bfloat16 (DEVICE, row-major, K contiguous; K, lda, ldb multiples of 8, 16-byte
 * aligned) and C FP32 (DEVICE, ldc).  op: 0 store, 1 accumulate, 2 atomic add (required when
 * split_k > 1: K is split across split_k blocks whose partial products are added atomically).
 * Asynchronous.  LBM_EINVAL for sizes or alignments it does not support. */
int lbm_nn_gemm_bf16(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C,
                     int ldc, int op, int split_k, void *stream);

/* The same product on the 5th-generation tensor cores (tcgen05.mma with the accumulator in tensor
 * memory; 128-row tiles, N tile 32/64/128 picked from N).  trans_c != 0 stores element (m, n) at
 * C[n*ldc + m].  split_k as above.  err: DEVICE int, set to 1 if a bounded internal wait ran out
 * (the result is then incomplete).  Asynchronous. */
int lbm_nn_gemm_bf16_tc05(int M, int N, int K, const void *A, int lda, const void *B, int ldb,
                          float *C, int ldc, int op, int trans_c, int split_k, int *err, void *stream);

/* 3x3 convolution (padding 1) of the FP32 inputs x1 [c1][H][W] ++ x2 [c2][H][W] (x2 may be NULL
 * with c2 = 0) as an implicit GEMM on the tcgen05 tensor cores: C[p][n] (op)= sum_k A[p][k] Wt[n][k]
 * with A the pixel-major im2col, k = ci*9 + ky*3 + kx, zeros outside the image and past
 * (c1 + c2)*9, each value rounded to BF16; A is never written to memory (each thread gathers one
 * pixel row of a 128 x 64 tile into shared memory).  Wt: DEVICE [N][K] BF16, K a multiple of 8 and
 * >= (c1 + c2)*9, 16-byte aligned; N <= 256.  C, op, trans_c, err as lbm_nn_gemm_bf16_tc05 with
 * M = H*W.  Bitwise equal to that GEMM on the explicit im2col.  No counterpart in the paper (the
 * warm start's convolutions).  Asynchronous.  Errors: LBM_EINVAL (shapes, NULL), LBM_ECUDA. */
int lbm_nn_conv3x3_bf16_tc05(const float *x1, int c1, const float *x2, int c2, int H, int W, int K,
                             const void *Wt, int N, float *C, int ldc, int op, int trans_c, int *err,
                             void *stream);

/* Weights of lbm_nn_conv3x3_bf16_tc05's layout (Wt [N][ldk] BF16, k = c*9 + ky*3 + kx, c < C) in
 * the tap-major layout of lbm_nn_conv3x3_bf16_tma: Wtap[n][tap*Cp + c] = Wt[n][c*9 + tap], tap =
 * ky*3 + kx, zero for C <= c < Cp, Cp = C rounded up to a multiple of 64.  Wtap: DEVICE, N*9*Cp
 * BF16, 16-byte aligned.  Asynchronous.  Errors: LBM_EINVAL (NULL, C or N < 1, ldk < 9 C),
 * LBM_ECUDA. */
int lbm_nn_weights_tap_major(const void *Wt, int ldk, int C, int N, void *Wtap, void *stream);

/* The same 3x3 convolution as lbm_nn_conv3x3_bf16_tc05 with the gather moved off the SM: one
 * kernel writes the input channels-last in BF16 (xs: DEVICE scratch of H*W*Cp BF16, 16-byte
 * aligned, Cp = (c1 + c2) rounded up to 64, zero padded; rounding as the explicit im2col), then
 * the tcgen05 GEMM runs with K ordered tap-major (k = tap*Cp + c) and fetches each 128-pixel x
 * 64-channel A tile as one 3-D TMA box shifted by the tap's offset (zeros outside the image).
 * Wtap: DEVICE [N][9*Cp] BF16 from lbm_nn_weights_tap_major.  C, op, trans_c, err as
 * lbm_nn_gemm_bf16_tc05 with M = H*W.  H*W must be a multiple of 128 and W a multiple or a divisor
 * of 128.  The products and their BF16 operands are those of the explicit path; only the order
 * of the FP32 sums differs.  No counterpart in the paper (the warm start's convolutions).
 * Asynchronous.  Errors: LBM_EINVAL (shapes, NULL, alignment; nothing launched), LBM_ECUDA. */
int lbm_nn_conv3x3_bf16_tma(const float *x1, int c1, const float *x2, int c2, int H, int W,
                            const void *Wtap, int N, float *C, int ldc, int op, int trans_c, void *xs,
                            int *err, void *stream);

/* ------------------------------------------------------------------ checkpoint */

/* Write / read the complete state (header with nx, ny, dtype, tau, U, flags, step; the stored
 * populations; the Eq. 6 snapshot and last results).  lbm_load requires a file written for the
 * same nx, ny and dtype (LBM_EIO otherwise).  A run continued from a checkpoint is bitwise
 * identical to an uninterrupted one.  Synchronising. */
int lbm_save(lbm_ctx *ctx, const char *path);
int lbm_load(lbm_ctx *ctx, const char *path);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
