/*
 * lks.h -- C ABI of the B300 lattice-kinetic-scheme solver with grid-separated moving rigid bodies
 * and its exact discrete adjoint ("4D Topology optimization of moving rigid bodies in fluid flows",
 * Tanabe, Yaji, Ushijima).
 *
 * Conventions for every entry point
 *  - Lattice units: grid spacing and time step are 1.  Positions are offsets in analysis cells.
 *  - Arrays are flat, x fastest: a field over an (nx, ny, nz) grid is indexed (z*ny + y)*nx + x;
 *    a design array over (ndx, ndy, ndz) likewise.  Knot arrays are (K, d) row-major; per-step arrays
 *    are (Nt+1, d) row-major.
 *  - Entry points without the _dev suffix take HOST pointers and copy in and out themselves.
 *    Entry points with the _dev suffix take DEVICE pointers of the current device and a cudaStream_t
 *    passed as void* (NULL = the legacy default stream); they are asynchronous with respect to the host
 *    unless stated otherwise.
 *  - The library owns all of its device state (fields, checkpoints, history, reduction slots); it is
 *    allocated in lks_create and freed in lks_destroy.  The caller owns every array it passes; no pointer
 *    passed in is retained after the call returns.
 *  - Every call returns an lks_status.  On error the outputs are left untouched and a message is
 *    available from lks_last_error_string.  A context is not thread-safe: one host thread at a time.
 */
#ifndef LKS_H
#define LKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LKS_ABI_VERSION 3

typedef enum lks_status {
    LKS_OK = 0,
    LKS_EINVAL = -1,     /* bad parameters, sizes or pointers */
    LKS_ENOMEM = -2,     /* a device or host allocation failed */
    LKS_ECUDA = -3,      /* a CUDA runtime call failed (including "no device") */
    LKS_ESTATE = -4,     /* call order violated (e.g. adjoint before forward) */
    LKS_EUNSTABLE = -5,  /* non-finite velocity or |u| > u_crit seen during a forward sweep */
    LKS_ETIMEOUT = -6    /* a bounded device-side wait expired */
} lks_status;

enum { LKS_D2Q9 = 9, LKS_D3Q15 = 15 };                         /* Sec. 2.2 velocity sets */
enum { LKS_MAP_LINEAR = 0, LKS_MAP_COSINE = 1 };               /* Sec. 2.3 transfer kernel w(r) */
enum { LKS_FP64 = 0, LKS_FP32 = 1 };                           /* state precision (accumulators FP64) */
enum { LKS_CKPT_FULL = 0, LKS_CKPT_SQRT = 1, LKS_CKPT_REVOLVE = 2 };
enum { LKS_MODE_JOINT = 0, LKS_MODE_SHAPE = 1, LKS_MODE_MOTION = 2 };
enum { LKS_OBJ_FLOW = 0, LKS_OBJ_OAR = 1 };
enum { LKS_ADJ_DISCRETE = 0, LKS_ADJ_ALKS = 1 };                /* reverse sweep: exact discrete adjoint or Sec. 2.5 */

/*
 * Problem parameters (plain data, versioned by `size`).  Fill with lks_default_params, then set fields.
 *
 *  lattice        LKS_D2Q9 (2D) or LKS_D3Q15 (3D), Sec. 2.2.
 *  n[3]           analysis grid; n[2] = 1 in 2D.
 *  periodic[3]    1: periodic axis; 0: wall planes at index 0 and n-1 (u imposed, p streamed), Sec. 2.2.
 *  wall_velocity  [axis][side][component] velocity of each wall plane (side 0 = index 0).
 *  nu             lattice kinematic viscosity; A = 3/4 - 9 nu / 2 (Sec. 2.2).  Requires 0 < nu.
 *  kappa_max, q   Eq. kappa_ref: kappa^ref = kappa_max q g / ((1 - g) + q).
 *  nd[3]          inner design grid (nd[2] = 1 in 2D); margin: zero-kappa fluid margin per side (Sec. 2.3).
 *  map_kernel     LKS_MAP_LINEAR (hat, w = max(0, 1-|r|)) or LKS_MAP_COSINE (Sec. 2.3 w(r), |r| <= 2).
 *  base_center    analysis coordinates of the design-grid centre at zero offset; NaN = grid centre.
 *  probe_lo/hi    objective box O_target [lo, hi) (wall nodes excluded); direction: n of Eq. objective1.
 *  phi_var        phi of Eq. objective1, the weight of the variance: J1 = E - phi_var V, with E and V the mean
 *                 and variance of n.u over the fluid nodes of O_target and steps 1..Nt; 0 = the mean E alone.
 *                 Any finite value.
 *  objective      LKS_OBJ_FLOW: J1 of Eq. objective1 (probe box, direction, phi_var).  LKS_OBJ_OAR: J2 of Eq.
 *                 objective2, J2 = F_L + w_D F_D + w_T T, with F_L the mean over steps 1..Nt of
 *                 sum_D F_x / |D|, F_D the sum over steps of u^G_y sum_D F_y / (drag_span |D|) and T the sum
 *                 over steps of omega sum_D (r_x F_y - r_y F_x) / (2 pi l_m |D|), where F = kappa^ref (u^ref -
 *                 u^S,ref) is the Brinkman force density on the design grid, u^ref the velocity mapped back onto
 *                 it, r = x^ref - x^G the arm and D the inner design grid.  Without rotation (K_w = 0) T is zero.
 *  w_D, drag_span weight of F_D and x_2^max - x_2^min (cells, > 0) of Eq. objective2 (LKS_OBJ_OAR only).
 *  w_T, l_m       weight of T and the moment arm l_m (cells, > 0) of Eq. objective2 (LKS_OBJ_OAR with a rotating
 *                 body; ignored without rotation).
 *  Nt, K          time steps and motion knots (knot k at step k Nt/(K-1)); K >= 2.
 *  R_t            temporal filter radius in steps (Eq. chi_filtered), > 0.
 *  filter_R       density filter radius in design cells (Eq. filtering); <= 1 means identity.
 *  beta, eta      Heaviside projection (Eq. projection); beta = 0 means identity.
 *  precision      LKS_FP64 (plain FP64 state) or LKS_FP32 (FP32 state/stencil, FP64 objective and
 *                 sensitivity accumulation).
 *  ckpt           LKS_CKPT_FULL (every state kept), LKS_CKPT_SQRT (checkpoints every ceil(sqrt Nt) steps),
 *                 LKS_CKPT_REVOLVE (binomial schedule with ckpt_slots checkpoints, or as many as fit
 *                 in ckpt_bytes when ckpt_slots = 0).  When the slots hold every segment boundary (and, under a
 *                 byte budget, a second recompute history fits too) the schedule is the sqrt one, and the reverse
 *                 sweep is pipelined like LKS_CKPT_SQRT's.
 *  seg_len        recompute-segment length for REVOLVE (0 = automatic).
 *  mode           which gradients lks_adjoint produces (the others are returned as zeros).
 *  u_crit         stability limit on |u| checked every forward step (<= 0 disables); LKS_EUNSTABLE.
 *  tile_rows      step-kernel variant of the forward sweep.  D2Q9: 1 or 2 = row tiles of 28 x 8 or 28 x 16
 *                 nodes staged in shared memory; 3 = two steps per launch on 24 x 8 row tiles; 4, 8 or 16 (16:
 *                 LKS_FP32 only) = warp-column kernels with that many grid rows per warp; 32 or 64 = vectorised
 *                 warp columns (two columns per lane, even n[0] only) with that many rows.  D3Q15: 1 =
 *                 shared-memory tiles of 32 x 4 x 4 nodes; 8 or 16 = z-marching kernels with that many planes per
 *                 block; 32 or 64 = separable z-marching kernels with 16 or 32 planes of 32 x 8 columns; 96 =
 *                 separable forward with 16 planes of 32 x 16 columns (forward only); LKS_FP32 only: 128 or 160 =
 *                 plane-pair kernels (two planes per FP32x2 instruction) with 16 or 32 planes of 32 x 8 columns
 *                 per block, 192 = the plane-pair adjoint with 64 planes (tile_rows_adj only).  The plane-pair
 *                 blocks whose input region lies inside the grid in x and y (n[0] a multiple of 4) fetch their
 *                 planes by tensor (TMA) copies that complete on shared-memory barriers; each wait for them is
 *                 bounded (one second), and an expired wait makes the block leave and the context report
 *                 LKS_ETIMEOUT.  Environment read by lks_create: LKS_NO_TMA=1 turns the tensor copies off (every
 *                 block copies per thread; same results bit for bit), LKS_WAIT_NS sets the bound in ns, and the
 *                 diagnostic LKS_WAIT_PROBE=1 makes every such block first wait on a barrier that nothing
 *                 completes (the wait expires: a test of the timeout path).
 *                 0 = autotune at lks_create: times every choice on the context's buffers, then the fastest
 *                 one-step forward/adjoint pairs launched side by side; the forward sweep takes the fastest
 *                 forward, the pipelined sqrt(N) sweep and batch instances the fastest side-by-side pair
 *                 (cached per process; lks_get_stats reports the choices).
 *  tile_rows_adj  adjoint step-kernel variant when tile_rows != 0 (same codes); 0 = tile_rows.
 *  tile_rows_rec  forward variant of the recomputation in lks_adjoint when tile_rows != 0; 0 = tile_rows.
 *                 tile_rows_adj and tile_rows_rec must be 0 when tile_rows = 0 (all three autotuned).
 *  K_w, R_w       rotating body (Sec. 2.3-2.5): K_w >= 2 angle knots (radians, lks_set_angle_knots; knot k at step
 *                 k Nt/(K_w-1)) filtered with radius R_w steps (Eq. psi_filtered) and interpolated to theta_n, with
 *                 omega_n = theta_n - theta_{n-1}; theta turns the x-y components of the body about an axis parallel
 *                 to z through x^G (Eqs. rigid_body_position, rigid_body_velocity).  K_w = 0: translation only.  With a
 *                 rotating body the forward sweep runs step-kernel variant 1 (tile_rows 0 or 1), the footprint box
 *                 on x and y covers the design grid at any angle (it must fit in one period of a periodic axis), and
 *                 the objective must be LKS_OBJ_FLOW.
 *  adjoint        LKS_ADJ_DISCRETE: the exact discrete adjoint of the forward sweep (the gradient of J as computed).
 *                 LKS_ADJ_ALKS: the paper's continuous adjoint, the ALKS of Sec. 2.5 (Eqs. ap_tmp-as: adjoint moments
 *                 p~, u~ and the symmetric s~ carried as state, explicit Brinkman source), an approximation of the
 *                 gradient; objective LKS_OBJ_FLOW with phi_var = 0 and a translating body only, no adjoint terminal
 *                 state.
 */
typedef struct lks_params {
    uint32_t size;
    int32_t lattice;
    int32_t n[3];
    int32_t periodic[3];
    double wall_velocity[3][2][3];
    double nu;
    double kappa_max;
    double q;
    int32_t nd[3];
    int32_t margin;
    int32_t map_kernel;
    double base_center[3];
    int32_t probe_lo[3];
    int32_t probe_hi[3];
    double direction[3];
    int32_t Nt;
    int32_t K;
    double R_t;
    double filter_R;
    double beta;
    double eta;
    int32_t precision;
    int32_t ckpt;
    int32_t ckpt_slots;
    int32_t seg_len;
    int64_t ckpt_bytes;
    int32_t mode;
    double u_crit;
    int32_t tile_rows;
    int32_t tile_rows_adj;
    int32_t tile_rows_rec;
    double phi_var;
    int32_t objective;
    int32_t reserved_obj;
    double w_D;
    double drag_span;
    int32_t K_w;
    int32_t adjoint;
    double R_w;
    double w_T;
    double l_m;
} lks_params;

typedef struct lks_ctx lks_ctx;

/* Counters of the last forward / adjoint (for measurement). */
typedef struct lks_stats {
    int64_t forward_steps;     /* LKS steps run by the last lks_forward */
    int64_t recompute_steps;   /* LKS steps re-run by the last lks_adjoint */
    int64_t adjoint_steps;     /* adjoint steps run by the last lks_adjoint */
    int64_t kernel_launches;   /* kernels launched by the last forward + adjoint pair */
    int64_t device_bytes;      /* device memory held by the context */
    int32_t ckpt_slots;        /* checkpoints in use */
    int32_t seg_len;           /* recompute segment length */
    int32_t tile_rows_fwd;     /* step-kernel variants (tile_rows codes) of the forward sweep, */
    int32_t tile_rows_adj;     /* the adjoint steps */
    int32_t tile_rows_rec;     /* and the recomputation in lks_adjoint */
    int32_t pipelined;         /* 1: the reverse sweep runs the recomputation beside the adjoint chain */
    /* With lks_set_timing(ctx, 1): device time (CUDA events on the launching stream) of the last call pair. */
    double ms_forward_steps;   /* the Nt forward-step kernels of lks_forward */
    double ms_recompute_steps; /* forward-step kernels re-run by lks_adjoint */
    double ms_adjoint_steps;   /* the adjoint-step kernels */
    double ms_total;           /* whole lks_forward + lks_adjoint device time */
} lks_stats;

/* Fill *p with defaults for a 2D D2Q9 problem (size set, base_center NaN, everything else valid). */
int lks_default_params(lks_params* p);

/* Validate *p, allocate all device state on the current device.  *out is set only on LKS_OK. */
int lks_create(const lks_params* p, lks_ctx** out);

/* Free a context (NULL is a no-op).  Waits for the context's outstanding work. */
void lks_destroy(lks_ctx* ctx);

/* Human-readable text of the last error on ctx (never NULL), and of a status code. */
const char* lks_last_error_string(const lks_ctx* ctx);
const char* lks_strerror(int status);

/*
 * Forward solve (Algorithm 1, filters and forward time loop; objective Eq. objective1):
 *   gamma[nd]      design variables on the inner design grid, in [0, 1];
 *   pos_knots[K*d] body-centre offsets (cells) at the knots;
 *   J              objective J1 = E - phi_var V: E the time-space mean of n.u over O_target, V its variance
 *                  (rectangle rule over steps 1..Nt; FP64 accumulation of per-block partials in a fixed order).
 * Keeps what the adjoint needs (checkpoints).  Host-pointer variant blocks until J is on the host.
 */
int lks_forward(lks_ctx* ctx, const double* gamma, const double* pos_knots, double* J);
int lks_forward_dev(lks_ctx* ctx, const double* d_gamma, const double* d_pos_knots, double* d_J, void* stream);

/*
 * Status of the last forward: waits for it to finish, then LKS_EUNSTABLE if it saw a non-finite velocity or |u| > u_crit
 * (the check of lks_params.u_crit), LKS_OK otherwise; LKS_ESTATE before the first forward.  The _dev forward and
 * adjoint calls do not wait for the forward, so this is where their callers learn of an unstable sweep.  It also
 * waits for the device and returns LKS_ETIMEOUT (before LKS_EUNSTABLE) once any bounded device-side wait of the
 * context's kernels has expired; that status stays set for the context's lifetime, and lks_forward and lks_adjoint
 * return it too (the _dev adjoint then fills its outputs with NaN).
 */
int lks_get_status(lks_ctx* ctx);

/*
 * Adjoint solve (Algorithm 1, reverse loop; shape sensitivity Eq. dJdgamma, motion sensitivity Eq. dJdchi,
 * as the exact discrete adjoint of the forward), then the chain rules through the filters:
 *   dJ_dgamma[nd]     dJ/dgamma on the inner design grid;
 *   dJ_dpos[K*d]      dJ/dpos_knots.
 * Needs a preceding lks_forward on the same context (LKS_ESTATE otherwise).  With LKS_CKPT_REVOLVE the
 * reverse sweep reuses the forward's checkpoint slots, so every lks_adjoint needs its own lks_forward.
 * If that forward was unstable, lks_adjoint returns LKS_EUNSTABLE with its outputs untouched, and lks_adjoint_dev,
 * which does not wait for the forward (it is enqueued behind it on the stream), fills both outputs with NaN;
 * lks_get_status reports the instability.
 */
int lks_adjoint(lks_ctx* ctx, double* dJ_dgamma, double* dJ_dpos);
int lks_adjoint_dev(lks_ctx* ctx, double* d_dJ_dgamma, double* d_dJ_dpos, void* stream);

/* Density filter of Eq. filtering on the inner design grid (out = W gamma) and its transpose.  The transpose stages
 * its input divided by the row sums in a buffer of the context: transposes on one context that may overlap on the
 * GPU (different streams without ordering) race; order them on one stream. */
int lks_density_filter_dev(lks_ctx* ctx, const double* d_in, double* d_out, void* stream);
int lks_density_filter_T_dev(lks_ctx* ctx, const double* d_in, double* d_out, void* stream);

/* Heaviside projection of Eq. projection: out = P(in), dout = dP/din (either output may be NULL). */
int lks_projection_dev(int64_t count, double beta, double eta, const double* d_in, double* d_out,
                       double* d_dout, void* stream);

/* One normalised projected-gradient step of an optimiser loop around lks_forward / lks_adjoint (the ascent step
 * of the plain optimisation driver; Sec. 3 uses MMA, which is not part of this library):
 *     x_i <- min(hi, max(lo, x_i + step * g_i / max_j |g_j|)),  i < count,
 * with x left unchanged when g is zero everywhere.  Device pointers, on `stream`; lo <= hi and a finite step are
 * required (LKS_EINVAL otherwise).  One block of the GPU does the work: meant for design grids and knot arrays. */
int lks_gradient_step_dev(int64_t count, double step, const double* d_g, double* d_x, double lo, double hi,
                          void* stream);

/* Temporal motion filter of Eq. chi_filtered over the knots (K x d) and its transpose. */
int lks_motion_filter_dev(lks_ctx* ctx, const double* d_knots, double* d_filtered, void* stream);
int lks_motion_filter_T_dev(lks_ctx* ctx, const double* d_in, double* d_out, void* stream);

/* Per-step offsets s[(Nt+1) x d] by linear interpolation of filtered knots and u^G_n = s_n - s_{n-1}
 * (Eq. u_g as a backward difference; u^G_0 = u^G_1); and the transpose (s-bar, u^G-bar) -> knot-bar. */
int lks_interp_positions_dev(lks_ctx* ctx, const double* d_filtered, double* d_s, double* d_uG, void* stream);
int lks_interp_positions_T_dev(lks_ctx* ctx, const double* d_gs, const double* d_guG, double* d_out, void* stream);

/*
 * Batched parameter study: `count` independent problems (any mix of grid sizes, viscosities, gradient modes and
 * designs, one common Nt) advanced together.  Every instance owns a context (its own autotuned tiles); the
 * forward sweeps of all instances are captured into one CUDA graph, and so are their reverse sweeps, in which
 * each instance's kernel chains are independent branches that the GPU runs concurrently.  Pointer arguments are
 * arrays of `count` pointers (device pointers for _dev); d_J / J hold `count` values.  Errors name the
 * failing instance in lks_batch_last_error.
 */
typedef struct lks_batch lks_batch;
int lks_batch_create(int count, const lks_params* params, lks_batch** out);
void lks_batch_destroy(lks_batch* b);
lks_ctx* lks_batch_context(lks_batch* b, int index);
const char* lks_batch_last_error(const lks_batch* b);
int lks_batch_forward_dev(lks_batch* b, const double* const* d_gamma, const double* const* d_pos_knots, double* d_J,
                          void* stream);
int lks_batch_adjoint_dev(lks_batch* b, double* const* d_dJ_dgamma, double* const* d_dJ_dpos, void* stream);

/* Host-pointer variants of the five calls above (same kernels, same layouts; the arrays are host memory).  Each
 * copies its inputs to device memory allocated for the call, runs the device variant on the default stream,
 * copies the results back and frees the copies: synchronous, and not for callers that cannot allocate.
 * lks_projection needs no context; either of out and dout may be NULL (not both). */
int lks_density_filter(lks_ctx* ctx, const double* in, double* out);
int lks_density_filter_T(lks_ctx* ctx, const double* in, double* out);
int lks_projection(int64_t count, double beta, double eta, const double* in, double* out, double* dout);
int lks_motion_filter(lks_ctx* ctx, const double* knots, double* filtered);
int lks_motion_filter_T(lks_ctx* ctx, const double* in, double* out);
int lks_interp_positions(lks_ctx* ctx, const double* filtered, double* s, double* uG);
int lks_interp_positions_T(lks_ctx* ctx, const double* gs, const double* guG, double* out);

/* Final state (p_Nt, u_Nt) of the last forward, as FP64: p[N], u[d*N] (component-major); still available after
 * that forward's adjoint.  Synchronous.  LKS_ESTATE before the first forward. */
int lks_get_state(lks_ctx* ctx, double* p, double* u);

/* Initial state (p_0, u_0) of every following lks_forward, host FP64 in the layout of lks_get_state (p is the
 * pressure itself, not p - 1/3).  This is the warm start of the periodic approximation (Sec. 3.3): the final
 * state of one optimisation iteration starts the next.  The values are used as given, wall nodes included.
 * p = u = NULL restores the default (p = 1/3, u = 0, wall nodes at their wall velocity).  Discards captured
 * graphs; the next lks_adjoint needs a new lks_forward.  Synchronous. */
int lks_set_initial_state(lks_ctx* ctx, const double* p, const double* u);

/* Terminal adjoint state of every following lks_adjoint: (lam_p, lam_u), host FP64 in the layout of lks_get_state
 * (lam_p[N], lam_u[d*N]), is added to dJ/d(p_Nt, u_Nt) before the reverse sweep.  This is the adjoint half of the
 * periodic approximation (Sec. 3.3): the adjoint state at n = 0 of one optimisation iteration (lks_get_adjoint_initial)
 * ends the reverse sweep of the next, as the final flow state starts its forward sweep (lks_set_initial_state).
 * lam_p = lam_u = NULL removes it.  Discards captured graphs; the next lks_adjoint needs a new lks_forward.
 * Synchronous. */
int lks_set_adjoint_terminal(lks_ctx* ctx, const double* lam_p, const double* lam_u);

/* Adjoint state lambda_0 = dJ/d(p_0, u_0) of the last adjoint (the gradient of J with respect to the initial state),
 * as FP64 in the layout of lks_get_state.  Waits for the device.  LKS_ESTATE before the first adjoint. */
int lks_get_adjoint_initial(lks_ctx* ctx, double* lam_p, double* lam_u);

/* Rotating body: the K_w angle knots (radians, host) of every following forward (all zero until set); LKS_EINVAL when
 * the context has K_w = 0.  Synchronous.  dJ/d(angle knots) of the last adjoint, K_w values (zeros with
 * LKS_MODE_SHAPE), and the per-step dJ/dtheta_n, dJ/domega_n ((Nt+1) values each).  Synchronous. */
int lks_set_angle_knots(lks_ctx* ctx, const double* aknots);
int lks_get_angle_gradient(lks_ctx* ctx, double* dJ_daknots);
int lks_get_step_angle_sensitivities(lks_ctx* ctx, double* dJ_dtheta, double* dJ_domega);
/* theta_n and omega_n = theta_n - theta_{n-1} of the last forward ((Nt+1) values each; Eqs. psi_filtered, theta,
 * omega), and the transposed chain from per-step sensitivities (g_theta, g_omega, (Nt+1) each) to the K_w angle knots
 * (difference^T, interpolation^T, filter^T): what an optimiser needs for a constraint on omega such as G3 of Eq.
 * constraint3.  Host pointers, synchronous. */
int lks_get_angles(lks_ctx* ctx, double* theta, double* omega);
int lks_angles_T(lks_ctx* ctx, const double* g_theta, const double* g_omega, double* g_aknots);

/* Per-step motion sensitivities of the last adjoint, dJ/ds_n and dJ/du^G_n, each (Nt+1) x d. Synchronous. */
int lks_get_step_sensitivities(lks_ctx* ctx, double* dJ_ds, double* dJ_duG);

/* The two terms of Eq. objective1 for the last forward: *E the mean of n.u, *V its variance (both over the
 * fluid nodes of O_target and steps 1..Nt), so that J = E - phi_var V.  The squares are summed only when
 * phi_var != 0; with phi_var = 0, *V is NaN.  With objective LKS_OBJ_OAR these are still the probe box's flow terms
 * (J is J2).  Synchronous.  LKS_ESTATE before the first forward; LKS_EINVAL for a NULL pointer. */
int lks_get_objective_terms(lks_ctx* ctx, double* E, double* V);

/* Counters of the last forward / adjoint. */
int lks_get_stats(const lks_ctx* ctx, lks_stats* out);

/* Enable (1) or disable (0) CUDA-event timing of the step kernels.  When enabled, lks_adjoint[_dev]
 * synchronizes its stream at the end to read the events. */
int lks_set_timing(lks_ctx* ctx, int enable);

/* Enable (1, the default) or disable (0) CUDA-graph replay of the forward and reverse sweeps.  With graphs
 * on, the first lks_forward / lks_adjoint of a context capture their kernel sequence (all buffers belong to
 * the context, so the sequence is fixed) and later calls replay it.  Results are identical either way.
 * Changing the setting discards the captured graphs and requires a new lks_forward. */
int lks_set_graphs(lks_ctx* ctx, int enable);

/*
 * Density filter (same arithmetic as lks_density_filter_dev) that performs no memory allocation of any kind.
 * The paper has no counterpart: it exists for callers that cannot call cudaMalloc or create a context,
 * e.g. code that runs under a host framework owning the whole device memory pool, or code that must not
 * take the latency or the failure modes of an allocation inside its loop.
 *
 *   nd[3]   design grid extents (nd[2] = 1 in 2D); nd[0]*nd[1]*nd[2] <= LKS_NOALLOC_FILTER_MAX, else LKS_EINVAL.
 *   R       filter radius in design cells (<= 1: identity copy), 0 <= R <= 32.
 *   d_in, d_out  device arrays of that many doubles (x fastest), owned by the caller; may not alias.
 *
 * Its scratch (the per-node weight sums) is a fixed file-scope device array of LKS_NOALLOC_FILTER_MAX
 * doubles (8 MiB) that every GPU loading the library holds until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the device current; make that
 * first call before any stream capture on the device.  All calls share the array and each call overwrites
 * the entries it uses, so calls whose kernels may overlap on the GPU (different streams without ordering)
 * race and give undefined results: order them on one stream.  Asynchronous on `stream`.  Error text:
 * lks_noalloc_last_error().
 */
#define LKS_NOALLOC_FILTER_MAX (1 << 20)
int lks_density_filter_noalloc(const int32_t nd[3], double R, const double* d_in, double* d_out, void* stream);
const char* lks_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LKS_H */
