/*
 * fga.h -- C ABI of the GB300 (sm_103a) frozen Gaussian approximation library.
 *
 * The library computes the frozen Gaussian approximation (FGA) of the acoustic
 * wave equation u_tt = c(x)^2 Laplace(u), u(0) = f0, u_t(0) = f1 (Theory
 * section, Eqs. wave, f0, f1) in the three steps of the Algorithm section:
 *   fga_decompose   -- FBI transform of f0, f1 (Eq. psi, Initial wavefield
 *                      decomposition section), branch split and thresholding
 *                      into the set of frozen Gaussians;
 *   fga_propagate   -- RK4 on the ray equations (Eqs. hamiltonian,
 *                      characline), the dynamic ray equations (Eqs. dzQ, dzP),
 *                      the amplitude equation (Eq. a_formu, Z of Eq. op_zZ) and
 *                      the action S, up to time T (Numerical test section: RK4);
 *   fga_reconstruct -- the Gaussian sum of Eq. recons on the grid.
 *
 * Conventions
 *   * Grids: x_i = origin + i*h per axis, arrays C-contiguous with the last axis
 *     fastest. The velocity, the initial data and the output share one grid.
 *   * Pointers marked "host or device" may point to either; the library asks
 *     the CUDA driver which it is. Device pointers must be on the current
 *     device. The caller owns every pointer it passes; the plan owns all the
 *     device memory it allocates and frees it in fga_destroy.
 *   * All work is issued on the plan's stream. fga_decompose synchronises that
 *     stream once (it reads the Gaussian counts back to size later launches);
 *     the other calls return before the device finishes, except when a host
 *     output pointer is given, in which case they wait for the copy.
 *   * Errors never abort or print: every call returns an fga_status and, on
 *     failure, records a message retrievable with fga_last_error. After a
 *     failure in a device-side step the plan is marked failed and every later
 *     call except fga_destroy / fga_last_error returns FGA_ERR_STATE.
 *   * A plan is not thread-safe; distinct plans are independent.
 *   * Only the + branch is propagated: for real f0, f1 the - branch terms are
 *     the complex conjugates of the + branch terms at -p (the p-grid is
 *     symmetric), so u = 2 Re(sum over the + branch).
 */
#ifndef FGA_H
#define FGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fga_plan_s* fga_plan_t;

typedef enum {
  FGA_OK = 0,
  FGA_ERR_INVALID = 1,  /* bad argument or configuration */
  FGA_ERR_OOM = 2,      /* a device allocation failed */
  FGA_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  FGA_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
  FGA_ERR_STATE = 5,    /* call out of order, or the plan failed earlier */
  FGA_ERR_NUMERIC = 6,  /* a ray met |P| = 0, det Z = 0 or a non-finite value */
  FGA_ERR_CAPACITY = 7  /* a fixed capacity of the plan was exceeded */
} fga_status;

typedef enum {
  FGA_FP64 = 0,         /* every step in FP64 */
  FGA_MIXED_TF32X3 = 1, /* the two contractions on the tensor cores, operands split into a
                           TF32 head and tail, hi*hi + hi*lo + lo*hi accumulated in FP32:
                           stage 2 of the FBI (the branch split in FP32 on its
                           accumulators; psi kept as FP32 pairs) and the reconstruction
                           (phase anchored in FP64). Stage 1 of the FBI runs in FP32 on
                           the CUDA cores (its output is stage 2's split operand); the
                           selection (on the exactly widened values), the rays and the
                           final sum over segments stay FP64. 2D grids with open axes
                           only. */
  FGA_MIXED_BF16X3 = 2  /* reserved (rejected by fga_plan) */
} fga_precision;

typedef struct {
  int dim;            /* 1, 2 or 3 (3: FP64 only; psi is held for every active q, so
                         large boxes need nq x prod(n_b) x 32 bytes of device memory) */
  int64_t n[3];       /* grid points per axis (>= 4) */
  double h[3];        /* grid spacing per axis (> 0) */
  double origin[3];   /* first grid point per axis */
  int periodic[3];    /* 1: axis is periodic (box = one period, n % q_stride == 0) */
  int nshots;         /* number of independent sets of initial data (>= 1) */
  const double* eps;  /* host [nshots]: FGA width parameter eps > 0 (a length) */
  const int* q_stride;/* host [nshots][dim] q-grid stride in grid points, or NULL:
                         round(0.5 sqrt(eps)/h) (reduced to divide n on periodic axes) */
  const int* box;     /* host [nshots][dim] FBI box points (even), or NULL:
                         ceil(12 sqrt(eps)/h) rounded up to a multiple of 32; n on
                         periodic axes (where any given value must equal n) */
  double T;           /* final time >= 0 */
  double dt;          /* RK4 step; T/dt must be an integer (to within 1e-9) below 2^31 */
  double kappa;       /* reconstruction window half-width in units of sqrt(eps) */
  double tau;         /* relative threshold: keep |psi+| >= tau * max|psi+-| */
  int precision;      /* fga_precision */
  int integrate_exited; /* 0 (default): a ray stops once its window has left an open
                           axis for good (|Q_k - edge| > kappa sqrt(eps) + 2 h_k outside
                           the grid with P_k pointing away; beyond the spline's clamped
                           margin c does not vary along that axis, so P_k keeps its sign
                           and the Gaussian never touches the grid again: the field is
                           unchanged, its stored state is the state at exit).
                           1: every ray is integrated to T. */
  int64_t keep_n;     /* 0: select by tau. > 0: keep, per shot, the keep_n largest |psi+|
                         over the valid (q, p) instead (ties by q index, then p index);
                         the - branch holds the mirror set, so each branch has keep_n
                         Gaussians (the N-largest selection of the paper's experiment) */
  int z_method;       /* how d_zQ and d_zP (Z of Eq. op_zZ) are obtained (fga_z_method):
                         FGA_Z_DYNAMIC (0): the dynamic ray equations (Eqs. dzQ, dzP);
                         FGA_Z_DIVIDED (1): central divided differences across 4d auxiliary
                         rays started at (q +- dq_k e_k, p) and (q, p +- dp_k e_k), integrated
                         with the ray by the same RK4 (the alternative named after Eq.
                         op_zZ); dq_k = dz_eta s_k h_k and dp_k = dz_eta times the p-grid
                         spacing of the shot. 1D and 2D; no receivers (so no fga_grad) */
  double dz_eta;      /* FGA_Z_DIVIDED: offsets as a fraction of the q- and p-grid spacings,
                         0 < dz_eta < 1 (at 1 the auxiliary rays would start at the
                         neighbouring grid points, which for p one step from 0 include
                         the left-out p = 0 where H = c|P| is singular). Ignored otherwise */
  int interp;         /* fga_interp: FGA_BSPLINE_APPROX (0): the velocity samples are the
                         spline coefficients (c(x) smooths them; the default).
                         FGA_BSPLINE_INTERP (1): the coefficients are the samples passed
                         through fga_spline_prefilter, so that c(x_i) = c_i at every grid
                         point (between the points the interpolant can undershoot where the
                         samples jump; the samples must be > 0, the rays need c > 0 where
                         they go); fga_grad then returns dJ/dc with respect to the samples */
} fga_config;

typedef enum {
  FGA_Z_DYNAMIC = 0,
  FGA_Z_DIVIDED = 1
} fga_z_method;

typedef enum {
  FGA_BSPLINE_APPROX = 0,
  FGA_BSPLINE_INTERP = 1
} fga_interp;

/* Create a plan: validate cfg, copy the velocity (host or device, [n...] FP64,
 * every value finite and > 0) to the device as the cubic B-spline coefficients
 * of the medium c(x) = sum_i c_i prod_k beta3((x_k - origin_k)/h_k - i_k) (indices
 * clamped on open axes, wrapped on periodic ones; with FGA_BSPLINE_INTERP the
 * coefficients are fga_spline_prefilter of the samples), and bind the CUDA stream
 * (a cudaStream_t; NULL = the legacy default stream).
 * Errors: FGA_ERR_INVALID (cfg, velocity <= 0 or NaN), FGA_ERR_OOM, FGA_ERR_CUDA. */
fga_status fga_plan(const fga_config* cfg, const double* velocity, void* stream,
                    fga_plan_t* out);

/* Step 1 (Eq. psi and the Initial wavefield decomposition section). u0, u1:
 * host or device, [nshots][n...] FP64. For every shot: the FBI transforms
 *   psi_j(q,p) = prod_k h_k sum_{j in box} f_j(q + r_j) w(r_j) exp(-i p.r_j/eps)
 * over the q-grid q = origin + s*m*h and the p-grid p = 2 pi eps m/(n_b h),
 * m = -n_b/2+1 .. n_b/2-1 (p = 0 left out), w the Gaussian window
 * exp(-|r|^2/(2 eps)) (periodised on periodic axes); the branch split
 * psi+ = 1/2 (psi_0 + i eps psi_1/(c(q)|p|)); and the selection of every (q,p)
 * with |psi+| >= tau * max|psi+|. counts_host (or NULL): host [nshots], the
 * number of Gaussians kept per shot. Synchronises the plan's stream.
 * Errors: FGA_ERR_INVALID (NULL data), FGA_ERR_OOM, FGA_ERR_CUDA, FGA_ERR_STATE. */
fga_status fga_decompose(fga_plan_t plan, const double* u0, const double* u1,
                         int64_t* counts_host);

/* Step 2. Integrates every kept Gaussian from (Q,P) = (q,p), d_zQ = I,
 * d_zP = -iI, a = 2^{d/2}, S = 0 to time T with T/dt classical RK4 steps (with
 * FGA_Z_DIVIDED: (Q,P), its auxiliary rays, a and S; the stored d_zQ, d_zP are then
 * the divided differences at the final time).
 * Errors: FGA_ERR_STATE (no decomposition yet), FGA_ERR_CUDA. A ray that meets
 * |P| = 0, det Z = 0 or a non-finite value is reported as FGA_ERR_NUMERIC by
 * the next call that synchronises (fga_reconstruct, fga_sync). */
fga_status fga_propagate(fga_plan_t plan);

/* Step 3 (Eq. recons). u_out: host or device, [nshots][n...] FP64, receives
 *   u(x) = 2 Re sum_{g in G+} W a_g psi_g (2 pi eps)^{-3d/2} exp(i S_g/eps)
 *            exp(i P_g.(x - Q_g)/eps - |x - Q_g|^2/(2 eps))
 * with every term cut to the window |x_k - Q_k| <= kappa sqrt(eps) on each axis
 * (all images on periodic axes) and W = prod_k (s_k h_k)(2 pi eps/(n_b,k h_k))
 * the phase-space cell of one Gaussian. Errors: FGA_ERR_STATE (not propagated),
 * FGA_ERR_INVALID, FGA_ERR_OOM, FGA_ERR_CUDA, FGA_ERR_NUMERIC. */
fga_status fga_reconstruct(fga_plan_t plan, double* u_out);

/* Receivers for traces: the field of Eq. recons (Re u, as fga_reconstruct writes it)
 * at the points xr (host or device, [nrx][dim] FP64, inside the grid, open axes only;
 * not with FGA_Z_DIVIDED)
 * at the record times t_m = m * record_every * dt, m = 0 .. T/(record_every dt)
 * (record_every must divide T/dt). fga_propagate then accumulates the traces while it
 * integrates the rays. nrx = 0 removes the receivers. Errors: FGA_ERR_INVALID,
 * FGA_ERR_OOM, FGA_ERR_CUDA. */
fga_status fga_set_receivers(fga_plan_t plan, int64_t nrx, const double* xr,
                             int64_t record_every);

/* Traces of the last fga_propagate: host or device [nshots][nrec][nrx] FP64,
 * nrec = T/(record_every dt) + 1. Synchronises the plan's stream. The sum over
 * Gaussians is accumulated with atomic additions, so the last bits may differ between
 * runs. Errors: FGA_ERR_STATE (no receivers or no propagation since they were set). */
fga_status fga_traces(fga_plan_t plan, double* traces);

/* Adjoint (gradient with respect to the velocity samples). With the set of Gaussians
 * of the last fga_decompose held fixed, computes
 *   grad[i] = sum_{s,m,r} residual[s][m][r] * d traces[s][m][r] / d c_i
 * for the traces of fga_traces (so for J = 1/2 sum (traces - data)^2 the residual is
 * traces - data and grad = dJ/dc). c_i are the velocity samples, which are the spline
 * coefficients of the medium; c enters through the rays (c, grad c, Hessian of c in
 * Eqs. characline, dzQ, dzP, a_formu) and through c(q) in the branch split (Eq. psi).
 * The derivative is that of the computed traces (discrete adjoint of the RK4 scheme; the
 * ray states are recorded or checkpointed as fga_set_adjoint_checkpointing says).
 * residual: host or device [nshots][nrec][nrx]; grad: host or device [n...], overwritten.
 * Rays that left the grid for good contribute nothing after they stop (as in the
 * forward). Needs fga_set_receivers and fga_propagate. Synchronises the stream.
 * Errors: FGA_ERR_STATE, FGA_ERR_INVALID, FGA_ERR_OOM, FGA_ERR_CUDA. */
fga_status fga_grad(fga_plan_t plan, const double* residual, double* grad);

/* fga_propagate followed by fga_reconstruct into device memory, replayed as one CUDA
 * graph: the ray, binning and reconstruction launches are captured on the plan's stream
 * (which must not be the legacy default stream) and replayed on later calls; the graph
 * is captured again when the Gaussian count, a buffer or u_dev changes. The first call
 * on a plan runs the two steps eagerly (it sets up the lazily initialised resources).
 * Results are identical to the two calls. Errors: FGA_ERR_STATE (not decomposed),
 * FGA_ERR_INVALID (host u_dev, default stream), FGA_ERR_CUDA. */
fga_status fga_run_graph(fga_plan_t plan, double* u_dev);

/* Autotuner (batching). Picks, by timing on this plan's own decomposed data, (0) the
 * number of resident blocks per SM of the persistent ray kernel and (2) its register
 * budget (variant 0: up to 255 registers per thread; 1: 168, so that 3 blocks of 128
 * fit an SM), both on a short integration of at most 64 steps, and (1) the split-K
 * segment length of the reconstruction gather (Gaussians per (tile, segment) work item;
 * 5 powers of two: 256 ... 4096 in FP64, 128 ... 2048 on the tensor cores, where the
 * FP32 accumulation of longer segments costs accuracy), then runs the full fga_propagate and fga_reconstruct with them into
 * the device buffer u_dev. Blocks the host until done. The choice stays with the plan
 * and is written to choice[3] when choice is not NULL. Ray states are identical for
 * every choice; the field changes only by the order of the FP64 (or FP32 tensor-core)
 * partial sums. Errors: FGA_ERR_STATE (not decomposed), FGA_ERR_INVALID (host u_dev),
 * FGA_ERR_OOM, FGA_ERR_CUDA. */
fga_status fga_autotune(fga_plan_t plan, double* u_dev, int64_t* choice);

/* The plan's current tuning, choice[3] as written by fga_autotune (blocks per SM, 0 =
 * occupancy maximum; segment length in Gaussians actually used, which is raised above
 * the set one when the partial tiles of a large batch would exceed 4 GiB; ray kernel
 * variant). */
fga_status fga_tuning(fga_plan_t plan, int64_t* choice);

/* Sets the tuning (e.g. one found earlier for the same workload): 0 <= choice[0] <= 64,
 * 0 <= choice[1] <= 2^20 (0 meaning the default for both), choice[2] in {0, 1}.
 * FGA_ERR_INVALID otherwise. */
fga_status fga_set_tuning(fga_plan_t plan, const int64_t* choice);

/* Waits for the plan's stream and reports any device-side error flag. */
fga_status fga_sync(fga_plan_t plan);

/* Frees everything the plan owns. NULL is accepted. */
fga_status fga_destroy(fga_plan_t plan);

const char* fga_status_string(fga_status s);
/* Message of the last failure on this plan ("" if none); NULL plan: the last
 * failure of fga_plan itself. The string lives until the next call. */
const char* fga_last_error(fga_plan_t plan);

/* ---- inspection (tests and diagnostics; each synchronises the stream) ---- */

/* Number of kept Gaussians of a shot (-1 before fga_decompose). */
int64_t fga_count(fga_plan_t plan, int shot);

/* The q-grid, p-grid and FBI box sizes of a shot: nq[dim], np[dim], nb[dim],
 * s[dim] (any may be NULL). np counts every p index j = m + n_b/2, j in [0, n_b). */
fga_status fga_shot_grid(fga_plan_t plan, int shot, int64_t* nq, int64_t* np, int64_t* nb,
                         int64_t* s);

/* psi+ over the whole q-grid x p-grid of a shot, host [n_q][n_p][2] (re, im),
 * p index j = m + n_b/2 in C order; zero outside the data's support and at the
 * left-out p values. max_abs (or NULL): max |psi+| of the shot. */
fga_status fga_psi(fga_plan_t plan, int shot, double* psi_host, double* max_abs);

/* The kept Gaussians of a shot in their stored order: host arrays of length
 * fga_count(shot): qidx (flat q-grid index), pidx (flat p-grid index), psi [2]. */
fga_status fga_gaussians(fga_plan_t plan, int shot, int64_t* qidx, int64_t* pidx,
                         double* psi);

/* Ray state after fga_propagate, host arrays over the shot's Gaussians:
 * Q,P [G][dim]; A = d_zQ, B = d_zP [G][dim][dim][2] ((j,k) = d_{z_j} Q_k);
 * a [G][2]; S [G]. Any pointer may be NULL. */
fga_status fga_state(fga_plan_t plan, int shot, double* Q, double* P, double* A, double* B,
                     double* a, double* S);

/* Ray steps integrated by the last fga_propagate, summed over all Gaussians
 * (G * T/dt when every ray is integrated to T; fewer when exited rays stop);
 * -1 before the first propagation. Synchronises the plan's stream. */
int64_t fga_ray_steps(fga_plan_t plan);

/* Per-stage device times in ms of the last decompose/propagate/reconstruct
 * (CUDA events on the plan's stream): out[0..4] = FBI, selection, rays,
 * binning, reconstruction; and the number of kernel launches issued by the
 * library since the plan was created. */
fga_status fga_stage_times(fga_plan_t plan, double* ms5, int64_t* launches);

/* ---- reconstruction without any device allocation ----
 *
 * The paper has no counterpart of this call; it exists for callers that cannot
 * allocate device memory (code running where cudaMalloc is off limits, such as
 * a host callback or a layer whose device memory is all owned by someone else,
 * or a caller that has budgeted every byte of the device). It is fga_reconstruct
 * for one set of propagated Gaussians given by the caller, with the scratch the
 * plan would allocate (tile offsets and per-tile Gaussian lists, 8.3 MiB) held in
 * one fixed file-scope device array instead. Every GPU that loads the library
 * holds that array until the process exits.
 *
 *   u(x) = Re sum_g coef_g prod_k X_k,   X_k = exp(i P_k (x_k - Q_k)/eps
 *                                                - (x_k - Q_k)^2/(2 eps))
 * cut to |x_k - Q_k| <= kappa sqrt(eps) on each axis (all images on periodic
 * axes). With coef_g = 2 W a_g psi_g (2 pi eps)^{-3d/2} exp(i S_g/eps) this is the
 * field fga_reconstruct writes for one shot.
 *
 * dim (1 or 2), n, h, origin, periodic: the output grid (as in fga_config); eps, kappa > 0.
 * qp: device, [2*dim][nG] FP64: rows Q_0..Q_{dim-1} then P_0..P_{dim-1}.
 * coef: device, [nG][2] FP64 (re, im). u: device, [n...] FP64, overwritten.
 * stream: a cudaStream_t (NULL = legacy default stream).
 *
 * Limits: the grid may have at most 16384 tiles (64 x 64 points in 2D, 256 in
 * 1D); larger grids get FGA_ERR_CAPACITY. Any nG < 2^31 is accepted: the
 * Gaussians are processed in chunks whose tile lists fit 2^21 entries.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine) and waits for its stream before returning (it reads a status word).
 * Its first call on a device looks up the array's device address on that
 * device; make that first call before any stream capture on the device. The
 * address is kept for the life of the process: after a cudaDeviceReset of that
 * device the kept address is stale, so do not call this entry point again in a
 * process that has reset the device.
 * Every call uses the same array and leaves its contents behind (the call
 * clears what must start at zero): calls that overlap on the GPU -- on two
 * streams, or from two host threads -- race on it and must be serialised.
 * Errors: FGA_ERR_INVALID (arguments, host pointers, pointers to another GPU's
 * memory), FGA_ERR_CAPACITY,
 * FGA_ERR_CUDA; the message is returned by fga_last_error(NULL). */
fga_status fga_reconstruct_static(int dim, const int64_t* n, const double* h, const double* origin,
                                  const int* periodic, double eps, double kappa, int64_t nG,
                                  const double* qp, const double* coef, double* u, void* stream);

/* The interpolating prefilter of the medium (host only; no CUDA call). Given samples
 * c_i on the grid (host, [n...] FP64, C order), writes the coefficients C (host, may be
 * the same array) of the clamped / wrapped cubic B-spline of fga_plan that interpolates
 * them: along every axis, one tridiagonal system per grid line,
 *   (C_{i-1} + 4 C_i + C_{i+1})/6 = c_i,
 * whose end rows on an open axis are those of the clamped spline itself,
 * (5 C_0 + C_1)/6 = c_0 and (C_{n-2} + 5 C_{n-1})/6 = c_{n-1}, and which wraps on a
 * periodic axis (solved by the Thomas algorithm, with the Sherman-Morrison correction
 * on periodic axes). Every such system is symmetric, so the map is its own adjoint
 * (fga_grad uses it to turn dJ/dC into dJ/dc).
 * dim 1..3, n[k] >= 4. Errors: FGA_ERR_INVALID (message via fga_last_error(NULL)). */
fga_status fga_spline_prefilter(int dim, const int64_t* n, const int* periodic,
                                const double* samples, double* coef);

/* The whole method -- fga_decompose, fga_propagate and fga_reconstruct of every shot
 * -- as one CUDA graph (batching of the Algorithm section's three steps: a captured
 * sequence of launches, each over all shots, with no host synchronisation and the
 * Gaussian counts kept on the device). u0, u1: device [nshots][grid] (as
 * fga_decompose); u_dev: device [nshots][grid], overwritten with Re u (as
 * fga_reconstruct).
 * The first call (and any call after an eager fga_decompose, or with other buffers)
 * runs the three steps eagerly -- that is its result -- to learn each shot's active q
 * rectangle and counts, sizes the Gaussian list, the tile lists and the binning for
 * 1.25 x those counts, and captures the graph; later calls replay it and return at
 * once. In the replay the counts, segment offsets and the total G are computed on the
 * device and every launch sizes itself from them within those capacities. If later
 * data need more (more Gaussians, longer tile lists) or give other active q
 * rectangles (a different support), the replay stays within its buffers, and the next
 * call that reads the device status (fga_sync, or one with a host output) fails with
 * FGA_ERR_CAPACITY and marks the plan failed. After a replay fga_count and the other
 * inspection calls report the replay's counts (they read them back, which waits for
 * the stream).
 * Needs a stream other than the legacy default stream, the dynamic-ray Z and no
 * receivers (FGA_ERR_INVALID otherwise); FGA_ERR_CUDA on a capture failure. */
fga_status fga_run_pipeline(fga_plan_t plan, const double* u0, const double* u1, double* u_dev);

/* Budget of the bounded waits in the tensor-core kernels (FGA_MIXED_TF32X3: FBI stage 2
 * and the reconstruction), as polls of the completion barrier of the previous chunk of
 * MMAs before the CTA gives up (no counterpart in the paper: failure detection of the
 * library). tries < 0 restores the defaults (2^22 polls, seconds); 0 makes every such
 * wait give up at once, which exercises the give-up path. A CTA that gives up issues no
 * further MMA, waits for its one outstanding commit with the default budget, releases
 * its tensor memory and sets the plan's status word; the next fga_sync (or call with a
 * host output) returns FGA_ERR_TIMEOUT and marks the plan failed.
 * Errors: FGA_ERR_INVALID (tries >= 2^32), FGA_ERR_STATE. */
fga_status fga_set_wait_budget(fga_plan_t plan, int64_t tries);

/* How fga_grad keeps the ray states for its reverse sweep (no counterpart in the paper:
 * the memory/recomputation trade-off of the discrete adjoint). mode 0 (the default):
 * every state and RK4 stage state of each resident thread's ray is recorded by the
 * forward pass when that takes at most half of the free device memory (4 (nsteps + 1)
 * states of nfields doubles per resident thread of the adjoint kernel, kept by the plan
 * for later calls), else mode 1's scheme. mode 1: checkpoints every
 * kseg = ceil(sqrt(nsteps)) steps, and each segment's states recomputed from its
 * checkpoint during the reverse sweep (one more forward step per ray step, about
 * 5 (kseg + 1) states per thread). Both give the same gradient up to the order of the
 * atomic additions. Errors: FGA_ERR_INVALID (mode not 0 or 1), FGA_ERR_STATE. */
fga_status fga_set_adjoint_checkpointing(fga_plan_t plan, int mode);

/* Measured fused multiply-add throughput of the current GPU (no counterpart in the
 * paper: the roofline denominator of the FP64-bound kernels). bits = 64 (DFMA) or 32
 * (FFMA); each of 8 blocks of 256 threads per SM runs 8 independent FMA chains for
 * iters x 16 rounds, timed with CUDA events on the legacy default stream after one
 * warm-up launch (the call synchronises the device's default stream and allocates
 * 64 KiB for the duration of the call). tflops (host) = 2 flop per FMA / time;
 * ms (host) = the timed launch. Errors: FGA_ERR_INVALID, FGA_ERR_CUDA (message via
 * fga_last_error(NULL)). */
fga_status fga_fma_peak(int bits, int iters, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* FGA_H */
