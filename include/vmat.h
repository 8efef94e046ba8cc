/*
 * vmat.h - C ABI of the B300 column-generation VMAT optimiser.
 *
 * The library solves the treatment-plan model of Men, Romeijn, Jia and Jiang
 * ("Ultra-fast treatment plan optimization for volumetric modulated arc
 * therapy"), Sec. 2.1, Eq. 3:
 *
 *     min_{y, A_k}  sum_j F(z_j) + gamma * G(y)
 *     s.t.  z_j = sum_k y_k sum_{i in A_k} D_ij,   y_k >= 0,
 *
 * with the one-sided quadratic voxel cost F of Eq. 1 and the dose-rate
 * smoothing G of Eq. 2, by column generation (Sec. 2.2): a pricing step picks
 * the most promising deliverable aperture among beams that have none yet, and
 * a master problem re-optimises the intensities y by gradient projection.
 *
 * Conventions
 *  - Beams k = 0..N-1 are sorted by angle theta_k (degrees, strictly
 *    increasing in [0, 360)).  Each beam has an MLC of R leaf rows x C
 *    columns; beamlet i = (k*R + r)*C + c.  Voxel j indexes the caller's grid.
 *  - An aperture is one open interval [l, r) of columns per leaf row
 *    (0 <= l <= r <= C; l == r is a closed row).
 *  - "_dev" pointers are CUDA device pointers owned by the caller (for
 *    instance torch tensors); the library never frees them.  "_host"
 *    pointers are ordinary host memory owned by the caller.
 *  - Every call is enqueued on the context's stream and is synchronous on
 *    return (the stream is synchronised before returning) unless stated.
 *  - Every call returns a vmat_status; nothing is thrown across the ABI.
 *    On failure vmat_last_error() gives a message.  A context is not
 *    thread-safe: use one context per host thread.
 *  - Device waits inside the library's kernels are bounded: a wait that runs
 *    out returns VMAT_ETIMEOUT instead of hanging.
 */
#ifndef VMAT_H
#define VMAT_H

#include <stdint.h>

#if defined(__GNUC__)
#define VMAT_API __attribute__((visibility("default")))
#else
#define VMAT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VMAT_OK = 0,
  VMAT_EINVAL = 1,   /* bad argument: sizes, unsorted CSR, non-finite value, bad state for the call */
  VMAT_ENOMEM = 2,   /* device allocation failed */
  VMAT_ECUDA = 3,    /* a CUDA runtime call failed */
  VMAT_ENOTCONV = 4, /* master problem hit max_iters before the KKT tolerance (results still written) */
  VMAT_ETIMEOUT = 5, /* a bounded device wait ran out */
  VMAT_ESTATE = 6    /* no feasible aperture / no free beam left */
} vmat_status;

/* Storage type of D on the device.  F16/BF16 store each beamlet's row scaled
 * by s_i = max_j D_ij (FP32 scale kept per beamlet) and accumulate in FP32. */
typedef enum { VMAT_F64 = 0, VMAT_F32 = 1, VMAT_F16 = 2, VMAT_BF16 = 3 } vmat_dtype;

typedef struct vmat_ctx vmat_ctx;

/* The planning problem (Sec. 2.1).  All pointers are host memory, read
 * during vmat_create only. */
typedef struct {
  int32_t n_vox;               /* |V|, voxels of the grid */
  int32_t n_angles;            /* N */
  int32_t n_rows, n_cols;      /* R, C: MLC leaf rows and beamlet columns */
  const double *theta_deg;     /* [N] beam angles, strictly increasing in [0, 360) */
  const uint8_t *struct_id;    /* [n_vox] structure of each voxel, < n_struct */
  int32_t n_struct;            /* entries of T/alpha/beta (<= 256) */
  const double *T;             /* [n_struct] threshold / prescription T_j (Eq. 1) */
  const double *alpha;         /* [n_struct] underdose weight alpha_j >= 0 (Eq. 1) */
  const double *beta;          /* [n_struct] overdose weight beta_j >= 0 (Eq. 1) */
  double gamma;                /* smoothing weight gamma >= 0 (Eq. 3) */
  int32_t cyclic;              /* 1: G and leaf limits run round the ring of beams; 0: path of Eq. 2 */
  int32_t max_leaf_step;       /* leaf travel limit s: columns per angle step (>= C: unconstrained) */
  int64_t nnz;                 /* non-zeros of D */
  const int64_t *row_ptr;      /* [B+1] beamlet-major CSR of D, B = N*R*C */
  const int32_t *vox_idx;      /* [nnz] voxel of each entry, strictly ascending within a row */
  vmat_dtype val_dtype;        /* VMAT_F64 or VMAT_F32: type of val */
  const void *val;             /* [nnz] D_ij, finite and > 0 */
} vmat_problem;

/* Size information of a context. */
typedef struct {
  int32_t n_vox, n_active;     /* grid voxels; voxels with at least one entry of D */
  int32_t n_angles, n_rows, n_cols;
  int64_t n_beamlets, nnz;
  int32_t n_columns;           /* apertures in the current plan */
  int64_t device_bytes;        /* device memory held by the context */
  vmat_dtype d_dtype;
  int32_t master_grid, master_block; /* launch shape of the master kernel */
  int64_t n_launches;          /* kernels this context has launched so far */
  double master_ms[4];         /* master kernel, cumulative device time (ms) in: gradient
                                  pass + its reduction, step, direction pass, line search */
  int64_t master_syncs;        /* cumulative grid-wide barriers of the master kernel */
  double master_wait_ms;       /* cumulative time (ms) CTA 0 spent at those barriers between its
                                  own arrival and the release (part of master_ms) */
  int64_t master_pg_iters;     /* cumulative projected-gradient iterations (accepted steps) */
  int64_t master_rejected;     /* cumulative trial steps the acceptance test cut back */
  int32_t subtile_voxels;      /* voxels per subtile of the aperture-dose columns */
  int32_t n_subtiles;          /* subtiles per column (padded active voxels / subtile_voxels) */
  int64_t tile_entries[2];     /* union entries of the row tiles of D used by the batched
                                  products (voxel-major, beamlet-major; 0 until built) */
  int64_t price_calls[2];      /* FP32 price products so far: [0] in the live-voxel form,
                                  [1] in total (see vmat_set_price_path) */
  int64_t price_live_entries;  /* entries of D read by the live-voxel calls so far */
} vmat_info;

/* Copy the problem to the device and build every storage form of D:
 * beamlet-major CSR and a voxel-major transpose (rows sorted by beamlet),
 * both over the compacted set of voxels D touches, in d_dtype (VMAT_F32,
 * VMAT_F16 or VMAT_BF16).  cuda_stream: a cudaStream_t (NULL: the legacy
 * default stream) on which every later call is enqueued.  Validates the
 * problem (sizes, sorted rows, finite positive values, sorted angles) and
 * returns VMAT_EINVAL on any violation.  *out is NULL on failure. */
VMAT_API vmat_status vmat_create(const vmat_problem *prob, vmat_dtype d_dtype, void *cuda_stream,
                        vmat_ctx **out);
VMAT_API void vmat_destroy(vmat_ctx *ctx);
/* Last error message of ctx (ctx NULL: of the last failed vmat_create).
 * Valid until the next call on that context. */
VMAT_API const char *vmat_last_error(const vmat_ctx *ctx);
VMAT_API vmat_status vmat_get_info(const vmat_ctx *ctx, vmat_info *out);

/* Dose of a beamlet fluence (Sec. 2.1): z_j = sum_i D_ij x_i for all grid
 * voxels, with the voxel cost of Eq. 1.  x_dev [B] float; z_dev [n_vox]
 * float or NULL; fprime_dev [n_vox] float F'(z_j) or NULL; cost_host: sum_j
 * F(z_j) reduced in FP64, or NULL. */
VMAT_API vmat_status vmat_dose(vmat_ctx *ctx, const float *x_dev, float *z_dev, float *fprime_dev,
                      double *cost_host);

/* Beamlet prices (Sec. 2.2: the KKT conditions give each beamlet the price
 * dF/dx_i): g_i = sum_j D_ij f_j for every beamlet of a beam with
 * angle_mask_dev[k] != 0 (angle_mask_dev NULL: all beams).  f_dev [n_vox]
 * float (typically F'(z)); g_dev [B] float; entries of masked-out beams are
 * not written. */
VMAT_API vmat_status vmat_price(vmat_ctx *ctx, const float *f_dev, const uint8_t *angle_mask_dev,
                       float *g_dev);

/* One aperture: beam and leaf pair per row. */
typedef struct {
  int32_t angle;     /* beam index k */
  double price;      /* total price of the aperture (sum of its row values) */
  double runner_up;  /* least price of any other free beam (INFINITY if none) */
  int16_t *l, *r;    /* [n_rows] host arrays, caller-allocated */
} vmat_column;

/* Pricing subproblem (Sec. 2.2): for every beam without an aperture, the
 * deliverable aperture of least total price under the leaf-travel limits to
 * the nearest beams with apertures, found by one left-to-right pass per leaf
 * row; returns the beam of least price (ties: lowest index).  g_dev [B]
 * float prices.  Row values and their prefix sums are formed in FP32 in
 * column order; the aperture price sums the rows in FP64 in row order.
 * VMAT_ESTATE if no beam is free or a row has no feasible interval. */
VMAT_API vmat_status vmat_pricing_select(vmat_ctx *ctx, const float *g_dev, vmat_column *out);

/* Add an aperture to the plan: builds its column of the aperture-dose matrix
 * M[:, k] = sum_{i in A_k} D_i,: , marks the beam occupied and records its
 * leaves; y_k starts at 0.  The leaves must satisfy 0 <= l <= r <= C (the
 * leaf-travel limits are not re-checked: replay of a recorded plan is
 * allowed).  VMAT_EINVAL if the beam already has an aperture. */
VMAT_API vmat_status vmat_add_column(vmat_ctx *ctx, const vmat_column *col);

/* Master problem (Sec. 2.2): minimise Eq. 3 over y >= 0 with the current
 * apertures fixed, y_k = 0 for beams without one, by projected gradient
 * (second Barzilai-Borwein step, exact line search on [0,1]).  Stops when
 * rho = max_k |min(y_k, df/dy_k)| <= kkt_tol * max(rho_start, rho_ref) or
 * after max_iters iterations (VMAT_ENOTCONV; y is still written).  y_host
 * [N] in: warm start (NULL: keep the context's y), out: solution (NULL: not
 * copied).  cost/kkt/iters (each may be NULL): final objective (FP64), final
 * rho, iterations used. */
VMAT_API vmat_status vmat_master_step(vmat_ctx *ctx, int32_t max_iters, double kkt_tol, double rho_ref,
                             double *y_host, double *cost, double *kkt, int32_t *iters);

/* Current plan dose z = sum_k y_k M[:, k] on the grid: z_dev [n_vox] float. */
VMAT_API vmat_status vmat_plan_dose(vmat_ctx *ctx, float *z_dev);

/* Clear the plan (apertures, y, dose) so a new column generation can start
 * on the same D. */
VMAT_API vmat_status vmat_reset(vmat_ctx *ctx);

typedef struct {
  int32_t n_iters;             /* column-generation iterations (<= N) */
  int32_t master_max_iters;    /* per master problem */
  double kkt_tol;              /* relative KKT tolerance of each master problem */
  const int32_t *forced_angle; /* NULL, or [n_iters] beams to take instead of the pricing result (replay) */
  const int16_t *forced_l;     /* [n_iters*R] leaves of the forced apertures */
  const int16_t *forced_r;
} vmat_colgen_opts;

typedef struct {              /* caller-allocated host arrays (any may be NULL) */
  int32_t *angle_order;       /* [n_iters] beam added at each iteration */
  int16_t *l, *r;             /* [N*R] final leaves (rows of beams without an aperture: 0) */
  double *y;                  /* [N] final intensities */
  double *price;              /* [n_iters] price of the chosen aperture (pricing result) */
  double *runner_up;          /* [n_iters] least price of the other free beams */
  double *cost;               /* [n_iters] objective after each master problem */
  double *kkt;                /* [n_iters] final rho of each master problem */
  int32_t *master_iters;      /* [n_iters] */
  double *phase_ms;           /* [n_iters*4] device time (ms) of each iteration's phases:
                                 prices, pricing, aperture column, master problem;
                                 written only while profiling is on */
  int32_t *col_subtiles;      /* [n_iters] subtiles holding a nonzero of each added column
                                 (the master kernel streams only those) */
  int32_t *priced_angle;      /* [n_iters] beam the pricing chose at each iteration; equals
                                 angle_order except in replay, where the forced aperture is
                                 added instead and this records the library's own choice on
                                 the replayed state */
  int16_t *priced_l, *priced_r; /* [n_iters*R] leaves of that choice, iteration-major */
} vmat_colgen_result;

/* Column generation (Sec. 2.2, Fig. 1) from the context's current plan:
 * n_iters times {prices of the free beams from F'(z); pricing; add column;
 * master problem}.  The master problems stop at kkt_tol relative to
 * max(rho_start, rho of the plan's first master problem).  The whole loop
 * runs on the device; the host reads the records once at the end.  With
 * forced_angle set (replay) iteration t adds the forced aperture, while
 * price/runner_up/priced_* still record what the pricing itself chose on
 * that state (decision-by-decision comparison with another solver's plan).
 * VMAT_ENOTCONV if some master problem hit its limit (records still
 * written). */
VMAT_API vmat_status vmat_colgen_run(vmat_ctx *ctx, const vmat_colgen_opts *opts,
                            vmat_colgen_result *res);

/* Profiling: with on != 0, vmat_colgen_run brackets each phase of every
 * iteration with CUDA events on the context's stream and reports the device
 * times in vmat_colgen_result.phase_ms.  Off by default. */
VMAT_API vmat_status vmat_set_profiling(vmat_ctx *ctx, int32_t on);

/* Batched dose of 32 fluence vectors (the differentiable forward):
 * Z[j][b] = sum_i D_ij X[i][b], X_dev [B][32] float row-major, Z_dev
 * [n_vox][32] float; cost_host [32] (or NULL): sum_j F(Z[j][b]) in FP64;
 * fprime_dev [n_vox][32] float F'(Z) or NULL. */
VMAT_API vmat_status vmat_dose_batch32(vmat_ctx *ctx, const float *X_dev, float *Z_dev, float *fprime_dev,
                              double *cost_host);

/* Batched adjoint: G[i][b] = w[b] * sum_j D_ij Fp[j][b] for all beamlets,
 * Fp_dev [n_vox][32] float, w_dev [32] float per-vector weights (NULL: all
 * 1; the backward pass passes the incoming gradient), G_dev [B][32] float. */
VMAT_API vmat_status vmat_price_batch32(vmat_ctx *ctx, const float *Fp_dev, const float *w_dev,
                                        float *G_dev);

/* Aperture maps for 32 intensity vectors (the differentiable forward with
 * respect to aperture intensities, Eq. 3): X = A Y with X[i][b] = Y[k][b] if
 * beamlet i = (k*R + r)*C + c is open in beam k (l[k*R+r] <= c < r[k*R+r]),
 * else 0.  l_dev, r_dev [N*R] int16 device; Y_dev [N][32], X_dev [B][32]
 * float row-major. */
VMAT_API vmat_status vmat_aperture_fluence_batch32(vmat_ctx *ctx, const int16_t *l_dev,
                                                   const int16_t *r_dev, const float *Y_dev,
                                                   float *X_dev);
/* Its adjoint: GY[k][b] = sum over the open beamlets i of beam k of GX[i][b]
 * (rows, then columns, in order), plus, if Y_dev is not NULL, the gradient of
 * gamma*G(Y) (Eq. 2) times w[b] (w_dev [32] or NULL: 1).  GX_dev [B][32],
 * Y_dev [N][32], GY_dev [N][32] float. */
VMAT_API vmat_status vmat_aperture_adjoint_batch32(vmat_ctx *ctx, const int16_t *l_dev,
                                                   const int16_t *r_dev, const float *GX_dev,
                                                   const float *Y_dev, const float *w_dev,
                                                   float *GY_dev);
/* The differentiable forward in aperture intensities (Eq. 3) for 32
 * intensity vectors on fixed apertures: X = A Y (as
 * vmat_aperture_fluence_batch32; X_dev [B][32] float, written), Z = D^T X
 * (Z_dev [n_vox][32] float), F'(Z) (fprime_dev [n_vox][32] float, or NULL)
 * and cost_host [32] = sum_j F(Z[j][b]) + gamma * G(Y[:, b]), both parts
 * reduced in FP64 (Eq. 1 and Eq. 2, ring if the context is cyclic). */
VMAT_API vmat_status vmat_aperture_dose_cost_batch32(vmat_ctx *ctx, const int16_t *l_dev,
                                                     const int16_t *r_dev, const float *Y_dev,
                                                     float *X_dev, float *Z_dev, float *fprime_dev,
                                                     double *cost_host);
/* Smoothing term of Eq. 2 (ring if the context is cyclic) for 32 intensity
 * vectors: G_host [32] (FP64) and, if dG_dev is not NULL, dG/dY [N][32]. */
VMAT_API vmat_status vmat_smoothing_batch32(vmat_ctx *ctx, const float *Y_dev, double *G_host,
                                            float *dG_dev);

/* Master-kernel CTA budget of a plan: tile its persistent master kernel for
 * at most max_ctas co-resident CTAs (0: every SM).  Used to run several plans'
 * master kernels side by side on disjoint SMs.  The plan must have no
 * columns (call vmat_reset first); re-allocates the aperture-dose matrix. */
VMAT_API vmat_status vmat_set_master_budget(vmat_ctx *ctx, int32_t max_ctas);

/* Method of the master problem (Sec. 2.2 solves it by the gradient
 * projection method).
 * VMAT_MASTER_PROJECTED_GRADIENT (default): the paper's method, with a
 *   Barzilai-Borwein step and an exact line search on [0, 1].
 * VMAT_MASTER_PROJECTED_NEWTON: not in the paper; a second-order member of
 *   the same family (projected Newton).  Each iteration forms the Hessian of
 *   Eq. 3 on the free set F = {y > 0 or g < 0} (the aperture columns' Gram
 *   matrix weighted by 2 alpha_j or 2 beta_j, plus the smoothing term's
 *   Laplacian) on the GPU, drops the variables at zero that the Newton step
 *   would push below zero, scales the step to the longest one in [0, 1] that
 *   keeps y >= 0 (ratio test) and then takes the same exact line search;
 *   where the factorisation fails or the step does not descend it takes the
 *   gradient-projection step.  Same stopping rule, same optimum; far fewer
 *   iterations on ill-conditioned columns (a per-variable projection of the
 *   Newton step, tried as well, needs 2-10x more iterations).
 * Switchable at any time (no re-tiling); VMAT_EINVAL for an unknown method or
 * if the variant's shared memory does not fit the current launch shape. */
typedef enum {
  VMAT_MASTER_PROJECTED_GRADIENT = 0,
  VMAT_MASTER_PROJECTED_NEWTON = 1
} vmat_master_method;
VMAT_API vmat_status vmat_set_master_method(vmat_ctx *ctx, int32_t method);

/* Arithmetic of the master problem's iterate.  extended = 0 (default): the
 * dose excess e = z - T of every voxel is an FP32 value carried by the
 * updates e += t w and recomputed from y every 16th iteration with
 * compensated sums; gradients are compensated FP32 dot products.  Its
 * rounding floor lets the relative KKT residual reach about 1e-9.
 * extended = 1: e, F'(z) and each structure's T, alpha and beta are float
 * pairs (about 48 bits), the gradient dot products take F' as a pair, and y
 * moves by exactly the FP32 step and direction that the excess moves by;
 * the floor drops to about 1e-12 at roughly 1.3x the time per iteration.
 * For comparisons with an FP64 solver decision by decision.  Available up
 * to 16 active voxels per master thread (about 1.2M active voxels);
 * VMAT_EINVAL beyond that or if the variant does not fit an SM.  Read by
 * every later master launch. */
VMAT_API vmat_status vmat_set_master_precision(vmat_ctx *ctx, int32_t extended);

/* Price of a beam in the pricing subproblem (Sec. 2.2).  on = 0 (default):
 * the least summed beamlet price of a feasible aperture, as the paper states
 * it.  on = 1: that sum plus gamma * dG/dy_k of Eq. 2 at the current y, which
 * makes it the exact reduced cost (the derivative of Eq. 3 along the new
 * column): for a beam without an aperture (y_k = 0) the added term is
 * -2 gamma (y_{k-1} / gap_left + y_{k+1} / gap_right), gaps in degrees, the
 * wrap pair on a ring, computed in FP64 and added after the row sum.  The
 * aperture of each beam is unchanged (the term is constant per beam); only
 * the choice of beam and the recorded prices change.  Read by every pricing
 * enqueued after the call (a batch re-captures its graph when it changes).
 * VMAT_EINVAL unless on is 0 or 1. */
VMAT_API vmat_status vmat_set_price_smoothing(vmat_ctx *ctx, int32_t on);

/* How the FP32 beamlet prices g = D f (Sec. 2.2) are formed, in vmat_price
 * and in every pricing of vmat_colgen_run (the extended-precision master
 * keeps its own FP64 row products).  Eq. 1 is one-sided, so at a master
 * solution F'(z_j) = 0 for all but a few percent of the voxels.
 *   VMAT_PRICE_AUTO (default): per call, on the device, the live-voxel form
 *     when the voxel-major rows of the voxels with f_j != 0 hold at most 1/16
 *     of D's entries, else the row products;
 *   VMAT_PRICE_ROWS: always the beamlet-major row products (warp per row,
 *     FP32 sums in the row's stored order);
 *   VMAT_PRICE_LIVE: always the live-voxel form: only the voxel-major rows
 *     with f_j != 0 are read; each product D_ij f_j (exact in FP64) is
 *     rounded to a fixed-point step 2^-S and summed in a 64-bit integer per
 *     beamlet, S chosen per call from max_j |f_j| and the largest row sum of
 *     D so that no sum overflows.  Integer sums do not depend on the order
 *     of the adds, so the result is deterministic; its error before the one
 *     rounding to FP32 is below 1e-15 of max|f| x (largest row sum).  A
 *     non-finite f falls back to the row products.
 * Read by every call enqueued after it (a batch re-captures its graph when it
 * changes).  VMAT_EINVAL for another value. */
#define VMAT_PRICE_AUTO 0
#define VMAT_PRICE_ROWS 1
#define VMAT_PRICE_LIVE 2
VMAT_API vmat_status vmat_set_price_path(vmat_ctx *ctx, int32_t path);

/* Dose-rate feasibility of the final plan (Sec. 3).  Eq. 2 only penalises
 * the dose-rate variation between neighbouring beams; as a hard limit the
 * paper raises gamma and re-optimises the intensities of the final apertures
 * until the plan is feasible.  Feasible: for every pair of neighbouring beams
 * (the wrap pair too when cyclic; beams without an aperture count with y = 0)
 * |y_k' - y_k| / gap <= max_rate, gap in degrees.  The paper gives no limit:
 * max_rate (intensity units per degree, >= 0) is the caller's.  Each round
 * multiplies gamma by gamma_factor (> 1) and solves the master problem again
 * from the current y (gradient-projection or projected-Newton method as set,
 * kkt_tol and the plan's reference residual as in vmat_colgen_run), at most
 * max_rounds rounds (0: only check).  Out (each may be NULL): y_host [N]
 * final intensities (also the plan's y), gamma_out the final gamma,
 * rounds_out rounds taken, violation_out max over pairs of |dy|/gap -
 * max_rate (<= 0 when feasible), cost_out Eq. 3 at the end with the final
 * gamma.  The context keeps its own gamma.  VMAT_ENOTCONV if the limit is
 * still exceeded after max_rounds (outputs written). */
VMAT_API vmat_status vmat_dose_rate_feasibility(vmat_ctx *ctx, double max_rate, double gamma_factor,
                                                int32_t max_rounds, int32_t master_max_iters,
                                                double kkt_tol, double *y_host, double *gamma_out,
                                                int32_t *rounds_out, double *violation_out,
                                                double *cost_out);

/* Plan quality (the evaluation behind Fig. 2; not part of the optimisation):
 * dose-volume histogram counts per structure of a dose vector z_dev [n_vox]
 * float on the device (e.g. from vmat_plan_dose).  Voxel j goes to bin
 * floor(z_j * s) of its structure, s = n_bins / dose_max rounded to FP32
 * once, the product in FP32, clamped to [0, n_bins - 1] (the last bin holds
 * doses >= dose_max too).  counts_host [n_struct * n_bins] int64, structure
 * major, host memory; exact integer counts.  VMAT_EINVAL for dose_max <= 0,
 * n_bins outside 1..4096, or more than 24,576 structure bins in all. */
VMAT_API vmat_status vmat_dvh(vmat_ctx *ctx, const float *z_dev, double dose_max, int32_t n_bins,
                              int64_t *counts_host);

/* ---- many independent plans (planning throughput; not in the paper) ----
 * A batch groups existing contexts (not owned).  Every plan's master kernel
 * gets a CTA budget (its SM "tokens"); a list schedule decides which plans
 * run side by side, and each plan starts after the plans whose tokens it
 * takes over, so plans that overlap always hold disjoint SMs.  The whole run
 * (reset + all iterations of every plan) is captured once into a CUDA graph
 * with those dependencies and replayed with one launch.  While a plan
 * belongs to a batch its context runs on a stream of the batch. */
typedef struct vmat_batch vmat_batch;
VMAT_API vmat_status vmat_batch_create(vmat_ctx *const *plans, int32_t n_plans, void *cuda_stream,
                                       vmat_batch **out);
VMAT_API void vmat_batch_destroy(vmat_batch *b);
VMAT_API const char *vmat_batch_last_error(const vmat_batch *b);
/* SM share (1..SMs): plan p's master kernel gets max(SMs / share, the CTAs
 * that keep it at <= 16 voxels per thread) CTAs, at most SMs.  Plans are
 * placed largest estimated work (active voxels x beams per CTA) first, each
 * on the SM tokens that free up earliest.  share = 1 runs the plans one after
 * another on the whole GPU.  VMAT_EINVAL if share is out of range or a plan
 * does not fit the GPU. */
VMAT_API vmat_status vmat_batch_configure(vmat_batch *b, int32_t share);
/* Autotuner: times a captured trial run of the first trial_iters iterations
 * of every plan for shares 1, 2, 3 and 4 (ms_out [4], -1 where not tried)
 * and configures the fastest (share_out). */
VMAT_API vmat_status vmat_batch_tune(vmat_batch *b, int32_t trial_iters, int32_t master_max_iters,
                                     double kkt_tol, int32_t *share_out, double *ms_out);
/* The batch's list schedule, exposed for testing (host only, no GPU):
 * n plans with CTA budgets budget [n] (1..sms) and estimated work est [n]
 * (>= 0) on sms SM tokens.  Out: order [n] capture order (decreasing est,
 * stable); ndep [n] and deps [n*n] (row p, first ndep[p] entries) the plans
 * each plan must wait for; tokens [n*sms] (or NULL) 1 where plan p holds
 * token t.  Any two plans holding a common token are ordered by the
 * dependencies, so plans that may overlap hold disjoint tokens.
 * VMAT_EINVAL on bad sizes. */
VMAT_API vmat_status vmat_list_schedule(int32_t n, const int32_t *budget, const double *est,
                                        int32_t sms, int32_t *order, int32_t *ndep, int32_t *deps,
                                        uint8_t *tokens);
/* Run every plan's full column generation (one aperture per beam) from an
 * empty plan as one graph launch.  res [n_plans] as for vmat_colgen_run
 * (phase_ms unused), plan_ms [n_plans] time from the launch to each plan's
 * end, total_ms the whole launch (either may be NULL).  The graph is captured
 * on the first run and again whenever the arguments or a plan's settings
 * (gamma, master method, smoothing-aware pricing) changed since. */
VMAT_API vmat_status vmat_batch_colgen_run(vmat_batch *b, int32_t master_max_iters, double kkt_tol,
                                           vmat_colgen_result *res, double *plan_ms,
                                           double *total_ms);

/* Dose and voxel cost without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not let a
 * library allocate GPU memory (a host framework that owns a fixed device pool
 * and forbids cudaMalloc behind its back, a service that may not allocate
 * while it serves plans, an embedded integration that sizes every buffer up
 * front).  It needs no context: the caller passes the voxel-major D as CSR
 * over its n_vox voxels (row_ptr_dev [n_vox+1] int64, beamlet_dev [nnz]
 * int32 beamlet of each entry, val_dev [nnz] float D_ij), the fluence x_dev
 * [B] float, struct_id_dev [n_vox] uint8 (< n_struct) and params_dev
 * [3*n_struct] double (the voxel cost's per-structure thresholds T, then its
 * underdose weights alpha, then its overdose weights beta), and gets z_dev
 * [n_vox] float and fprime_dev [n_vox] float F'(z) (either may be NULL) and
 * cost_dev [1] double = sum_j F(z_j) reduced in FP64 in a fixed order.  A
 * voxel whose structure id is >= n_struct gets F' = NaN and makes the cost
 * NaN (its parameters are not read).  Everything is enqueued on cuda_stream (a cudaStream_t, NULL: legacy
 * default stream) and the call returns without waiting.
 * Its only scratch, one FP64 partial cost per 8 voxels, is a file-scope
 * __device__ array of 65,536 doubles (512 KiB) that every GPU loading the
 * library keeps until the process exits; n_vox above 524,288 is rejected
 * with VMAT_EINVAL.  All calls share that array and it keeps the last call's
 * contents, so calls that may overlap on the GPU (different streams, or
 * different threads) race and must be serialised by the caller.  The first
 * call on each device looks up the array's device address (with that device
 * current) and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call this entry point on a device
 * after cudaDeviceReset of that device (the kept address belongs to the old
 * context).  Errors are reported by vmat_last_error(NULL). */
VMAT_API vmat_status vmat_dose_cost_noalloc(int32_t n_vox, const int64_t *row_ptr_dev,
                                            const int32_t *beamlet_dev, const float *val_dev,
                                            const float *x_dev, const uint8_t *struct_id_dev,
                                            const double *params_dev, int32_t n_struct,
                                            float *z_dev, float *fprime_dev, double *cost_dev,
                                            void *cuda_stream);

/* Self-test of the bounded device waits (no counterpart in the method):
 * launches the master kernel's grid barrier with every CTA but one waiting
 * for a CTA that never arrives, each wait limited to wait_seconds.  Returns
 * VMAT_ETIMEOUT when the waits ran out as designed (the context stays
 * usable), VMAT_OK if skip_one == 0 and the barrier completed normally. */
VMAT_API vmat_status vmat_selftest_grid_wait(vmat_ctx *ctx, int32_t skip_one, double wait_seconds);

#ifdef __cplusplus
}
#endif
#endif /* VMAT_H */
