/*
 * lp.h -- C ABI of liblp.so, the GB300 (sm_103a) hot path of the Lagrangian
 * particle (LP) method of Yuan, Zepeda Aguilar, Naitlho and Samulyak,
 * "Massively-Parallel Lagrangian Particle Code and Applications" (Sec. 2).
 *
 * The library advances the compressible Euler equations in Lagrangian form
 * (Sec. 2.1, Eqs. mass, momentum, energy, eos) for an ideal gas, one particle
 * per fluid parcel, with the per-step algorithm of Sec. 2.2:
 *   neighbour search on a space-filling-curve ordering   -> lp_build_neighbors
 *   GFD least-squares derivatives (Eq. linear_system_axb) -> lp_gfd_derivs,
 *                                                           lp_onesided_derivs
 *   Lax-Wendroff / upwind rates, state estimator, limiter
 *   blend and particle mover (Eq. timeIntegrate)          -> lp_step
 *
 * Conventions for every entry point
 *   - Pointers named "device" are CUDA device pointers; "host" pointers are
 *     ordinary host memory.  Particle and field buffers are owned by the caller
 *     and never freed by the library.  The context owns its scratch (sort
 *     buffers, cell tables, neighbour lists) and frees it in lp_destroy.
 *   - Work is enqueued asynchronously on the given CUDA stream (0 = legacy
 *     default stream).  Host-side argument errors return immediately without
 *     enqueuing anything.  Conditions found on the device (capacity overflow,
 *     ill-conditioned stencils, non-finite states) are accumulated in a device
 *     status word that lp_get_stats reads; no entry point aborts or traps.
 *   - A context must not be used from two host threads at once.
 *   - Positions, state and time are float64 structure-of-arrays.
 */
#ifndef LP_H
#define LP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lp_stream;   /* a cudaStream_t */

typedef enum {
    LP_OK = 0,
    LP_ERR_ARG = 1,        /* invalid argument (null pointer, bad size or mode) */
    LP_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    LP_ERR_CAPACITY = 3,   /* n exceeds the context capacity */
    LP_ERR_ILLCOND = 4,    /* a stencil had no usable fit (see lp_stats) */
    LP_ERR_NONFINITE = 5,  /* a non-finite state or time step was produced */
    LP_ERR_TIMEOUT = 6,    /* a bounded device wait gave up */
    LP_ERR_STATE = 7       /* entry point called in the wrong order */
} lp_status;

enum { LP_PREC_FP32 = 0,   /* fits in FP32 with FP64 redo of ill-conditioned stencils */
       LP_PREC_FP64 = 1 }; /* every fit in FP64 */

enum { LP_RADIUS_FIXED = 0,   /* j is a neighbour of i iff |x_j - x_i| <= radius */
       LP_RADIUS_VOLUME = 1,  /* ... iff |x_j - x_i| <= kappa (m_i V_i)^(1/dim) */
       LP_RADIUS_KSIDE = 2 }; /* 1D only: k_per_side nearest on each side */

enum { LP_LIM_FLAGGED = 0,  /* phi(r_s) where the estimator flags, pure LW elsewhere */
       LP_LIM_PAPER = 1,    /* phi(r_s) at every particle */
       LP_LIM_LW = 2,       /* Lax-Wendroff only (phi = 1) */
       LP_LIM_UW = 3 };     /* upwind only (phi = 0) */

enum { LP_EST_PLAIN = 0,    /* state estimator of Sec. 2.1 */
       LP_EST_MLP = 1 };    /* learned estimator, plain estimator as fallback */

enum { LP_OUT_F32 = 0, LP_OUT_F64 = 1 };

/*
 * Method and layout parameters (host struct, copied by lp_create).
 *   dim            1, 2 or 3.
 *   precision      LP_PREC_*.
 *   radius_mode    LP_RADIUS_*; radius / kappa as the mode needs.
 *   k_max          neighbour capacity per particle, 1..80; which neighbours
 *                  are kept when more lie inside the radius: see `select`.
 *   k_side         one-sided stencil size per half-space (Sec. 2.2 step 5
 *                  uses 8 in 3D), 1..16.
 *   k_per_side     LP_RADIUS_KSIDE only, 1..8.
 *   gamma          ideal-gas exponent, > 1.
 *   limiter, estimator   LP_LIM_*, LP_EST_*.
 *   flat_eps, active_frac, s_ref[5]   state-estimator constants: a field whose
 *                  one-sided derivatives d satisfy max|d| * ell <= flat_eps *
 *                  max(|s|, s_ref) is treated as locally constant (r = 1); axes
 *                  with max(|s_l|,|s_r|) < active_frac * (largest over axes) are
 *                  ignored.  Field order V, u_1..u_dim, P.
 *   tau32, tau64   FP32 fits whose min|R_kk|/max|R_kk| (column-scaled) falls
 *                  below tau32 are redone in FP64; below tau64 (FP64) the
 *                  second-order fit is replaced by the first-order one.
 *   periodic[3], box_lo[3], box_hi[3]   periodic axes use the minimum image
 *                  and wrap moved particles; a periodic box must be a cube and
 *                  periodic on all dim axes (LP_ERR_ARG otherwise).
 *   n_fluid        particles whose id >= n_fluid are frozen boundary
 *                  particles: neighbours of others, never updated or moved.
 *   capacity       largest n any call will pass (scratch is sized for it).
 *   max_level      finest cell level of the Morton cell tables (0 = automatic, <= 17).
 *   mlp_tau_lo     LP_EST_MLP: a particle whose learned flag probability is
 *                  below this is treated as unflagged (pure Lax-Wendroff) without
 *                  its one-sided fits; otherwise the plain estimator decides.
 *   mlp_audit      LP_EST_MLP: also run the plain estimator on every particle and
 *                  count the skipped particles it would have flagged (the miss
 *                  count in lp_stats); the update still follows the learned call.
 *   max_sims       most simulations one lp_step_batched call advances (0 or 1:
 *                  one).  2D keys keep 21 bits per axis; 3D keys with several
 *                  simulations keep min(21, (64 - ceil(log2 max_sims)) / 3).
 *   refine         the FP32 central fit's correction pass (one step of the
 *                  semi-normal equations on the first solution's residual):
 *                  LP_REFINE_AUTO (0, the default) where min|R_kk|/max|R_kk| <
 *                  refine_ratio, i.e. where cond(A)^2 u of the normal
 *                  equations is not negligible; LP_REFINE_ALWAYS (1);
 *                  LP_REFINE_NEVER (2).  On the jittered-lattice GFD workload
 *                  AUTO and ALWAYS give the same gradients (error 2.5e-6; a
 *                  well-conditioned stencil's correction rounds away), NEVER
 *                  1.8e-4; on the 2M gas cloud AUTO corrects ~3% of the
 *                  stencils and its state after a step is within 2e-7 of
 *                  ALWAYS's.
 *   refine_ratio   LP_REFINE_AUTO threshold (0: 0.1).
 *   select         which k_max neighbours are kept when more lie inside the
 *                  radius (Sec. 2.2 step 4): LP_SELECT_NEAREST (0) the k_max
 *                  nearest by (d^2, id); LP_SELECT_OCTANT (1) round robin over
 *                  the octants (quadrants in 2D) of the offsets, nearest first
 *                  in each, so that the list covers all directions.  Either way
 *                  the list is stored in (d^2, id) order, and with at most k_max
 *                  inside the radius the two agree.  LP_SELECT_OCTANT needs dim
 *                  2 or 3 and a radius (not LP_RADIUS_KSIDE).
 *   reserved       0.
 *   t_end          end time (0: none).  When a step is given the device time t
 *                  (lp_step's `t`), its time step is clipped to t_end - t, so the
 *                  last step ends at t_end; a simulation already at t_end takes
 *                  a step of 0 (its state does not change).
 */
typedef struct {
    int32_t dim;
    int32_t precision;
    int32_t radius_mode;
    int32_t k_max;
    int32_t k_side;
    int32_t k_per_side;
    int32_t limiter;
    int32_t estimator;
    double gamma;
    double radius;
    double kappa;
    double flat_eps;
    double active_frac;
    double s_ref[5];
    double tau32;
    double tau64;
    int32_t periodic[3];
    int32_t max_level;
    double box_lo[3];
    double box_hi[3];
    int64_t n_fluid;
    int64_t capacity;
    double mlp_tau_lo;
    int32_t mlp_audit;
    int32_t max_sims;
    int32_t refine;
    double refine_ratio;
    int32_t select;
    int32_t reserved;
    double t_end;
} lp_config;

enum { LP_SELECT_NEAREST = 0, LP_SELECT_OCTANT = 1 };

enum { LP_REFINE_AUTO = 0, LP_REFINE_ALWAYS = 1, LP_REFINE_NEVER = 2 };

/* Caller-owned device particle arrays (SoA, float64; id uint32).  Unused axes
 * (>= dim) may be NULL. */
typedef struct {
    int64_t n;
    double *x[3];
    double *V;        /* specific volume 1/rho */
    double *u[3];
    double *P;
    double *m;        /* particle mass (never modified, only permuted) */
    uint32_t *id;
} lp_particles;

/* Read-only view of the context-owned neighbour lists (device pointers),
 * valid until the next call that rebuilds them. */
typedef struct {
    int64_t n;
    int32_t k_max;             /* row stride of idx */
    int32_t pad;
    const uint32_t *count;     /* [n] list length, <= k_max */
    const uint32_t *total;     /* [n] neighbours inside the radius before truncation,
                                  saturated at 4 k_max */
    const uint32_t *idx;       /* [n][k_max] indices into the permuted particle arrays,
                                  in (d^2, id) order */
    const double *d2min;       /* [n] squared distance of the nearest neighbour */
    const uint64_t *keys;      /* [n] Morton keys of the permuted particles */
} lp_neighbors;

/* Counters accumulated since the last lp_reset_stats (host struct). */
typedef struct {
    double dt;                 /* last time step used */
    int64_t steps;
    int64_t n_flagged;         /* particle-steps flagged by the estimator */
    int64_t n_fp64_redo;       /* FP32 fits redone in FP64 */
    int64_t n_linear;          /* fits that fell back to first order */
    int64_t n_nofit;           /* fits with no usable system (derivatives zero) */
    int64_t n_overflow;        /* particles with more than k_max neighbours */
    int64_t n_nonfinite;       /* non-finite states produced */
    int64_t n_mlp_uncertain;   /* learned-estimator calls deferred to the plain one */
    uint32_t max_count;        /* largest neighbour count seen */
    uint32_t status;           /* OR of LP_ERR_* bits (1 << code) seen on the device */
    int64_t kernel_launches;   /* kernels this context launched (host-side count) */
    int64_t n_mlp_skip;        /* particle-steps the learned estimator declared unflagged */
    int64_t n_mlp_miss;        /* ... of which the plain estimator flags (audit mode) */
    int64_t n_query_fallback;  /* particles of the last neighbour build listed by the warp-per-particle
                                  query (more than 64 neighbours, or a tile spread over too many cells) */
    int64_t n_refined;         /* FP32 central fits of lp_step that ran the correction pass */
} lp_stats;

typedef struct lp_ctx lp_ctx;

/* Create a context for cfg (validated; LP_ERR_ARG on a bad field). Allocates
 * scratch for cfg->capacity particles on the current CUDA device. */
lp_status lp_create(const lp_config *cfg, lp_ctx **out);

/* Free the context and its scratch. NULL is accepted. */
lp_status lp_destroy(lp_ctx *ctx);

/*
 * Sec. 2.2 steps 2-4: Morton keys of the positions (the Z-curve order of
 * Sec. 2.2 "Space-filling curve"), radix sort, permutation of every particle
 * array IN PLACE into that order, cell tables, and the neighbour query
 * {j != i : |x_j - x_i| <= R_i} ordered by (d^2, id) and truncated to k_max.
 * FP64 distances with the fixed operation order ((dx*dx + dy*dy) + dz*dz)
 * decide membership and order, so the lists are exact.
 * out (host struct) receives the view of the lists.
 */
lp_status lp_build_neighbors(lp_ctx *ctx, lp_particles *p, lp_neighbors *out, lp_stream stream);

/*
 * Central second-order GFD derivatives (Sec. 2.1, Eq. linear_system_axb and its
 * 1D/3D analogues) of nfields fields on the lists of the last
 * lp_build_neighbors (whose permuted particles p must be).  fields: host array
 * of nfields device pointers (float64 [n], in the permuted order).
 * derivs: device [nfields][n][n_u] of out_dtype, n_u = 2/5/9 for dim 1/2/3,
 * unknowns ordered (d_1.., d_11.., mixed d_12, d_13, d_23).
 * status: optional device uint32 [n] of per-particle fit flags
 * (1 linear fallback, 2 no fit, 8 FP64 redo).
 */
lp_status lp_gfd_derivs(lp_ctx *ctx, const lp_particles *p, const double *const *fields,
                        int32_t nfields, int32_t out_dtype, void *derivs, uint32_t *status,
                        lp_stream stream);

/*
 * One-sided first derivatives (Sec. 2.1, the left/right derivatives of the
 * upwind scheme): for each axis k and side (0 left, 1 right) the first k_side
 * list members with x_jk on that side are fitted to first order and component
 * k kept; with fewer than dim members the central derivative is used.
 * derivs: device float64 [n][dim][2][nfields].
 */
lp_status lp_onesided_derivs(lp_ctx *ctx, const lp_particles *p, const double *const *fields,
                             int32_t nfields, double *derivs, lp_stream stream);

/*
 * One LP time step (Sec. 2.2 steps 2-6): neighbours, fits, Lax-Wendroff and
 * upwind rates, state estimator, limiter blend
 *   s^{n+1} = s^n + dt (UW - phi (UW - LW))
 * and the mover x^{n+1} = x^n + dt (u^n + u^{n+1}) / 2 (Eq. timeIntegrate).
 * p is permuted into Morton order and advanced in place.
 *   dt > 0 : that step;  dt <= 0 : dt = cfl * min_i ell_i / c_i on the device
 *            (ell_i nearest-neighbour distance, c_i = sqrt(gamma P_i V_i)).
 *   t      : optional device float64 scalar, incremented by dt on the device.
 *   diag   : optional device outputs (any may be NULL): flag uint8 [n],
 *            phi float32 [n][nf], r float32 [n][nf] (nf = dim + 2),
 *            features float32 [n][8] (see lp_mlp_*), gate_p float32 [n].
 */
typedef struct {
    uint8_t *flag;
    float *phi;
    float *r;
    float *features;   /* float32 [n][8]: the learned estimator's inputs */
    float *gate_p;     /* float32 [n]: LP_EST_MLP only, the learned estimator's
                          probability that the particle is flagged (a particle
                          below mlp_tau_lo skips the plain estimator); frozen
                          boundary particles get 0; not written otherwise */
} lp_step_diag;

lp_status lp_step(lp_ctx *ctx, lp_particles *p, double dt, double cfl, double *t,
                  const lp_step_diag *diag, lp_stream stream);

/*
 * lp_step on particles in HOST memory (single-simulation contexts).  The host
 * arrays of h are copied into a device copy the context owns (allocated at
 * capacity on the first call): positions, m and V on `stream`, the other
 * fields on a second stream of the context while the keys are sorted.  When
 * every array of h is page-locked (cudaHostAlloc / cudaHostRegister), the
 * step's kernels write the new, Morton-ordered state straight into them, so
 * no copy back follows the step; otherwise it is copied back on `stream`.
 * Either way h holds on completion of `stream` what lp_step leaves in p.
 * h must not be read or written by the host until then.  t and diag are
 * device pointers as for lp_step.  LP_ERR_STATE for a batched context.
 */
lp_status lp_step_host(lp_ctx *ctx, lp_particles *h, double dt, double cfl, double *t,
                       const lp_step_diag *diag, lp_stream stream);

/*
 * Copy the lists of the last lp_build_neighbors / lp_step into caller-owned
 * device buffers (any may be NULL): count/total uint32 [n], idx uint32
 * [n][k_max], d2min float64 [n], keys uint64 [n] (Morton keys of the permuted
 * particles).  Enqueued on `stream`.
 */
lp_status lp_export_neighbors(lp_ctx *ctx, uint32_t *count, uint32_t *total, uint32_t *idx,
                              double *d2min, uint64_t *keys, lp_stream stream);

/*
 * All-octant coverage check of the central stencils (Sec. 2.1: the
 * second-order stencils are meant to include particles from all 8 octants).
 * For every particle of the last neighbour build (key order, as
 * lp_export_neighbors), gap[i] = 1 when its list misses one of the 2^dim
 * sign patterns of the offsets x_j - x_i (an offset of exactly 0 counted as
 * positive), else 0; gap (device, n bytes) may be null.  *n_gap (host) = the
 * number of such particles.  The signs come from the float hi/lo offsets the
 * fits use.  Synchronises `stream`.  LP_ERR_STATE when the lists are stale,
 * LP_ERR_ARG in the k-per-side mode.
 */
lp_status lp_octant_coverage(lp_ctx *ctx, uint8_t *gap, int64_t *n_gap, lp_stream stream);

/*
 * Synchronise `stream` and read the quantisation cube of the last build into
 * host out[5] = {lo_0, lo_1, lo_2, L, finest level}: Morton coordinates are
 * q_k = floor((x_k - lo_k) * 2^21 / L), clamped to [0, 2^21 - 1].
 */
lp_status lp_grid_info(lp_ctx *ctx, double *out, lp_stream stream);

/*
 * Learned state estimator (no counterpart in the paper beyond the plain
 * estimator it imitates): an 8 -> 32 (ReLU) -> 1 (sigmoid) network on eight
 * dimensionless stencil features of each particle (from its central fit: the
 * scaled |grad P|, |grad V|, |Hess P|, |Hess V|, divergence over sound speed,
 * largest rise and fall of P over the neighbours, relative residual of the P
 * fit; each transformed as log(1 + 10|f|), the divergence keeping its sign).
 * BF16 weights with FP32 accumulation on the device, FP32 master weights.
 * Parameters (LP_MLP_NPARAM floats): W1[32][8] row-major, b1[32], w2[32], b2.
 *   lp_mlp_set_params   upload master weights (host), reset Adam.
 *   lp_mlp_get_params   download master weights and/or the BF16 values (host).
 *   lp_mlp_grad         loss and gradient of the mean class-weighted BCE
 *                       (weight pos_weight on y = 1) over n samples X [n][8],
 *                       y [n] (device), at the BF16 weights; grad [NPARAM] and
 *                       loss [1] are device float32.
 *   lp_mlp_adam_step    one Adam step (beta 0.9/0.999, eps 1e-8) with grad (device).
 *   lp_mlp_train        minibatch Adam over the samples in order, `epochs` passes;
 *                       epoch_loss (host, may be NULL) gets the mean batch loss.
 *   lp_mlp_infer        probabilities p [n] (device) for features X.
 */
#define LP_MLP_NPARAM 321
lp_status lp_mlp_set_params(lp_ctx *ctx, const float *params);
lp_status lp_mlp_get_params(lp_ctx *ctx, float *master, float *bf16_as_float);
lp_status lp_mlp_grad(lp_ctx *ctx, const float *X, const float *y, int64_t n, double pos_weight,
                      float *grad, float *loss, lp_stream stream);
lp_status lp_mlp_adam_step(lp_ctx *ctx, const float *grad, double lr, lp_stream stream);
lp_status lp_mlp_train(lp_ctx *ctx, const float *X, const float *y, int64_t n, int32_t epochs,
                       int32_t batch, double lr, double pos_weight, float *epoch_loss, lp_stream stream);
lp_status lp_mlp_infer(lp_ctx *ctx, const float *X, int64_t n, float *p, lp_stream stream);

/*
 * Phase timing.  With profiling on, every entry point records CUDA events on
 * its stream around each phase; lp_phase_times synchronises the stream and
 * adds, per phase, the elapsed milliseconds and launch count since the last
 * reset into host out_ms[LP_NPHASES] / out_launches[LP_NPHASES] (either may be
 * NULL), then clears them.  lp_phase_name(k) is the phase's static name.
 */
enum { LP_PH_GRID = 0, LP_PH_SORT = 1, LP_PH_GATHER = 2, LP_PH_TABLES = 3, LP_PH_QUERY = 4,
       LP_PH_CFL = 5, LP_PH_FIT = 6, LP_PH_FIT64 = 7,
       LP_PH_HOST_IN = 8,     /* lp_step_host: copies on the caller's stream, and the
                                 wait for the second stream's copies before the gather */
       LP_PH_HOST_OUT = 9,    /* lp_step_host on pageable arrays: the copy back */
       LP_NPHASES = 10 };
lp_status lp_set_profiling(lp_ctx *ctx, int32_t on);
lp_status lp_phase_times(lp_ctx *ctx, double *out_ms, int64_t *out_launches, lp_stream stream);
const char *lp_phase_name(int32_t phase);

/*
 * Morton keys of n positions and their sort order, computed without allocating
 * any device memory.  The paper has no counterpart: this serves callers that
 * cannot allocate device memory at the point they need the key order -- a host
 * application whose own pool owns all device memory and forbids other
 * allocations, or a latency-critical loop that cannot afford cudaMalloc's
 * implicit device-wide synchronisation.
 *
 * Computes what lp_build_neighbors computes for its keys and order with a
 * default configuration (non-periodic bounding cube, keys sorted by their cell
 * bits down to level 9 in 3D / 13 in 2D, ties in input order; 1D: the exact
 * order of x): keys_out[i] is the key of the i-th particle in sorted order and
 * perm_out[i] its input index.  x0..x2: device float64 [n] (unused axes may be
 * NULL); keys_out uint64 [n], perm_out uint32 [n]: caller-owned device buffers.
 *
 * Scratch: one fixed device array inside the library, sized for
 * LP_NOALLOC_MAX_N particles (about 6 MiB), which every GPU that loads the
 * library holds until the process exits.  n > LP_NOALLOC_MAX_N returns
 * LP_ERR_CAPACITY without enqueuing anything.  Each call made outside stream
 * capture looks up the array's device address on the current device (no
 * allocation; this also follows a cudaDeviceReset); a call on a capturing
 * stream uses the address of the last call outside capture on that device, so
 * make one call on each device before any stream capture (LP_ERR_CUDA
 * otherwise).  All calls
 * share the one array: calls whose work overlaps on the GPU (different streams,
 * or different host threads) race and corrupt each other's results, so
 * serialise them.  No cudaMalloc, cudaFree or allocating library routine is
 * called.
 */
#define LP_NOALLOC_MAX_N 262144
lp_status lp_sort_keys_noalloc(int32_t dim, int64_t n, const double *x0, const double *x1,
                               const double *x2, uint64_t *keys_out, uint32_t *perm_out,
                               lp_stream stream);

/*
 * Reservoir inflow through a nozzle inlet (Sec. 4, "Supersonic jets for
 * LPWA": a nozzle attached to a high-pressure reservoir, modelled by a
 * boundary condition at the inlet).  The inflow state follows the three
 * hypotheses printed there:
 *   P_inf   the mean pressure of the fluid particles near the inlet (those
 *           within `radius` of the axis and within `sample_depth` past the
 *           inlet plane); the reservoir pressure P_res on the first call;
 *   rho_inf the reservoir's entropy: P_res / rho_res^gamma = P_inf / rho_inf^gamma;
 *   u_inf   along the axis, from the enthalpy balance with the reservoir at
 *           rest: u_inf^2 / 2 + c_inf^2 / (gamma - 1) = c_res^2 / (gamma - 1),
 *           c^2 = gamma P / rho; no transverse component.
 * Injected particles sit on a square lattice of in-plane spacing `spacing`
 * clipped to the inlet disk (npat points per layer), each with mass `mass`, so
 * a layer's axial thickness is h_z = mass / (rho_inf spacing^2).  The axial
 * distance the inflow has travelled accumulates u_inf dt (dt: the last
 * lp_step's time step, 0 before the first step); each whole h_z of it
 * becomes one layer of fluid particles past the inlet, appended at the end of
 * the particle arrays with ids first_id + (layer index) npat + point.  Each
 * layer's lattice is shifted in-plane by a counter-based fraction of the
 * spacing (Weyl sequence of the layer index).  `ghost_layers` layers of frozen
 * reservoir particles (ids from ghost_id, which must be >= the configuration's
 * n_fluid) lie behind the inlet plane with the inflow state: appended on the
 * first call and rewritten (by id) on every call.
 *
 * p: device particle arrays with room for `capacity` particles, p->n in use.
 * On return *n_out = the new count (p->n plus what was appended).  When that
 * would exceed `capacity`, nothing is appended or advanced and
 * LP_ERR_CAPACITY is returned (grow the arrays, lp_reserve, call again).
 * info (host, may be NULL) receives the inflow state of this call.
 * Synchronises `stream` (the host reads the number of layers decided on the
 * device).  Every call must pass the same inlet; LP_ERR_ARG otherwise.
 */
typedef struct {
    double center[3];       /* centre of the inlet disk (on the inlet plane) */
    int32_t axis;           /* the inflow runs along +axis (0, 1, 2; 3D only) */
    int32_t ghost_layers;   /* reservoir layers behind the inlet, >= 0 */
    double radius;          /* inlet radius */
    double spacing;         /* in-plane lattice spacing of injected particles */
    double mass;            /* mass of each injected particle */
    double P_res, rho_res;  /* reservoir pressure and density */
    double sample_depth;    /* depth of the region whose mean pressure is P_inf */
    uint32_t first_id;      /* ids of injected fluid particles count up from here */
    uint32_t ghost_id;      /* ids of the reservoir ghosts count up from here */
} lp_inlet;

typedef struct {
    double P_inf, rho_inf, u_inf, c_inf;   /* the inflow state of this call */
    double h_z;                            /* axial thickness of a layer */
    double travel;                         /* inflow distance not yet a whole layer */
    int64_t layers;                        /* layers appended by this call */
    int64_t layers_total;                  /* layers appended since the first call */
    int64_t npat;                          /* particles per layer */
    int64_t sampled;                       /* fluid particles averaged into P_inf */
} lp_inflow_info;

lp_status lp_inflow(lp_ctx *ctx, lp_particles *p, int64_t capacity, const lp_inlet *inlet, int64_t *n_out,
                    lp_inflow_info *info, lp_stream stream);

/*
 * Outflow (Sec. 2.2 step 1: outflow boundaries delete particles): removes the
 * particles whose position is outside [lo_k, hi_k] on some axis k < dim, or
 * not finite, keeping the others in their order (stable, in place in p's
 * arrays); *n_out receives the count that remains.  The neighbour lists of the
 * last build are dropped.  lo, hi: host double[3].  Synchronises `stream`.
 */
lp_status lp_remove_outside(lp_ctx *ctx, lp_particles *p, const double *lo, const double *hi, int64_t *n_out,
                            lp_stream stream);

/*
 * Grow (or shrink) the context's scratch to `capacity` particles (at least the
 * n of the last build).  The neighbour lists of the last build are dropped (the
 * next call that needs them must rebuild) and a captured graph is discarded.
 * Synchronises the device.  No counterpart in the paper: the capacity growth
 * that particle insertion needs.
 */
lp_status lp_reserve(lp_ctx *ctx, int64_t capacity);

/*
 * Free-surface ghost particles (Sec. 2.2 step 3: where a free boundary
 * condition applies and a particle's neighbours are incomplete in some of the
 * axis directions, ghost particles are generated to complete them).  The
 * paper defers their placement and state; the reading here:
 *   - the neighbour lists of p are built (as lp_build_neighbors: p is permuted
 *     into key order);
 *   - direction (axis k, side s) of a fluid particle (id < n_fluid) with at
 *     least one neighbour is incomplete when fewer than `min_per_side` list
 *     members have an FP64 offset along k of sign s (0 counts on neither side);
 *   - each incomplete direction gets one ghost at x + s sqrt(d2min) e_k (the
 *     nearest-neighbour distance), with the particle's m, V and u, pressure
 *     `p_ghost` (0: vacuum) and id ghost_base + 2 dim id + 2k + (s > 0);
 *   - the ghosts are appended after the p->n particles in (particle, axis,
 *     side) order; *n_out = p->n + their count.
 * Ghosts are frozen in lp_step (ghost_base must be >= the configuration's
 * n_fluid, and ghost_base + 2 dim n_fluid <= 2^32, else LP_ERR_ARG); remove
 * them after the step with lp_remove_ghosts(ctx, p, ghost_base, ...).
 * Non-periodic, single-simulation contexts only (LP_ERR_ARG); min_per_side in
 * 1..k_max.  When p->n + ghosts > capacity (or capacity exceeds the context's)
 * nothing is appended and LP_ERR_CAPACITY is returned.  Synchronises `stream`
 * (the ghost count is read back).  The neighbour lists are stale afterwards.
 */
lp_status lp_free_surface_ghosts(lp_ctx *ctx, lp_particles *p, int64_t capacity, int32_t min_per_side,
                                 double p_ghost, uint32_t ghost_base, int64_t *n_out, lp_stream stream);

/*
 * Deletes the particles with id >= first_id (ghosts), keeping the order of the
 * others; *n_out = the count kept.  Synchronises `stream`; the neighbour lists
 * are stale afterwards.  LP_ERR_ARG for batched contexts.
 */
lp_status lp_remove_ghosts(lp_ctx *ctx, lp_particles *p, uint32_t first_id, int64_t *n_out, lp_stream stream);

/*
 * One LP step of nsim independent simulations stored back to back in p: the
 * particles of simulation s are [offsets[s], offsets[s+1]) (offsets: device
 * int64 [nsim + 1], offsets[0] = 0, offsets[nsim] = p->n; nsim <= max_sims).
 * One sort, one set of cell tables and one launch per phase serve all of
 * them: a key carries its simulation above the Morton bits, so every
 * simulation's particles stay at the same offsets after the step.  Each
 * simulation has its own bounding cube and its own CFL step (dt <= 0); the
 * periodic box of the configuration is shared.  t: optional device float64
 * [nsim], advanced by each simulation's step.  Otherwise as lp_step.
 */
lp_status lp_step_batched(lp_ctx *ctx, lp_particles *p, const int64_t *offsets, int32_t nsim,
                          double dt, double cfl, double *t, const lp_step_diag *diag,
                          lp_stream stream);

/*
 * CUDA-graph form of a step.  lp_graph_capture records one lp_step_batched
 * call (same arguments) on `stream` -- which must be a created stream, not the
 * legacy default stream -- into an executable graph kept by the context, without
 * running it; lp_graph_launch replays that step on `stream`.  The particle,
 * offsets and t buffers are captured by address and must stay valid; the
 * neighbour build of the previous step must already have run on this context
 * (LP_ERR_STATE otherwise), because each step clears the cell-table entries of
 * the one before.  Profiling must be off while capturing.
 */
lp_status lp_graph_capture(lp_ctx *ctx, lp_particles *p, const int64_t *offsets, int32_t nsim, double dt,
                           double cfl, double *t, lp_stream stream);
lp_status lp_graph_launch(lp_ctx *ctx, lp_stream stream);

/*
 * Schedules (no counterpart in the paper: implementation choices with
 * identical results), as bit flags.
 *   fit + update pass:
 *     LP_SCHED_FUSED  one kernel runs the whole per-particle update (central
 *                     fit, LW rates, one-sided fits, estimator, blend, mover).
 *     LP_SCHED_SPLIT  a first kernel runs the central fit, the LW rates and the
 *                     learned gate, finishes the particles the gate clears, and
 *                     appends the rest (with their central first derivatives
 *                     and LW rates) to a compacted list; a second kernel runs
 *                     the one-sided fits, estimator and blend over that list.
 *   neighbour query:
 *     (default)            one warp per 32 key-ordered particles (tiles), with
 *                          the per-particle kernel for the particles a tile
 *                          leaves (more than 64 neighbours, scattered groups).
 *     LP_SCHED_QUERY_WARP  one warp per particle for every particle.
 *   work distribution (same results):
 *     LP_SCHED_QUEUE_QUERY the tile kernel runs as a grid of resident blocks
 *                          whose warps take their next tile of 32 particles
 *                          from a device work counter (a warp work queue)
 *                          instead of one tile per warp of the launch.
 *     LP_SCHED_QUEUE_FIT   likewise for the SPLIT schedule's two kernels
 *                          (32 particles, then 32 list entries, per take);
 *                          FP32 path.
 * The default is SPLIT with the learned estimator, FUSED otherwise, and tiles.
 * A graph captured by lp_graph_capture keeps the schedule it was captured with.
 */
#define LP_SCHED_FUSED 0
#define LP_SCHED_SPLIT 1
#define LP_SCHED_QUERY_WARP 2
#define LP_SCHED_QUEUE_QUERY 4
#define LP_SCHED_QUEUE_FIT 8
lp_status lp_set_schedule(lp_ctx *ctx, int32_t schedule);   /* LP_ERR_ARG on unknown bits */
lp_status lp_get_schedule(lp_ctx *ctx, int32_t *schedule);

/*
 * Autotuner: runs the neighbour build and CFL step of lp_step_batched (same
 * arguments; t is not advanced), then times the neighbour query under each
 * query schedule and the fit pass under each fit schedule (`reps` timed
 * launches after one warm-up, CUDA events on `stream`), selects the faster of
 * each, and writes the mean times in milliseconds to out_ms[0] (fit FUSED),
 * out_ms[1] (fit SPLIT), out_ms[2] (query tiles), out_ms[3] (query per
 * particle), out_ms[4] (query tiles, LP_SCHED_QUEUE_QUERY) and out_ms[5] (fit
 * SPLIT | LP_SCHED_QUEUE_FIT; 0 on the FP64 path, where it is not offered)
 * when out_ms (host, LP_AUTOTUNE_TIMES doubles) is not null.  Entries of
 * schedules that do not apply (the query schedules of 1D and k-per-side
 * neighbourhoods) are 0.  The particle state is
 * not changed (the timed fit passes write to scratch buffers the call
 * allocates and frees); the counters, the device time steps (lp_dt_device) and
 * the launch tally are restored.  Synchronises `stream`.  LP_ERR_STATE while
 * profiling is on.
 */
#define LP_AUTOTUNE_TIMES 6
lp_status lp_autotune(lp_ctx *ctx, lp_particles *p, const int64_t *offsets, int32_t nsim, double dt, double cfl,
                      int32_t reps, double *out_ms, lp_stream stream);

/* Device time step of the last lp_step (device float64 scalar owned by ctx;
 * one per simulation after lp_step_batched). */
const double *lp_dt_device(lp_ctx *ctx);

/* Synchronise `stream`, read the counters into *out (host). */
lp_status lp_get_stats(lp_ctx *ctx, lp_stats *out, lp_stream stream);
lp_status lp_reset_stats(lp_ctx *ctx, lp_stream stream);

/* Human-readable name of a status code (static string). */
const char *lp_status_string(lp_status s);

/* Library version string (static). */
const char *lp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LP_H */
