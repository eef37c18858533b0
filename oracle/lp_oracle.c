/*
 * lp_oracle.c -- plain, slow FP64 CPU oracle for the hot path of the
 * Lagrangian particle (LP) method (Yuan, Zepeda Aguilar, Naitlho, Samulyak,
 * "Massively-Parallel Lagrangian Particle Code and Applications").
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product path (the CUDA
 * library under paper_2206_11998_gb300/) never links, loads or calls it, and
 * the two share no code.
 *
 * Everything here is FP64 with IEEE round-to-nearest and no FMA contraction
 * (built with -ffp-contract=off), written as the plain definition of each
 * step, one particle at a time:
 *
 *   lpo_morton_keys     Morton (Z-curve) keys of quantised positions
 *                       (Sec. 2.2, "Space-filling curve").
 *   lpo_neighbors       neighbour set {j != i : |x_j - x_i| <= R_i} ordered by
 *                       (d^2, id) and truncated to the nearest or to an
 *                       octant-balanced selection (Sec. 2.2 steps 3-4).
 *   lpo_gfd_central     second-order GFD least-squares fit, Eq. (linear_system_axb)
 *                       generalised to 1D/3D, solved by Householder QR with
 *                       column pivoting (Sec. 2.1).
 *   lpo_gfd_onesided    first-order fits on half-space stencils for the
 *                       left/right derivatives of the upwind scheme (Sec. 2.1).
 *   lpo_step            one LP time step: Lax-Wendroff and upwind rates, state
 *                       estimator, limiter blend, particle mover (Sec. 2.1,
 *                       Eqs. eq_upwind_V/u/P, the Lax-Wendroff expansions, the
 *                       blend, the estimator r, the limiter phi, Eq. timeIntegrate).
 *   lpo_cfl_dt          CFL time step (the paper gives none; see the reading below).
 *   lpo_riemann_exact   exact Riemann solution of the ideal-gas shock tube
 *                       (textbook; the Sod check of the full scheme).
 *   lpo_free_surface_ghosts  ghost particles completing free-surface
 *                       neighbourhoods (Sec. 2.2 step 3).
 *   lpo_inflow_state    reservoir inflow state at a nozzle inlet (Sec. 4).
 *   lpo_mlp_*           FP64 forward/backward/Adam of the 8-32-1 estimator MLP.
 *
 * Readings where the paper is silent (the 3D forms are deferred to the 2018
 * LP paper, which is not available) are stated at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* configuration (mirrored by the ctypes Structure in oracle/__init__.py)    */
/* ------------------------------------------------------------------------ */

enum { LPO_RADIUS_FIXED = 0, LPO_RADIUS_VOLUME = 1, LPO_RADIUS_KSIDE = 2 };
enum { LPO_LIM_FLAGGED = 0, LPO_LIM_PAPER = 1, LPO_LIM_LW = 2, LPO_LIM_UW = 3 };

typedef struct {
    int32_t dim;          /* 1, 2 or 3 */
    int32_t radius_mode;  /* LPO_RADIUS_* */
    double gamma;         /* ideal-gas exponent */
    double radius;        /* fixed-radius mode: R */
    double kappa;         /* volume mode: R_i = kappa (m_i V_i)^(1/dim) */
    int32_t k_max;        /* neighbour list capacity */
    int32_t k_side;       /* one-sided stencil size (8 in the paper, Sec. 2.2 step 5) */
    int32_t k_per_side;   /* 1D k-per-side mode: neighbours taken on each side */
    int32_t limiter;      /* LPO_LIM_* */
    double flat_eps;      /* estimator flatness floor */
    double active_frac;   /* estimator: axes below this fraction of the largest are ignored */
    double s_ref[5];      /* per-field reference magnitude for the flatness floor */
    int32_t periodic[3];
    int32_t pad0;
    double box_lo[3];
    double box_hi[3];
    double rank_tol;      /* numerical-rank threshold on |R_kk| / |R_00| */
    int64_t n_fluid;      /* particles with id >= n_fluid are frozen boundary particles */
    int32_t select;       /* LPO_SELECT_*: which k_max are kept when more lie inside the radius */
    int32_t pad1;
} lpo_config;

enum { LPO_SELECT_NEAREST = 0, LPO_SELECT_OCTANT = 1 };

#define LPO_MAXN 9      /* unknowns of the 3D second-order fit */
#define LPO_MAXF 5      /* fields V, u_1..u_d, P */

/* status bits written per particle */
#define LPO_ST_LINEAR_FALLBACK 1u   /* second-order system rank deficient: first-order fit used */
#define LPO_ST_NO_FIT          2u   /* first-order system rank deficient too: derivatives zero */
#define LPO_ST_OVERFLOW        4u   /* more than k_max neighbours inside the radius */
#define LPO_ST_REJECTED        8u   /* update not admissible (V or P <= 0, non-finite): not applied */

/* ------------------------------------------------------------------------ */
/* Morton keys (Sec. 2.2, space-filling Z-curve)                              */
/* ------------------------------------------------------------------------ */

/*
 * Quantise each coordinate to `bits` bits inside a cube of edge L anchored at
 * lo: q = floor((x - lo) * (2^bits / L)), clamped to [0, 2^bits - 1].  The key
 * interleaves the bits of (q_0, q_1, q_2) most-significant first, axis 0 taking
 * the lowest bit of each triple.  Written bit by bit, as the definition.
 */
void lpo_morton_keys(int32_t dim, int64_t n, const double *const *x,
                     const double *lo, double L, int32_t bits, uint64_t *key)
{
    double inv = ldexp(1.0, bits) / L;
    uint64_t qmax = (1ull << bits) - 1ull;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t q[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) {
            double t = (x[k][i] - lo[k]) * inv;
            double f = floor(t);
            uint64_t v;
            if (!(f > 0.0)) v = 0;              /* also catches NaN */
            else if (f >= (double)qmax) v = qmax;
            else v = (uint64_t)f;
            q[k] = v;
        }
        uint64_t k64 = 0;
        for (int b = bits - 1; b >= 0; --b)
            for (int k = dim - 1; k >= 0; --k)
                k64 = (k64 << 1) | ((q[k] >> b) & 1ull);
        key[i] = k64;
    }
}

/* ------------------------------------------------------------------------ */
/* neighbour search (Sec. 2.2 steps 3-4)                                     */
/* ------------------------------------------------------------------------ */

/* offset x_j - x_i on axis k, minimum image on periodic axes */
static double offset(const lpo_config *c, const double *const *x, int k, int64_t i, int64_t j)
{
    double dx = x[k][j] - x[k][i];
    if (c->periodic[k]) {
        double L = c->box_hi[k] - c->box_lo[k];
        double h = 0.5 * L;
        if (dx > h) dx = dx - L;
        else if (dx < -h) dx = dx + L;
    }
    return dx;
}

/* squared distance, summed in axis order: ((dx*dx + dy*dy) + dz*dz) */
static double dist2(const lpo_config *c, const double *const *x, int64_t i, int64_t j)
{
    double d0 = offset(c, x, 0, i, j);
    double d2 = d0 * d0;
    if (c->dim > 1) { double d1 = offset(c, x, 1, i, j); d2 = d2 + d1 * d1; }
    if (c->dim > 2) { double d3 = offset(c, x, 2, i, j); d2 = d2 + d3 * d3; }
    return d2;
}

/*
 * Membership j in N(i):  d2 <= R_i^2.  In the volume mode R_i = kappa (m_i V_i)^(1/dim)
 * (the local particle spacing scaled by kappa); the test is taken without a root:
 *   dim 3: (d2*d2)*d2 <= k6 * (w*w),   dim 2: d2*d2 <= k4 * (w*w),   dim 1: d2 <= k2 * (w*w),
 * with w = m_i V_i, k2 = kappa*kappa, k4 = k2*k2, k6 = (k2*k2)*k2.
 */
static int inside(const lpo_config *c, double d2, double w)
{
    if (c->radius_mode == LPO_RADIUS_FIXED) {
        double R2 = c->radius * c->radius;
        return d2 <= R2;
    }
    double k2 = c->kappa * c->kappa;
    double ww = w * w;
    if (c->dim == 3) {
        double k6 = (k2 * k2) * k2;
        return (d2 * d2) * d2 <= k6 * ww;
    } else if (c->dim == 2) {
        double k4 = k2 * k2;
        return d2 * d2 <= k4 * ww;
    }
    return d2 <= k2 * ww;
}

typedef struct { double d2; uint32_t id; int64_t j; int64_t rank; } cand_t;

static int cand_cmp(const void *a, const void *b)
{
    const cand_t *p = (const cand_t *)a, *q = (const cand_t *)b;
    if (p->d2 < q->d2) return -1;
    if (p->d2 > q->d2) return 1;
    if (p->id < q->id) return -1;
    if (p->id > q->id) return 1;
    return 0;
}

/* (rank, d2, id) order of the octant-balanced selection */
static int cand_rank_cmp(const void *a, const void *b)
{
    const cand_t *p = (const cand_t *)a, *q = (const cand_t *)b;
    if (p->rank < q->rank) return -1;
    if (p->rank > q->rank) return 1;
    return cand_cmp(a, b);
}

/* octant (quadrant in 2D) of x_j seen from x_i: bit k set when the offset
 * along axis k (minimum image on a periodic axis) is >= 0 */
static int octant_of(const lpo_config *c, const double *const *x, int64_t i, int64_t j)
{
    int o = 0;
    for (int k = 0; k < c->dim; ++k)
        if (offset(c, x, k, i, j) >= 0.0) o |= 1 << k;
    return o;
}

/*
 * Octant-balanced selection (Sec. 2.2 step 4: the top members of a list are
 * to contain neighbours from all directions, not only the nearest).  Reading:
 * buf[0..nc) holds the in-radius set in (d2, id) order and nc > k_max.  Each
 * member gets its rank within its octant in that order; the k_max kept are
 * the first k_max by (rank, d2, id), i.e. round robin over the octants,
 * nearest first in each, an octant that runs out giving its turn to the
 * others.  They are returned in buf[0..k_max) in (d2, id) order.
 */
static void select_octant_balanced(const lpo_config *c, const double *const *x, int64_t i,
                                   cand_t *buf, int64_t nc)
{
    int64_t seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t t = 0; t < nc; ++t) buf[t].rank = seen[octant_of(c, x, i, buf[t].j)]++;
    qsort(buf, (size_t)nc, sizeof(cand_t), cand_rank_cmp);
    qsort(buf, (size_t)c->k_max, sizeof(cand_t), cand_cmp);
}

/* index order by (x_0, index), used by the window pre-filter */
static const double *g_sort_x0;
static int idx_cmp_x0(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    if (g_sort_x0[i] < g_sort_x0[j]) return -1;
    if (g_sort_x0[i] > g_sort_x0[j]) return 1;
    return (i < j) ? -1 : (i > j);
}

/*
 * Neighbour lists of the query particles q[0..nq-1] (indices into the inputs).
 *
 * out_idx[r*k_max + t] holds the t-th neighbour (input index) of query r in
 * (d2, id) order, out_count[r] = min(#inside, k_max); when more than k_max lie
 * inside, the k_max nearest are kept (LPO_SELECT_NEAREST) or the octant-
 * balanced selection of select_octant_balanced (LPO_SELECT_OCTANT),
 * out_total[r] = min(#inside, 4 k_max) (the count saturates there),
 * out_d2min[r] = d2 of the nearest neighbour (INFINITY if none).
 *
 * 1D k-per-side mode (radius_mode 2): the k_per_side nearest with x_j < x_i and
 * the k_per_side nearest with x_j > x_i, each side by (d2, id); coincident
 * particles belong to neither side.  The union is then ordered by (d2, id).
 *
 * use_window != 0 restricts candidates to |x_j0 - x_i0| <= R_i (1 + 1e-6) on a
 * copy sorted by x_0 before the exact test (a pre-filter that drops nothing the
 * exact test keeps: fl(dx*dx) <= fl(d2) because rounding is monotone).  It is
 * not used on a periodic axis 0 or in the k-per-side mode.
 */
int lpo_neighbors(const lpo_config *c, int64_t n, const double *const *x,
                  const double *V, const double *m, const uint32_t *id,
                  int64_t nq, const int64_t *q, int32_t use_window,
                  uint32_t *out_count, uint32_t *out_total, int64_t *out_idx,
                  double *out_d2min)
{
    int64_t *order = NULL;
    int window = use_window && !c->periodic[0] && c->radius_mode != LPO_RADIUS_KSIDE;
    if (window) {
        order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        if (!order) return -1;
        for (int64_t i = 0; i < n; ++i) order[i] = i;
        g_sort_x0 = x[0];
        qsort(order, (size_t)n, sizeof(int64_t), idx_cmp_x0);
    }
    int err = 0;
#pragma omp parallel
    {
        cand_t *buf = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
        if (!buf) {
#pragma omp atomic write
            err = -1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < nq; ++r) {
            if (!buf) continue;
            int64_t i = q[r];
            double w = m[i] * V[i];
            int64_t nc = 0;
            if (c->radius_mode == LPO_RADIUS_KSIDE) {
                /* left and right sides separately */
                int64_t nl = 0, nr;
                for (int64_t j = 0; j < n; ++j) {
                    if (j == i) continue;
                    double dx = offset(c, x, 0, i, j);
                    if (dx < 0.0) { buf[nl].d2 = dx * dx; buf[nl].id = id[j]; buf[nl].j = j; ++nl; }
                }
                qsort(buf, (size_t)nl, sizeof(cand_t), cand_cmp);
                if (nl > c->k_per_side) nl = c->k_per_side;
                nr = nl;
                for (int64_t j = 0; j < n; ++j) {
                    if (j == i) continue;
                    double dx = offset(c, x, 0, i, j);
                    if (dx > 0.0) { buf[nr].d2 = dx * dx; buf[nr].id = id[j]; buf[nr].j = j; ++nr; }
                }
                qsort(buf + nl, (size_t)(nr - nl), sizeof(cand_t), cand_cmp);
                if (nr - nl > c->k_per_side) nr = nl + c->k_per_side;
                nc = nr;
            } else if (window) {
                double R;
                if (c->radius_mode == LPO_RADIUS_FIXED) R = c->radius;
                else R = c->kappa * pow(w, 1.0 / (double)c->dim);
                R = R * (1.0 + 1e-6) + 1e-300;
                double xlo = x[0][i] - R, xhi = x[0][i] + R;
                int64_t a = 0, b = n;  /* first with x0 >= xlo */
                while (a < b) { int64_t h = a + (b - a) / 2; if (x[0][order[h]] < xlo) a = h + 1; else b = h; }
                for (int64_t t = a; t < n && x[0][order[t]] <= xhi; ++t) {
                    int64_t j = order[t];
                    if (j == i) continue;
                    double d2 = dist2(c, x, i, j);
                    if (inside(c, d2, w)) { buf[nc].d2 = d2; buf[nc].id = id[j]; buf[nc].j = j; ++nc; }
                }
            } else {
                for (int64_t j = 0; j < n; ++j) {
                    if (j == i) continue;
                    double d2 = dist2(c, x, i, j);
                    if (inside(c, d2, w)) { buf[nc].d2 = d2; buf[nc].id = id[j]; buf[nc].j = j; ++nc; }
                }
            }
            qsort(buf, (size_t)nc, sizeof(cand_t), cand_cmp);
            const double d2min = nc > 0 ? buf[0].d2 : INFINITY;
            if (c->select == LPO_SELECT_OCTANT && c->radius_mode != LPO_RADIUS_KSIDE && nc > c->k_max)
                select_octant_balanced(c, x, i, buf, nc);
            int64_t keep = nc < c->k_max ? nc : c->k_max;
            for (int64_t t = 0; t < keep; ++t) out_idx[r * c->k_max + t] = buf[t].j;
            for (int64_t t = keep; t < c->k_max; ++t) out_idx[r * c->k_max + t] = -1;
            out_count[r] = (uint32_t)keep;
            out_total[r] = (uint32_t)(nc < 4 * (int64_t)c->k_max ? nc : 4 * (int64_t)c->k_max);
            out_d2min[r] = d2min;
        }
        free(buf);
    }
    free(order);
    return err;
}

/* ------------------------------------------------------------------------ */
/* least squares by Householder QR with column pivoting (Sec. 2.1)           */
/* ------------------------------------------------------------------------ */

/*
 * min ||A x - b||_2 for nrhs right-hand sides.  A is m x n column-major
 * (A[j*m + i]), B is m x nrhs column-major; both are overwritten.  Columns are
 * first scaled to unit 2-norm (the minimiser is unchanged by column scaling),
 * then factored A P = Q R by Householder reflections, choosing at each step the
 * remaining column of largest norm.  The numerical rank is the number of
 * leading |R_kk| > rank_tol * |R_00|.  Returns 0 and X (n x nrhs, X[r*n + j])
 * when the rank is n, otherwise -1 (X untouched).
 */
static int lsq_qrcp(int m, int n, double *A, int nrhs, double *B, double rank_tol, double *X)
{
    double scale[LPO_MAXN];
    int perm[LPO_MAXN];
    if (m < n) return -1;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += A[j * m + i] * A[j * m + i];
        s = sqrt(s);
        if (!(s > 0.0)) return -1;
        scale[j] = s;
        for (int i = 0; i < m; ++i) A[j * m + i] /= s;
        perm[j] = j;
    }
    double r00 = 0.0;
    for (int k = 0; k < n; ++k) {
        /* pivot: remaining column with the largest norm over rows k..m-1 */
        int p = k;
        double best = -1.0;
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += A[j * m + i] * A[j * m + i];
            if (s > best) { best = s; p = j; }
        }
        if (p != k) {
            for (int i = 0; i < m; ++i) { double t = A[k * m + i]; A[k * m + i] = A[p * m + i]; A[p * m + i] = t; }
            int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
        }
        /* Householder reflector H = I - beta v v^T mapping A[k:,k] to alpha e_1 */
        double norm = sqrt(best);
        double akk = A[k * m + k];
        double alpha = (akk >= 0.0) ? -norm : norm;
        if (k == 0) r00 = fabs(alpha);
        if (!(fabs(alpha) > rank_tol * r00) || norm == 0.0) return -1;
        double v[64 * 4];
        double *vv = v;
        double *vheap = NULL;
        if (m > 256) { vheap = (double *)malloc(sizeof(double) * (size_t)m); vv = vheap; }
        for (int i = k; i < m; ++i) vv[i] = A[k * m + i];
        vv[k] = akk - alpha;
        double vtv = 0.0;
        for (int i = k; i < m; ++i) vtv += vv[i] * vv[i];
        double beta = (vtv > 0.0) ? 2.0 / vtv : 0.0;
        for (int j = k + 1; j < n; ++j) {
            double w = 0.0;
            for (int i = k; i < m; ++i) w += vv[i] * A[j * m + i];
            w *= beta;
            for (int i = k; i < m; ++i) A[j * m + i] -= w * vv[i];
        }
        for (int r = 0; r < nrhs; ++r) {
            double w = 0.0;
            for (int i = k; i < m; ++i) w += vv[i] * B[r * m + i];
            w *= beta;
            for (int i = k; i < m; ++i) B[r * m + i] -= w * vv[i];
        }
        A[k * m + k] = alpha;
        for (int i = k + 1; i < m; ++i) A[k * m + i] = 0.0;
        free(vheap);
    }
    /* back substitution R y = Q^T b, then undo pivoting and scaling */
    for (int r = 0; r < nrhs; ++r) {
        double y[LPO_MAXN];
        for (int k = n - 1; k >= 0; --k) {
            double s = B[r * m + k];
            for (int j = k + 1; j < n; ++j) s -= A[j * m + k] * y[j];
            y[k] = s / A[k * m + k];
        }
        for (int k = 0; k < n; ++k) X[r * n + perm[k]] = y[k] / scale[perm[k]];
    }
    return 0;
}

/* number of unknowns of the second-order fit in dim dimensions */
static int n_second(int dim) { return dim == 1 ? 2 : (dim == 2 ? 5 : 9); }

/*
 * Row of the GFD system for offset d (Sec. 2.1, Eq. linear_system_axb; the 2D
 * row [h, k, h^2/2, k^2/2, hk] of the paper, and its 1D and 3D analogues):
 *   1D: [h, h^2/2]
 *   2D: [h, k, h^2/2, k^2/2, h k]
 *   3D: [dx, dy, dz, dx^2/2, dy^2/2, dz^2/2, dx dy, dx dz, dy dz]
 * The unknowns are, in the same order, the first derivatives, the pure second
 * derivatives and the mixed second derivatives at the centre particle.
 */
static void gfd_row(int dim, const double *d, double *row)
{
    if (dim == 1) { row[0] = d[0]; row[1] = 0.5 * d[0] * d[0]; return; }
    if (dim == 2) {
        row[0] = d[0]; row[1] = d[1];
        row[2] = 0.5 * d[0] * d[0]; row[3] = 0.5 * d[1] * d[1];
        row[4] = d[0] * d[1];
        return;
    }
    row[0] = d[0]; row[1] = d[1]; row[2] = d[2];
    row[3] = 0.5 * d[0] * d[0]; row[4] = 0.5 * d[1] * d[1]; row[5] = 0.5 * d[2] * d[2];
    row[6] = d[0] * d[1]; row[7] = d[0] * d[2]; row[8] = d[1] * d[2];
}

/*
 * Central second-order GFD fit of particle i on its neighbour list nb[0..cnt-1]
 * for nf fields.  out[f*n_u + u] receives derivative u of field f.  When the
 * second-order system is rank deficient the first-order system (columns
 * dx..) is solved instead and the second derivatives are zero; when that is
 * rank deficient too every derivative is zero.  Returns the status bits.
 */
static uint32_t central_fit(const lpo_config *c, const double *const *x, const double *const *F, int nf,
                            int64_t i, const int64_t *nb, int cnt, double *out)
{
    int dim = c->dim, nu = n_second(dim);
    int m = cnt;
    double *A = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * LPO_MAXN);
    double *B = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * LPO_MAXF);
    double X[LPO_MAXN * LPO_MAXF];
    uint32_t st = 0;
    for (int f = 0; f < nf * nu; ++f) out[f] = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        int n = pass == 0 ? nu : dim;
        for (int r = 0; r < m; ++r) {
            int64_t j = nb[r];
            double d[3], row[LPO_MAXN];
            for (int k = 0; k < dim; ++k) d[k] = offset(c, x, k, i, j);
            gfd_row(dim, d, row);
            for (int u = 0; u < n; ++u) A[u * m + r] = row[u];
            for (int f = 0; f < nf; ++f) B[f * m + r] = F[f][j] - F[f][i];
        }
        if (lsq_qrcp(m, n, A, nf, B, c->rank_tol, X) == 0) {
            for (int f = 0; f < nf; ++f)
                for (int u = 0; u < n; ++u) out[f * nu + u] = X[f * n + u];
            break;
        }
        st |= pass == 0 ? LPO_ST_LINEAR_FALLBACK : LPO_ST_NO_FIT;
    }
    free(A);
    free(B);
    return st;
}

/*
 * One-sided first derivatives (Sec. 2.1: left/right derivatives of the upwind
 * scheme from the left/right semi-spheres in each dimension).  For axis k and
 * side s (0 = left, x_jk < x_ik; 1 = right, x_jk > x_ik; offsets exactly 0 are
 * on neither side) the stencil is the first k_side entries of the neighbour
 * list on that side; the first-order system [dx .. ] is solved in least squares
 * and component k kept.  With fewer than dim stencil members, or a
 * rank-deficient system, the central derivative of axis k is used.
 * out[(k*2 + s)*nf + f].
 */
static void onesided_fit(const lpo_config *c, const double *const *x, const double *const *F, int nf,
                         int64_t i, const int64_t *nb, int cnt, const double *central, double *out)
{
    int dim = c->dim, nu = n_second(dim);
    int ks = c->k_side;
    double *A = (double *)malloc(sizeof(double) * (size_t)(ks > 0 ? ks : 1) * 3);
    double *B = (double *)malloc(sizeof(double) * (size_t)(ks > 0 ? ks : 1) * LPO_MAXF);
    double X[3 * LPO_MAXF];
    for (int k = 0; k < dim; ++k) {
        for (int s = 0; s < 2; ++s) {
            int64_t sel[256];
            int ns = 0;
            for (int r = 0; r < cnt && ns < ks && ns < 256; ++r) {
                double dk = offset(c, x, k, i, nb[r]);
                if ((s == 0 && dk < 0.0) || (s == 1 && dk > 0.0)) sel[ns++] = nb[r];
            }
            int ok = -1;
            if (ns >= dim) {
                for (int r = 0; r < ns; ++r) {
                    for (int a = 0; a < dim; ++a) A[a * ns + r] = offset(c, x, a, i, sel[r]);
                    for (int f = 0; f < nf; ++f) B[f * ns + r] = F[f][sel[r]] - F[f][i];
                }
                ok = lsq_qrcp(ns, dim, A, nf, B, c->rank_tol, X);
            }
            for (int f = 0; f < nf; ++f)
                out[(k * 2 + s) * nf + f] = (ok == 0) ? X[f * dim + k] : central[f * nu + k];
        }
    }
    free(A);
    free(B);
}

/* ------------------------------------------------------------------------ */
/* state estimator and limiter (Sec. 2.1)                                    */
/* ------------------------------------------------------------------------ */

/*
 * Limiter phi(r) (Sec. 2.1): 1.25 exp(1 - sqrt r) for r < 3/2,
 * 1.25 exp(-9/2 (sqrt r - 1)^2) for r > 3/2.  The paper leaves r = 3/2 open;
 * it takes the first branch.  phi(inf) = 0.
 */
double lpo_phi(double r)
{
    if (isinf(r)) return 0.0;
    double sr = sqrt(r);
    if (r <= 1.5) return 1.25 * exp(1.0 - sr);
    return 1.25 * exp(-4.5 * (sr - 1.0) * (sr - 1.0));
}

/*
 * Estimator of one field (Sec. 2.1): per axis k, r_k = inf if s_kl s_kr <= 0,
 * else (s_kr/s_kl + s_kl/s_kr)/2.  Reading for several axes: axes whose larger
 * one-sided magnitude is below active_frac of the largest over all axes are
 * ignored, and r is the maximum over the others.  A field whose one-sided
 * derivatives are all below the flatness floor (max|s_k| * ell <= flat_eps * S,
 * S = max(|s_i|, s_ref)) is locally constant and gets r = 1.
 */
static double estimator_r(int dim, const double *sl, const double *sr, double ell, double s_i,
                          double s_ref, double flat_eps, double active_frac)
{
    double G = 0.0;
    for (int k = 0; k < dim; ++k) {
        double g = fmax(fabs(sl[k]), fabs(sr[k]));
        if (g > G) G = g;
    }
    double S = fmax(fabs(s_i), s_ref);
    if (G * ell <= flat_eps * S) return 1.0;
    double r = 1.0;
    for (int k = 0; k < dim; ++k) {
        double g = fmax(fabs(sl[k]), fabs(sr[k]));
        if (g < active_frac * G) continue;
        double rk;
        if (sl[k] * sr[k] <= 0.0) rk = INFINITY;
        else rk = 0.5 * (sr[k] / sl[k] + sl[k] / sr[k]);
        if (rk > r) r = rk;
    }
    return r;
}

/* estimator_r of one field, exported so that the tests can pin it directly */
double lpo_estimator_r(int32_t dim, const double *sl, const double *sr, double ell, double s_i,
                       double s_ref, double flat_eps, double active_frac)
{
    return estimator_r(dim, sl, sr, ell, s_i, s_ref, flat_eps, active_frac);
}

/* ------------------------------------------------------------------------ */
/* one LP step                                                              */
/* ------------------------------------------------------------------------ */

/*
 * Rates of the unsplit Lax-Wendroff scheme for an ideal gas, all coefficients at
 * t^n.  The paper prints the 1D form and defers 2D/3D to the 2018 LP paper; the
 * multi-D form here follows its own recipe: differentiate V_t = V div u,
 * u_t = -V grad P, P_t = -gamma P div u once more in time and exchange material
 * and spatial derivatives with D(d_k f)/Dt = d_k(Df/Dt) - (d_k u_m)(d_m f):
 *   V_tt   = V (div u)^2 - V S2 - V gradV.gradP - V^2 lap P
 *   u_i,tt = (gamma-1) V (div u) d_i P + V sum_m (d_i u_m)(d_m P) + gamma V P d_i(div u)
 *   P_tt   = gamma^2 P (div u)^2 + gamma P S2 + gamma P (gradV.gradP + V lap P)
 * with S2 = sum_{k,m} (d_k u_m)(d_m u_k).  In 1D these are the paper's second
 * time derivatives; its printed u update carries -V u_x P_x where the derived
 * u_tt gives +gamma V u_x P_x, and the derivation is followed.
 * LW_s = s_t + dt/2 s_tt.
 * cd[f*nu + u]: central derivatives; field order V, u_1..u_d, P.
 */
static void lw_rates(int dim, double gamma, double dt, double V, const double *u, double P,
                     const double *cd, double *lw)
{
    int nu = n_second(dim);
    const double *dV = cd;
    const double *dP = cd + (dim + 1) * nu;
    double J[3][3];          /* J[a][b] = d_b u_a */
    double gdiv[3];          /* d_c (div u) = sum_a d_c d_a u_a */
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) J[a][b] = cd[(1 + a) * nu + b];
    /* second-derivative slot of (c, a) in the unknown ordering */
    for (int cc = 0; cc < dim; ++cc) {
        double s = 0.0;
        for (int a = 0; a < dim; ++a) {
            int slot;
            if (cc == a) slot = dim + a;                      /* pure second derivative */
            else {
                int lo = cc < a ? cc : a, hi = cc < a ? a : cc;
                /* mixed: 2D -> 4; 3D: (0,1)->6, (0,2)->7, (1,2)->8 */
                slot = (dim == 2) ? 4 : (lo == 0 ? (hi == 1 ? 6 : 7) : 8);
            }
            s += cd[(1 + a) * nu + slot];
        }
        gdiv[cc] = s;
    }
    double divu = 0.0, S2 = 0.0, gVgP = 0.0, lapP = 0.0;
    for (int a = 0; a < dim; ++a) divu += J[a][a];
    for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) S2 += J[a][b] * J[b][a];
    for (int k = 0; k < dim; ++k) gVgP += dV[k] * dP[k];
    for (int k = 0; k < dim; ++k) lapP += dP[dim + k];

    double Vt = V * divu;
    double Vtt = V * divu * divu - V * S2 - V * gVgP - V * V * lapP;
    lw[0] = Vt + 0.5 * dt * Vtt;
    for (int i = 0; i < dim; ++i) {
        double uPt = 0.0;
        for (int mm = 0; mm < dim; ++mm) uPt += J[mm][i] * dP[mm];
        double ut = -V * dP[i];
        double utt = (gamma - 1.0) * V * divu * dP[i] + V * uPt + gamma * V * P * gdiv[i];
        lw[1 + i] = ut + 0.5 * dt * utt;
    }
    double Pt = -gamma * P * divu;
    double Ptt = gamma * gamma * P * divu * divu + gamma * P * S2 + gamma * P * (gVgP + V * lapP);
    lw[dim + 1] = Pt + 0.5 * dt * Ptt;
    (void)u;
}

/*
 * First-order upwind rates (Sec. 2.1, Eqs. eq_upwind_V, eq_upwind_u, eq_upwind_P),
 * K = gamma P / V for the ideal gas (Eq. Kdef with e = P V / (gamma - 1)).  The
 * paper prints 1D; the multi-D reading applies the 1D operator along each axis
 * k with the normal velocity u_k and sums the contributions to V_t and P_t:
 *   V_t   = sum_k [ V/2 (u_k,kr + u_k,kl) - V/(2 sqrt K) (P_kr - P_kl) ]
 *   u_k,t = V sqrt(K)/2 (u_k,kr - u_k,kl) - V/2 (P_kr + P_kl)
 *   P_t   = sum_k [ -V K/2 (u_k,kr + u_k,kl) + V sqrt(K)/2 (P_kr - P_kl) ]
 * os[(k*2 + s)*nf + f] one-sided derivatives (s = 0 left, 1 right).
 */
static void uw_rates(int dim, double gamma, double V, double P, const double *os, int nf, double *uw)
{
    double K = gamma * P / V;
    double sK = sqrt(K);
    double Vt = 0.0, Pt = 0.0;
    for (int k = 0; k < dim; ++k) {
        double ul = os[(k * 2 + 0) * nf + 1 + k], ur = os[(k * 2 + 1) * nf + 1 + k];
        double Pl = os[(k * 2 + 0) * nf + dim + 1], Pr = os[(k * 2 + 1) * nf + dim + 1];
        Vt += 0.5 * V * (ur + ul) - V / (2.0 * sK) * (Pr - Pl);
        uw[1 + k] = 0.5 * V * sK * (ur - ul) - 0.5 * V * (Pr + Pl);
        Pt += -0.5 * V * K * (ur + ul) + 0.5 * V * sK * (Pr - Pl);
    }
    uw[0] = Vt;
    uw[dim + 1] = Pt;
}

/*
 * One LP time step (Sec. 2.2 steps 3-6 and Sec. 2.1) for the query particles
 * q[0..nq-1], given the full state at t^n and the step dt.  Each query's new
 * state depends only on the state at t^n of the particle and of its neighbours.
 *
 * Per fluid particle (id < n_fluid; boundary particles are copied unchanged):
 *   neighbours, central fit of V, u, P, one-sided fits, LW and UW rates,
 *   estimator r_s per field, phi_s, and the blend of Sec. 2.1
 *     s^{n+1} = s^n + dt (UW - phi (UW - LW)),
 *   with phi by limiter mode: PAPER phi(r_s); FLAGGED phi(r_s) when any field
 *   has r_s > 3/2 and 1 (pure Lax-Wendroff) otherwise; LW 1; UW 0.
 *   Then the mover, Eq. timeIntegrate: x^{n+1} = x^n + dt/2 (u^n + u^{n+1}),
 *   wrapped into the box on periodic axes.
 *
 * forced_phi (may be NULL): nq x nf; a finite entry replaces the oracle's own
 * phi for that particle and field (used only for particles whose discrete
 * decision is within round-off of a threshold).
 * Outputs per query: xn[k][r], Vn, un[k], Pn, flag, phi_out[r*nf+f], r_out[r*nf+f],
 * status.
 */
int lpo_step(const lpo_config *c, int64_t n, const double *const *x, const double *V,
             const double *const *u, const double *P, const double *m, const uint32_t *id,
             double dt, int64_t nq, const int64_t *q, const double *forced_phi,
             double *const *xn, double *Vn, double *const *un, double *Pn,
             uint8_t *flag, double *phi_out, double *r_out, uint32_t *status)
{
    int dim = c->dim, nf = dim + 2, nu = n_second(dim);
    const double *F[LPO_MAXF];
    F[0] = V;
    for (int k = 0; k < dim; ++k) F[1 + k] = u[k];
    F[dim + 1] = P;
    int kmax = c->k_max;
    uint32_t *cnt = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nq > 0 ? nq : 1));
    uint32_t *tot = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nq > 0 ? nq : 1));
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nq > 0 ? nq : 1) * (size_t)kmax);
    double *d2m = (double *)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1));
    if (!cnt || !tot || !nb || !d2m) { free(cnt); free(tot); free(nb); free(d2m); return -1; }
    int rc = lpo_neighbors(c, n, x, V, m, id, nq, q, 1, cnt, tot, nb, d2m);
    if (rc != 0) { free(cnt); free(tot); free(nb); free(d2m); return rc; }

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nq; ++r) {
        int64_t i = q[r];
        double cd[LPO_MAXF * LPO_MAXN], os[3 * 2 * LPO_MAXF];
        double lw[LPO_MAXF], uw[LPO_MAXF], phi[LPO_MAXF], rs[LPO_MAXF], s0[LPO_MAXF], s1[LPO_MAXF];
        uint32_t st = tot[r] > (uint32_t)kmax ? LPO_ST_OVERFLOW : 0u;
        for (int f = 0; f < nf; ++f) s0[f] = F[f][i];
        if ((int64_t)id[i] >= c->n_fluid) {
            for (int k = 0; k < dim; ++k) xn[k][r] = x[k][i];
            Vn[r] = V[i]; for (int k = 0; k < dim; ++k) un[k][r] = u[k][i]; Pn[r] = P[i];
            flag[r] = 0;
            for (int f = 0; f < nf; ++f) { phi_out[r * nf + f] = 1.0; r_out[r * nf + f] = 1.0; }
            status[r] = st;
            continue;
        }
        st |= central_fit(c, x, F, nf, i, nb + r * kmax, (int)cnt[r], cd);
        onesided_fit(c, x, F, nf, i, nb + r * kmax, (int)cnt[r], cd, os);
        lw_rates(dim, c->gamma, dt, V[i], NULL, P[i], cd, lw);
        uw_rates(dim, c->gamma, V[i], P[i], os, nf, uw);

        /* estimator per field */
        double ell = sqrt(d2m[r]);
        int any = 0;
        for (int f = 0; f < nf; ++f) {
            double sl[3], sr[3];
            for (int k = 0; k < dim; ++k) { sl[k] = os[(k * 2 + 0) * nf + f]; sr[k] = os[(k * 2 + 1) * nf + f]; }
            rs[f] = estimator_r(dim, sl, sr, ell, s0[f], c->s_ref[f], c->flat_eps, c->active_frac);
            if (rs[f] > 1.5) any = 1;
        }
        for (int f = 0; f < nf; ++f) {
            double p;
            switch (c->limiter) {
            case LPO_LIM_PAPER: p = lpo_phi(rs[f]); break;
            case LPO_LIM_LW: p = 1.0; break;
            case LPO_LIM_UW: p = 0.0; break;
            default: p = any ? lpo_phi(rs[f]) : 1.0; break;
            }
            if (forced_phi && isfinite(forced_phi[r * nf + f])) p = forced_phi[r * nf + f];
            phi[f] = p;
            s1[f] = s0[f] + dt * (uw[f] - p * (uw[f] - lw[f]));
        }
        /* safeguard (not in the paper): an update that leaves V or P non-positive
         * or a field non-finite is not applied; the particle keeps its state */
        int admissible = s1[0] > 0.0 && s1[dim + 1] > 0.0;
        for (int f = 0; f < nf; ++f) admissible = admissible && isfinite(s1[f]);
        if (!admissible) {
            for (int f = 0; f < nf; ++f) s1[f] = s0[f];
            st |= 8u;
        }
        Vn[r] = s1[0];
        for (int k = 0; k < dim; ++k) un[k][r] = s1[1 + k];
        Pn[r] = s1[dim + 1];
        for (int k = 0; k < dim; ++k) {
            double xk = x[k][i] + 0.5 * dt * (u[k][i] + s1[1 + k]);
            if (c->periodic[k]) {
                double L = c->box_hi[k] - c->box_lo[k];
                if (xk >= c->box_hi[k]) xk = xk - L;
                else if (xk < c->box_lo[k]) xk = xk + L;
            }
            xn[k][r] = xk;
        }
        flag[r] = (uint8_t)any;
        for (int f = 0; f < nf; ++f) { phi_out[r * nf + f] = phi[f]; r_out[r * nf + f] = rs[f]; }
        status[r] = st;
    }
    free(cnt); free(tot); free(nb); free(d2m);
    (void)nu;
    return 0;
}

/*
 * Central derivatives of nf arbitrary fields for the query particles, using
 * neighbour lists from lpo_neighbors (nb: nq x k_max input indices, cnt: list
 * lengths).  out[(f*nq + r)*n_u + u].  status[r]: LPO_ST_* bits.
 */
int lpo_gfd_central(const lpo_config *c, const double *const *x, int32_t nf, const double *const *F,
                    int64_t nq, const int64_t *q, const uint32_t *cnt, const int64_t *nb,
                    double *out, uint32_t *status)
{
    int nu = n_second(c->dim);
    if (nf < 1 || nf > LPO_MAXF) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nq; ++r) {
        double cd[LPO_MAXF * LPO_MAXN];
        status[r] = central_fit(c, x, F, nf, q[r], nb + r * c->k_max, (int)cnt[r], cd);
        for (int f = 0; f < nf; ++f)
            for (int u = 0; u < nu; ++u) out[((int64_t)f * nq + r) * nu + u] = cd[f * nu + u];
    }
    return 0;
}

/*
 * One-sided derivatives for the query particles (same conventions as above).
 * out[((r*dim + k)*2 + s)*nf + f].
 */
int lpo_gfd_onesided(const lpo_config *c, const double *const *x, int32_t nf, const double *const *F,
                     int64_t nq, const int64_t *q, const uint32_t *cnt, const int64_t *nb, double *out)
{
    int nu = n_second(c->dim);
    if (nf < 1 || nf > LPO_MAXF) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nq; ++r) {
        double cd[LPO_MAXF * LPO_MAXN];
        central_fit(c, x, F, nf, q[r], nb + r * c->k_max, (int)cnt[r], cd);
        onesided_fit(c, x, F, nf, q[r], nb + r * c->k_max, (int)cnt[r], cd, out + r * c->dim * 2 * nf);
    }
    (void)nu;
    return 0;
}

/*
 * CFL step.  The paper does not state its time-step rule; the reading here is
 * dt = cfl * min_i ell_i / c_i over fluid particles, ell_i the distance to the
 * nearest neighbour and c_i = sqrt(gamma P_i V_i) the sound speed of the ideal
 * gas.  d2min holds ell_i^2 per particle (INFINITY when it has no neighbour).
 */
double lpo_cfl_dt(const lpo_config *c, int64_t n, const double *V, const double *P,
                  const uint32_t *id, const double *d2min, double cfl)
{
    double best = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)id[i] >= c->n_fluid || isinf(d2min[i])) continue;
        double ell = sqrt(d2min[i]);
        double cs = sqrt(c->gamma * P[i] * V[i]);
        double t = ell / cs;
        if (t < best) best = t;
    }
    return cfl * best;
}

/* ------------------------------------------------------------------------ */
/* exact Riemann solver for the ideal-gas shock tube (textbook)              */
/* ------------------------------------------------------------------------ */

/* pressure function of one side: jump in velocity across the wave joining the
 * side state (rho, p, c) to pressure ps; shock if ps > p, rarefaction otherwise */
static void wave_fn(double g, double ps, double rho, double p, double cs, double *f, double *df)
{
    if (ps > p) {
        double A = 2.0 / ((g + 1.0) * rho), B = (g - 1.0) / (g + 1.0) * p;
        double s = sqrt(A / (ps + B));
        *f = (ps - p) * s;
        *df = s * (1.0 - 0.5 * (ps - p) / (ps + B));
    } else {
        double e = (g - 1.0) / (2.0 * g);
        *f = 2.0 * cs / (g - 1.0) * (pow(ps / p, e) - 1.0);
        *df = 1.0 / (rho * cs) * pow(ps / p, -(g + 1.0) / (2.0 * g));
    }
}

/*
 * Star state of the Riemann problem: p* solves fL(p) + fR(p) + (uR - uL) = 0 by
 * Newton's method from the two-rarefaction estimate; u* = (uL + uR)/2 +
 * (fR(p*) - fL(p*))/2.  Returns the iteration count.
 */
int lpo_riemann_star(double g, double rL, double uL, double pL, double rR, double uR, double pR,
                     double *ps_out, double *us_out)
{
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    double e = (g - 1.0) / (2.0 * g);
    double p = pow((cL + cR - 0.5 * (g - 1.0) * (uR - uL)) /
                   (cL / pow(pL, e) + cR / pow(pR, e)), 1.0 / e);
    if (!(p > 0.0)) p = 1e-8;
    int it;
    for (it = 1; it <= 100; ++it) {
        double fL, dL, fR, dR;
        wave_fn(g, p, rL, pL, cL, &fL, &dL);
        wave_fn(g, p, rR, pR, cR, &fR, &dR);
        double pn = p - (fL + fR + (uR - uL)) / (dL + dR);
        if (pn < 1e-14) pn = 1e-14;
        double ch = 2.0 * fabs(pn - p) / (pn + p);
        p = pn;
        if (ch < 1e-15) break;
    }
    double fL, dL, fR, dR;
    wave_fn(g, p, rL, pL, cL, &fL, &dL);
    wave_fn(g, p, rR, pR, cR, &fR, &dR);
    *ps_out = p;
    *us_out = 0.5 * (uL + uR) + 0.5 * (fR - fL);
    return it;
}

/*
 * Exact solution at positions xs[0..n-1] and time t > 0 of the ideal-gas
 * Riemann problem with the discontinuity at x0 (left state for x < x0).
 * Writes density, velocity and pressure.
 */
void lpo_riemann_exact(double g, double rL, double uL, double pL, double rR, double uR, double pR,
                       double x0, double t, int64_t n, const double *xs,
                       double *rho, double *vel, double *pre)
{
    double ps, us;
    lpo_riemann_star(g, rL, uL, pL, rR, uR, pR, &ps, &us);
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    double gm = (g - 1.0) / (g + 1.0);
    for (int64_t i = 0; i < n; ++i) {
        double S = (xs[i] - x0) / t;
        double r, uu, pp;
        if (S <= us) {                                    /* left of the contact */
            if (ps > pL) {                                /* left shock */
                double SL = uL - cL * sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g));
                if (S <= SL) { r = rL; uu = uL; pp = pL; }
                else { r = rL * (ps / pL + gm) / (gm * ps / pL + 1.0); uu = us; pp = ps; }
            } else {                                      /* left rarefaction */
                double cs = cL * pow(ps / pL, (g - 1.0) / (2.0 * g));
                double SH = uL - cL, ST = us - cs;
                if (S <= SH) { r = rL; uu = uL; pp = pL; }
                else if (S >= ST) { r = rL * pow(ps / pL, 1.0 / g); uu = us; pp = ps; }
                else {
                    double a = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * cL) * (uL - S);
                    r = rL * pow(a, 2.0 / (g - 1.0));
                    uu = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + S);
                    pp = pL * pow(a, 2.0 * g / (g - 1.0));
                }
            }
        } else {                                          /* right of the contact */
            if (ps > pR) {                                /* right shock */
                double SR = uR + cR * sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g));
                if (S >= SR) { r = rR; uu = uR; pp = pR; }
                else { r = rR * (ps / pR + gm) / (gm * ps / pR + 1.0); uu = us; pp = ps; }
            } else {                                      /* right rarefaction */
                double cs = cR * pow(ps / pR, (g - 1.0) / (2.0 * g));
                double SH = uR + cR, ST = us + cs;
                if (S >= SH) { r = rR; uu = uR; pp = pR; }
                else if (S <= ST) { r = rR * pow(ps / pR, 1.0 / g); uu = us; pp = ps; }
                else {
                    double a = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * cR) * (uR - S);
                    r = rR * pow(a, 2.0 / (g - 1.0));
                    uu = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + S);
                    pp = pR * pow(a, 2.0 * g / (g - 1.0));
                }
            }
        }
        rho[i] = r; vel[i] = uu; pre[i] = pp;
    }
}

/*
 * The eight inputs of the learned state estimator for the query particles,
 * from each particle's central fit (see central_fit), its nearest-neighbour
 * distance ell, and the differences b_j = P_j - P_i over its list:
 *   f0 = ell |grad P| / P          f1 = ell |grad V| / V
 *   f2, f3 = for P and V: the largest, over axes k whose |d_k s| is at least
 *            half the largest, of ell |d_kk s| / (|d_k s| + ell |d_kk s|)
 *   f4 = ell div u / c, c = sqrt(gamma P V)
 *   f5 = max_j b_j / P             f6 = -min_j b_j / P   (extremes include 0)
 *   f7 = sqrt(sum_j res_j^2 / sum_j b_j^2), res = residual of the P fit
 * each mapped to log(1 + 10 |f|), f4 keeping its sign.  out[r*8 + k].
 */
int lpo_features(const lpo_config *c, int64_t n, const double *const *x, const double *V,
                 const double *const *u, const double *P, const double *m, const uint32_t *id,
                 int64_t nq, const int64_t *q, double *out)
{
    int dim = c->dim, nf = dim + 2, nu = n_second(dim);
    const double *F[LPO_MAXF];
    F[0] = V;
    for (int k = 0; k < dim; ++k) F[1 + k] = u[k];
    F[dim + 1] = P;
    int kmax = c->k_max;
    uint32_t *cnt = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nq > 0 ? nq : 1));
    uint32_t *tot = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nq > 0 ? nq : 1));
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nq > 0 ? nq : 1) * (size_t)kmax);
    double *d2m = (double *)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1));
    if (!cnt || !tot || !nb || !d2m) { free(cnt); free(tot); free(nb); free(d2m); return -1; }
    int rc = lpo_neighbors(c, n, x, V, m, id, nq, q, 1, cnt, tot, nb, d2m);
    if (rc != 0) { free(cnt); free(tot); free(nb); free(d2m); return rc; }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nq; ++r) {
        int64_t i = q[r];
        double cd[LPO_MAXF * LPO_MAXN];
        const int64_t *lst = nb + r * kmax;
        central_fit(c, x, F, nf, i, lst, (int)cnt[r], cd);
        const double *dV = cd, *dP = cd + (dim + 1) * nu;
        double gP = 0, gV = 0, hP = 0, hV = 0, divu = 0;
        for (int k = 0; k < dim; ++k) {
            gP += dP[k] * dP[k];
            gV += dV[k] * dV[k];
            hP += dP[dim + k] * dP[dim + k];
            hV += dV[dim + k] * dV[dim + k];
            divu += cd[(1 + k) * nu + k];
        }
        for (int s2 = 2 * dim; s2 < nu; ++s2) {
            hP += 2.0 * dP[s2] * dP[s2];
            hV += 2.0 * dV[s2] * dV[s2];
        }
        double bmin = 0, bmax = 0, ssb = 0, ssr = 0;
        for (int t = 0; t < (int)cnt[r]; ++t) {
            int64_t j = lst[t];
            double d[3], row[LPO_MAXN];
            for (int k = 0; k < dim; ++k) d[k] = offset(c, x, k, i, j);
            gfd_row(dim, d, row);
            double b = P[j] - P[i];
            double fit = 0;
            for (int s2 = 0; s2 < nu; ++s2) fit += row[s2] * dP[s2];
            if (b < bmin) bmin = b;
            if (b > bmax) bmax = b;
            ssb += b * b;
            ssr += (b - fit) * (b - fit);
        }
        double ell = sqrt(d2m[r]), Pi = P[i], Vi = V[i];
        double cs = sqrt(c->gamma * Pi * Vi);
        double f[8];
        f[0] = ell * sqrt(gP) / Pi;
        f[1] = ell * sqrt(gV) / Vi;
        for (int w = 0; w < 2; ++w) {
            const double *dd = w == 0 ? dP : dV;
            double gmax = 0.0, best = 0.0;
            for (int k = 0; k < dim; ++k) gmax = fmax(gmax, fabs(dd[k]));
            for (int k = 0; k < dim; ++k) {
                double g = fabs(dd[k]);
                if (g < 0.5 * gmax) continue;
                double h = ell * fabs(dd[dim + k]);
                double rr = (g + h) > 0.0 ? h / (g + h) : 0.0;
                best = fmax(best, rr);
            }
            f[2 + w] = best;
        }
        (void)hP; (void)hV;
        f[4] = ell * divu / cs;
        f[5] = bmax / Pi;
        f[6] = -bmin / Pi;
        f[7] = ssb > 0 ? sqrt(ssr / ssb) : 0.0;
        for (int k = 0; k < 8; ++k) {
            double t = log1p(10.0 * fabs(f[k]));
            out[r * 8 + k] = (k == 4 && f[k] < 0) ? -t : t;
        }
    }
    free(cnt); free(tot); free(nb); free(d2m);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* reservoir inflow state (Sec. 4, the nozzle inlet boundary condition)      */
/* ------------------------------------------------------------------------ */

/*
 * Free-surface ghost particles (Sec. 2.2 step 3: where the free boundary
 * condition applies and a particle's neighbourhood is incomplete in one of
 * the 2 dim axis directions, ghost particles complete it).  The paper leaves
 * the ghosts' placement and state to the 2018 LP paper; reading:
 *   - direction (k, s) of fluid particle i (id < n_fluid) is incomplete when
 *     fewer than min_per_side members of its neighbour list (lpo_neighbors
 *     with this configuration) have an offset along axis k of sign s (offsets
 *     exactly 0 count on neither side, as for the one-sided stencils);
 *     particles with no neighbour at all get no ghosts;
 *   - the ghost of (i, k, s) sits at x_i + s ell_i e_k, ell_i = sqrt(d2) of
 *     i's nearest neighbour, with i's mass, specific volume and velocity and
 *     the pressure p_ghost (0: vacuum), and id ghost_base + 2 dim id_i + 2k +
 *     (s > 0), so that ids stay distinct and ghosts (ids >= n_fluid) are
 *     frozen in a step.
 * Ghosts are written in the order (particle index, k, side -, +) to out_*
 * (capacity max_out); returns their count, or -1 when max_out is too small
 * or memory runs out.
 */
int64_t lpo_free_surface_ghosts(const lpo_config *c, int64_t n, const double *const *x, const double *V,
                                const double *const *u, const double *m, const uint32_t *id,
                                int32_t min_per_side, double p_ghost, uint32_t ghost_base, int64_t max_out,
                                double *const *out_x, double *out_V, double *const *out_u, double *out_P,
                                double *out_m, uint32_t *out_id)
{
    int64_t *q = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    uint32_t *cnt = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t *tot = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1) * (size_t)c->k_max);
    double *d2m = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t ng = -1;
    if (!q || !cnt || !tot || !nb || !d2m) goto done;
    for (int64_t i = 0; i < n; ++i) q[i] = i;
    if (lpo_neighbors(c, n, x, V, m, id, n, q, 1, cnt, tot, nb, d2m) != 0) goto done;
    ng = 0;
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)id[i] >= c->n_fluid || cnt[i] == 0) continue;
        const double ell = sqrt(d2m[i]);
        for (int k = 0; k < c->dim; ++k) {
            int neg = 0, pos = 0;
            for (uint32_t t = 0; t < cnt[i]; ++t) {
                const double dx = offset(c, x, k, i, nb[i * c->k_max + t]);
                if (dx < 0.0) ++neg;
                else if (dx > 0.0) ++pos;
            }
            for (int side = 0; side < 2; ++side) {
                if ((side ? pos : neg) >= min_per_side) continue;
                if (ng >= max_out) { ng = -1; goto done; }
                for (int a = 0; a < c->dim; ++a) out_x[a][ng] = x[a][i];
                out_x[k][ng] = side ? x[k][i] + ell : x[k][i] - ell;
                for (int a = 0; a < c->dim; ++a) out_u[a][ng] = u[a][i];
                out_V[ng] = V[i];
                out_P[ng] = p_ghost;
                out_m[ng] = m[i];
                out_id[ng] = ghost_base + (uint32_t)(2 * c->dim) * id[i] + (uint32_t)(2 * k + side);
                ++ng;
            }
        }
    }
done:
    free(q); free(cnt); free(tot); free(nb); free(d2m);
    return ng;
}

/*
 * The state of particles entering a nozzle from a reservoir at rest (P_res,
 * rho_res), given the inflow pressure P_inf (the mean pressure near the
 * inlet): the reservoir's entropy, P_res / rho_res^gamma = P_inf / rho_inf^gamma,
 * gives rho_inf; the enthalpy balance u_res^2/2 + c_res^2/(gamma-1) =
 * u_inf^2/2 + c_inf^2/(gamma-1) with u_res = 0 and c^2 = gamma P / rho gives
 * u_inf (0 where the inflow pressure is not below the reservoir's).
 */
void lpo_inflow_state(double gamma, double P_res, double rho_res, double P_inf, double *rho_inf, double *u_inf)
{
    double rho = rho_res * pow(P_inf / P_res, 1.0 / gamma);
    double c2_res = gamma * P_res / rho_res;
    double c2 = gamma * P_inf / rho;
    double w = 2.0 / (gamma - 1.0) * (c2_res - c2);
    *rho_inf = rho;
    *u_inf = w > 0.0 ? sqrt(w) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* learned state estimator: 8 -> 32 (ReLU) -> 1 (sigmoid), FP64              */
/* ------------------------------------------------------------------------ */

#define MLP_IN 8
#define MLP_H 32

/*
 * Forward pass for n samples: h = relu(W1 x + b1), z = w2 . h + b2, p = sigmoid(z).
 * W1 is row-major H x IN (W1[j*IN + k]).  Writes z and p.
 */
void lpo_mlp_forward(int64_t n, const double *X, const double *W1, const double *b1,
                     const double *w2, double b2, double *z, double *p)
{
    for (int64_t s = 0; s < n; ++s) {
        double acc = b2;
        for (int j = 0; j < MLP_H; ++j) {
            double a = b1[j];
            for (int k = 0; k < MLP_IN; ++k) a += W1[j * MLP_IN + k] * X[s * MLP_IN + k];
            double h = a > 0.0 ? a : 0.0;
            acc += w2[j] * h;
        }
        z[s] = acc;
        p[s] = 1.0 / (1.0 + exp(-acc));
    }
}

/*
 * Mean class-weighted binary cross-entropy and its gradient:
 *   L = (1/n) sum_s c_s [ -y_s log p_s - (1 - y_s) log(1 - p_s) ],
 *   c_s = pos_weight for y_s = 1, 1 otherwise,
 * with dL/dz_s = c_s (p_s - y_s) / n, back-propagated through the two layers
 * (ReLU derivative taken as 0 at a = 0).  Returns L; gradients are overwritten.
 */
double lpo_mlp_loss_grad(int64_t n, const double *X, const double *y, double pos_weight,
                         const double *W1, const double *b1, const double *w2, double b2,
                         double *gW1, double *gb1, double *gw2, double *gb2)
{
    double L = 0.0;
    memset(gW1, 0, sizeof(double) * MLP_H * MLP_IN);
    memset(gb1, 0, sizeof(double) * MLP_H);
    memset(gw2, 0, sizeof(double) * MLP_H);
    *gb2 = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        double a[MLP_H], h[MLP_H];
        double zz = b2;
        for (int j = 0; j < MLP_H; ++j) {
            double t = b1[j];
            for (int k = 0; k < MLP_IN; ++k) t += W1[j * MLP_IN + k] * X[s * MLP_IN + k];
            a[j] = t;
            h[j] = t > 0.0 ? t : 0.0;
            zz += w2[j] * h[j];
        }
        double cw = y[s] > 0.5 ? pos_weight : 1.0;
        /* log(sigmoid(z)) = -log1p(exp(-z)), log(1 - sigmoid(z)) = -log1p(exp(z)) */
        double lp = zz >= 0.0 ? -log1p(exp(-zz)) : zz - log1p(exp(zz));
        double lq = zz >= 0.0 ? -zz - log1p(exp(-zz)) : -log1p(exp(zz));
        L += cw * (-y[s] * lp - (1.0 - y[s]) * lq);
        double pz = 1.0 / (1.0 + exp(-zz));
        double dz = cw * (pz - y[s]) / (double)n;
        *gb2 += dz;
        for (int j = 0; j < MLP_H; ++j) {
            gw2[j] += dz * h[j];
            double da = a[j] > 0.0 ? dz * w2[j] : 0.0;
            gb1[j] += da;
            for (int k = 0; k < MLP_IN; ++k) gW1[j * MLP_IN + k] += da * X[s * MLP_IN + k];
        }
    }
    return L / (double)n;
}

/*
 * One Adam update (Kingma & Ba) of np parameters at step t (1-based):
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 */
void lpo_adam(int64_t np, double *w, const double *g, double *mo, double *ve, int64_t t,
              double lr, double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < np; ++i) {
        mo[i] = beta1 * mo[i] + (1.0 - beta1) * g[i];
        ve[i] = beta2 * ve[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = mo[i] / c1, vh = ve[i] / c2;
        w[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* number of OpenMP threads the oracle uses (1 without OpenMP) */
int lpo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void lpo_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
