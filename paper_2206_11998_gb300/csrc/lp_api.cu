// lp_api.cu -- the C ABI of liblp.so (include/lp.h): context management,
// argument checks, and the order of the phases of one LP step (Sec. 2.2).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lp_fit_kern.cuh"

using namespace lp;

namespace {

#define LP_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return LP_ERR_CUDA;             \
    } while (0)

template <typename P>
cudaError_t dalloc(P** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

// the buffers sized by the particle capacity n (sorted copies, records,
// neighbour lists, sort ping-pong, fit-schedule lists), allocated at
// lp_create and again by lp_reserve
cudaError_t alloc_n_buffers(lp_ctx* c, int64_t n)
{
    const int dim = c->dc.dim;
    c->hist_blocks = (n + RS_TILE_KEYS - 1) / RS_TILE_KEYS;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (r != cudaSuccess && e == cudaSuccess) e = r; };
    A(dalloc(&c->keys[0], n * 8)); A(dalloc(&c->keys[1], n * 8));
    A(dalloc(&c->vals[0], n * 4)); A(dalloc(&c->vals[1], n * 4));
    A(dalloc(&c->hist, (size_t)RS_BINS * (c->hist_blocks + 1) * 4));   // block counts + digit totals
    for (int k = 0; k < dim; ++k) { A(dalloc(&c->sx[k], n * 8)); A(dalloc(&c->su[k], n * 8)); }
    A(dalloc(&c->sV, n * 8)); A(dalloc(&c->sP, n * 8)); A(dalloc(&c->sm, n * 8)); A(dalloc(&c->sid, n * 4));
    A(dalloc(&c->rec, (size_t)n * REC_F4 * sizeof(float4)));
    A(dalloc(&c->pos4, (size_t)n * 2 * sizeof(float4)));
    A(dalloc(&c->nb_count, n * 4)); A(dalloc(&c->nb_total, n * 4));
    A(dalloc(&c->nb_idx, (size_t)n * c->cfg.k_max * 4)); A(dalloc(&c->nb_d2min, n * 8));
    A(dalloc(&c->sim_of, c->dc.nsim_max > 1 ? n * 4 : 4));
    A(dalloc(&c->redo_list, n * 4));
    A(dalloc(&c->plain_list, n * 4));
    A(dalloc(&c->refine_list, n * 4));
    A(dalloc(&c->mid, (size_t)n * MidN<3>::v * (c->cfg.precision == LP_PREC_FP32 ? 4 : 8)));
    return e;
}

void free_n_buffers(lp_ctx* c)
{
    void** ptrs[] = {(void**)&c->keys[0], (void**)&c->keys[1], (void**)&c->vals[0], (void**)&c->vals[1],
                     (void**)&c->hist, (void**)&c->sx[0], (void**)&c->sx[1], (void**)&c->sx[2], (void**)&c->su[0],
                     (void**)&c->su[1], (void**)&c->su[2], (void**)&c->sV, (void**)&c->sP, (void**)&c->sm,
                     (void**)&c->sid, (void**)&c->rec, (void**)&c->pos4, (void**)&c->nb_count,
                     (void**)&c->nb_total, (void**)&c->nb_idx, (void**)&c->nb_d2min, (void**)&c->sim_of,
                     (void**)&c->redo_list, (void**)&c->plain_list, (void**)&c->refine_list, (void**)&c->mid,
                     (void**)&c->stage_buf};
    for (void** p : ptrs) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
}

void free_all(lp_ctx* c)
{
    void* ptrs[] = {c->keys[0], c->keys[1], c->vals[0], c->vals[1], c->hist, c->sx[0], c->sx[1], c->sx[2],
                    c->sV, c->su[0], c->su[1], c->su[2], c->sP, c->sm, c->sid, c->rec, c->pos4, c->cells, c->nb_count, c->nb_total,
                    c->nb_idx, c->nb_d2min, c->grid, c->dt_dev, c->dt_min, c->counters, c->redo_list,
                    c->plain_list, c->refine_list, c->mid, c->ext, c->grange, c->level_off_dev, c->sim_of,
                    c->mlp_master, c->mlp_bf16, c->mlp_m1, c->mlp_m2, c->mlp_grad, c->mlp_loss, c->stage_buf,
                    c->in_pattern, c->in_state, c->in_part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

lp_status check_cfg(const lp_config* g)
{
    if (!g) return LP_ERR_ARG;
    if (g->dim < 1 || g->dim > 3) return LP_ERR_ARG;
    if (g->precision != LP_PREC_FP32 && g->precision != LP_PREC_FP64) return LP_ERR_ARG;
    if (g->radius_mode < 0 || g->radius_mode > 2) return LP_ERR_ARG;
    if (g->radius_mode == LP_RADIUS_KSIDE && (g->dim != 1 || g->k_per_side < 1 || g->k_per_side > 8 ||
                                              g->k_max < 2 * g->k_per_side))
        return LP_ERR_ARG;
    if (g->radius_mode == LP_RADIUS_FIXED && !(g->radius > 0.0)) return LP_ERR_ARG;
    if (g->radius_mode == LP_RADIUS_VOLUME && !(g->kappa > 0.0)) return LP_ERR_ARG;
    if (g->k_max < 1 || g->k_max > KMAX) return LP_ERR_ARG;
    if (g->k_side < 1 || g->k_side > 16) return LP_ERR_ARG;
    if (!(g->gamma > 1.0)) return LP_ERR_ARG;
    if (g->limiter < 0 || g->limiter > 3) return LP_ERR_ARG;
    if (g->estimator != LP_EST_PLAIN && g->estimator != LP_EST_MLP) return LP_ERR_ARG;
    if (g->estimator == LP_EST_MLP && (g->limiter != LP_LIM_FLAGGED || !(g->mlp_tau_lo >= 0.0) ||
                                       !(g->mlp_tau_lo <= 1.0)))
        return LP_ERR_ARG;
    if (g->capacity < 1 || g->capacity > (int64_t)0x7fffffff) return LP_ERR_ARG;
    if (!(g->tau32 >= 0.0) || !(g->tau64 >= 0.0)) return LP_ERR_ARG;
    double L = -1.0;
    int nper = 0;
    for (int k = 0; k < g->dim; ++k) nper += g->periodic[k] ? 1 : 0;
    if (nper != 0 && nper != g->dim) return LP_ERR_ARG;   // periodic on every axis or on none
    for (int k = 0; k < g->dim; ++k) {
        if (!g->periodic[k]) continue;
        double e = g->box_hi[k] - g->box_lo[k];
        if (!(e > 0.0)) return LP_ERR_ARG;
        if (L > 0.0 && e != L) return LP_ERR_ARG;   // a periodic box must be a cube
        L = e;
    }
    if (g->max_level < 0 || g->max_level > 17) return LP_ERR_ARG;
    if (g->max_sims < 0 || g->max_sims > (1 << 20)) return LP_ERR_ARG;
    if (g->max_sims > 1 && g->dim == 1) return LP_ERR_ARG;   // 1D keys are the raw order of x
    if (g->refine < LP_REFINE_AUTO || g->refine > LP_REFINE_NEVER || !(g->refine_ratio >= 0.0)) return LP_ERR_ARG;
    if (g->select != LP_SELECT_NEAREST && g->select != LP_SELECT_OCTANT) return LP_ERR_ARG;
    if (g->select == LP_SELECT_OCTANT && (g->dim < 2 || g->radius_mode == LP_RADIUS_KSIDE)) return LP_ERR_ARG;
    if (g->reserved != 0) return LP_ERR_ARG;
    if (!(g->t_end >= 0.0) || isinf(g->t_end)) return LP_ERR_ARG;
    return LP_OK;
}

lp_status check_particles(const lp_ctx* c, const lp_particles* p)
{
    if (!p) return LP_ERR_ARG;
    if (p->n < 0) return LP_ERR_ARG;
    if (p->n > c->cap) return LP_ERR_CAPACITY;
    if (p->n == 0) return LP_OK;   // nothing is read or written
    int d = c->dc.dim;
    for (int k = 0; k < d; ++k)
        if (!p->x[k] || !p->u[k]) return LP_ERR_ARG;
    if (!p->V || !p->P || !p->m || !p->id) return LP_ERR_ARG;
    return LP_OK;
}

// the first nf of the F fields a fit kernel reads, into the fit records
__global__ void k_split_fields(int64_t n, int nf, int F, const double* f0, const double* f1, const double* f2,
                               const double* f3, const double* f4, float4* rec)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* f[5] = {f0, f1, f2, f3, f4};
    float* r = reinterpret_cast<float*>(rec + i * REC_F4);
    for (int q = 0; q < nf; ++q) split(f[q][i], r[rec_fh(q, F)], r[rec_fl(q, F)]);
}

// dt_s = cfl * sqrt(min_i d2min_i / (gamma P_i V_i)) over the fluid particles of
// simulation s (one simulation: a grid-stride loop; several: one particle per
// thread, reduced over the warp when its particles share a simulation)
__global__ void k_cfl(int64_t n, DevCfg c, const double* d2min, const double* P, const double* V,
                      const uint32_t* id, const uint64_t* keys, int key_shift, unsigned long long* dtmin)
{
    // The smallest quotient d2 / cs2 is kept as the pair (bn, bd) and compared
    // by cross-multiplication, d2 bd < bn cs2 (both sides positive): two FP64
    // multiplications per particle instead of a division, which is a sequence
    // of FP64 operations on a GPU with little FP64 throughput.  The one
    // division comes at the end, per warp.  (The comparison rounds: between
    // two quotients within a few ulp either may win, far inside the accuracy
    // the step's Delta t is held to.)
    // The tests compare the bit patterns as integers: for doubles that are
    // not negative and not NaN the order of the patterns is the order of the
    // values, and an integer comparison does not occupy the FP64 units
    // (finite positive values below 2^1024 have patterns below 0x7ff0...).
    constexpr long long INF_BITS = 0x7ff0000000000000ll;
    double bn = INFINITY, bd = 1.0;
    uint32_t sim = 0;
    bool many = c.nsim_max > 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (many) sim = (uint32_t)(keys[i] >> key_shift);
        const double d2 = d2min[i];
        const long long d2b = __double_as_longlong(d2);
        // fluid, 0 <= d2 < inf (-0 has the sign bit and is left out with the negatives)
        if ((int64_t)id[i] < c.n_fluid && d2b >= 0 && d2b < INF_BITS) {
            const double cs2 = (c.gamma * P[i]) * V[i];
            const long long cb = __double_as_longlong(cs2);
            if (cb > 0 && cb < INF_BITS &&
                __double_as_longlong(d2 * bd) < __double_as_longlong(bn * cs2)) { bn = d2; bd = cs2; }
        }
        if (many) break;
    }
    uint32_t s0 = __shfl_sync(0xffffffffu, sim, 0);
    if (__all_sync(0xffffffffu, sim == s0)) {
        for (int o = 16; o > 0; o >>= 1) {
            const double on = __shfl_xor_sync(0xffffffffu, bn, o), od = __shfl_xor_sync(0xffffffffu, bd, o);
            if (__double_as_longlong(on * bd) < __double_as_longlong(bn * od)) { bn = on; bd = od; }
        }
        if ((threadIdx.x & 31) != 0) return;
    }
    const double best = bn / bd;
    if (best >= 0.0 && best < INFINITY) atomicMin(dtmin + sim, (unsigned long long)__double_as_longlong(best));
}

__global__ void k_dt_finalize(int nsim, double cfl, double dt_fixed, double t_end, const unsigned long long* dtmin,
                              double* dt, double* t, unsigned long long* counters)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsim) return;
    double v;
    if (dt_fixed > 0.0) v = dt_fixed;
    else v = cfl * sqrt(__longlong_as_double((long long)dtmin[s]));
    if (!(v > 0.0) || isinf(v) || isnan(v)) {
        atomicOr(reinterpret_cast<unsigned int*>(counters + C_STATUS), ST_NONFINITE);
        v = 0.0;
    }
    // the last step ends at t_end (a simulation already there does not move)
    if (t && t_end > 0.0) {
        const double rem = fmax(__dsub_rn(t_end, t[s]), 0.0);
        if (v >= rem) {
            dt[s] = rem;
            t[s] = fmax(t[s], t_end);
            if (s == 0) counters[C_STEPS] += 1;
            return;
        }
    }
    dt[s] = v;
    if (t) t[s] += v;
    if (s == 0) counters[C_STEPS] += 1;
}

void fill_fit_args(lp_ctx* c, FitArgs& a, int64_t n)
{
    memset(&a, 0, sizeof(a));
    a.c = c->dc;
    a.n = n;
    a.count = c->nb_count;
    a.idx = c->nb_idx;
    a.d2min = c->nb_d2min;
    for (int k = 0; k < 3; ++k) {
        int kk = k < c->dc.dim ? k : 0;
        a.sx[k] = c->sx[kk];
    }
    a.rec = c->rec;
    a.sid = c->sid;
    a.sm = c->sm;
    a.counters = c->counters;
    a.redo_list = c->redo_list;
    a.list = nullptr;
    a.list_len = c->counters + C_REDO_LEN;
    a.keys = c->keys_sorted;
    a.key_shift = c->dc.dim * c->dc.mbits;
    a.plain_list = c->plain_list;
    a.plain_len = c->counters + C_PLAIN_LEN;
    a.refine_list = c->refine_list;
    a.refine_len = c->counters + C_REFINE_LEN;
    a.queue = c->counters + C_QUEUE_CENTRAL;      // and C_QUEUE_PLAIN after it
    a.mid = c->mid;
    a.mid_cap = c->cap;
    a.plain_ident = 0;
}

constexpr int EV_PAIRS = LP_NPHASES * 4;

cudaError_t flush_events(lp_ctx* c)
{
    for (int q = 0; q < c->ev_used; ++q) {
        cudaError_t e = cudaEventSynchronize(c->ev[2 * q + 1]);
        if (e != cudaSuccess) return e;
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, c->ev[2 * q], c->ev[2 * q + 1]);
        if (e != cudaSuccess) return e;
        c->phase_ms[c->ev_phase[q]] += ms;
    }
    c->ev_used = 0;
    return cudaSuccess;
}

// phase bracket: counts launches always, records events when profiling
struct Phase {
    lp_ctx* c;
    int ph;
    int launches;
    cudaStream_t s;
    int slot;
    Phase(lp_ctx* c_, int ph_, int launches_, cudaStream_t s_) : c(c_), ph(ph_), launches(launches_), s(s_), slot(-1)
    {
        c->launches += launches;
        c->phase_launches[ph] += launches;
        if (c->profiling) {
            if (c->ev_used == EV_PAIRS) flush_events(c);
            slot = c->ev_used++;
            c->ev_phase[slot] = ph;
            cudaEventRecord(c->ev[2 * slot], s);
        }
    }
    ~Phase()
    {
        if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], s);
    }
};

}  // namespace

namespace lp {

cudaError_t run_cfl(lp_ctx* c, int64_t n, double cfl, double dt_fixed, double* t, cudaStream_t s)
{
    int nsim = c->nsim;
    cudaError_t e = cudaMemsetAsync(c->dt_min, 0x7f, sizeof(unsigned long long) * nsim, s);   // large positive
    if (e != cudaSuccess) return e;
    if (dt_fixed <= 0.0 && n > 0) {
        int64_t nb_ = (n + 255) / 256;
        unsigned blocks = nsim > 1 ? (unsigned)nb_ : (unsigned)(nb_ < 152 * 8 ? nb_ : 152 * 8);
        k_cfl<<<blocks, 256, 0, s>>>(n, c->dc, c->nb_d2min, c->sP, c->sV, c->sid, c->keys_sorted,
                                     c->dc.dim * c->dc.mbits, c->dt_min);
    }
    k_dt_finalize<<<(unsigned)((nsim + 127) / 128), 128, 0, s>>>(nsim, cfl, dt_fixed, c->cfg.t_end, c->dt_min,
                                                                c->dt_dev, t, c->counters);
    return cudaGetLastError();
}

}  // namespace lp

namespace {

// the fit + update pass of one step: the main pass over all particles (fused,
// or split into central and plain kernels), then, after an FP32 pass, the FP64
// redo of the particles it listed
lp_status run_fit(lp_ctx* c, FitArgs a, const StepOut& o, int sched, cudaStream_t s)
{
    const bool split = (sched & LP_SCHED_SPLIT) != 0;
    const int dim = c->dc.dim;
    if (split) LP_CUDA(cudaMemsetAsync(c->counters + C_PLAIN_LEN, 0, 8, s));
    // with no learned gate every fitted particle takes the plain stage: its
    // slot is its index, and the plain kernel keeps the key order (slots of
    // particles without a plain stage stay all ones)
    if (split && !o.features && c->dc.estimator != LP_EST_MLP && a.n > 0) {
        a.plain_ident = 1;
        LP_CUDA(cudaMemsetAsync(c->plain_list, 0xff, (size_t)a.n * 4, s));
    }
    if (c->dc.precision == LP_PREC_FP32) {
        LP_CUDA(cudaMemsetAsync(c->counters + C_REDO_LEN, 0, 8, s));
        const bool defer = split && c->dc.refine == LP_REFINE_AUTO;
        if (defer) LP_CUDA(cudaMemsetAsync(c->counters + C_REFINE_LEN, 0, 8, s));
        {
            Phase ph(c, LP_PH_FIT, split ? (defer ? 3 : 2) : 1, s);
            if (split && (sched & LP_SCHED_QUEUE_FIT)) LP_CUDA(launch_step_split_queue_f32(dim, a, o, s));
            else LP_CUDA(split ? launch_step_split_f32(dim, a, o, s) : launch_step_f32(dim, a, o, s));
        }
        a.list = c->redo_list;
        Phase ph(c, LP_PH_FIT64, 1, s);
        LP_CUDA(launch_step_f64(dim, a, o, s));
    } else {
        Phase ph(c, LP_PH_FIT64, split ? 2 : 1, s);
        LP_CUDA(split ? launch_step_split_f64(dim, a, o, s) : launch_step_f64(dim, a, o, s));
    }
    return LP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* lp_version(void) { return "lp-gb300 0.1 (sm_103a)"; }

const char* lp_status_string(lp_status s)
{
    switch (s) {
    case LP_OK: return "ok";
    case LP_ERR_ARG: return "invalid argument";
    case LP_ERR_CUDA: return "CUDA runtime error";
    case LP_ERR_CAPACITY: return "particle count exceeds context capacity";
    case LP_ERR_ILLCOND: return "stencil without a usable fit";
    case LP_ERR_NONFINITE: return "non-finite state or time step";
    case LP_ERR_TIMEOUT: return "bounded device wait timed out";
    case LP_ERR_STATE: return "entry point called out of order";
    }
    return "unknown status";
}

lp_status lp_create(const lp_config* cfg, lp_ctx** out)
{
    if (!out) return LP_ERR_ARG;
    *out = nullptr;
    lp_status st = check_cfg(cfg);
    if (st != LP_OK) return st;
    lp_ctx* c = (lp_ctx*)calloc(1, sizeof(lp_ctx));
    if (!c) return LP_ERR_CUDA;
    c->cfg = *cfg;
    if (c->cfg.tau32 == 0.0) c->cfg.tau32 = 1e-3;
    if (c->cfg.tau64 == 0.0) c->cfg.tau64 = 1e-12;
    DevCfg& d = c->dc;
    d.dim = cfg->dim;
    d.precision = cfg->precision;
    d.radius_mode = cfg->radius_mode;
    d.k_max = cfg->k_max;
    d.k_side = cfg->k_side;
    d.k_per_side = cfg->k_per_side;
    d.limiter = cfg->limiter;
    d.estimator = cfg->estimator;
    d.refine = cfg->refine;
    d.refine_ratio = cfg->refine_ratio > 0.0 ? cfg->refine_ratio : 0.1;
    d.select = cfg->select;
    d.mlp_tau_lo = (float)cfg->mlp_tau_lo;
    d.mlp_audit = cfg->mlp_audit ? 1 : 0;
    d.nsim_max = cfg->max_sims > 1 ? cfg->max_sims : 1;
    c->schedule = cfg->estimator == LP_EST_MLP ? LP_SCHED_SPLIT : LP_SCHED_FUSED;
    int simbits = 0;
    while ((1 << simbits) < d.nsim_max) ++simbits;
    d.mbits = (cfg->dim == 3 && d.nsim_max > 1) ? (64 - simbits) / 3 : MORTON_BITS;
    if (d.mbits > MORTON_BITS) d.mbits = MORTON_BITS;
    d.gamma = cfg->gamma;
    d.radius = cfg->radius;
    d.kappa = cfg->kappa;
    d.radius_f = (float)cfg->radius;
    d.radius2_f = (float)(cfg->radius * cfg->radius);
    d.kappa_f = (float)cfg->kappa;
    d.flat_eps = cfg->flat_eps;
    d.active_frac = cfg->active_frac;
    d.tau32 = c->cfg.tau32;
    d.tau64 = c->cfg.tau64;
    for (int f = 0; f < 5; ++f) d.s_ref[f] = cfg->s_ref[f];
    for (int k = 0; k < 3; ++k) {
        d.periodic[k] = k < cfg->dim ? cfg->periodic[k] : 0;
        d.box_lo[k] = cfg->box_lo[k];
        d.box_hi[k] = cfg->box_hi[k];
        d.Lper[k] = cfg->box_hi[k] - cfg->box_lo[k];
        d.Lper_h[k] = (float)d.Lper[k];
        d.Lper_l[k] = (float)(d.Lper[k] - (double)d.Lper_h[k]);
    }
    d.n_fluid = cfg->n_fluid;
    c->cap = cfg->capacity;
    cudaGetDevice(&c->device);
    // cell tables: levels 0..lmax_cap, 2^(dim l) entries each
    int dim = cfg->dim;
    bool batched = d.nsim_max > 1;
    if (dim == 1) c->lmax_cap = 0;
    else c->lmax_cap = cfg->max_level > 0 ? cfg->max_level : (dim == 3 ? (batched ? 6 : 9) : (batched ? 8 : 13));
    if (c->lmax_cap > d.mbits) c->lmax_cap = d.mbits;
    int64_t off = 0;
    for (int l = 0; l <= MAX_LEVELS; ++l) {
        c->level_off[l] = off;
        if (l <= c->lmax_cap && dim > 1) off += (int64_t)d.nsim_max << (dim * l);
    }
    c->table_entries = dim > 1 ? off : 1;
    // sort bits: the simulation and the cells down to level lmax_cap
    sort_bit_range(dim, d.mbits, c->lmax_cap, simbits, c->sort_lo_bit, c->sort_hi_bit);
    bool ok = alloc_n_buffers(c, c->cap) == cudaSuccess;
    auto A = [&](cudaError_t e) { if (e != cudaSuccess) ok = false; };
    A(dalloc(&c->cells, (size_t)c->table_entries * 8));
    int ns = d.nsim_max;
    A(dalloc(&c->grid, sizeof(Grid) * ns)); A(dalloc(&c->dt_dev, 8 * ns));
    A(dalloc(&c->dt_min, 8 * ns)); A(dalloc(&c->ext, 64 * (size_t)ns)); A(dalloc(&c->grange, 8));
    A(dalloc(&c->level_off_dev, sizeof(int64_t) * (MAX_LEVELS + 1)));
    A(dalloc(&c->counters, C_COUNT * 8));
    A(dalloc(&c->mlp_master, MLP_NPARAM * 4)); A(dalloc(&c->mlp_bf16, MLP_NPARAM * 2));
    A(dalloc(&c->mlp_m1, MLP_NPARAM * 4)); A(dalloc(&c->mlp_m2, MLP_NPARAM * 4));
    A(dalloc(&c->mlp_grad, MLP_NPARAM * 4)); A(dalloc(&c->mlp_loss, 4));
    if (ok) {
        A(cudaMemset(c->cells, 0, (size_t)c->table_entries * 8));
        A(cudaMemset(c->counters, 0, C_COUNT * 8));
        A(cudaMemset(c->dt_dev, 0, 8 * ns));
        A(cudaMemcpy(c->level_off_dev, c->level_off, sizeof(int64_t) * (MAX_LEVELS + 1), cudaMemcpyHostToDevice));
        for (int q = 0; q < 2 * EV_PAIRS && ok; ++q) A(cudaEventCreate(&c->ev[q]));
        A(query_init());
        A(cudaDeviceSynchronize());
    }
    if (!ok) {
        free_all(c);
        free(c);
        return LP_ERR_CUDA;
    }
    *out = c;
    return LP_OK;
}

lp_status lp_reserve(lp_ctx* c, int64_t capacity)
{
    if (!c || capacity < 1 || capacity > (int64_t)0x7fffffff || capacity < c->n_lists) return LP_ERR_ARG;
    LP_CUDA(cudaDeviceSynchronize());
    free_n_buffers(c);
    c->cap = capacity;
    c->cfg.capacity = capacity;
    if (alloc_n_buffers(c, capacity) != cudaSuccess) {
        free_n_buffers(c);
        c->cap = 0;
        return LP_ERR_CUDA;
    }
    // the tables still hold the last build's entries, whose keys are gone
    LP_CUDA(cudaMemset(c->cells, 0, (size_t)c->table_entries * 8));
    c->tables_dirty = 0;
    c->n_lists = 0;
    if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
    if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
    LP_CUDA(cudaDeviceSynchronize());
    return LP_OK;
}

lp_status lp_destroy(lp_ctx* c)
{
    if (!c) return LP_OK;
    cudaDeviceSynchronize();
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (int q = 0; q < 2 * EV_PAIRS; ++q)
        if (c->ev[q]) cudaEventDestroy(c->ev[q]);
    if (c->ev_host_start) cudaEventDestroy(c->ev_host_start);
    if (c->ev_host_in) cudaEventDestroy(c->ev_host_in);
    if (c->ev_host_fields) cudaEventDestroy(c->ev_host_fields);
    if (c->ev_sorted) cudaEventDestroy(c->ev_sorted);
    if (c->ev_fields_done) cudaEventDestroy(c->ev_fields_done);
    if (c->aux) cudaStreamDestroy(c->aux);
    free_all(c);
    free(c);
    return LP_OK;
}

static lp_status build(lp_ctx* c, lp_particles* p, cudaStream_t s)
{
    int64_t n = p->n;
    bool tables = c->dc.dim > 1;
    if (c->tables_dirty) {   // clear the previous build's table entries
        Phase ph(c, LP_PH_TABLES, tables && c->n_lists > 0 ? 1 : 0, s);
        LP_CUDA(fill_tables(c, c->n_lists, true, s));
        c->tables_dirty = 0;
    }
    c->n_lists = 0;
    c->lists_stale = 0;
    if (n == 0) return LP_OK;
    {
        Phase ph(c, LP_PH_GRID, 4 + (c->nsim > 1 ? 1 : 0), s);
        LP_CUDA(build_grid(c, p, s));
        LP_CUDA(make_keys(c, p, s));
    }
    {
        Phase ph(c, LP_PH_SORT, 3 * radix_passes(c), s);
        LP_CUDA(radix_sort(c, n, s));
    }
    if (c->gather_wait) {
        Phase ph(c, LP_PH_HOST_IN, 0, s);
        LP_CUDA(cudaStreamWaitEvent(s, c->gather_wait, 0));
    }
    {
        Phase ph(c, LP_PH_GATHER, 2, s);
        LP_CUDA(c->fields_wait ? gather_geometry(c, p, s) : gather(c, p, s));
    }
    if (c->fields_wait) {
        // the fields, gathered on the copy stream behind their copies from the
        // host, while the tables and the query run here
        LP_CUDA(cudaEventRecord(c->ev_sorted, s));
        LP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_sorted, 0));
        LP_CUDA(gather_fields(c, p, c->aux));
        LP_CUDA(cudaEventRecord(c->ev_fields_done, c->aux));
        c->launches += 1;
    }
    {
        Phase ph(c, LP_PH_TABLES, tables ? 1 : 0, s);
        LP_CUDA(fill_tables(c, n, false, s));
        c->tables_dirty = tables ? 1 : 0;
    }
    {
        Phase ph(c, LP_PH_QUERY, query_launches(c), s);
        LP_CUDA(query_neighbors(c, n, s));
    }
    if (c->fields_wait) {          // the fields, gathered while the query ran
        Phase ph(c, LP_PH_HOST_IN, 0, s);
        LP_CUDA(cudaStreamWaitEvent(s, c->ev_fields_done, 0));
    }
    c->n_lists = n;
    return LP_OK;
}

lp_status lp_build_neighbors(lp_ctx* c, lp_particles* p, lp_neighbors* out, lp_stream stream)
{
    if (!c) return LP_ERR_ARG;
    c->nsim = 1;
    c->offsets = nullptr;
    lp_status st = check_particles(c, p);
    if (st != LP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = build(c, p, s);
    if (st != LP_OK) return st;
    if (p->n > 0) {
        Phase ph(c, LP_PH_GATHER, 1, s);
        LP_CUDA(scatter_back(c, p, s));
    }
    if (out) {
        out->n = p->n;
        out->k_max = c->dc.k_max;
        out->pad = 0;
        out->count = c->nb_count;
        out->total = c->nb_total;
        out->idx = c->nb_idx;
        out->d2min = c->nb_d2min;
        out->keys = c->keys_sorted;
    }
    return LP_OK;
}

lp_status lp_gfd_derivs(lp_ctx* c, const lp_particles* p, const double* const* fields, int32_t nfields,
                        int32_t out_dtype, void* derivs, uint32_t* status, lp_stream stream)
{
    if (!c || !p || !fields || !derivs || nfields < 1) return LP_ERR_ARG;
    if (out_dtype != LP_OUT_F32 && out_dtype != LP_OUT_F64) return LP_ERR_ARG;
    if (c->n_lists != p->n || c->lists_stale) return LP_ERR_STATE;
    for (int f = 0; f < nfields; ++f)
        if (!fields[f]) return LP_ERR_ARG;
    int64_t n = p->n;
    if (n == 0) return LP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int dim = c->dc.dim;
    bool fp32 = c->dc.precision == LP_PREC_FP32;
    for (int f0 = 0; f0 < nfields;) {
        int F = (dim == 3 && nfields - f0 == 1) ? 1 : 5;
        int real = nfields - f0 < F ? nfields - f0 : F;
        FitArgs a;
        fill_fit_args(c, a, n);
        for (int q = 0; q < 5; ++q) a.fd[q] = fields[f0 + (q < real ? q : 0)];
        DerivOut o;
        o.out = derivs;
        o.out_f64 = out_dtype == LP_OUT_F64;
        o.f_first = f0;
        o.f_real = real;
        o.status = status;
        if (fp32) {
            {
                Phase ph(c, LP_PH_GATHER, 1, s);
                k_split_fields<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
                    n, F, F, a.fd[0], a.fd[1], a.fd[2], a.fd[3], a.fd[4], c->rec);
            }
            LP_CUDA(cudaMemsetAsync(c->counters + C_REDO_LEN, 0, 8, s));
            {
                Phase ph(c, LP_PH_FIT, 1, s);
                LP_CUDA(launch_derivs_f32(dim, F, a, o, s));
            }
            a.list = c->redo_list;
            Phase ph(c, LP_PH_FIT64, 1, s);
            LP_CUDA(launch_derivs_f64(dim, F, a, o, s));
        } else {
            Phase ph(c, LP_PH_FIT64, 1, s);
            LP_CUDA(launch_derivs_f64(dim, F, a, o, s));
        }
        f0 += real;
    }
    // the neighbour lists stay valid; the split copies of the state are
    // rebuilt by the next lp_step
    return LP_OK;
}

lp_status lp_onesided_derivs(lp_ctx* c, const lp_particles* p, const double* const* fields, int32_t nfields,
                             double* derivs, lp_stream stream)
{
    if (!c || !p || !fields || !derivs || nfields < 1 || nfields > 5) return LP_ERR_ARG;
    if (c->n_lists != p->n || c->lists_stale) return LP_ERR_STATE;
    for (int f = 0; f < nfields; ++f)
        if (!fields[f]) return LP_ERR_ARG;
    int64_t n = p->n;
    if (n == 0) return LP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int dim = c->dc.dim;
    FitArgs a;
    fill_fit_args(c, a, n);
    for (int q = 0; q < 5; ++q) a.fd[q] = fields[q < nfields ? q : 0];
    if (c->dc.precision == LP_PREC_FP32) {
        {
            Phase ph(c, LP_PH_GATHER, 1, s);
            k_split_fields<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
                n, 5, 5, a.fd[0], a.fd[1], a.fd[2], a.fd[3], a.fd[4], c->rec);
        }
        LP_CUDA(cudaMemsetAsync(c->counters + C_REDO_LEN, 0, 8, s));
        {
            Phase ph(c, LP_PH_FIT, 1, s);
            LP_CUDA(launch_onesided_f32(dim, a, derivs, nfields, s));
        }
        a.list = c->redo_list;
        Phase ph(c, LP_PH_FIT64, 1, s);
        LP_CUDA(launch_onesided_f64(dim, a, derivs, nfields, s));
    } else {
        Phase ph(c, LP_PH_FIT64, 1, s);
        LP_CUDA(launch_onesided_f64(dim, a, derivs, nfields, s));
    }
    return LP_OK;
}

}  // extern "C"

namespace {

// everything of a step before the fit pass: checks, neighbour build, CFL step;
// fills the fit pass's arguments.  *n_out = 0 when there is nothing to fit.
lp_status step_prologue(lp_ctx* c, lp_particles* p, const int64_t* offsets, int32_t nsim, double dt, double cfl,
                        double* t, const lp_step_diag* diag, cudaStream_t s, FitArgs& a, StepOut& o, int64_t* n_out)
{
    *n_out = 0;
    if (!c) return LP_ERR_ARG;
    lp_status st = check_particles(c, p);
    if (st != LP_OK) return st;
    if (nsim < 1 || nsim > c->dc.nsim_max || (nsim > 1 && !offsets)) return LP_ERR_ARG;
    if (!(dt > 0.0) && !(cfl > 0.0)) return LP_ERR_ARG;
    if (c->dc.estimator == LP_EST_MLP && !c->mlp_ready) return LP_ERR_STATE;
    if (isnan(dt) || isinf(dt)) return LP_ERR_ARG;
    c->nsim = nsim;
    c->offsets = nsim > 1 ? offsets : nullptr;
    st = build(c, p, s);
    if (st != LP_OK) return st;
    int64_t n = p->n;
    {
        Phase ph(c, LP_PH_CFL, (dt <= 0.0 && n > 0) ? 2 : 1, s);
        LP_CUDA(run_cfl(c, n, cfl, dt, t, s));
    }
    if (n == 0) return LP_OK;
    int dim = c->dc.dim;
    fill_fit_args(c, a, n);
    a.fd[0] = c->sV;
    for (int k = 0; k < dim; ++k) a.fd[1 + k] = c->su[k];
    a.fd[dim + 1] = c->sP;
    for (int q = dim + 2; q < 5; ++q) a.fd[q] = c->sV;
    memset(&o, 0, sizeof(o));
    for (int k = 0; k < 3; ++k) {
        o.x[k] = p->x[k < dim ? k : 0];
        o.u[k] = p->u[k < dim ? k : 0];
    }
    o.V = p->V; o.P = p->P; o.m = p->m; o.id = p->id;
    if (diag) {
        o.flag = diag->flag; o.phi = diag->phi; o.r = diag->r; o.features = diag->features;
        o.gate_p = diag->gate_p;
    }
    a.mlp_w = reinterpret_cast<const __nv_bfloat16*>(c->mlp_bf16);
    o.dt = c->dt_dev;
    *n_out = n;
    return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_step_batched(lp_ctx* c, lp_particles* p, const int64_t* offsets, int32_t nsim, double dt, double cfl,
                          double* t, const lp_step_diag* diag, lp_stream stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    FitArgs a;
    StepOut o;
    int64_t n = 0;
    lp_status st = step_prologue(c, p, offsets, nsim, dt, cfl, t, diag, s, a, o, &n);
    if (st != LP_OK || n == 0) return st;
    return run_fit(c, a, o, c->schedule, s);
}

lp_status lp_step_host(lp_ctx* c, lp_particles* h, double dt, double cfl, double* t, const lp_step_diag* diag,
                       lp_stream stream)
{
    if (!c) return LP_ERR_ARG;
    if (c->dc.nsim_max > 1) return LP_ERR_STATE;
    lp_status st = check_particles(c, h);
    if (st != LP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int dim = c->dc.dim;
    const int64_t n = h->n;
    if (!c->stage_buf) {            // first call: the device copy at capacity, the copy stream
        const size_t cap = (size_t)c->cap;
        LP_CUDA(cudaMalloc(&c->stage_buf, cap * 8 * (2 * (size_t)dim + 3) + cap * 4));
        double* q = c->stage_buf;
        memset(&c->stage, 0, sizeof(c->stage));
        for (int k = 0; k < dim; ++k) { c->stage.x[k] = q; q += cap; c->stage.u[k] = q; q += cap; }
        c->stage.V = q; q += cap;
        c->stage.P = q; q += cap;
        c->stage.m = q; q += cap;
        c->stage.id = reinterpret_cast<uint32_t*>(q);
        LP_CUDA(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
        LP_CUDA(cudaEventCreateWithFlags(&c->ev_host_start, cudaEventDisableTiming));
        LP_CUDA(cudaEventCreateWithFlags(&c->ev_host_in, cudaEventDisableTiming));
        LP_CUDA(cudaEventCreateWithFlags(&c->ev_host_fields, cudaEventDisableTiming));
        LP_CUDA(cudaEventCreateWithFlags(&c->ev_sorted, cudaEventDisableTiming));
        LP_CUDA(cudaEventCreateWithFlags(&c->ev_fields_done, cudaEventDisableTiming));
    }
    // pinned (page-locked) host arrays: the step writes the new state straight
    // into them; otherwise into the device copy, then copied back
    const void* arrs[4 + 2 * 3] = {h->V, h->P, h->m, h->id};
    for (int k = 0; k < dim; ++k) { arrs[4 + k] = h->x[k]; arrs[4 + dim + k] = h->u[k]; }
    bool direct = true;
    for (int q = 0; q < 4 + 2 * dim; ++q) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, arrs[q]) != cudaSuccess) { cudaGetLastError(); direct = false; break; }
        if (at.type != cudaMemoryTypeHost || !at.devicePointer) { direct = false; break; }
    }
    lp_particles g = c->stage;
    g.n = n;
    const size_t b8 = (size_t)n * 8;
    if (n > 0) {
        // what the keys need (the positions) on the caller's stream; on the
        // copy stream, after everything before this step, what the query needs
        // next (m, V, id: the gather of the geometry waits for them) and then
        // what only the fit needs (u, P: gathered after the query)
        {
            Phase ph(c, LP_PH_HOST_IN, 0, s);
            for (int k = 0; k < dim; ++k) LP_CUDA(cudaMemcpyAsync(g.x[k], h->x[k], b8, cudaMemcpyHostToDevice, s));
        }
        LP_CUDA(cudaEventRecord(c->ev_host_start, s));
        LP_CUDA(cudaStreamWaitEvent(c->aux, c->ev_host_start, 0));
        LP_CUDA(cudaMemcpyAsync(g.m, h->m, b8, cudaMemcpyHostToDevice, c->aux));
        LP_CUDA(cudaMemcpyAsync(g.V, h->V, b8, cudaMemcpyHostToDevice, c->aux));
        LP_CUDA(cudaMemcpyAsync(g.id, h->id, (size_t)n * 4, cudaMemcpyHostToDevice, c->aux));
        LP_CUDA(cudaEventRecord(c->ev_host_in, c->aux));
        c->gather_wait = c->ev_host_in;
        for (int k = 0; k < dim; ++k) LP_CUDA(cudaMemcpyAsync(g.u[k], h->u[k], b8, cudaMemcpyHostToDevice, c->aux));
        LP_CUDA(cudaMemcpyAsync(g.P, h->P, b8, cudaMemcpyHostToDevice, c->aux));
        LP_CUDA(cudaEventRecord(c->ev_host_fields, c->aux));
        c->fields_wait = c->ev_host_fields;
    }
    FitArgs a;
    StepOut o;
    int64_t nn = 0;
    st = step_prologue(c, &g, nullptr, 1, dt, cfl, t, diag, s, a, o, &nn);
    if (c->gather_wait) {           // (a no-op when the gathers already waited for the copies)
        cudaStreamWaitEvent(s, c->gather_wait, 0);
        c->gather_wait = nullptr;
    }
    if (c->fields_wait) {
        cudaStreamWaitEvent(s, c->fields_wait, 0);
        c->fields_wait = nullptr;
    }
    if (st != LP_OK || nn == 0) return st;
    if (direct) {
        cudaPointerAttributes at;
        auto dev = [&](const void* hp) -> void* {
            return cudaPointerGetAttributes(&at, hp) == cudaSuccess ? at.devicePointer : nullptr;
        };
        for (int k = 0; k < 3; ++k) {
            o.x[k] = static_cast<double*>(dev(h->x[k < dim ? k : 0]));
            o.u[k] = static_cast<double*>(dev(h->u[k < dim ? k : 0]));
        }
        o.V = static_cast<double*>(dev(h->V));
        o.P = static_cast<double*>(dev(h->P));
        o.m = static_cast<double*>(dev(h->m));
        o.id = static_cast<uint32_t*>(dev(h->id));
    }
    st = run_fit(c, a, o, c->schedule, s);
    if (st != LP_OK || direct) return st;
    Phase ph(c, LP_PH_HOST_OUT, 0, s);
    for (int k = 0; k < dim; ++k) {
        LP_CUDA(cudaMemcpyAsync(h->x[k], g.x[k], b8, cudaMemcpyDeviceToHost, s));
        LP_CUDA(cudaMemcpyAsync(h->u[k], g.u[k], b8, cudaMemcpyDeviceToHost, s));
    }
    LP_CUDA(cudaMemcpyAsync(h->V, g.V, b8, cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaMemcpyAsync(h->P, g.P, b8, cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaMemcpyAsync(h->m, g.m, b8, cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaMemcpyAsync(h->id, g.id, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    return LP_OK;
}

lp_status lp_set_schedule(lp_ctx* c, int32_t schedule)
{
    if (!c || (schedule & ~(LP_SCHED_SPLIT | LP_SCHED_QUERY_WARP | LP_SCHED_QUEUE_QUERY | LP_SCHED_QUEUE_FIT)) != 0)
        return LP_ERR_ARG;
    c->schedule = schedule;
    return LP_OK;
}

lp_status lp_get_schedule(lp_ctx* c, int32_t* schedule)
{
    if (!c || !schedule) return LP_ERR_ARG;
    *schedule = c->schedule;
    return LP_OK;
}

lp_status lp_autotune(lp_ctx* c, lp_particles* p, const int64_t* offsets, int32_t nsim, double dt, double cfl,
                      int32_t reps, double* out_ms, lp_stream stream)
{
    if (!c || reps < 1) return LP_ERR_ARG;
    if (c->profiling) return LP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    // the counters and the launch tally are put back afterwards: tuning is not a step
    unsigned long long saved[C_COUNT];
    LP_CUDA(cudaMemcpyAsync(saved, c->counters, sizeof(saved), cudaMemcpyDeviceToHost, s));
    double* dt_saved = (double*)malloc(sizeof(double) * c->dc.nsim_max);
    if (!dt_saved) return LP_ERR_CUDA;
    if (cudaMemcpyAsync(dt_saved, c->dt_dev, sizeof(double) * c->dc.nsim_max, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        free(dt_saved);
        return LP_ERR_CUDA;
    }
    struct FreeOnExit { double* p; ~FreeOnExit() { free(p); } } dt_guard{dt_saved};
    const int64_t launches0 = c->launches;
    int64_t ph_launches0[LP_NPHASES];
    memcpy(ph_launches0, c->phase_launches, sizeof(ph_launches0));
    FitArgs a;
    StepOut o;
    int64_t n = 0;
    lp_status st = step_prologue(c, p, offsets, nsim, dt, cfl, nullptr, nullptr, s, a, o, &n);
    if (st != LP_OK) return st;
    // fit FUSED, fit SPLIT, query tiles, query per particle, query tiles from
    // the work queue, fit SPLIT from the work queues (FP32)
    double ms[LP_AUTOTUNE_TIMES] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (n > 0) {
        // the fit pass reads the sorted copies and writes only its outputs, so it
        // can be repeated; outputs go to scratch so that the state is untouched
        const int dim = c->dc.dim;
        double* scratch = nullptr;
        uint32_t* sid = nullptr;
        if (cudaMalloc(&scratch, (size_t)n * 8 * (2 * dim + 3)) != cudaSuccess) return LP_ERR_CUDA;
        if (cudaMalloc(&sid, (size_t)n * 4) != cudaSuccess) { cudaFree(scratch); return LP_ERR_CUDA; }
        for (int k = 0; k < 3; ++k) {
            o.x[k] = scratch + (size_t)n * (k < dim ? k : 0);
            o.u[k] = scratch + (size_t)n * (dim + (k < dim ? k : 0));
        }
        o.V = scratch + (size_t)n * (2 * dim);
        o.P = scratch + (size_t)n * (2 * dim + 1);
        o.m = scratch + (size_t)n * (2 * dim + 2);
        o.id = sid;
        cudaEvent_t e0 = c->ev[0], e1 = c->ev[1];
        lp_status rs = LP_OK;
        auto timed = [&](auto&& body, double& out) {
            if (body() != LP_OK) return LP_ERR_CUDA;            // warm-up
            if (cudaEventRecord(e0, s) != cudaSuccess) return LP_ERR_CUDA;
            for (int r = 0; r < reps; ++r)
                if (body() != LP_OK) return LP_ERR_CUDA;
            float f = 0.0f;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&f, e0, e1) != cudaSuccess)
                return LP_ERR_CUDA;
            out = f / reps;
            return LP_OK;
        };
        // the query rewrites the same lists whichever schedule runs it
        const int keep = c->schedule;
        if (c->dc.radius_mode != LP_RADIUS_KSIDE && c->dc.dim > 1) {
            const int qs[3] = {0, LP_SCHED_QUERY_WARP, LP_SCHED_QUEUE_QUERY};
            const int qslot[3] = {2, 3, 4};
            for (int q = 0; q < 3 && rs == LP_OK; ++q) {
                c->schedule = qs[q];
                rs = timed([&] { return query_neighbors(c, n, s) == cudaSuccess ? LP_OK : LP_ERR_CUDA; },
                           ms[qslot[q]]);
            }
        }
        c->schedule = keep;
        const bool fp32 = c->dc.precision == LP_PREC_FP32;
        const int fs[3] = {LP_SCHED_FUSED, LP_SCHED_SPLIT, LP_SCHED_SPLIT | LP_SCHED_QUEUE_FIT};
        const int fslot[3] = {0, 1, 5};
        for (int f = 0; f < (fp32 ? 3 : 2) && rs == LP_OK; ++f)
            rs = timed([&] { return run_fit(c, a, o, fs[f], s); }, ms[fslot[f]]);
        cudaStreamSynchronize(s);
        cudaFree(scratch);
        cudaFree(sid);
        if (rs != LP_OK) return rs;
        // the fastest fit schedule, and the fastest query schedule
        int sched = LP_SCHED_FUSED;
        double best = ms[0];
        if (ms[1] < best) { sched = LP_SCHED_SPLIT; best = ms[1]; }
        if (fp32 && ms[5] > 0.0 && ms[5] < best) sched = LP_SCHED_SPLIT | LP_SCHED_QUEUE_FIT;
        if (ms[2] > 0.0) {
            double qbest = ms[2];
            int qsched = 0;
            if (ms[3] > 0.0 && ms[3] < qbest) { qsched = LP_SCHED_QUERY_WARP; qbest = ms[3]; }
            if (ms[4] > 0.0 && ms[4] < qbest) qsched = LP_SCHED_QUEUE_QUERY;
            sched |= qsched;
        }
        c->schedule = sched;
    }
    LP_CUDA(cudaMemcpyAsync(c->counters, saved, sizeof(saved), cudaMemcpyHostToDevice, s));
    LP_CUDA(cudaMemcpyAsync(c->dt_dev, dt_saved, sizeof(double) * c->dc.nsim_max, cudaMemcpyHostToDevice, s));
    LP_CUDA(cudaStreamSynchronize(s));
    c->launches = launches0;
    memcpy(c->phase_launches, ph_launches0, sizeof(ph_launches0));
    if (out_ms)
        for (int q = 0; q < LP_AUTOTUNE_TIMES; ++q) out_ms[q] = ms[q];
    return LP_OK;
}

lp_status lp_export_neighbors(lp_ctx* c, uint32_t* count, uint32_t* total, uint32_t* idx, double* d2min,
                              uint64_t* keys, lp_stream stream)
{
    if (!c) return LP_ERR_ARG;
    int64_t n = c->n_lists;
    if (n == 0) return LP_OK;
    if (c->lists_stale) return LP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (count) LP_CUDA(cudaMemcpyAsync(count, c->nb_count, n * 4, cudaMemcpyDeviceToDevice, s));
    if (total) LP_CUDA(cudaMemcpyAsync(total, c->nb_total, n * 4, cudaMemcpyDeviceToDevice, s));
    if (idx) LP_CUDA(cudaMemcpyAsync(idx, c->nb_idx, (size_t)n * c->dc.k_max * 4, cudaMemcpyDeviceToDevice, s));
    if (d2min) LP_CUDA(cudaMemcpyAsync(d2min, c->nb_d2min, n * 8, cudaMemcpyDeviceToDevice, s));
    if (keys) LP_CUDA(cudaMemcpyAsync(keys, c->keys_sorted, n * 8, cudaMemcpyDeviceToDevice, s));
    return LP_OK;
}

lp_status lp_grid_info(lp_ctx* c, double* out, lp_stream stream)
{
    if (!c || !out) return LP_ERR_ARG;
    Grid g;
    cudaStream_t s = (cudaStream_t)stream;
    LP_CUDA(cudaMemcpyAsync(&g, c->grid, sizeof(Grid), cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaStreamSynchronize(s));
    out[0] = g.lo[0]; out[1] = g.lo[1]; out[2] = g.lo[2]; out[3] = g.L; out[4] = (double)g.lmax;
    return LP_OK;
}

lp_status lp_set_profiling(lp_ctx* c, int32_t on)
{
    if (!c) return LP_ERR_ARG;
    c->profiling = on ? 1 : 0;
    return LP_OK;
}

lp_status lp_phase_times(lp_ctx* c, double* out_ms, int64_t* out_launches, lp_stream stream)
{
    if (!c) return LP_ERR_ARG;
    LP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    LP_CUDA(flush_events(c));
    for (int q = 0; q < LP_NPHASES; ++q) {
        if (out_ms) out_ms[q] = c->phase_ms[q];
        if (out_launches) out_launches[q] = c->phase_launches[q];
        c->phase_ms[q] = 0.0;
        c->phase_launches[q] = 0;
    }
    return LP_OK;
}

const char* lp_phase_name(int32_t ph)
{
    static const char* names[LP_NPHASES] = {"grid+keys", "radix-sort", "gather", "cell-tables",
                                            "neighbor-query", "cfl", "fit+update", "fit+update-fp64",
                                            "host-in", "host-out"};
    return (ph >= 0 && ph < LP_NPHASES) ? names[ph] : "unknown";
}

lp_status lp_step(lp_ctx* c, lp_particles* p, double dt, double cfl, double* t, const lp_step_diag* diag,
                  lp_stream stream)
{
    return lp_step_batched(c, p, nullptr, 1, dt, cfl, t, diag, stream);
}

lp_status lp_graph_capture(lp_ctx* c, lp_particles* p, const int64_t* offsets, int32_t nsim, double dt, double cfl,
                           double* t, lp_stream stream)
{
    if (!c || !p || !stream) return LP_ERR_ARG;
    if (c->profiling) return LP_ERR_STATE;
    if (c->n_lists != p->n || c->lists_stale || (c->dc.dim > 1 && !c->tables_dirty)) return LP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
    if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
    int64_t before = c->launches;
    LP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    lp_status st = lp_step_batched(c, p, offsets, nsim, dt, cfl, t, nullptr, stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != LP_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return LP_ERR_CUDA;
    c->graph = g;
    if (cudaGraphInstantiate(&c->graph_exec, g, 0) != cudaSuccess) return LP_ERR_CUDA;
    c->graph_launches = c->launches - before;
    c->launches = before;           // nothing ran yet
    return LP_OK;
}

lp_status lp_graph_launch(lp_ctx* c, lp_stream stream)
{
    if (!c) return LP_ERR_ARG;
    if (!c->graph_exec) return LP_ERR_STATE;
    LP_CUDA(cudaGraphLaunch(c->graph_exec, (cudaStream_t)stream));
    c->launches += c->graph_launches;
    return LP_OK;
}

const double* lp_dt_device(lp_ctx* c) { return c ? c->dt_dev : nullptr; }

lp_status lp_get_stats(lp_ctx* c, lp_stats* out, lp_stream stream)
{
    if (!c || !out) return LP_ERR_ARG;
    unsigned long long h[C_COUNT];
    double dt = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    LP_CUDA(cudaMemcpyAsync(h, c->counters, sizeof(h), cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaMemcpyAsync(&dt, c->dt_dev, 8, cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaStreamSynchronize(s));
    memset(out, 0, sizeof(*out));
    out->dt = dt;
    out->steps = (int64_t)h[C_STEPS];
    out->n_flagged = (int64_t)h[C_FLAGGED];
    out->n_fp64_redo = (int64_t)h[C_FP64];
    out->n_linear = (int64_t)h[C_LINEAR];
    out->n_nofit = (int64_t)h[C_NOFIT];
    out->n_overflow = (int64_t)h[C_OVERFLOW];
    out->n_nonfinite = (int64_t)h[C_NONFINITE];
    out->n_mlp_uncertain = (int64_t)h[C_MLP_UNCERTAIN];
    out->max_count = (uint32_t)h[C_MAXCOUNT];
    out->status = (uint32_t)h[C_STATUS];
    out->kernel_launches = c->launches;
    out->n_mlp_skip = (int64_t)h[C_MLP_SKIP];
    out->n_mlp_miss = (int64_t)h[C_MLP_MISS];
    out->n_query_fallback = (int64_t)h[C_QFB_LEN];
    out->n_refined = (int64_t)h[C_REFINED];
    return LP_OK;
}

lp_status lp_reset_stats(lp_ctx* c, lp_stream stream)
{
    if (!c) return LP_ERR_ARG;
    LP_CUDA(cudaMemsetAsync(c->counters, 0, C_COUNT * 8, (cudaStream_t)stream));
    return LP_OK;
}

}  // extern "C"
