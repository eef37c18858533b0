// lp_internal.cuh -- device-side building blocks shared by the liblp.so
// translation units (never by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lp.h"
#include "lp_split.h"

namespace lp {

constexpr int KMAX = 80;          // largest k_max the kernels accept
constexpr int MORTON_BITS = 21;   // bits per axis of a Morton key (one simulation)
constexpr int MAX_LEVELS = 22;    // cell levels 0..21
constexpr int NB_WARPS = 6;       // warps per block of the neighbour query (static smem <= 48 KB)
constexpr int NB_CAP = 128;       // candidate buffer per warp (a power of two: the sort's size)
// The per-particle query compacts its buffer once more than NB_CAP - 32 entries
// are held and then appends up to 32: the compacted entries (k_max; with the
// octant selection fewer than k_max + 8) must leave that room.
static_assert((NB_CAP & (NB_CAP - 1)) == 0 && KMAX + 8 <= NB_CAP - 32, "per-particle buffer too small for KMAX");
// packed fit record of F <= 5 fields: floats [0,3) position hi, [3,6)
// position lo, [6,8) hi and lo of the last field (P in a step), then hi, lo of
// fields 0..F-2 from float 8 on -- so the first 32 bytes hold the positions and
// the last field
constexpr int REC_F4 = 4;
constexpr int REC_XH = 0, REC_XL = 3;
__host__ __device__ constexpr int rec_fh(int f, int F) { return f == F - 1 ? 6 : 8 + 2 * f; }
__host__ __device__ constexpr int rec_fl(int f, int F) { return f == F - 1 ? 7 : 9 + 2 * f; }

// status bits kept in the device status word (1 << lp_status)
constexpr uint32_t ST_CAPACITY = 1u << LP_ERR_CAPACITY;
constexpr uint32_t ST_ILLCOND = 1u << LP_ERR_ILLCOND;
constexpr uint32_t ST_NONFINITE = 1u << LP_ERR_NONFINITE;
constexpr uint32_t ST_ARG = 1u << LP_ERR_ARG;

// per-particle fit flags (lp_gfd_derivs status output)
constexpr uint32_t FIT_LINEAR = 1u, FIT_NONE = 2u, FIT_FP64 = 8u;

// device counters (unsigned long long each)
enum Counter {
    C_FLAGGED = 0, C_FP64, C_LINEAR, C_NOFIT, C_OVERFLOW, C_NONFINITE, C_MLP_UNCERTAIN,
    C_MAXCOUNT, C_STATUS, C_REDO_LEN, C_STEPS, C_MLP_SKIP, C_MLP_MISS, C_PLAIN_LEN, C_QFB_LEN, C_REFINED,
    C_REFINE_LEN, C_QUEUE_TILE, C_QUEUE_CENTRAL, C_QUEUE_PLAIN, C_OCT_GAP, C_COUNT
};

// method constants as the kernels see them
struct DevCfg {
    int dim, precision, radius_mode, k_max, k_side, k_per_side, limiter, estimator, refine;
    int select;           // LP_SELECT_*
    double refine_ratio;
    int mlp_audit;
    float mlp_tau_lo;
    int mbits;            // bits per axis of the Morton part of a key
    int nsim_max;         // simulations per batched call (1: a single simulation)
    int periodic[3];
    double gamma, radius, kappa, flat_eps, active_frac, tau32, tau64;
    double s_ref[5];
    double box_lo[3], box_hi[3];
    double Lper[3];       // box_hi - box_lo on periodic axes
    float Lper_h[3], Lper_l[3];
    float radius_f, radius2_f, kappa_f;   // float copies: (float)radius, (float)(radius^2), (float)kappa
    int64_t n_fluid;
};

// the float query radius of a particle from RN(m) and RN(V): kappa (m V)^(1/dim)
// (volume mode) or R (fixed mode); 0 for a non-finite or negative volume.
// Written once per build into the fourth component of the particle's float4
// position (hi part).
__device__ inline float query_radius_ff(const DevCfg& c, int dim, float mf, float Vf)
{
    float Rf;
    if (c.radius_mode == LP_RADIUS_FIXED) Rf = c.radius_f;
    else {
        float wf = mf * Vf;
        if (!(wf > 0.0f)) wf = 0.0f;
        const float r = dim == 3 ? cbrtf(wf) : (dim == 2 ? sqrtf(wf) : wf);
        Rf = c.kappa_f * r;
    }
    if (!(Rf >= 0.0f) || isinf(Rf)) Rf = 0.0f;
    return Rf;
}

// grid parameters computed on the device every build
struct Grid {
    double lo[3];         // quantisation origin
    double L;             // cube edge
    double inv;           // 2^mbits / L
    int lmin, lmax;       // cell levels in use
    float lo_h[3], lo_l[3];   // origin as float hi/lo (FP32 query set-up)
    float inv_f, L_f;
};

// ---------------------------------------------------------------------------
// Morton helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__host__ __device__ inline uint64_t spread2(uint64_t v)
{
    v &= 0xffffffffull;
    v = (v | (v << 16)) & 0x0000ffff0000ffffull;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}

template <int DIM>
__host__ __device__ inline uint64_t morton(const uint32_t* q)
{
    if (DIM == 3) return spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    if (DIM == 2) return spread2(q[0]) | (spread2(q[1]) << 1);
    return q[0];
}

// total order of doubles as unsigned integers (-0 is mapped to +0)
// LSD radix sort of the Morton keys: RS_BITS-bit digits over tiles of
// RS_TILE_KEYS keys (block counts and digit totals: RS_BINS x (tiles + 1) words)
constexpr int RS_BITS = 9;
constexpr int RS_BINS = 1 << RS_BITS;
constexpr int RS_TILE_KEYS = 2048;

// bits [lo, hi) of a key the sort orders by: the simulation index and the cell
// bits down to table level lmax_cap (every bit in 1D), in whole digits
inline void sort_bit_range(int dim, int mbits, int lmax_cap, int simbits, int& lo, int& hi)
{
    if (dim == 1) { lo = 0; hi = 64; return; }
    hi = dim * mbits + simbits;
    const int need = dim * lmax_cap + simbits;
    lo = hi - RS_BITS * ((need + RS_BITS - 1) / RS_BITS);
    if (lo < 0) lo = 0;
}

__device__ inline uint64_t order_key(double x)
{
    if (x == 0.0) x = 0.0;
    uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// ---------------------------------------------------------------------------
// exact FP64 geometry, fixed operation order (no contraction)
// ---------------------------------------------------------------------------
__device__ inline double offset64(const DevCfg& c, int k, double xi, double xj)
{
    double dx = __dsub_rn(xj, xi);
    if (c.periodic[k]) {
        double L = c.Lper[k];
        double h = __dmul_rn(0.5, L);
        if (dx > h) dx = __dsub_rn(dx, L);
        else if (dx < -h) dx = __dadd_rn(dx, L);
    }
    return dx;
}

// neighbour membership for squared distance d2 and w = m_i V_i
__device__ inline bool inside64(const DevCfg& c, int dim, double d2, double w)
{
    if (c.radius_mode == LP_RADIUS_FIXED) {
        double R2 = __dmul_rn(c.radius, c.radius);
        return d2 <= R2;
    }
    double k2 = __dmul_rn(c.kappa, c.kappa);
    double ww = __dmul_rn(w, w);
    if (dim == 3) {
        double k6 = __dmul_rn(__dmul_rn(k2, k2), k2);
        return __dmul_rn(__dmul_rn(d2, d2), d2) <= __dmul_rn(k6, ww);
    }
    if (dim == 2) {
        double k4 = __dmul_rn(k2, k2);
        return __dmul_rn(d2, d2) <= __dmul_rn(k4, ww);
    }
    return d2 <= __dmul_rn(k2, ww);
}

// split a double into float hi + float lo (x ~ hi + lo): h = RN(x), l =
// RN(x - h), by integer operations where lp_split.h handles the value, by FP64
// conversions and a subtraction elsewhere (the same results)
__device__ inline void split(double x, float& h, float& l)
{
    if (split_exact(x, h, l)) return;
    h = __double2float_rn(x);
    l = __double2float_rn(__dsub_rn(x, (double)h));
}

// RN(x) as a float (integer operations where lp_split.h handles the value)
__device__ inline float to_float_rn(double x)
{
    float h;
    return round_exact(x, h) ? h : __double2float_rn(x);
}

// 32 bytes (two float4) from a 32-byte-aligned global address that the kernel
// only reads, as one 256-bit load: a lane gathering a record from a random
// address costs the L1 one wavefront per load instruction, so one wide load
// instead of two halves that cost
__device__ __forceinline__ void ldg256(const float4* p, float4& lo, float4& hi)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
        : "l"(p));
}

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ inline unsigned lane_id() { return threadIdx.x & 31u; }

__device__ inline void count_add(unsigned long long* ctr, int which, unsigned long long v)
{
    if (v) atomicAdd(ctr + which, v);
}

// one atomic per warp: counts the active lanes with pred set
__device__ inline void warp_count(unsigned long long* ctr, int which, bool pred)
{
    unsigned m = __activemask();
    unsigned b = __ballot_sync(m, pred);
    if (b && (int)(threadIdx.x & 31u) == __ffs(m) - 1) atomicAdd(ctr + which, (unsigned long long)__popc(b));
}

}  // namespace lp

// ---------------------------------------------------------------------------
// context (host-side object, device buffers)
// ---------------------------------------------------------------------------
struct lp_ctx {
    lp_config cfg;
    lp::DevCfg dc;
    int64_t cap;
    int device;
    int lmax_cap;             // finest level a table is allocated for
    int sort_lo_bit, sort_hi_bit;
    int64_t level_off[lp::MAX_LEVELS + 1];
    int64_t table_entries;
    // sort
    uint64_t* keys[2];
    uint32_t* vals[2];
    uint32_t* hist;           // [256][max_blocks]
    int64_t hist_blocks;
    // sorted copies of the state
    double* sx[3];
    double* sV;
    double* su[3];
    double* sP;
    double* sm;
    uint32_t* sid;
    float4* rec;              // packed per-particle fit record, REC_F4 float4 each
    float4* pos4;             // [n][2] position hi / lo as float4 (neighbour query)
    // cell tables, neighbour lists
    unsigned long long* cells;
    uint32_t* nb_count;
    uint32_t* nb_total;
    uint32_t* nb_idx;
    double* nb_d2min;
    uint64_t* keys_sorted;    // points at keys[0] or keys[1] after the sort
    uint32_t* perm_sorted;    // matching permutation (sorted position -> input index)
    // grid, time step, counters
    lp::Grid* grid;               // one per simulation
    double* dt_dev;               // one per simulation
    unsigned long long* dt_min;   // per simulation: bit pattern of min(d2 / c^2)
    unsigned long long* ext;      // per simulation: 8 extent words
    int* grange;                  // [2] table levels in use over all simulations
    int64_t* level_off_dev;
    uint32_t* sim_of;             // simulation of each particle (input order)
    const int64_t* offsets;       // batched call: device [nsim + 1] (null: one simulation)
    int nsim;                     // simulations of the current call
    unsigned long long* counters;
    uint32_t* redo_list;
    // split fit schedule: compacted plain-stage list and intermediate record,
    // and the list of FP32 central fits deferred to the correction kernel
    uint32_t* plain_list;
    uint32_t* refine_list;
    void* mid;
    int schedule;                 // LP_SCHED_FUSED / LP_SCHED_SPLIT
    // lp_step_host: device copy of the caller's host particles, a second stream
    // for the copies that overlap the key sort, and the event the gather waits on
    lp_particles stage;
    double* stage_buf;
    cudaStream_t aux;
    cudaEvent_t ev_host_start, ev_host_in;
    cudaEvent_t gather_wait;      // when set, build() waits for it before the (geometry) gather
    cudaEvent_t fields_wait;      // when set, build() gathers in two stages and waits for this
                                  // one before the fields (u, P), after the neighbour query
    cudaEvent_t ev_host_fields, ev_sorted, ev_fields_done;
    int64_t n_lists;          // n of the last neighbour build (0: none)
    int lists_stale;          // lp_remove_outside ran since: the lists no longer describe the particles
    int tables_dirty;         // tables hold entries of the last build
    double reduce_min_w;
    // learned estimator: FP32 master weights, BF16 copy used by the kernels, Adam
    float* mlp_master;
    void* mlp_bf16;
    float* mlp_m1;
    float* mlp_m2;
    float* mlp_grad;
    float* mlp_loss;
    int64_t mlp_step;
    int mlp_ready;
    // reservoir inflow (lp_inflow): the in-plane lattice of a layer [in_npat][2],
    // the device state (committed and next), the sampling partial sums, and
    // the inlet of the first call
    double* in_pattern;
    int64_t in_npat;
    double* in_state;
    double* in_part;
    int in_ghosts;                // reservoir ghosts were appended
    lp_inlet in_cfg;
    // captured step
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
    int64_t graph_launches;       // kernels in one replay
    // launch accounting and optional phase timing
    int64_t launches;
    int profiling;
    cudaEvent_t ev[2 * LP_NPHASES * 4];
    int ev_used;                      // events recorded since the last read
    int ev_phase[LP_NPHASES * 4];
    double phase_ms[LP_NPHASES];
    int64_t phase_launches[LP_NPHASES];
};

namespace lp {
// launchers implemented in the .cu files
cudaError_t build_grid(lp_ctx* c, const lp_particles* p, cudaStream_t s);
cudaError_t make_keys(lp_ctx* c, const lp_particles* p, cudaStream_t s);
int radix_passes(const lp_ctx* c);
cudaError_t radix_sort(lp_ctx* c, int64_t n, cudaStream_t s);
cudaError_t gather(lp_ctx* c, const lp_particles* p, cudaStream_t s);
cudaError_t gather_geometry(lp_ctx* c, const lp_particles* p, cudaStream_t s);
cudaError_t gather_fields(lp_ctx* c, const lp_particles* p, cudaStream_t s);
cudaError_t fill_tables(lp_ctx* c, int64_t n, bool clear, cudaStream_t s);
cudaError_t query_neighbors(lp_ctx* c, int64_t n, cudaStream_t s);
cudaError_t query_init();   // once per context: kernel attributes
int query_launches(const lp_ctx* c);   // kernels one query launches
cudaError_t scatter_back(lp_ctx* c, lp_particles* p, cudaStream_t s);
cudaError_t split_fields(lp_ctx* c, int64_t n, const double* const* f, int nf, cudaStream_t s);
cudaError_t run_derivs(lp_ctx* c, int64_t n, const double* const* f, int nf, int out_dtype,
                       void* out, uint32_t* status, cudaStream_t s);
cudaError_t run_onesided(lp_ctx* c, int64_t n, const double* const* f, int nf, double* out,
                         cudaStream_t s);
cudaError_t run_cfl(lp_ctx* c, int64_t n, double cfl, double dt_fixed, double* t, cudaStream_t s);
cudaError_t run_step(lp_ctx* c, lp_particles* p, const lp_step_diag* diag, cudaStream_t s);
}  // namespace lp
