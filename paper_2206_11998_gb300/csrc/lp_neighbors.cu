// lp_neighbors.cu -- Sec. 2.2 steps 3-4: neighbour lists
//   N(i) = {j != i : |x_j - x_i| <= R_i}, ordered by (d^2, id), first k_max kept.
//
// One warp per particle.  The particle queries the finest cell level whose edge
// is at least R_i, i.e. at most 3 cells per axis; the cells' key-sorted ranges
// come from the dense per-level tables, so candidates of a cell are contiguous
// and the 32 lanes read them coalesced.  Distances are first taken in FP32 from
// split (hi, lo) coordinates, which carry the offsets to ~3 ulp relative; only
// candidates within a rounding band of the radius, and entries whose order is
// within rounding of a neighbour's, are decided with the exact FP64 distance
// ((dx*dx + dy*dy) + dz*dz, no contraction), so the lists are bit-exact.
#include <algorithm>

#include "lp_internal.cuh"

namespace lp {

namespace {

constexpr float TOL_R = 4e-6f;   // relative band around R^2 decided in FP64
constexpr float TOL_T = 4e-6f;   // relative gap below which two entries are re-ordered in FP64

struct QueryArgs {
    DevCfg c;
    int64_t n;
    const Grid* g;            // one per simulation
    const uint64_t* keys;     // key-sorted keys: simulation = key >> (dim mbits)
    const int64_t* level_off;
    const unsigned long long* cells;
    const double* sx[3];
    const float4* pos4;       // [n][2]: position hi (xyz) and float radius (w), lo (xyz, 0)
    const double* sm;
    const double* sV;
    const uint32_t* sid;
    uint32_t* count;
    uint32_t* total;
    uint32_t* idx;
    double* d2min;
    unsigned long long* counters;
    // the per-particle kernel runs over this list (null: every particle)
    const uint32_t* list;
    const unsigned long long* list_len;
    // the tile kernel appends the particles it leaves here
    uint32_t* fb_list;
    unsigned long long* fb_len;
    // the persistent tile kernel's work counter (zero at launch)
    unsigned long long* queue;
};

template <int DIM>
__device__ inline double exact_d2(const QueryArgs& a, int64_t i, int64_t j)
{
    double d0 = offset64(a.c, 0, a.sx[0][i], a.sx[0][j]);
    double d2 = __dmul_rn(d0, d0);
    if (DIM > 1) { double d1 = offset64(a.c, 1, a.sx[1][i], a.sx[1][j]); d2 = __dadd_rn(d2, __dmul_rn(d1, d1)); }
    if (DIM > 2) { double d3 = offset64(a.c, 2, a.sx[2][i], a.sx[2][j]); d2 = __dadd_rn(d2, __dmul_rn(d3, d3)); }
    return d2;
}

constexpr int FCAP = 256;          // cells per frontier (current / next) per warp
constexpr uint32_t DESC_MIN = 64;  // cells with more particles than this are split into children

struct WarpBuf {
    unsigned long long key[NB_CAP];   // float bits of d2 << 32 | id
    uint32_t j[NB_CAP];
    double d64[NB_CAP];
    uint32_t tie[NB_CAP / 32];        // bit e: entry e is within rounding of entry e-1
    uint32_t cstart[32];
    uint32_t cexcl[32];
    unsigned long long front[2][FCAP];   // packed (level, unwrapped cell coordinates)
};

__device__ inline float key_d2(unsigned long long k) { return __uint_as_float((uint32_t)(k >> 32)); }

// frontier cell: level l in bits 58..62; per axis k the wrapped coordinate
// w_k in [0, 2^l) (17 bits at 17k) and the periodic image shift s_k in
// {-1, 0, 1} (2 bits at 51 + 2k); the unwrapped coordinate is w_k + s_k 2^l.
// A child keeps the shift: 2 (w + s 2^l) + b = (2w + b) + s 2^(l+1).
__device__ inline unsigned long long pack_cell(int l, const int (&w)[3], const int (&sh)[3])
{
    unsigned long long e = (unsigned long long)l << 58;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e |= (unsigned long long)(w[k] & 0x1ffff) << (17 * k);
        e |= (unsigned long long)(max(-1, min(1, sh[k])) + 1) << (51 + 2 * k);
    }
    return e;
}
__device__ inline void unpack_cell(unsigned long long e, int& l, int (&w)[3], int (&sh)[3])
{
    l = (int)((e >> 58) & 31u);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        w[k] = (int)((e >> (17 * k)) & 0x1ffffull);
        sh[k] = (int)((e >> (51 + 2 * k)) & 3ull) - 1;
    }
}

// Sort buf[0..m) by (d2, id) exactly; returns nothing, buffer sorted in place.
template <int DIM>
__device__ void sort_exact(const QueryArgs& a, WarpBuf& b, int m, int64_t i)
{
    unsigned lane = lane_id();
    int P = 32;
    while (P < m) P <<= 1;
    for (int e = m + (int)lane; e < P; e += 32) { b.key[e] = ~0ull; b.j[e] = 0xffffffffu; }
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int e = lane; e < P; e += 32) {
                int p = e ^ jj;
                if (p > e) {
                    bool up = (e & k) == 0;
                    unsigned long long ke = b.key[e], kp = b.key[p];
                    if ((ke > kp) == up) {
                        b.key[e] = kp; b.key[p] = ke;
                        uint32_t t = b.j[e]; b.j[e] = b.j[p]; b.j[p] = t;
                    }
                }
            }
            __syncwarp();
        }
    }
    // entries whose float distances are within rounding of a neighbour's; the
    // runs are fixed here, before any entry moves
    bool any = false;
    for (int e0 = 0; e0 < P; e0 += 32) {
        int e = e0 + (int)lane;
        bool tp = false, tn = false;
        if (e < m) {
            float d = key_d2(b.key[e]);
            tp = e > 0 && d <= key_d2(b.key[e - 1]) * (1.0f + TOL_T);
            tn = e + 1 < m && key_d2(b.key[e + 1]) <= d * (1.0f + TOL_T);
            if (tp || tn) { b.d64[e] = exact_d2<DIM>(a, i, b.j[e]); any = true; }
        }
        unsigned bits = __ballot_sync(0xffffffffu, tp);
        if (lane == 0) b.tie[e0 >> 5] = bits;
    }
    if (!__any_sync(0xffffffffu, any)) return;
    __syncwarp();
    if (lane == 0) {
        int e = 0;
        while (e < m) {
            int f = e + 1;
            while (f < m && ((b.tie[f >> 5] >> (f & 31)) & 1u)) ++f;
            // insertion sort of the run [e, f) by (exact d2, id)
            for (int q = e + 1; q < f; ++q) {
                unsigned long long kq = b.key[q];
                uint32_t jq = b.j[q];
                double dq = b.d64[q];
                int r = q - 1;
                while (r >= e) {
                    double dr = b.d64[r];
                    bool gt = dr > dq || (dr == dq && (uint32_t)b.key[r] > (uint32_t)kq);
                    if (!gt) break;
                    b.key[r + 1] = b.key[r]; b.j[r + 1] = b.j[r]; b.d64[r + 1] = b.d64[r];
                    --r;
                }
                b.key[r + 1] = kq; b.j[r + 1] = jq; b.d64[r + 1] = dq;
            }
            e = f;
        }
    }
    __syncwarp();
}

// Octree-style traversal of the per-level cell tables.  Cells start at the
// finest level whose edge is >= R (at most 3 per axis) and are classified
// lane-parallel from their box distances (in quantised units, with margins
// that cover the float rounding):
//   outside the radius                         -> skipped
//   nearest point beyond the current k_max-th distance (no kept neighbour
//   possible): entirely inside -> counted whole; otherwise counted by scanning
//   or split
//   large (> DESC_MIN particles, finer level available) -> split into children
//   otherwise                                  -> candidates scanned
// Split cells go to the next frontier, processed once the current one is done,
// so the k_max-th distance found so far prunes them.
// own position and radius terms of particle i, and the start cells of its
// query (written to b.front[0]): the cells of the finest level whose edge is
// at least half the radius that meet the radius's box.  Shared by both
// per-particle queries.
struct QueryStart {
    float hxi[3], lxi[3], tq[3];   // position (hi, lo) and quantised position
    float inv;                     // quantised units per length
    float R2f, Rq, Rout, Rin;      // squared radius; radius and box margins, quantised units
    int ncells;                    // start cells in b.front[0]
    uint64_t sim;
};

template <int DIM>
__device__ __forceinline__ void query_start(const QueryArgs& a, WarpBuf& b, int64_t i, QueryStart& st)
{
    unsigned lane = lane_id();
    const DevCfg& c = a.c;
    const int mb = c.mbits;
    const uint64_t sim = c.nsim_max > 1 ? (a.keys[i] >> (DIM * mb)) : 0ull;
    st.sim = sim;
    const Grid& g = a.g[sim];

    // own position and radius, all in FP32 (FP64 warp instructions are costly
    // on this part: one occupies a sub-partition's FP64 pipe for ~64 cycles)
    const float inv = g.inv_f;
    st.inv = inv;
    const float4 pih = a.pos4[2 * i], pil = a.pos4[2 * i + 1];
    st.hxi[0] = pih.x; st.hxi[1] = pih.y; st.hxi[2] = pih.z;
    st.lxi[0] = pil.x; st.lxi[1] = pil.y; st.lxi[2] = pil.z;
#pragma unroll
    for (int k = 0; k < DIM; ++k) st.tq[k] = ((st.hxi[k] - g.lo_h[k]) + (st.lxi[k] - g.lo_l[k])) * inv;   // quantised units, error < 1
    const float Rf = pih.w;                          // query_radius_ff, written by the gather
    st.R2f = (c.radius_mode == LP_RADIUS_FIXED) ? c.radius2_f : Rf * Rf;
    float Rc = Rf * (1.0f + 1e-5f);
    const float Rq = Rc * inv;
    st.Rq = Rq;
    st.Rout = Rf * inv * (1.0f + 2e-5f) + 2.0f;   // boxes beyond: no neighbour
    st.Rin = Rf * inv * (1.0f - 2e-5f) - 2.0f;    // boxes within: all neighbours
    if (lane == 0) {   // the minimum image needs R < L/2 on periodic axes
#pragma unroll
        for (int k = 0; k < DIM; ++k)
            if (c.periodic[k] && 2.0f * Rq >= ldexpf(1.0f, mb))
                atomicOr(reinterpret_cast<unsigned int*>(a.counters + C_STATUS), ST_ARG);
    }

    // start level: finest with cell edge L / 2^l >= Rc / 2 (at most 5 cells per axis)
    float Lf = g.L_f;
    float Rh = 0.5f * Rc;
    int l0 = Rh > 0.0f ? (int)floorf(log2f(Lf / Rh)) : g.lmax;
    while (l0 > 0 && ldexpf(Lf, -l0) < Rh) --l0;
    l0 = max(g.lmin, min(l0, g.lmax));
    long long ncell_axis = 1ll << l0;
    const float cell_scale = ldexpf(1.0f, -(mb - l0));
    long long clo[3] = {0, 0, 0};
    int nc[3] = {1, 1, 1};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        long long a0 = (long long)floorf((st.tq[k] - Rq - 2.0f) * cell_scale);
        long long a1 = (long long)floorf((st.tq[k] + Rq + 2.0f) * cell_scale);
        if (!c.periodic[k]) {
            a0 = max(0ll, min(a0, ncell_axis - 1));
            a1 = max(0ll, min(a1, ncell_axis - 1));
        } else if (a1 - a0 + 1 > ncell_axis) {
            a1 = a0 + ncell_axis - 1;
        }
        clo[k] = a0;
        nc[k] = (int)(a1 - a0 + 1);
    }
    int ncells = nc[0] * nc[1] * nc[2];
    if (ncells > FCAP) {   // cannot happen with cell edge >= radius / 2; recorded, never silent
        if (lane == 0) atomicOr(reinterpret_cast<unsigned int*>(a.counters + C_STATUS), ST_ILLCOND);
        ncells = FCAP;
    }
    for (int t = lane; t < ncells; t += 32) {
        int u = t;
        int wv[3] = {0, 0, 0}, shv[3] = {0, 0, 0};
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            long long v = clo[k] + (u % nc[k]);     // unwrapped (periodic axes: within one period)
            u /= nc[k];
            long long wr = ((v % ncell_axis) + ncell_axis) % ncell_axis;
            wv[k] = (int)wr;
            shv[k] = (int)((v - wr) / ncell_axis);
        }
        b.front[0][t] = pack_cell(l0, wv, shv);
    }
    __syncwarp();
    st.ncells = ncells;
}

template <int DIM>
__device__ void query_one(const QueryArgs& a, WarpBuf& b, int64_t i)
{
    unsigned lane = lane_id();
    const DevCfg& c = a.c;
    const int mb = c.mbits;
    const uint64_t sim = c.nsim_max > 1 ? (a.keys[i] >> (DIM * mb)) : 0ull;
    const Grid& g = a.g[sim];
    unsigned lt = (1u << lane) - 1u;
    QueryStart st;
    query_start<DIM>(a, b, i, st);
    const float* hxi = st.hxi;
    const float* lxi = st.lxi;
    const float* tq = st.tq;
    const float inv = st.inv;
    const float R2f = st.R2f, Rout = st.Rout, Rin = st.Rin;
    const int ncells = st.ncells;

    const uint32_t total_cap = 4u * (uint32_t)c.k_max;   // the count before truncation saturates here
    int m = 0;                     // entries in the buffer
    uint32_t whole = 0;            // particles of cells counted whole (per lane)
    uint32_t scanned_in = 0;       // scanned candidates inside the radius (warp-uniform)
    float cut = INFINITY;          // entries beyond this (float d2) can no longer be kept
    float cutq = INFINITY;         // the same distance in quantised units, with margin
    int cur = 0, ncur = ncells;
    while (ncur > 0) {
        int nnext = 0;
        for (int base0 = 0; base0 < ncur; base0 += 32) {
            uint32_t counted = scanned_in;
            {
                uint32_t wsum = whole;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
                counted += wsum;
            }
            const bool count_done = counted >= total_cap;   // further cells matter only if keepable
            // ---- classify one batch of cells, one lane per cell
            int e = base0 + (int)lane;
            uint32_t cs = 0, cn = 0;
            int act = 0;           // 0 nothing to scan, 1 scan, 2 scan for the count only, 3 split
            bool beyond = false;   // no particle of the cell can be kept
            int l = 0, wv[3] = {0, 0, 0}, shv[3] = {0, 0, 0};
            if (e < ncur) {
                unpack_cell(b.front[cur][e], l, wv, shv);
                uint32_t q[3] = {0, 0, 0};
                float size = ldexpf(1.0f, mb - l);
                float period = ldexpf(1.0f, mb);
                float dmin2 = 0.0f, dmax2 = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    q[k] = (uint32_t)wv[k];
                    float lo = (float)wv[k] * size + (float)shv[k] * period, hi = lo + size;
                    float dn = fmaxf(0.0f, fmaxf(lo - tq[k], tq[k] - hi));
                    float df = fmaxf(tq[k] - lo, hi - tq[k]);
                    dmin2 += dn * dn;
                    dmax2 += df * df;
                }
                uint64_t code = (sim << (DIM * l)) | morton<DIM>(q);
                unsigned long long ent = a.cells[a.level_off[l] + (int64_t)code];
                cs = (uint32_t)ent;
                uint32_t ce = (uint32_t)(ent >> 32);
                cn = ce > cs ? ce - cs : 0;
                float dmin = sqrtf(dmin2), dmax = sqrtf(dmax2);
                bool splittable = cn > DESC_MIN && l < g.lmax;
                beyond = dmin > cutq;
                if (cn == 0 || dmin >= Rout) act = 0;
                else if (beyond && (count_done || dmax <= Rin)) {
                    if (!count_done) whole += cn;
                    act = 0;
                }
                else if (splittable) act = 3;
                else act = beyond ? 2 : 1;
            }
            // ---- split cells: children into the next frontier; a cell that does
            // not fit waits there unsplit; with no room at all it is scanned
            const int nchild = 1 << DIM;
            unsigned sm_ = __ballot_sync(0xffffffffu, act == 3);
            int room = (FCAP - nnext) / nchild;
            int nsplit = min(__popc(sm_), max(room, 0));
            if (act == 3) {
                int rank = __popc(sm_ & lt);
                if (rank < room) {
                    int pos = nnext + rank * nchild;
                    for (int ch = 0; ch < nchild; ++ch) {
                        int cw[3] = {2 * wv[0] + (ch & 1), DIM > 1 ? 2 * wv[1] + ((ch >> 1) & 1) : 0,
                                     DIM > 2 ? 2 * wv[2] + ((ch >> 2) & 1) : 0};
                        b.front[cur ^ 1][pos + ch] = pack_cell(l + 1, cw, shv);
                    }
                    act = 0;
                }
            }
            int after = nnext + nsplit * nchild;
            unsigned wait_ = __ballot_sync(0xffffffffu, act == 3);
            if (act == 3) {
                int rank = __popc(wait_ & lt);
                if (after + rank < FCAP) {
                    b.front[cur ^ 1][after + rank] = pack_cell(l, wv, shv);
                    act = 0;
                } else {
                    act = beyond ? 2 : 1;
                }
            }
            nnext = min(FCAP, after + __popc(wait_));
            // ---- scanned cells: flatten their candidates over the lanes
            uint32_t cnt = (act == 1 || act == 2) ? cn : 0;
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += v;
            }
            uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
            unsigned co = __ballot_sync(0xffffffffu, act == 2);
            b.cstart[lane] = cs;
            b.cexcl[lane] = incl - cnt;
            __syncwarp();
            for (uint32_t base = 0; base < T; base += 32) {
                if (m > NB_CAP - 32) {
                    sort_exact<DIM>(a, b, m, i);
                    m = min(m, c.k_max);
                    if (m == c.k_max) {
                        cut = key_d2(b.key[m - 1]) * (1.0f + TOL_T);
                        cutq = sqrtf(cut) * inv * (1.0f + 2e-5f) + 1.0f;
                    }
                }
                uint32_t t = base + lane;
                bool in = false, keep = false;
                float d2f = 0.0f;
                uint32_t j = 0;
                if (t < T) {
                    int lo = 0, hi = 31;       // the last cell with cexcl <= t
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (b.cexcl[mid] <= t) lo = mid; else hi = mid - 1;
                    }
                    j = b.cstart[lo] + (t - b.cexcl[lo]);
                    bool count_only = (co >> lo) & 1u;
                    if ((int64_t)j != i) {
                        float4 ph, pl;
                        ldg256(a.pos4 + 2 * (int64_t)j, ph, pl);
                        float hj[3] = {ph.x, ph.y, ph.z}, lj[3] = {pl.x, pl.y, pl.z};
#pragma unroll
                        for (int k = 0; k < DIM; ++k) {
                            float dh = hj[k] - hxi[k];
                            float dl = lj[k] - lxi[k];
                            if (c.periodic[k]) {
                                if (dh > 0.5f * c.Lper_h[k]) { dh -= c.Lper_h[k]; dl -= c.Lper_l[k]; }
                                else if (dh < -0.5f * c.Lper_h[k]) { dh += c.Lper_h[k]; dl += c.Lper_l[k]; }
                            }
                            float d = dh + dl;
                            d2f = fmaf(d, d, d2f);
                        }
                        if (d2f <= R2f * (1.0f - TOL_R)) in = true;
                        else if (d2f <= R2f * (1.0f + TOL_R))
                            in = inside64(c, DIM, exact_d2<DIM>(a, i, j), __dmul_rn(a.sm[i], a.sV[i]));
                        keep = in && !count_only && d2f <= cut;
                    }
                }
                scanned_in += __popc(__ballot_sync(0xffffffffu, in));
                unsigned km = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    int pos = m + __popc(km & lt);
                    b.key[pos] = ((unsigned long long)__float_as_uint(d2f) << 32) | a.sid[j];
                    b.j[pos] = j;
                }
                m += __popc(km);
                __syncwarp();
            }
            __syncwarp();
        }
        cur ^= 1;
        ncur = nnext;
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) whole += __shfl_xor_sync(0xffffffffu, whole, o);
    uint32_t inside_total = whole + scanned_in;
    sort_exact<DIM>(a, b, m, i);
    int cnt = min(m, c.k_max);
    for (int e = lane; e < cnt; e += 32) a.idx[i * (int64_t)c.k_max + e] = b.j[e];
    if (lane == 0) {
        a.count[i] = (uint32_t)cnt;
        a.total[i] = min(inside_total, total_cap);
        // the exact squared distance to the nearest entry (the CFL step's ell^2)
        a.d2min[i] = cnt > 0 ? exact_d2<DIM>(a, i, b.j[0]) : INFINITY;
        if (inside_total > (uint32_t)c.k_max) atomicAdd(a.counters + C_OVERFLOW, 1ull);
        atomicMax(a.counters + C_MAXCOUNT, (unsigned long long)inside_total);
    }
    __syncwarp();
}

// Octant (quadrant in 2D) of x_j seen from x_i: bit k set when the FP64
// offset along axis k (minimum image on a periodic axis) is >= 0.  It is read
// from the split float parts of both positions (h = RN(x), l = RN(x - h)).
// Both roundings are monotonic, so h_j > h_i implies x_j > x_i, and with equal
// high parts l_j > l_i implies it too (and < likewise): the offset's sign is
// read from the first part that differs, exactly.  Where both parts are equal,
// and on periodic axes, the FP64 offset decides.  The octant query tests many
// candidates per particle, and FP64 arithmetic is scarce on this GPU.
template <int DIM>
__device__ inline int octant_split(const QueryArgs& a, int64_t i, int64_t j, const float (&hi)[3],
                                   const float (&li)[3], const float (&hj)[3], const float (&lj)[3])
{
    int o = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        bool ge;
        if (!a.c.periodic[k] && hj[k] != hi[k]) ge = hj[k] > hi[k];
        else if (!a.c.periodic[k] && lj[k] != li[k]) ge = lj[k] > li[k];
        else ge = offset64(a.c, k, a.sx[k][i], a.sx[k][j]) >= 0.0;
        if (ge) o |= 1 << k;
    }
    return o;
}

__device__ inline uint32_t warp_sum_u32(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ranks of the entries b.key/b.j[0..m) (sorted by (d2, id)) within their
// octants; entry e's rank and octant go to the lane e % 32 of chunk e / 32
// through the callback, called by all lanes once per chunk
template <int DIM, typename F>
__device__ inline void octant_ranks(const QueryArgs& a, WarpBuf& b, int m, int64_t i, const float (&hi)[3],
                                    const float (&li)[3], F&& fn)
{
    const unsigned lane = lane_id(), lt = (1u << lane) - 1u;
    uint32_t carry[1 << DIM];
#pragma unroll
    for (int q = 0; q < (1 << DIM); ++q) carry[q] = 0;
    for (int e0 = 0; e0 < m; e0 += 32) {
        const int e = e0 + (int)lane;
        const bool valid = e < m;
        int o = -1;
        if (valid) {
            const uint32_t j = b.j[e];
            float4 ph, pl;
            ldg256(a.pos4 + 2 * (int64_t)j, ph, pl);
            const float hj[3] = {ph.x, ph.y, ph.z}, lj[3] = {pl.x, pl.y, pl.z};
            o = octant_split<DIM>(a, i, j, hi, li, hj, lj);
        }
        uint32_t rank = 0;
#pragma unroll
        for (int q = 0; q < (1 << DIM); ++q) {
            const unsigned bq = __ballot_sync(0xffffffffu, o == q);
            if (o == q) rank = carry[q] + (uint32_t)__popc(bq & lt);
            carry[q] += (uint32_t)__popc(bq);
        }
        fn(e0, valid, o, rank);
    }
}

// Octant-balanced selection (LP_SELECT_OCTANT; Sec. 2.2 step 4: the top
// members of a neighbour list cover all directions).  When more than k_max
// particles lie inside the radius, the k_max kept are the first by (rank, d2,
// id), the rank of a member being its place in its octant's (d2, id) order:
// round robin over the octants, nearest first in each.  They are stored in
// (d2, id) order; with at most k_max inside, the list is the nearest-first one.
//   1. a traversal counts the members of each octant (n_o, needed up to k_max)
//      and in all (needed up to 4 k_max);
//   2. R is the smallest rank with sum_o min(n_o, R + 1) >= k_max: ranks below
//      R are all kept, rank R partly, so each octant needs only its
//      q_o = min(n_o, R + 1) nearest;
//   3. a second traversal keeps those (compacting the buffer to the quotas
//      whenever it fills and after each level of cells), and the final sorted
//      buffer gives the selection.
// Both traversals start at the start cells and split a cell with more than
// DESC_MIN particles into its children (processed as the next level), so
// that a dense region is visited only where it matters: the counting pass
// counts a cell that lies inside the radius and inside one octant without
// scanning it, and skips cells whose octants are all counted out once the
// total reached 4 k_max; the collecting pass skips cells farther than the
// current q_o-th member of each octant they meet.  A cell is in one octant
// when its box lies, with the quantisation margin, on one side of the
// particle along every axis.  Membership and order are decided as in
// query_one (float split distances, FP64 inside the rounding bands), octants
// on the FP64 offsets.
template <int DIM>
__device__ void query_one_octant(const QueryArgs& a, WarpBuf& b, int64_t i)
{
    const unsigned lane = lane_id(), lt = (1u << lane) - 1u;
    const DevCfg& c = a.c;
    const int mb = c.mbits;
    QueryStart st;
    query_start<DIM>(a, b, i, st);
    const Grid& g = a.g[st.sim];
    const uint32_t kmax = (uint32_t)c.k_max;
    constexpr int NO = 1 << DIM;
    constexpr unsigned ALL_O = (1u << NO) - 1u;
    // octants with bit k set (offset along k >= 0), per axis
    constexpr unsigned AXIS_SET[3] = {DIM == 3 ? 0xAAu : (DIM == 2 ? 0xAu : 0x2u), DIM == 3 ? 0xCCu : 0xCu, 0xF0u};
    enum { SKIP = 0, SCAN = 1, SPLIT = 2, WHOLE = 3 };
    // One traversal from the start cells.  pre() runs (all lanes) before each
    // batch of 32 cells; cls(dmin, dmax, touched, splittable) classifies a
    // non-empty cell within reach (one lane, no warp operations); whole(w,
    // touched, cn) is called by all lanes (w: this lane's cell is counted
    // whole); fn(in, j, d2f, octant) by all lanes for each scanned candidate;
    // level_end() by all lanes after each level.
    auto traverse = [&](auto&& pre, auto&& cls, auto&& whole, auto&& fn, auto&& level_end) {
        query_start<DIM>(a, b, i, st);
        int cur = 0, ncur = st.ncells;
        while (ncur > 0) {
            int nnext = 0;
            for (int base0 = 0; base0 < ncur; base0 += 32) {
                pre();
                const int e = base0 + (int)lane;
                uint32_t cs = 0, cn = 0;
                int act = SKIP, l = 0, wv[3] = {0, 0, 0}, shv[3] = {0, 0, 0};
                unsigned touched = 0u;
                if (e < ncur) {
                    unpack_cell(b.front[cur][e], l, wv, shv);
                    const float size = ldexpf(1.0f, mb - l), period = ldexpf(1.0f, mb);
                    uint32_t q[3] = {0u, 0u, 0u};
                    float dmin2 = 0.0f, dmax2 = 0.0f;
                    touched = ALL_O;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        q[k] = (uint32_t)wv[k];
                        const float lo = (float)wv[k] * size + (float)shv[k] * period, hi = lo + size;
                        const float dn = fmaxf(0.0f, fmaxf(lo - st.tq[k], st.tq[k] - hi));
                        const float df = fmaxf(st.tq[k] - lo, hi - st.tq[k]);
                        dmin2 += dn * dn;
                        dmax2 += df * df;
                        if (lo > st.tq[k] + 2.0f) touched &= AXIS_SET[k];          // every offset > 0
                        else if (hi < st.tq[k] - 2.0f) touched &= ~AXIS_SET[k];    // every offset < 0
                    }
                    const float dmin = sqrtf(dmin2), dmax = sqrtf(dmax2);
                    if (dmin < st.Rout) {
                        const uint64_t code = (st.sim << (DIM * l)) | morton<DIM>(q);
                        const unsigned long long ent = a.cells[a.level_off[l] + (int64_t)code];
                        cs = (uint32_t)ent;
                        const uint32_t ce = (uint32_t)(ent >> 32);
                        cn = ce > cs ? ce - cs : 0;
                        if (cn > 0) act = cls(dmin, dmax, touched, cn > DESC_MIN && l < g.lmax);
                    }
                }
                // split cells: children to the next level while there is room,
                // scanned otherwise
                constexpr int nchild = 1 << DIM;
                const unsigned sm = __ballot_sync(0xffffffffu, act == SPLIT);
                const int room = (FCAP - nnext) / nchild;
                if (act == SPLIT) {
                    const int rank = __popc(sm & lt);
                    if (rank < room) {
                        const int pos = nnext + rank * nchild;
                        for (int ch = 0; ch < nchild; ++ch) {
                            const int cw[3] = {2 * wv[0] + (ch & 1), DIM > 1 ? 2 * wv[1] + ((ch >> 1) & 1) : 0,
                                               DIM > 2 ? 2 * wv[2] + ((ch >> 2) & 1) : 0};
                            b.front[cur ^ 1][pos + ch] = pack_cell(l + 1, cw, shv);
                        }
                        act = SKIP;
                    } else {
                        act = SCAN;
                    }
                }
                nnext += min(__popc(sm), max(room, 0)) * nchild;
                whole(act == WHOLE, touched, cn);
                // scanned cells: their candidates over the lanes
                const uint32_t cnt = act == SCAN ? cn : 0u;
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((int)lane >= o) incl += v;
                }
                const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
                b.cstart[lane] = cs;
                b.cexcl[lane] = incl - cnt;
                __syncwarp();
                for (uint32_t base = 0; base < T; base += 32) {
                    const uint32_t t = base + lane;
                    bool in = false;
                    float d2f = 0.0f;
                    uint32_t j = 0;
                    int oct = 0;                   // octant of an in-radius candidate
                    if (t < T) {
                        int lo = 0, hi = 31;       // the last cell with cexcl <= t
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (b.cexcl[mid] <= t) lo = mid; else hi = mid - 1;
                        }
                        j = b.cstart[lo] + (t - b.cexcl[lo]);
                        if ((int64_t)j != i) {
                            float4 ph, pl;
                            ldg256(a.pos4 + 2 * (int64_t)j, ph, pl);
                            const float hj[3] = {ph.x, ph.y, ph.z}, lj[3] = {pl.x, pl.y, pl.z};
#pragma unroll
                            for (int k = 0; k < DIM; ++k) {
                                float dh = hj[k] - st.hxi[k];
                                float dl = lj[k] - st.lxi[k];
                                if (c.periodic[k]) {
                                    if (dh > 0.5f * c.Lper_h[k]) { dh -= c.Lper_h[k]; dl -= c.Lper_l[k]; }
                                    else if (dh < -0.5f * c.Lper_h[k]) { dh += c.Lper_h[k]; dl += c.Lper_l[k]; }
                                }
                                const float d = dh + dl;
                                d2f = fmaf(d, d, d2f);
                            }
                            if (d2f <= st.R2f * (1.0f - TOL_R)) in = true;
                            else if (d2f <= st.R2f * (1.0f + TOL_R))
                                in = inside64(c, DIM, exact_d2<DIM>(a, i, j), __dmul_rn(a.sm[i], a.sV[i]));
                            if (in) oct = octant_split<DIM>(a, i, j, st.hxi, st.lxi, hj, lj);
                        }
                    }
                    fn(in, j, d2f, oct);
                }
                __syncwarp();
            }
            level_end();
            cur ^= 1;
            ncur = nnext;
            __syncwarp();
        }
    };
    // ---- 1. members per octant (lane o holds octant o's count) and in all
    uint32_t cnt_o = 0, total = 0;
    unsigned sat = 0u;             // octants counted up to k_max (warp-uniform)
    bool total_done = false;       // total >= 4 k_max
    traverse(
        [&]() {
            sat = __ballot_sync(0xffffffffu, (int)lane < NO && cnt_o >= kmax) & ALL_O;
            total_done = total >= 4u * kmax;
        },
        [&](float dmin, float dmax, unsigned touched, bool splittable) -> int {
            if (total_done && (touched & ~sat) == 0u) return SKIP;
            if (__popc(touched) == 1 && dmax <= st.Rin) return WHOLE;
            return splittable ? SPLIT : SCAN;
        },
        [&](bool w, unsigned touched, uint32_t cn) {
            total += __reduce_add_sync(0xffffffffu, w ? cn : 0u);
#pragma unroll
            for (int q = 0; q < NO; ++q) {
                const uint32_t add = __reduce_add_sync(0xffffffffu, (w && touched == (1u << q)) ? cn : 0u);
                if ((int)lane == q) cnt_o += add;
            }
        },
        [&](bool in, uint32_t, float, int oct) {
            const int o = in ? oct : -1;
            total += (uint32_t)__popc(__ballot_sync(0xffffffffu, in));
#pragma unroll
            for (int q = 0; q < NO; ++q) {
                const unsigned bq = __ballot_sync(0xffffffffu, o == q);
                if ((int)lane == q) cnt_o += (uint32_t)__popc(bq);
            }
        },
        [&]() {});
    // ---- 2. the rank threshold and the quotas
    const uint32_t n_o = (int)lane < NO ? min(cnt_o, kmax) : 0u;
    uint32_t R = kmax, q_o = n_o, rem = 0;
    if (total > kmax) {
        R = 0;
        while (warp_sum_u32(min(n_o, R + 1)) < kmax) ++R;    // ends at R <= kmax - 1
        q_o = min(n_o, R + 1);
        rem = kmax - warp_sum_u32(min(n_o, R));              // rank-R members kept
    }
    const unsigned zero_q = __ballot_sync(0xffffffffu, (int)lane < NO && q_o == 0u) & ALL_O;
    // ---- 3. the q_o nearest of each octant
    int m = 0;
    unsigned full = 0u;            // octants holding q_o members (warp-uniform)
    float cut_o = INFINITY;        // lane o: float d2 bound of octant o's members, when full
    auto compact = [&]() {
        sort_exact<DIM>(a, b, m, i);
        int w = 0;
        unsigned nfull = 0u;
        float ncut = INFINITY;
        octant_ranks<DIM>(a, b, m, i, st.hxi, st.lxi, [&](int e0, bool valid, int o, uint32_t rank) {
            const int e = e0 + (int)lane;
            // every lane takes part in the shuffle (no short circuit before it)
            const uint32_t qo = __shfl_sync(0xffffffffu, q_o, o & 7);
            const bool keep = valid && rank < qo;
            const unsigned long long kk = valid ? b.key[e] : 0ull;
            const uint32_t jj = valid ? b.j[e] : 0u;
            // the last member an octant keeps sets its bound
            const bool last = keep && rank + 1u == qo;
#pragma unroll
            for (int q = 0; q < NO; ++q) {
                const unsigned bl = __ballot_sync(0xffffffffu, last && o == q);
                const float d = __shfl_sync(0xffffffffu, key_d2(kk), bl ? __ffs(bl) - 1 : 0);
                if (bl) {
                    nfull |= 1u << q;
                    if ((int)lane == q) ncut = d * (1.0f + TOL_T);
                }
            }
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) {
                const int pos = w + __popc(km & lt);
                b.key[pos] = kk;
                b.j[pos] = jj;
            }
            w += __popc(km);
            __syncwarp();
        });
        m = w;
        full = nfull;
        cut_o = ncut;
    };
    float cutq[NO];                // per octant, quantised units (warp-uniform)
    traverse(
        [&]() {
#pragma unroll
            for (int q = 0; q < NO; ++q) {
                const float cd = __shfl_sync(0xffffffffu, cut_o, q);
                cutq[q] = ((full >> q) & 1u) ? sqrtf(cd) * st.inv * (1.0f + 2e-5f) + 1.0f : INFINITY;
            }
        },
        [&](float dmin, float, unsigned touched, bool splittable) -> int {
            bool need = false;
#pragma unroll
            for (int q = 0; q < NO; ++q)
                if (((touched & ~zero_q) >> q) & 1u) need |= dmin <= cutq[q];
            if (!need) return SKIP;
            return splittable ? SPLIT : SCAN;
        },
        [&](bool, unsigned, uint32_t) {},
        [&](bool in, uint32_t j, float d2f, int oct) {
            const int o = in ? oct : 0;
            const uint32_t qo = __shfl_sync(0xffffffffu, q_o, o);   // every lane, then the test
            const float co = __shfl_sync(0xffffffffu, cut_o, o);
            const bool keep = in && qo > 0u && d2f <= co;
            if (m > NB_CAP - 32) compact();                      // warp-uniform
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = m + __popc(km & lt);
                b.key[pos] = ((unsigned long long)__float_as_uint(d2f) << 32) | a.sid[j];
                b.j[pos] = j;
            }
            m += __popc(km);
            __syncwarp();
        },
        [&]() {
            if (m > 0) compact();          // bounds for the next level
        });
    compact();                                               // m <= sum_o q_o, sorted
    // ---- the selection, in (d2, id) order: ranks below R, and the first rem of rank R
    int w = 0;
    uint32_t taken_r = 0;
    octant_ranks<DIM>(a, b, m, i, st.hxi, st.lxi, [&](int e0, bool valid, int, uint32_t rank) {
        const int e = e0 + (int)lane;
        const bool atR = valid && rank == R;
        const unsigned bR = __ballot_sync(0xffffffffu, atR);
        const bool keep = valid && (rank < R || (atR && taken_r + (uint32_t)__popc(bR & lt) < rem));
        taken_r += (uint32_t)__popc(bR);
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) a.idx[i * (int64_t)kmax + w + __popc(km & lt)] = b.j[e];
        w += __popc(km);
    });
    if (lane == 0) {
        a.count[i] = (uint32_t)w;
        a.total[i] = min(total, 4u * kmax);
        // the nearest member is kept (rank 0, nearest of the rank-0 members)
        a.d2min[i] = w > 0 ? exact_d2<DIM>(a, i, b.j[0]) : INFINITY;
        if (total > kmax) atomicAdd(a.counters + C_OVERFLOW, 1ull);
        atomicMax(a.counters + C_MAXCOUNT, (unsigned long long)total);
    }
    __syncwarp();
}

// warp per particle: every particle, or the particles of a list
template <int DIM>
__global__ void __launch_bounds__(NB_WARPS * 32) k_query(QueryArgs a)
{
    __shared__ WarpBuf bufs[NB_WARPS];
    const int w = threadIdx.x >> 5;
    WarpBuf& b = bufs[w];
    if (a.list) {
        const unsigned long long len = *a.list_len;
        for (unsigned long long t = (unsigned long long)blockIdx.x * NB_WARPS + w; t < len;
             t += (unsigned long long)gridDim.x * NB_WARPS)
            query_one<DIM>(a, b, (int64_t)a.list[t]);
    } else {
        const int64_t i = (int64_t)blockIdx.x * NB_WARPS + w;
        if (i < a.n) query_one<DIM>(a, b, i);
    }
}

// the octant-balanced selection (LP_SELECT_OCTANT), warp per particle: every
// particle, or the particles of a list.  A kernel of its own so that the
// nearest-first kernel keeps its register budget.
template <int DIM>
__global__ void __launch_bounds__(NB_WARPS * 32) k_query_octant(QueryArgs a)
{
    __shared__ WarpBuf bufs[NB_WARPS];
    const int w = threadIdx.x >> 5;
    WarpBuf& b = bufs[w];
    if (a.list) {
        const unsigned long long len = *a.list_len;
        for (unsigned long long t = (unsigned long long)blockIdx.x * NB_WARPS + w; t < len;
             t += (unsigned long long)gridDim.x * NB_WARPS)
            query_one_octant<DIM>(a, b, (int64_t)a.list[t]);
    } else {
        const int64_t i = (int64_t)blockIdx.x * NB_WARPS + w;
        if (i < a.n) query_one_octant<DIM>(a, b, i);
    }
}

// ---------------------------------------------------------------------------
// Tile kernel: one warp per 32 consecutive particles in key order.  The tile
// is cut into groups where consecutive particles lie more than TQ_GAP radii
// apart (jumps of the Morton curve) or belong to different simulations; each
// group is a compact region of space.  For a group:
//   1. the cells of one level (edge >= half the group's largest radius) within
//      reach of the group's bounding box are classified lane-parallel and the
//      non-empty ones compacted;
//   2. their particles are staged 32 at a time in shared memory as positions
//      relative to the group's first particle, and every lane tests each staged
//      candidate against its own particle with a margin that covers the
//      rounding of the relative coordinates (a prefilter: no neighbour is
//      lost), keeping the index of each hit in its own column of a shared list;
//   3. per particle, the warp recomputes the hits' distances exactly as the
//      per-particle kernel does (float hi/lo offsets; FP64 inside the rounding
//      band of the radius), sorts (float d2, index) with a register bitonic
//      network, re-orders near-tie runs by (FP64 d2, id) and writes the row.
// Particles with more than TQ_CAP hits, and groups whose region spans too many
// cells or candidates, are left to the per-particle kernel.
// ---------------------------------------------------------------------------
constexpr int TQ_WARPS = 4;
constexpr int TQ_CAP = 64;            // prefilter hits a lane keeps (two sort keys per lane)
constexpr int TQ_PAD = 33;            // column stride: a row read across lanes is conflict-free
constexpr int TQ_CELLS_MAX = 4096;    // cells a group's region may span
constexpr uint32_t TQ_CAND_MAX = 2048;   // candidates a group may test (fastest of 2048, 4096, 8192 on the gas cloud)
constexpr int TQ_KC = 256;            // non-empty cells a group may keep
constexpr float TQ_GAP = 2.0f;        // in radii
constexpr int TQ_SPLIT_MIN = 4;       // smallest half a too-large group is split into

struct TileBuf {
    uint32_t kj[TQ_CAP][TQ_PAD];      // prefilter hits, one column per lane
    unsigned long long kc[TQ_KC];     // kept cells: start | count << 32
    alignas(16) float cx[32];         // staged candidates: position relative to the group's origin,
    alignas(16) float cy[32];         // read four at a time by the prefilter
    alignas(16) float cz[32];
    uint32_t cj[32];                  // and index
};
static_assert(sizeof(TileBuf) % 16 == 0, "per-warp buffers keep the 16-byte alignment of cx, cy, cz");

__device__ inline float warp_minf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ inline float warp_maxf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ inline void list_append(const QueryArgs& a, bool pred, uint32_t v)
{
    unsigned m = __ballot_sync(0xffffffffu, pred);
    if (!m) return;
    unsigned lane = lane_id();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.fb_len, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (pred) a.fb_list[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// own position (hi, lo), quantised position, radius terms of particle i
template <int DIM>
struct TileLane {
    float hx[3], lx[3], tq[3];
    float Rf, R2f, Rq, Rout;
};

template <int DIM, bool PER>
__device__ inline void tile_lane(const QueryArgs& a, const Grid& g, int64_t i, TileLane<DIM>& t)
{
    const DevCfg& c = a.c;
    const float inv = g.inv_f;
    const float4 ph = a.pos4[2 * i], pl = a.pos4[2 * i + 1];
    t.hx[0] = ph.x; t.hx[1] = ph.y; t.hx[2] = ph.z;
    t.lx[0] = pl.x; t.lx[1] = pl.y; t.lx[2] = pl.z;
#pragma unroll
    for (int k = 0; k < 3; ++k) t.tq[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) t.tq[k] = ((t.hx[k] - g.lo_h[k]) + (t.lx[k] - g.lo_l[k])) * inv;
    const float Rf = ph.w;                           // query_radius_ff, written by the gather
    t.Rf = Rf;
    t.R2f = (c.radius_mode == LP_RADIUS_FIXED) ? c.radius2_f : Rf * Rf;
    t.Rq = Rf * (1.0f + 1e-5f) * inv;
    t.Rout = Rf * inv * (1.0f + 2e-5f) + 2.0f;
}

// float offset x_j - x_i along k from hi/lo parts (minimum image): the
// per-particle kernel's arithmetic, so both give the same float d2
template <bool PER>
__device__ inline float split_offset(const DevCfg& c, int k, float hj, float lj, float hi, float li)
{
    float dh = hj - hi;
    float dl = lj - li;
    if (PER && c.periodic[k]) {
        if (dh > 0.5f * c.Lper_h[k]) { dh -= c.Lper_h[k]; dl -= c.Lper_l[k]; }
        else if (dh < -0.5f * c.Lper_h[k]) { dh += c.Lper_h[k]; dl += c.Lper_l[k]; }
    }
    return dh + dl;
}

// ascending sort of P = 32 * W distinct 32-bit keys, element e = lane + 32 s
// held by lane in key[s].  Bitonic merges in the form whose compare-exchanges
// all point the same way: the first stage of the merge of two sorted runs of
// k/2 compares each element with its mirror in the k-block (partner e ^ (k-1)),
// the later stages with e ^ jj; the lower element takes the minimum.  So a
// lane's direction depends on one lane bit per stage (five predicates in all)
// instead of two.
template <int W>
__device__ inline void bitonic_keys(uint32_t (&key)[2])
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            const int mask = jj == (k >> 1) ? k - 1 : jj;
            const bool low = (lane & (unsigned)jj) == 0u;
#pragma unroll
            for (int s = 0; s < W; ++s) {
                const uint32_t pk = __shfl_xor_sync(0xffffffffu, key[s], mask);
                key[s] = low ? min(key[s], pk) : max(key[s], pk);
            }
        }
    }
    if (W == 2) {
        // the merge of the two sorted registers: mirror stage across them
        // (e ^ 63 is lane ^ 31 of the other register), then within each
        const uint32_t p0 = __shfl_xor_sync(0xffffffffu, key[1], 31);
        const uint32_t p1 = __shfl_xor_sync(0xffffffffu, key[0], 31);
        key[0] = min(key[0], p0);
        key[1] = max(key[1], p1);
#pragma unroll
        for (int jj = 16; jj > 0; jj >>= 1) {
            const bool low = (lane & (unsigned)jj) == 0u;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint32_t pk = __shfl_xor_sync(0xffffffffu, key[s], jj);
                key[s] = low ? min(key[s], pk) : max(key[s], pk);
            }
        }
    }
}

// one group of lanes of the tile (act); all 32 lanes take part.  false: the
// group's region spans too many cells or candidates, nothing was written (the
// caller splits the group or hands its particles to the per-particle kernel)
template <int DIM, bool PER>
__device__ bool tile_group(const QueryArgs& a, TileBuf& b, int64_t i, bool act, uint64_t sim,
                           const TileLane<DIM>& me)
{
    const unsigned lane = lane_id();
    const DevCfg& c = a.c;
    const int mb = c.mbits;
    const Grid& g = a.g[sim];
    if (PER && act) {
#pragma unroll
        for (int k = 0; k < DIM; ++k)
            if (c.periodic[k] && 2.0f * me.Rq >= ldexpf(1.0f, mb))
                atomicOr(reinterpret_cast<unsigned int*>(a.counters + C_STATUS), ST_ARG);
    }
    // bounding box of the group and its largest radius (quantised units)
    float bmin[3] = {0.0f, 0.0f, 0.0f}, bmax[3] = {0.0f, 0.0f, 0.0f};
    float ext = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        bmin[k] = warp_minf(act ? me.tq[k] : INFINITY);
        bmax[k] = warp_maxf(act ? me.tq[k] : -INFINITY);
        ext = fmaxf(ext, bmax[k] - bmin[k]);
    }
    const float Rqm = warp_maxf(act ? me.Rq : 0.0f);
    const float Routm = warp_maxf(act ? me.Rout : 0.0f);
    // finest table level whose cell edge 2^(mb - l) is at least half the radius
    const float Rh = 0.5f * Rqm;
    int l0 = g.lmax;
    while (l0 > g.lmin && ldexpf(1.0f, mb - l0) < Rh) --l0;
    const float size = ldexpf(1.0f, mb - l0);
    const float scale = ldexpf(1.0f, l0 - mb);
    const float period = ldexpf(1.0f, mb);
    const int naxis = 1 << l0;
    int clo[3] = {0, 0, 0}, nc[3] = {1, 1, 1};
    bool full[3] = {false, false, false};   // the region wraps a whole period on this axis
    long long ncells = 1;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        float lo_f = fmaxf(-16777216.0f, fminf(16777216.0f, (bmin[k] - Rqm - 2.0f) * scale));
        float hi_f = fmaxf(-16777216.0f, fminf(16777216.0f, (bmax[k] + Rqm + 2.0f) * scale));
        int a0 = (int)floorf(lo_f), a1 = (int)floorf(hi_f);
        if (!PER || !c.periodic[k]) {
            a0 = max(0, min(a0, naxis - 1));
            a1 = max(0, min(a1, naxis - 1));
        } else if (a1 - a0 + 1 > naxis) {
            // each cell once, at one of its images -- not necessarily the one
            // nearest the box, so this axis takes no part in the pruning
            a1 = a0 + naxis - 1;
            full[k] = true;
        }
        clo[k] = a0;
        nc[k] = a1 - a0 + 1;
        ncells = nc[k] < 1 ? 0 : ncells * nc[k];
    }
    if (ncells > TQ_CELLS_MAX) return false;     // a scattered group
    const int nct = (int)ncells;
    float rnc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) rnc[k] = 1.0f / (float)nc[k];
    // one lane per cell: the key-order range of cell e if it is within reach of the box
    auto cell_range = [&](int e, uint32_t& cs, uint32_t& cn) {
        cs = 0;
        cn = 0;
        if (e >= nct) return;
        int u = e;
        uint32_t q[3] = {0u, 0u, 0u};
        float dmin2 = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            int qt = (int)((float)u * rnc[k]);            // u / nc[k], corrected below
            int rm = u - qt * nc[k];
            if (rm < 0) { --qt; rm += nc[k]; } else if (rm >= nc[k]) { ++qt; rm -= nc[k]; }
            const int v = clo[k] + rm;
            u = qt;
            const int wr = v & (naxis - 1);
            const int sh = (v - wr) >> l0;          // periodic image (0 on other axes)
            const float lo = (float)wr * size + (float)sh * period;
            const float dn = full[k] ? 0.0f : fmaxf(0.0f, fmaxf(lo - bmax[k], bmin[k] - (lo + size)));
            dmin2 += dn * dn;
            q[k] = (uint32_t)wr;
        }
        if (sqrtf(dmin2) < Routm) {
            const uint64_t code = (sim << (DIM * l0)) | morton<DIM>(q);
            const unsigned long long ent = a.cells[a.level_off[l0] + (int64_t)code];
            cs = (uint32_t)ent;
            const uint32_t ce = (uint32_t)(ent >> 32);
            cn = ce > cs ? ce - cs : 0;
        }
    };
    // ---- 1. the group's candidate count (a dense region under a wide group is
    // cheaper per particle) and, while they fit, its non-empty cells compacted
    const unsigned lt = (1u << lane) - 1u;
    int nk = 0;                       // compacted cells in b.kc
    bool spill = false;               // more non-empty cells than b.kc holds
    {
        uint32_t ncand = 0;
        for (int base0 = 0; base0 < nct && ncand <= TQ_CAND_MAX; base0 += 32) {
            uint32_t cs, cn;
            cell_range(base0 + (int)lane, cs, cn);
            ncand += __reduce_add_sync(0xffffffffu, cn);
            const unsigned km = __ballot_sync(0xffffffffu, cn > 0);
            if (!spill && nk + __popc(km) > TQ_KC) spill = true;
            if (!spill) {
                if (cn > 0) b.kc[nk + __popc(km & lt)] = (unsigned long long)cs | ((unsigned long long)cn << 32);
                nk += __popc(km);
            }
        }
        if (ncand > TQ_CAND_MAX) return false;
    }
    __syncwarp();

    // ---- 2. prefilter: candidates relative to the group's first particle
    const int lead = __ffs(__ballot_sync(0xffffffffu, act)) - 1;
    float oh[3], ol[3], ri[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        oh[k] = __shfl_sync(0xffffffffu, me.hx[k], lead);
        ol[k] = __shfl_sync(0xffffffffu, me.lx[k], lead);
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) ri[k] = split_offset<PER>(c, k, me.hx[k], me.lx[k], oh[k], ol[k]);
    // rounding margin of the relative coordinates: each is within 2^-23 |r| of
    // the split value and |r| <= E / sqrt(dim) per axis, so the prefilter's d2
    // is within 2^-24 (7 d2 + 8 E |d|) of the true one; a true neighbour has
    // d2 <= R^2 <= R2f (1 + TOL_R), hence d2_prefilter <= thr
    float E = (ext + Rqm + size + 4.0f) / g.inv_f;
    if (PER) E = fmaxf(E, g.L_f);
    E *= DIM == 3 ? 1.7320508f : (DIM == 2 ? 1.4142136f : 1.0f);
    const float thr = me.R2f * (1.0f + TOL_R) + ldexpf(me.R2f + 4.0f * E * me.Rf, -20);
    float halfL[3], Lh[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { Lh[k] = c.Lper_h[k]; halfL[k] = 0.5f * c.Lper_h[k]; }
    // the group's box in the relative coordinates, and a bound on a candidate's
    // squared distance to it above every lane's threshold (the distance to the
    // box is at most the distance to any lane's particle; the margin covers the
    // rounding of both): candidates beyond it are not staged (open domains;
    // the minimum image of a periodic axis has no such box)
    float rlo[3] = {0.0f, 0.0f, 0.0f}, rhi[3] = {0.0f, 0.0f, 0.0f};
    float thr_box = INFINITY;
    if (!PER) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            rlo[k] = warp_minf(act ? ri[k] : INFINITY);
            rhi[k] = warp_maxf(act ? ri[k] : -INFINITY);
        }
        const float thm = warp_maxf(act ? thr : 0.0f);
        const float Rm = warp_maxf(act ? me.Rf : 0.0f);
        thr_box = thm + ldexpf(thm + 4.0f * E * Rm, -18);
    }
    uint32_t cnt = 0;                 // prefilter hits of this lane
    // candidates of the compacted cells b.kc[0..nk), 32 cells at a time
    auto scan_kept = [&](int nk) {
        for (int c0 = 0; c0 < nk; c0 += 32) {
            uint32_t cs = 0, cn = 0;
            if (c0 + (int)lane < nk) {
                const unsigned long long ent = b.kc[c0 + lane];
                cs = (uint32_t)ent;
                cn = (uint32_t)(ent >> 32);
            }
            uint32_t incl = cn;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += v;
            }
            const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t cex = incl - cn;       // this lane's cell: its first slot among the T
            for (uint32_t base = 0; base < T; base += 32) {
                const uint32_t t = base + lane;
                // slot t lies in the last non-empty cell whose first slot is <= t (first
                // slots of non-empty cells strictly increase): count the cells starting
                // before this batch, and those starting in it up to t by a bit mask
                const bool here = cn > 0 && cex >= base && cex - base < 32u;
                const uint32_t starts = __reduce_or_sync(0xffffffffu, here ? 1u << (cex - base) : 0u);
                const int before = __popc(__ballot_sync(0xffffffffu, cn > 0 && cex < base));
                const int cl = before - 1 + __popc(starts & (0xffffffffu >> (31u - lane)));   // in [0, 31]
                const uint32_t cs_t = __shfl_sync(0xffffffffu, cs, cl);
                const uint32_t cex_t = __shfl_sync(0xffffffffu, cex, cl);
                bool keep = false;
                float p[3] = {0.0f, 0.0f, 0.0f};
                uint32_t j = 0;
                if (t < T) {
                    j = cs_t + (t - cex_t);
                    float4 ph, pl;
                    ldg256(a.pos4 + 2 * (int64_t)j, ph, pl);
                    p[0] = split_offset<PER>(c, 0, ph.x, pl.x, oh[0], ol[0]);
                    if (DIM > 1) p[1] = split_offset<PER>(c, 1, ph.y, pl.y, oh[1], ol[1]);
                    if (DIM > 2) p[2] = split_offset<PER>(c, 2, ph.z, pl.z, oh[2], ol[2]);
                    float d2b = 0.0f;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        const float dk = fmaxf(0.0f, fmaxf(rlo[k] - p[k], p[k] - rhi[k]));
                        d2b = fmaf(dk, dk, d2b);
                    }
                    keep = PER || d2b <= thr_box;
                }
                // the kept candidates, compacted
                const unsigned km = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int sl = __popc(km & lt);
                    b.cx[sl] = p[0];
                    b.cy[sl] = p[1];
                    b.cz[sl] = p[2];
                    b.cj[sl] = j;
                }
                __syncwarp();
                const int nb = __popc(km);
                if (act && nb > 0) {
                    // bit q: staged candidate q passes the prefilter
                    uint32_t hits = 0;
                    if (PER) {
#pragma unroll 4
                        for (int qq = 0; qq < nb; ++qq) {
                            float d[3] = {b.cx[qq] - ri[0], b.cy[qq] - ri[1], b.cz[qq] - ri[2]};
#pragma unroll
                            for (int k = 0; k < DIM; ++k)
                                if (c.periodic[k]) {
                                    if (d[k] > halfL[k]) d[k] -= Lh[k];
                                    else if (d[k] < -halfL[k]) d[k] += Lh[k];
                                }
                            float d2 = d[0] * d[0];
                            if (DIM > 1) d2 = fmaf(d[1], d[1], d2);
                            if (DIM > 2) d2 = fmaf(d[2], d[2], d2);
                            hits |= (d2 <= thr ? 1u : 0u) << qq;
                        }
                    } else {
                        // four candidates per iteration, two per packed FP32 instruction
                        // (per component the same rounding as the scalar form).  The
                        // test d2 <= thr is the sign bit of RN(thr - d2), which is clear
                        // exactly when d2 <= thr (a NaN d2, from non-finite positions, may
                        // only add a hit that the exact pass rejects); a funnel shift
                        // appends it to miss, the earlier candidate in the higher bit
                        const float2 nx = make_float2(-ri[0], -ri[0]);
                        const float2 ny = make_float2(-ri[1], -ri[1]);
                        const float2 nz = make_float2(-ri[2], -ri[2]);
                        const float2 t2 = make_float2(thr, thr);
                        const float2 m1 = make_float2(-1.0f, -1.0f);
                        uint32_t miss = 0;
#pragma unroll 1
                        for (int qq = 0; qq < nb; qq += 4) {
                            const float4 X = *reinterpret_cast<const float4*>(&b.cx[qq]);
                            const float2 dxa = __fadd2_rn(make_float2(X.x, X.y), nx);
                            const float2 dxb = __fadd2_rn(make_float2(X.z, X.w), nx);
                            float2 d2a = __fmul2_rn(dxa, dxa);
                            float2 d2b = __fmul2_rn(dxb, dxb);
                            if (DIM > 1) {
                                const float4 Y = *reinterpret_cast<const float4*>(&b.cy[qq]);
                                const float2 dya = __fadd2_rn(make_float2(Y.x, Y.y), ny);
                                const float2 dyb = __fadd2_rn(make_float2(Y.z, Y.w), ny);
                                d2a = __ffma2_rn(dya, dya, d2a);
                                d2b = __ffma2_rn(dyb, dyb, d2b);
                            }
                            if (DIM > 2) {
                                const float4 Z = *reinterpret_cast<const float4*>(&b.cz[qq]);
                                const float2 dza = __fadd2_rn(make_float2(Z.x, Z.y), nz);
                                const float2 dzb = __fadd2_rn(make_float2(Z.z, Z.w), nz);
                                d2a = __ffma2_rn(dza, dza, d2a);
                                d2b = __ffma2_rn(dzb, dzb, d2b);
                            }
                            const float2 sa = __ffma2_rn(d2a, m1, t2);
                            const float2 sb = __ffma2_rn(d2b, m1, t2);
                            miss = __funnelshift_l(__float_as_uint(sa.x), miss, 1);
                            miss = __funnelshift_l(__float_as_uint(sa.y), miss, 1);
                            miss = __funnelshift_l(__float_as_uint(sb.x), miss, 1);
                            miss = __funnelshift_l(__float_as_uint(sb.y), miss, 1);
                        }
                        // nq candidates went in (nb rounded up to 4, at most 32): candidate
                        // q sits at bit nq - 1 - q; reversed and shifted, at bit q
                        const int nq = (nb + 3) & ~3;
                        hits = ~(__brev(miss) >> (32 - nq));
                        if (nb < 32) hits &= (1u << nb) - 1u;   // slots past nb hold no candidate
                    }
                    // append the hits to this lane's column, highest slot first (the
                    // particle itself is one of them: the exact pass below drops it,
                    // and sorts by (d2, id), so the column's order is free).  A lane
                    // whose hits overflow the column goes to the per-particle kernel,
                    // so then only the count matters
                    const uint32_t nh = (uint32_t)__popc(hits);
                    if (cnt + nh <= (uint32_t)TQ_CAP) {
                        uint32_t* col = &b.kj[cnt][lane];
                        while (hits) {
                            const int q = 31 - __clz(hits);
                            hits ^= 1u << q;
                            *col = b.cj[q];
                            col += TQ_PAD;
                        }
                    }
                    cnt += nh;
                }
                __syncwarp();
            }
        }
    };
    if (!spill) {
        scan_kept(nk);                // every kept cell is already in b.kc
    } else {
        // classify again, compacting the non-empty cells; scan whenever the
        // buffer of kept cells would overflow, and at the end
        nk = 0;
        for (int base0 = 0; base0 < nct; base0 += 32) {
            uint32_t cs, cn;
            cell_range(base0 + (int)lane, cs, cn);
            const unsigned km = __ballot_sync(0xffffffffu, cn > 0);
            if (nk + __popc(km) > TQ_KC) {
                __syncwarp();
                scan_kept(nk);
                nk = 0;
            }
            if (cn > 0) b.kc[nk + __popc(km & lt)] = (unsigned long long)cs | ((unsigned long long)cn << 32);
            nk += __popc(km);
        }
        __syncwarp();
        scan_kept(nk);
    }

    // ---- 3. per particle: exact membership, order, row
    const bool mine = act && cnt <= (uint32_t)TQ_CAP;
    list_append(a, act && !mine, (uint32_t)i);
    const uint32_t kmax = (uint32_t)c.k_max;
    uint32_t mx = 0, novf = 0;
    uint32_t near_j = 0xffffffffu;       // this lane's particle: its nearest entry (none: all ones)
    bool handed = false;                 // this lane's particle went to the per-particle kernel
    unsigned todo = __ballot_sync(0xffffffffu, mine);
    // the hits of the next particle are loaded while the current one is sorted
    uint32_t fj[2] = {0u, 0u};
    float4 fh[2], fl[2];
    auto fetch = [&](int p, int m) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int e = (int)lane + 32 * s;
            if (e < m) {
                fj[s] = b.kj[e][p];
                ldg256(a.pos4 + 2 * (int64_t)fj[s], fh[s], fl[s]);
            }
        }
    };
    int pn = todo ? __ffs(todo) - 1 : -1;
    int mn = pn >= 0 ? (int)__shfl_sync(0xffffffffu, cnt, pn) : 0;
    if (pn >= 0) fetch(pn, mn);
    while (pn >= 0) {
        const int p = pn, m = mn;
        todo &= todo - 1;
        const uint32_t cj[2] = {fj[0], fj[1]};
        const float4 ch[2] = {fh[0], fh[1]}, cl[2] = {fl[0], fl[1]};
        pn = todo ? __ffs(todo) - 1 : -1;
        mn = pn >= 0 ? (int)__shfl_sync(0xffffffffu, cnt, pn) : 0;
        if (pn >= 0) fetch(pn, mn);
        const int64_t ip = i - (int64_t)lane + p;
        float ph_[3], pl_[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ph_[k] = __shfl_sync(0xffffffffu, me.hx[k], p);
            pl_[k] = __shfl_sync(0xffffffffu, me.lx[k], p);
        }
        const float pR2 = __shfl_sync(0xffffffffu, me.R2f, p);
        // sort keys: float bits of d2 with the low 6 bits replaced by the slot,
        // so keys are distinct and ordered as the floats up to 2^-17 relative;
        // the slot brings index and exact float d2 back after the sort
        uint32_t key[2], jv[2] = {0xffffffffu, 0xffffffffu};
        key[0] = 0xffffffc0u | lane;
        key[1] = 0xffffffc0u | (lane + 32u);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int e = (int)lane + 32 * s;
            if (e < m && (int64_t)cj[s] != ip) {      // every hit but the particle itself
                const uint32_t j = cj[s];
                const float4 qh = ch[s];
                const float4 ql = cl[s];
                const float hj[3] = {qh.x, qh.y, qh.z}, lj[3] = {ql.x, ql.y, ql.z};
                float d2f = 0.0f;
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    const float dd = split_offset<PER>(c, k, hj[k], lj[k], ph_[k], pl_[k]);
                    d2f = fmaf(dd, dd, d2f);
                }
                bool in = d2f <= pR2 * (1.0f - TOL_R);
                if (!in && d2f <= pR2 * (1.0f + TOL_R))
                    in = inside64(c, DIM, exact_d2<DIM>(a, ip, j), __dmul_rn(a.sm[ip], a.sV[ip]));
                if (in) {
                    key[s] = (__float_as_uint(d2f) & ~63u) | (uint32_t)e;
                    jv[s] = j;
                }
            }
        }
        const uint32_t nin = (uint32_t)(__popc(__ballot_sync(0xffffffffu, key[0] < 0xffffffc0u)) +
                                        __popc(__ballot_sync(0xffffffffu, key[1] < 0xffffffc0u)));
        if (c.select == LP_SELECT_OCTANT && nin > kmax) {
            // the octant-balanced selection of more than k_max: the per-particle kernel
            if (lane == 0) a.fb_list[atomicAdd(a.fb_len, 1ull)] = (uint32_t)ip;
            if ((int)lane == p) handed = true;
            continue;
        }
        if (m <= 32) bitonic_keys<1>(key);
        else bitonic_keys<2>(key);
        {
            uint32_t js[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const unsigned slot = key[s] & 63u;
                const uint32_t j0 = __shfl_sync(0xffffffffu, jv[0], slot & 31u);
                const uint32_t j1 = __shfl_sync(0xffffffffu, jv[1], slot & 31u);
                js[s] = slot < 32u ? j0 : j1;
            }
            jv[0] = js[0]; jv[1] = js[1];
        }
        // runs of entries within rounding of their predecessor: exact order.
        // The test reads the keys' truncated d2 (below the float d2 by less
        // than 2^-17 relative).  A pair it leaves out is more than 2^-16 apart
        // there, so more than 2^-17 apart in float d2, far beyond the float's
        // error: its order is the exact one
        unsigned tie[2];
        {
            const float dv[2] = {__uint_as_float(key[0] & ~63u), __uint_as_float(key[1] & ~63u)};
            const float TOL_P = 1.52587890625e-05f;    // 2^-16
            const float prev0 = __shfl_up_sync(0xffffffffu, dv[0], 1);
            const float last0 = __shfl_sync(0xffffffffu, dv[0], 31);
            const float prev1 = __shfl_up_sync(0xffffffffu, dv[1], 1);
            const float pk1 = lane == 0 ? last0 : prev1;
            const bool t0 = lane > 0 && lane < nin && dv[0] <= prev0 * (1.0f + TOL_P);
            const bool t1 = lane + 32 < nin && dv[1] <= pk1 * (1.0f + TOL_P);
            tie[0] = __ballot_sync(0xffffffffu, t0);
            tie[1] = __ballot_sync(0xffffffffu, t1);
        }
        if (tie[0] | tie[1]) {
            // sorted indices to the column, runs re-sorted there by lane 0
#pragma unroll
            for (int s = 0; s < 2; ++s)
                if ((int)lane + 32 * s < (int)nin) b.kj[lane + 32 * s][p] = jv[s];
            __syncwarp();
            if (lane == 0) {
                int e = 1;
                while (e < (int)nin) {
                    if (!((tie[e >> 5] >> (e & 31)) & 1u)) { ++e; continue; }
                    const int s0 = e - 1;
                    int f = e + 1;
                    while (f < (int)nin && ((tie[f >> 5] >> (f & 31)) & 1u)) ++f;
                    for (int qq = s0 + 1; qq < f; ++qq) {
                        const uint32_t jq = b.kj[qq][p];
                        const double dq = exact_d2<DIM>(a, ip, jq);
                        const uint32_t iq = a.sid[jq];
                        int r = qq - 1;
                        while (r >= s0) {
                            const uint32_t jr = b.kj[r][p];
                            const double dr = exact_d2<DIM>(a, ip, jr);
                            if (dr < dq || (dr == dq && a.sid[jr] < iq)) break;
                            b.kj[r + 1][p] = jr;
                            --r;
                        }
                        b.kj[r + 1][p] = jq;
                    }
                    e = f;
                }
            }
            __syncwarp();
#pragma unroll
            for (int s = 0; s < 2; ++s)
                if ((int)lane + 32 * s < (int)nin) jv[s] = b.kj[lane + 32 * s][p];
            __syncwarp();
        }
        const uint32_t keep = min(nin, kmax);
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (lane + 32u * s < keep) a.idx[ip * (int64_t)kmax + lane + 32 * s] = jv[s];
        const uint32_t j0 = __shfl_sync(0xffffffffu, jv[0], 0);
        if ((int)lane == p) near_j = keep > 0 ? j0 : 0xffffffffu;
        if (lane == 0) {
            a.count[ip] = keep;
            a.total[ip] = min(nin, 4u * kmax);
        }
        mx = max(mx, nin);
        novf += nin > kmax ? 1u : 0u;
    }
    if (lane == 0) {
        if (novf) atomicAdd(a.counters + C_OVERFLOW, (unsigned long long)novf);
        if (mx) atomicMax(a.counters + C_MAXCOUNT, (unsigned long long)mx);
    }
    // the exact squared distance to each particle's nearest entry (the CFL
    // step's ell^2), every lane its own particle
    if (mine && !handed) a.d2min[i] = near_j != 0xffffffffu ? exact_d2<DIM>(a, i, near_j) : INFINITY;
    __syncwarp();
    return true;
}

// the tile of 32 key-ordered particles starting at i0 (< n), one warp
template <int DIM, bool PER>
__device__ __forceinline__ void tile_tile(const QueryArgs& a, TileBuf& b, int64_t i0)
{
    const unsigned lane = lane_id();
    const int64_t i = i0 + lane;
    const bool valid = i < a.n;
    const int mb = a.c.mbits;
    const uint64_t mysim = (valid && a.c.nsim_max > 1) ? (a.keys[i] >> (DIM * mb)) : 0ull;
    // groups: a new one starts at lane 0, at a change of simulation, and after
    // a jump of more than TQ_GAP radii between consecutive particles
    TileLane<DIM> t;
    if (valid) tile_lane<DIM, PER>(a, a.g[mysim], i, t);
    else {
#pragma unroll
        for (int k = 0; k < 3; ++k) { t.hx[k] = 0.0f; t.lx[k] = 0.0f; t.tq[k] = 0.0f; }
        t.Rf = t.R2f = t.Rq = t.Rout = 0.0f;
    }
    float tq[3] = {t.tq[0], t.tq[1], t.tq[2]};
    const float Rq = t.Rq;
    const uint64_t psim = __shfl_up_sync(0xffffffffu, mysim, 1);
    const float pRq = __shfl_up_sync(0xffffffffu, Rq, 1);
    float gap2 = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float d = tq[k] - __shfl_up_sync(0xffffffffu, tq[k], 1);
        gap2 = fmaf(d, d, gap2);
    }
    const float lim = TQ_GAP * fmaxf(Rq, pRq);
    const unsigned starts = __ballot_sync(0xffffffffu, valid && (lane == 0 || psim != mysim || !(gap2 <= lim * lim)));
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    unsigned rest = starts;
    while (rest) {                              // the groups, in turn
        const int s0 = __ffs(rest) - 1;
        rest &= rest - 1;
        const int s1 = rest ? __ffs(rest) - 1 : 32;
        const unsigned grp = vmask & ((s1 == 32 ? 0xffffffffu : ((1u << s1) - 1u)) & ~((1u << s0) - 1u));
        const uint64_t sim = __shfl_sync(0xffffffffu, mysim, s0);
        // a group whose region is too large is halved (by key order: the
        // halves are smaller regions) down to TQ_SPLIT_MIN particles; what is
        // still too large goes to the per-particle kernel
        unsigned stk[6];
        int sp = 0;
        stk[sp++] = grp;
        while (sp > 0) {
            const unsigned g = stk[--sp];
            if (tile_group<DIM, PER>(a, b, i, ((g >> lane) & 1u) != 0u, sim, t)) continue;
            const int pc = __popc(g);
            if (pc >= 2 * TQ_SPLIT_MIN && sp + 2 <= 6) {
                unsigned lo = 0, gg = g;                // the first pc / 2 members
                for (int q = 0; q < pc / 2; ++q) { lo |= gg & (0u - gg); gg &= gg - 1; }
                stk[sp++] = g & ~lo;
                stk[sp++] = lo;
            } else {
                list_append(a, ((g >> lane) & 1u) != 0u, (uint32_t)i);
            }
        }
    }
}

template <int DIM, bool PER>
__global__ void __launch_bounds__(TQ_WARPS * 32, 5) k_query_tile(QueryArgs a)
{
    extern __shared__ __align__(16) unsigned char tq_smem[];
    TileBuf& b = reinterpret_cast<TileBuf*>(tq_smem)[threadIdx.x >> 5];
    const int64_t i0 = ((int64_t)blockIdx.x * TQ_WARPS + (threadIdx.x >> 5)) * 32;
    if (i0 >= a.n) return;                      // whole warp
    tile_tile<DIM, PER>(a, b, i0);
}

// Persistent form (LP_SCHED_QUEUE_QUERY): a grid of resident blocks whose
// warps take their next tile from a.queue until none is left, so a warp whose
// tile was cheap takes another at once instead of holding its slot (and its
// shared-memory buffer) until the slowest warp of its block ends.
template <int DIM, bool PER>
__global__ void __launch_bounds__(TQ_WARPS * 32, 5) k_query_tile_q(QueryArgs a)
{
    extern __shared__ __align__(16) unsigned char tq_smem[];
    TileBuf& b = reinterpret_cast<TileBuf*>(tq_smem)[threadIdx.x >> 5];
    for (;;) {
        unsigned long long base = 0;
        if (lane_id() == 0) base = atomicAdd(a.queue, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= (unsigned long long)a.n) return;
        tile_tile<DIM, PER>(a, b, (int64_t)base);
        __syncwarp();                           // the buffer is reused by the next tile
    }
}

// 1D, k nearest per side on the exactly x-ordered particles
__global__ void k_query_kside(QueryArgs a)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const DevCfg& c = a.c;
    const int K = c.k_per_side;
    const int W = K + 4;
    double dl[8], dr[8];
    uint32_t il[8], ir[8], jl[8], jr[8];
    int nl = 0, nr = 0;
    double xi = a.sx[0][i];
    for (int side = 0; side < 2; ++side) {
        for (int s = 1; s <= W; ++s) {
            int64_t j = side == 0 ? i - s : i + s;
            if (c.periodic[0]) j = ((j % a.n) + a.n) % a.n;
            else if (j < 0 || j >= a.n) break;
            if (j == i) break;
            double dx = offset64(c, 0, xi, a.sx[0][j]);
            if ((side == 0 && !(dx < 0.0)) || (side == 1 && !(dx > 0.0))) continue;
            double d2 = __dmul_rn(dx, dx);
            uint32_t id = a.sid[j];
            double* D = side == 0 ? dl : dr;
            uint32_t* I = side == 0 ? il : ir;
            uint32_t* J = side == 0 ? jl : jr;
            int& cnt = side == 0 ? nl : nr;
            // insertion into the K smallest by (d2, id)
            int r = cnt < K ? cnt : K;
            if (cnt >= K && !(d2 < D[K - 1] || (d2 == D[K - 1] && id < I[K - 1]))) continue;
            if (cnt < K) ++cnt;
            r = cnt - 1;
            while (r > 0 && (D[r - 1] > d2 || (D[r - 1] == d2 && I[r - 1] > id))) {
                D[r] = D[r - 1]; I[r] = I[r - 1]; J[r] = J[r - 1];
                --r;
            }
            D[r] = d2; I[r] = id; J[r] = (uint32_t)j;
        }
    }
    // merge by (d2, id)
    int a_ = 0, b_ = 0, o = 0;
    double first = INFINITY;
    while (a_ < nl || b_ < nr) {
        bool takel = b_ >= nr || (a_ < nl && (dl[a_] < dr[b_] || (dl[a_] == dr[b_] && il[a_] < ir[b_])));
        double d = takel ? dl[a_] : dr[b_];
        uint32_t j = takel ? jl[a_++] : jr[b_++];
        if (o == 0) first = d;
        a.idx[i * (int64_t)c.k_max + o++] = j;
    }
    a.count[i] = (uint32_t)o;
    a.total[i] = (uint32_t)o;
    a.d2min[i] = first;
    atomicMax(a.counters + C_MAXCOUNT, (unsigned long long)o);
}

}  // namespace

// The all-octant coverage check of the central stencils (Sec. 2.1: the
// second-order stencils are meant to include particles from all 8 octants):
// per particle of the last build, whether its list misses one of the 2^dim
// sign patterns of the offsets (an offset of exactly 0 counted as positive),
// from the same float hi/lo offsets the fits use.  Thread per particle.
template <int DIM, bool PER>
__global__ void k_octant_coverage(int64_t n, DevCfg c, const float4* __restrict__ pos4,
                                  const uint32_t* __restrict__ count, const uint32_t* __restrict__ idx,
                                  uint8_t* gap, unsigned long long* ngap)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool g = false;
    if (i < n) {
        const float4 ih = pos4[2 * i], il = pos4[2 * i + 1];
        const float hi[3] = {ih.x, ih.y, ih.z}, li[3] = {il.x, il.y, il.z};
        const uint32_t cnt = count[i];
        unsigned mask = 0u;
        for (uint32_t t = 0; t < cnt; ++t) {
            const uint32_t j = idx[i * (int64_t)c.k_max + t];
            float4 qh, ql;
            ldg256(pos4 + 2 * (int64_t)j, qh, ql);
            const float hj[3] = {qh.x, qh.y, qh.z}, lj[3] = {ql.x, ql.y, ql.z};
            unsigned o = 0u;
#pragma unroll
            for (int k = 0; k < DIM; ++k)
                o |= (split_offset<PER>(c, k, hj[k], lj[k], hi[k], li[k]) >= 0.0f ? 1u : 0u) << k;
            mask |= 1u << o;
        }
        g = __popc(mask) < (1 << DIM);
        if (gap) gap[i] = g ? 1 : 0;
    }
    const unsigned b = __ballot_sync(0xffffffffu, g);
    if ((threadIdx.x & 31u) == 0u && b) atomicAdd(ngap, (unsigned long long)__popc(b));
}

cudaError_t query_neighbors(lp_ctx* c, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    QueryArgs a;
    a.c = c->dc;
    a.n = n;
    a.g = c->grid;
    a.keys = c->keys_sorted;
    a.level_off = c->level_off_dev;
    a.cells = c->cells;
    for (int k = 0; k < 3; ++k) {
        int kk = k < c->dc.dim ? k : 0;
        a.sx[k] = c->sx[kk];
    }
    a.pos4 = c->pos4;
    a.sm = c->sm; a.sV = c->sV; a.sid = c->sid;
    a.count = c->nb_count; a.total = c->nb_total; a.idx = c->nb_idx; a.d2min = c->nb_d2min;
    a.counters = c->counters;
    a.list = nullptr;
    a.list_len = nullptr;
    a.fb_list = c->redo_list;                  // capacity n: each particle is appended at most once
    a.fb_len = c->counters + C_QFB_LEN;
    a.queue = nullptr;
    if (c->dc.radius_mode == LP_RADIUS_KSIDE) {
        k_query_kside<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
        return cudaGetLastError();
    }
    const int dim = c->dc.dim;
    if (dim == 1) {
        k_query<1><<<(unsigned)((n + NB_WARPS - 1) / NB_WARPS), NB_WARPS * 32, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(c->counters + C_QFB_LEN, 0, 8, s);
    if (e != cudaSuccess) return e;
    const bool octant = c->dc.select == LP_SELECT_OCTANT;
    if (c->schedule & LP_SCHED_QUERY_WARP) {   // one warp per particle for every particle
        const unsigned wb = (unsigned)((n + NB_WARPS - 1) / NB_WARPS);
        if (octant) {
            if (dim == 3) k_query_octant<3><<<wb, NB_WARPS * 32, 0, s>>>(a);
            else k_query_octant<2><<<wb, NB_WARPS * 32, 0, s>>>(a);
        } else {
            if (dim == 3) k_query<3><<<wb, NB_WARPS * 32, 0, s>>>(a);
            else k_query<2><<<wb, NB_WARPS * 32, 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    // tiles first; the particles they leave go to the per-particle kernel
    const bool per = c->dc.periodic[0] || c->dc.periodic[1] || c->dc.periodic[2];
    const int64_t tiles = (n + 31) / 32;
    const unsigned tblocks = (unsigned)((tiles + TQ_WARPS - 1) / TQ_WARPS);
    const size_t smem = sizeof(TileBuf) * TQ_WARPS;
    if (c->schedule & LP_SCHED_QUEUE_QUERY) {
        // as many blocks as are resident at once, never more than the tiles need
        auto kq = dim == 3 ? (per ? k_query_tile_q<3, true> : k_query_tile_q<3, false>)
                           : (per ? k_query_tile_q<2, true> : k_query_tile_q<2, false>);
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kq, TQ_WARPS * 32, smem)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        const unsigned qb = (unsigned)std::min<int64_t>((int64_t)sms * per_sm, (int64_t)tblocks);
        a.queue = c->counters + C_QUEUE_TILE;
        if ((e = cudaMemsetAsync(a.queue, 0, 8, s)) != cudaSuccess) return e;
        kq<<<qb, TQ_WARPS * 32, smem, s>>>(a);
    } else if (dim == 3) {
        if (per) k_query_tile<3, true><<<tblocks, TQ_WARPS * 32, smem, s>>>(a);
        else k_query_tile<3, false><<<tblocks, TQ_WARPS * 32, smem, s>>>(a);
    } else {
        if (per) k_query_tile<2, true><<<tblocks, TQ_WARPS * 32, smem, s>>>(a);
        else k_query_tile<2, false><<<tblocks, TQ_WARPS * 32, smem, s>>>(a);
    }
    a.list = c->redo_list;
    a.list_len = c->counters + C_QFB_LEN;
    const unsigned fblocks = 152u * 4u;
    if (octant) {
        if (dim == 3) k_query_octant<3><<<fblocks, NB_WARPS * 32, 0, s>>>(a);
        else k_query_octant<2><<<fblocks, NB_WARPS * 32, 0, s>>>(a);
    } else {
        if (dim == 3) k_query<3><<<fblocks, NB_WARPS * 32, 0, s>>>(a);
        else k_query<2><<<fblocks, NB_WARPS * 32, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int query_launches(const lp_ctx* c)
{
    if (c->dc.radius_mode == LP_RADIUS_KSIDE) return 1;
    if (c->dc.dim == 1 || (c->schedule & LP_SCHED_QUERY_WARP)) return 1;
    return 2;
}

cudaError_t query_init()
{
    const int smem = (int)(sizeof(TileBuf) * TQ_WARPS);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_query_tile<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_query_tile<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_query_tile<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_query_tile<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_query_tile_q<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_query_tile_q<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_query_tile_q<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_query_tile_q<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace lp

using namespace lp;

extern "C" lp_status lp_octant_coverage(lp_ctx* c, uint8_t* gap, int64_t* n_gap, lp_stream stream)
{
    if (!c || !n_gap || c->dc.radius_mode == LP_RADIUS_KSIDE) return LP_ERR_ARG;
    if (c->lists_stale) return LP_ERR_STATE;
    *n_gap = 0;
    const int64_t n = c->n_lists;
    if (n == 0) return LP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* ctr = c->counters + C_OCT_GAP;
    if (cudaMemsetAsync(ctr, 0, 8, s) != cudaSuccess) return LP_ERR_CUDA;
    const bool per = c->dc.periodic[0] || c->dc.periodic[1] || c->dc.periodic[2];
    const unsigned gb = (unsigned)((n + 255) / 256);
    const int dim = c->dc.dim;
#define LP_COV_ARGS n, c->dc, c->pos4, c->nb_count, c->nb_idx, gap, ctr
    if (dim == 3) { if (per) k_octant_coverage<3, true><<<gb, 256, 0, s>>>(LP_COV_ARGS); else k_octant_coverage<3, false><<<gb, 256, 0, s>>>(LP_COV_ARGS); }
    else if (dim == 2) { if (per) k_octant_coverage<2, true><<<gb, 256, 0, s>>>(LP_COV_ARGS); else k_octant_coverage<2, false><<<gb, 256, 0, s>>>(LP_COV_ARGS); }
    else { if (per) k_octant_coverage<1, true><<<gb, 256, 0, s>>>(LP_COV_ARGS); else k_octant_coverage<1, false><<<gb, 256, 0, s>>>(LP_COV_ARGS); }
#undef LP_COV_ARGS
    c->launches += 1;
    unsigned long long h = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h, ctr, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LP_ERR_CUDA;
    *n_gap = (int64_t)h;
    return LP_OK;
}
