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
#include "lp_internal.cuh"

namespace lp {

namespace {

constexpr float TOL_R = 4e-6f;   // relative band around R^2 decided in FP64
constexpr float TOL_T = 4e-6f;   // relative gap below which two entries are re-ordered in FP64

struct QueryArgs {
    DevCfg c;
    int64_t n;
    const Grid* g;
    const int64_t* level_off;
    const unsigned long long* cells;
    const double* sx[3];
    const float* hx[3];
    const float* lx[3];
    const double* sm;
    const double* sV;
    const uint32_t* sid;
    uint32_t* count;
    uint32_t* total;
    uint32_t* idx;
    double* d2min;
    unsigned long long* counters;
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

struct WarpBuf {
    unsigned long long key[NB_CAP];   // float bits of d2 << 32 | id
    uint32_t j[NB_CAP];
    double d64[NB_CAP];
    uint32_t tie[NB_CAP / 32];        // bit e: entry e is within rounding of entry e-1
    uint32_t cstart[32];
    uint32_t cexcl[32];
};

__device__ inline float key_d2(unsigned long long k) { return __uint_as_float((uint32_t)(k >> 32)); }

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

template <int DIM>
__global__ void __launch_bounds__(NB_WARPS * 32) k_query(QueryArgs a)
{
    __shared__ WarpBuf bufs[NB_WARPS];
    unsigned lane = lane_id();
    int w = threadIdx.x >> 5;
    WarpBuf& b = bufs[w];
    int64_t i = (int64_t)blockIdx.x * NB_WARPS + w;
    if (i >= a.n) return;
    const DevCfg& c = a.c;
    const Grid& g = *a.g;
    unsigned lt = (1u << lane) - 1u;

    // own position and radius
    double xi[3];
    float hxi[3], lxi[3];
#pragma unroll
    for (int k = 0; k < DIM; ++k) { xi[k] = a.sx[k][i]; hxi[k] = a.hx[k][i]; lxi[k] = a.lx[k][i]; }
    double wi = __dmul_rn(a.sm[i], a.sV[i]);
    float Rf;
    if (c.radius_mode == LP_RADIUS_FIXED) Rf = (float)c.radius;
    else {
        float wf = (float)wi;
        float r = DIM == 3 ? cbrtf(wf) : (DIM == 2 ? sqrtf(wf) : wf);
        Rf = (float)c.kappa * r;
    }
    float R2f = (c.radius_mode == LP_RADIUS_FIXED) ? (float)(c.radius * c.radius) : Rf * Rf;
    float Rc = Rf * (1.0f + 1e-5f);

    // level: finest with cell edge L / 2^l >= Rc
    float Lf = (float)g.L;
    int l = (int)floorf(log2f(Lf / Rc));
    while (l > 0 && ldexpf(Lf, -l) < Rc) --l;
    l = max(g.lmin, min(l, g.lmax));
    double scale = ldexp(g.inv, -(MORTON_BITS - l));   // cells per unit length at level l
    long long ncell_axis = 1ll << l;

    long long clo[3] = {0, 0, 0};
    int nc[3] = {1, 1, 1};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double lo_t = floor(__dmul_rn(__dsub_rn(__dsub_rn(xi[k], (double)Rc), g.lo[k]), scale));
        double hi_t = floor(__dmul_rn(__dsub_rn(__dadd_rn(xi[k], (double)Rc), g.lo[k]), scale));
        long long a0 = (long long)lo_t, a1 = (long long)hi_t;
        if (!c.periodic[k]) {
            a0 = max(0ll, min(a0, ncell_axis - 1));
            a1 = max(0ll, min(a1, ncell_axis - 1));
            clo[k] = a0;
            nc[k] = (int)(a1 - a0 + 1);
        } else {
            long long span = a1 - a0 + 1;
            if (span > ncell_axis) span = ncell_axis;
            clo[k] = a0;
            nc[k] = (int)span;
        }
    }
    int ncells = nc[0] * nc[1] * nc[2];
    if (ncells > 32) {   // cannot happen with cell edge >= radius; recorded, never silent
        if (lane == 0) atomicOr(reinterpret_cast<unsigned int*>(a.counters + C_STATUS), ST_ILLCOND);
        ncells = 32;
    }

    // cell ranges, one lane per cell
    uint32_t cs = 0, cn = 0;
    if ((int)lane < ncells) {
        int t = lane;
        uint32_t q[3] = {0, 0, 0};
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            long long v = clo[k] + (t % nc[k]);
            t /= nc[k];
            if (c.periodic[k]) v = ((v % ncell_axis) + ncell_axis) % ncell_axis;
            q[k] = (uint32_t)v;
        }
        uint64_t code = morton<DIM>(q);
        unsigned long long e = a.cells[a.level_off[l] + (int64_t)code];
        cs = (uint32_t)e;
        uint32_t ce = (uint32_t)(e >> 32);
        cn = ce > cs ? ce - cs : 0;
    }
    uint32_t incl = cn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
    b.cstart[lane] = cs;
    b.cexcl[lane] = incl - cn;
    __syncwarp();

    int m = 0;                     // entries in the buffer
    uint32_t inside_total = 0;
    float cut = INFINITY;          // entries beyond this can no longer be kept
    int nce = min(ncells, 32);
    for (uint32_t base = 0; base < T; base += 32) {
        if (m > NB_CAP - 32) {
            sort_exact<DIM>(a, b, m, i);
            m = min(m, c.k_max);
            if (m == c.k_max) cut = key_d2(b.key[m - 1]) * (1.0f + TOL_T);
        }
        uint32_t t = base + lane;
        bool in = false;
        bool keep = false;
        float d2f = 0.0f;
        uint32_t j = 0;
        if (t < T) {
            int lo = 0, hi = nce - 1;      // last cell with cexcl <= t
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (b.cexcl[mid] <= t) lo = mid; else hi = mid - 1;
            }
            j = b.cstart[lo] + (t - b.cexcl[lo]);
            if ((int64_t)j != i) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    float dh = a.hx[k][j] - hxi[k];
                    float dl = a.lx[k][j] - lxi[k];
                    if (c.periodic[k]) {
                        if (dh > 0.5f * c.Lper_h[k]) { dh -= c.Lper_h[k]; dl -= c.Lper_l[k]; }
                        else if (dh < -0.5f * c.Lper_h[k]) { dh += c.Lper_h[k]; dl += c.Lper_l[k]; }
                    }
                    float d = dh + dl;
                    d2f = fmaf(d, d, d2f);
                }
                if (d2f <= R2f * (1.0f - TOL_R)) in = true;
                else if (d2f <= R2f * (1.0f + TOL_R)) in = inside64(c, DIM, exact_d2<DIM>(a, i, j), wi);
                keep = in && d2f <= cut;
            }
        }
        inside_total += __popc(__ballot_sync(0xffffffffu, in));
        unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int pos = m + __popc(km & lt);
            b.key[pos] = ((unsigned long long)__float_as_uint(d2f) << 32) | a.sid[j];
            b.j[pos] = j;
        }
        m += __popc(km);
        __syncwarp();
    }
    sort_exact<DIM>(a, b, m, i);
    int cnt = min(m, c.k_max);
    for (int e = lane; e < cnt; e += 32) a.idx[i * (int64_t)c.k_max + e] = b.j[e];
    if (lane == 0) {
        a.count[i] = (uint32_t)cnt;
        a.total[i] = inside_total;
        a.d2min[i] = cnt > 0 ? exact_d2<DIM>(a, i, b.j[0]) : INFINITY;
        if (inside_total > (uint32_t)c.k_max) atomicAdd(a.counters + C_OVERFLOW, 1ull);
        atomicMax(a.counters + C_MAXCOUNT, (unsigned long long)inside_total);
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

cudaError_t query_neighbors(lp_ctx* c, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    QueryArgs a;
    a.c = c->dc;
    a.n = n;
    a.g = c->grid;
    a.level_off = reinterpret_cast<const int64_t*>(c->dt_min + 16);
    a.cells = c->cells;
    for (int k = 0; k < 3; ++k) {
        int kk = k < c->dc.dim ? k : 0;
        a.sx[k] = c->sx[kk]; a.hx[k] = c->hx[kk]; a.lx[k] = c->lx[kk];
    }
    a.sm = c->sm; a.sV = c->sV; a.sid = c->sid;
    a.count = c->nb_count; a.total = c->nb_total; a.idx = c->nb_idx; a.d2min = c->nb_d2min;
    a.counters = c->counters;
    if (c->dc.radius_mode == LP_RADIUS_KSIDE) {
        k_query_kside<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
    } else {
        unsigned blocks = (unsigned)((n + NB_WARPS - 1) / NB_WARPS);
        if (c->dc.dim == 3) k_query<3><<<blocks, NB_WARPS * 32, 0, s>>>(a);
        else if (c->dc.dim == 2) k_query<2><<<blocks, NB_WARPS * 32, 0, s>>>(a);
        else k_query<1><<<blocks, NB_WARPS * 32, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lp
