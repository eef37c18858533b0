// lp_sort.cu -- Sec. 2.2 steps 2-3 on the GPU: bounding cube, Morton (Z-curve)
// keys, LSD radix sort, gather of the state into key order, and the per-level
// cell tables that stand in for the paper's octree.
#include <string.h>

#include <mutex>

#include "lp_internal.cuh"

namespace lp {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
static_assert(RS_TILE == RS_TILE_KEYS, "the histogram is sized for this tile");
static_assert(RS_BINS == 2 * RS_THREADS, "each thread owns two digits of the histogram");
constexpr uint32_t RS_MASK = RS_BINS - 1;


__device__ inline double from_order_key(unsigned long long k)
{
    uint64_t b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

constexpr int EXT_ITEMS = 16;

// order key of the double with bit pattern b (order_key without FP64
// instructions), and whether b is a NaN (NaNs take no part in an extent, as
// with fmin / fmax)
__device__ __forceinline__ uint64_t order_key_bits(uint64_t b)
{
    if ((b << 1) == 0) b = 0;                   // -0 as +0
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ bool is_nan_bits(uint64_t b) { return (b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull; }

constexpr uint64_t KEY_POS_INF = 0xfff0000000000000ull;   // order_key(+inf)
constexpr uint64_t KEY_NEG_INF = 0x000fffffffffffffull;   // order_key(-inf)

// extent of one run of particles, as order keys: lo[k], hi[k] of the
// coordinates and wlo, whi of m V
struct ExtKeys {
    uint64_t lo[3], hi[3], wlo, whi;
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int k = 0; k < 3; ++k) { lo[k] = KEY_POS_INF; hi[k] = KEY_NEG_INF; }
        wlo = KEY_POS_INF;
        whi = KEY_NEG_INF;
    }
    template <int DIM>
    __device__ __forceinline__ void add(const double* const (&xs)[3], int64_t i)
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const uint64_t b = (uint64_t)__double_as_longlong(xs[k][i]);
            if (is_nan_bits(b)) continue;
            const uint64_t q = order_key_bits(b);
            lo[k] = q < lo[k] ? q : lo[k];
            hi[k] = q > hi[k] ? q : hi[k];
        }
    }
    __device__ __forceinline__ void add_w(double w)
    {
        const uint64_t bw = (uint64_t)__double_as_longlong(w);
        if (!is_nan_bits(bw)) {
            const uint64_t q = order_key_bits(bw);
            wlo = q < wlo ? q : wlo;
            whi = q > whi ? q : whi;
        }
    }
    template <int DIM>
    __device__ void flush(unsigned long long* e) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            atomicMin(e + k, (unsigned long long)lo[k]);
            atomicMax(e + 3 + k, (unsigned long long)hi[k]);
        }
    }
    __device__ void flush_w(unsigned long long* e) const
    {
        atomicMin(e + 6, (unsigned long long)wlo);
        atomicMax(e + 7, (unsigned long long)whi);
    }
};

// the m V extent of the particles of a block (gather order, simulations
// kept together), to ext[8 s + 6..7] of their simulation s: reduced over each
// warp whose particles share a simulation, then over the block when all its
// warps do (one pair of atomics per block: the extent words are the same few
// addresses for every block, so their atomics would otherwise queue);
// atomics per warp or per lane otherwise.  Every thread of the block calls it
// (valid: this thread has a particle); blockDim.x <= 32 * EXT_WARPS.
constexpr int EXT_WARPS = 8;
__device__ __forceinline__ void block_w_extent(bool valid, double w, uint32_t sim, unsigned long long* ext)
{
    __shared__ uint64_t swlo[EXT_WARPS], swhi[EXT_WARPS];
    __shared__ uint32_t ssim[EXT_WARPS];
    ExtKeys r;
    r.init();
    if (valid) r.add_w(w);
    else sim = 0xffffffffu;
    const uint32_t s0 = __shfl_sync(0xffffffffu, sim, 0);
    const bool uniform = __all_sync(0xffffffffu, sim == s0 || sim == 0xffffffffu);
    const unsigned wid = threadIdx.x >> 5;
    if (uniform) {
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t a = __shfl_xor_sync(0xffffffffu, r.wlo, o);
            const uint64_t b = __shfl_xor_sync(0xffffffffu, r.whi, o);
            r.wlo = a < r.wlo ? a : r.wlo;
            r.whi = b > r.whi ? b : r.whi;
        }
    } else if (sim != 0xffffffffu) {
        r.flush_w(ext + 8 * (int64_t)sim);                  // a warp across simulations
    }
    if (lane_id() == 0) {
        ssim[wid] = uniform ? s0 : 0xfffffffeu;             // 0xfffffffe: flushed already
        swlo[wid] = r.wlo;
        swhi[wid] = r.whi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (int)((blockDim.x + 31) / 32);
        uint32_t sb = 0xffffffffu;
        bool one = true;
        for (int q = 0; q < nw; ++q) {
            const uint32_t sq = ssim[q];
            if (sq == 0xffffffffu) continue;                // no particle
            if (sq == 0xfffffffeu || (sb != 0xffffffffu && sq != sb)) { one = false; break; }
            sb = sq;
        }
        if (one) {
            if (sb != 0xffffffffu) {
                ExtKeys t;
                t.init();
                for (int q = 0; q < nw; ++q)
                    if (ssim[q] == sb) {
                        t.wlo = swlo[q] < t.wlo ? swlo[q] : t.wlo;
                        t.whi = swhi[q] > t.whi ? swhi[q] : t.whi;
                    }
                t.flush_w(ext + 8 * (int64_t)sb);
            }
        } else {
            for (int q = 0; q < nw; ++q) {
                ExtKeys t;
                t.init();
                t.wlo = swlo[q];
                t.whi = swhi[q];
                if (ssim[q] < 0xfffffffeu) t.flush_w(ext + 8 * (int64_t)ssim[q]);
            }
        }
    }
}

// ext[8 s + 0..2] min x_k, [8 s + 3..5] max x_k (order keys) of simulation s
// (the extent of m V, ext[8 s + 6..7], is taken by the gather, which reads m
// and V anyway: the keys need only the positions).  One simulation:
// grid-stride accumulation and a warp reduction; several: EXT_ITEMS particles
// per thread, reduced over the warp when the warp's particles share a
// simulation (they are stored by simulation), with atomics per run otherwise.
// The comparisons are integer ones on the order keys (FP64 min / max would
// run on the scarce FP64 units).
template <int DIM>
__global__ void k_reduce_extent(int64_t n, const double* __restrict__ x0,
                                const double* __restrict__ x1, const double* __restrict__ x2,
                                const uint32_t* __restrict__ sim_of, unsigned long long* ext)
{
    ExtKeys r;
    r.init();
    const double* const xs[3] = {x0, x1, x2};
    uint32_t sim = 0;
    if (!sim_of) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            r.add<DIM>(xs, i);
    } else {
        // EXT_ITEMS particles per thread (strided by the block size, so loads
        // stay coalesced); a change of simulation flushes the running extent
        sim = 0xffffffffu;
        const int64_t base = (int64_t)blockIdx.x * blockDim.x * EXT_ITEMS + threadIdx.x;
        for (int q = 0; q < EXT_ITEMS; ++q) {
            const int64_t i = base + (int64_t)q * blockDim.x;
            if (i >= n) break;
            const uint32_t si = sim_of[i];
            if (si != sim) {
                if (sim != 0xffffffffu) r.flush<DIM>(ext + 8 * (int64_t)sim);
                sim = si;
                r.init();
            }
            r.add<DIM>(xs, i);
        }
    }
    // over the warp when its particles share a simulation, then over the
    // block when all its warps do (one set of atomics per block: the extent
    // words are the same few addresses for every block); per lane otherwise
    __shared__ uint64_t slo[EXT_WARPS][3], shi[EXT_WARPS][3];
    __shared__ uint32_t ssim[EXT_WARPS];
    const uint32_t s0 = __shfl_sync(0xffffffffu, sim, 0);
    const bool uniform = __all_sync(0xffffffffu, sim == s0 || sim == 0xffffffffu);
    const unsigned wid = threadIdx.x >> 5;
    if (uniform) {
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const uint64_t a = __shfl_xor_sync(0xffffffffu, r.lo[k], o);
                const uint64_t b = __shfl_xor_sync(0xffffffffu, r.hi[k], o);
                r.lo[k] = a < r.lo[k] ? a : r.lo[k];
                r.hi[k] = b > r.hi[k] ? b : r.hi[k];
            }
        }
    } else if (sim != 0xffffffffu) {
        r.flush<DIM>(ext + 8 * (int64_t)sim);
    }
    if (lane_id() == 0) {
        ssim[wid] = uniform ? s0 : 0xfffffffeu;             // 0xfffffffe: flushed already
#pragma unroll
        for (int k = 0; k < DIM; ++k) { slo[wid][k] = r.lo[k]; shi[wid][k] = r.hi[k]; }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int nw = (int)((blockDim.x + 31) / 32);
    uint32_t sb = 0xffffffffu;
    bool one = true;
    for (int q = 0; q < nw; ++q) {
        const uint32_t sq = ssim[q];
        if (sq == 0xffffffffu) continue;                    // no particle
        if (sq == 0xfffffffeu || (sb != 0xffffffffu && sq != sb)) { one = false; break; }
        sb = sq;
    }
    for (int q = 0; q < nw; ++q) {
        const uint32_t sq = ssim[q];
        if (sq >= 0xfffffffeu) continue;
        ExtKeys t;
        t.init();
#pragma unroll
        for (int k = 0; k < DIM; ++k) { t.lo[k] = slo[q][k]; t.hi[k] = shi[q][k]; }
        if (one) {
            // merge every warp into the first, flushed once at the end
            for (int q2 = q + 1; q2 < nw; ++q2) {
                if (ssim[q2] != sb) continue;
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    t.lo[k] = slo[q2][k] < t.lo[k] ? slo[q2][k] : t.lo[k];
                    t.hi[k] = shi[q2][k] > t.hi[k] ? shi[q2][k] : t.hi[k];
                }
            }
            t.flush<DIM>(ext + 8 * (int64_t)sb);
            break;
        }
        t.flush<DIM>(ext + 8 * (int64_t)sq);
    }
}

__global__ void k_init_extent(unsigned long long* ext, int nsim)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 8 * nsim) {
        int w = t & 7;
        ext[t] = (w < 3 || w == 6) ? ~0ull : 0ull;
    }
}

// Bounding cube of each simulation (what the keys need).
__global__ void k_finalize_cube(DevCfg c, int nsim, const unsigned long long* ext_all, Grid* grids)
{
    int sim = blockIdx.x * blockDim.x + threadIdx.x;
    if (sim >= nsim) return;
    const unsigned long long* ext = ext_all + 8 * sim;
    Grid* g = grids + sim;
    double L = 0.0;
    for (int k = 0; k < c.dim; ++k) {
        double lo, ext_k;
        if (c.periodic[k]) { lo = c.box_lo[k]; ext_k = c.Lper[k]; }
        else { lo = from_order_key(ext[k]); ext_k = __dsub_rn(from_order_key(ext[3 + k]), lo); }
        g->lo[k] = lo;
        L = fmax(L, ext_k);
    }
    for (int k = c.dim; k < 3; ++k) g->lo[k] = 0.0;
    if (!(L > 0.0)) L = 1.0;
    g->L = L;
    g->inv = __ddiv_rn(ldexp(1.0, c.mbits), L);
    for (int k = 0; k < 3; ++k) split(g->lo[k], g->lo_h[k], g->lo_l[k]);
    g->inv_f = (float)g->inv;
    g->L_f = (float)L;
}

// The range of cell levels of each simulation, and over all of them (one
// block).  lmin is the finest level whose cell edge L / 2^l is at least the
// largest radius present; lmax the finest whose edge is at least half the
// smallest radius (the queries use cells down to half a radius).
constexpr int LEVEL_THREADS = 256;
__global__ void __launch_bounds__(LEVEL_THREADS) k_finalize_levels(DevCfg c, int lmax_cap, int nsim,
                                                                   const unsigned long long* ext_all, Grid* grids,
                                                                   int* grange)
{
    __shared__ int slo[LEVEL_THREADS], shi[LEVEL_THREADS];
    int lo_all = 1 << 20, hi_all = 0;
    for (int sim = threadIdx.x; sim < nsim; sim += LEVEL_THREADS) {
        const unsigned long long* ext = ext_all + 8 * sim;
        Grid* g = grids + sim;
        const double L = g->L;
        double rmin, rmax;
        if (c.radius_mode == LP_RADIUS_FIXED) { rmin = rmax = c.radius; }
        else {
            double wlo = from_order_key(ext[6]), whi = from_order_key(ext[7]);
            rmin = c.kappa * pow(wlo, 1.0 / c.dim);
            rmax = c.kappa * pow(whi, 1.0 / c.dim);
        }
        // margins wider than the per-particle float radius margin (1e-5) keep every
        // particle's level inside [lmin, lmax]
        rmin *= 1.0 - 1e-4;
        rmax *= 1.0 + 1e-4;
        if (!(rmin > 0.0)) rmin = L * ldexp(1.0, -lmax_cap);   // empty or degenerate simulation
        if (!(rmax > 0.0) || isinf(rmax)) rmax = L;
        int lmax = (int)floor(log2(2.0 * L / rmin));
        int lmin = (int)floor(log2(L / rmax));
        lmax = max(0, min(lmax, lmax_cap));
        lmin = max(0, min(lmin, lmax));
        g->lmax = lmax;
        g->lmin = lmin;
        lo_all = min(lo_all, lmin);
        hi_all = max(hi_all, lmax);
    }
    slo[threadIdx.x] = lo_all;
    shi[threadIdx.x] = hi_all;
    __syncthreads();
    for (int h = LEVEL_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            slo[threadIdx.x] = min(slo[threadIdx.x], slo[threadIdx.x + h]);
            shi[threadIdx.x] = max(shi[threadIdx.x], shi[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        grange[0] = slo[0];
        grange[1] = shi[0];
    }
}

// key = simulation << (DIM mbits) | Morton code of the quantised position
template <int DIM>
__global__ void k_keys(int64_t n, const double* __restrict__ x0, const double* __restrict__ x1,
                       const double* __restrict__ x2, const Grid* __restrict__ grids,
                       const uint32_t* __restrict__ sim_of, int mbits,
                       uint64_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (DIM == 1) {
        keys[i] = order_key(x0[i]);
        vals[i] = (uint32_t)i;
        return;
    }
    const double* xs[3] = {x0, x1, x2};
    uint32_t sim = sim_of ? sim_of[i] : 0u;
    const Grid* g = grids + sim;
    double inv = g->inv;
    const uint32_t qmax = (1u << mbits) - 1u;
    uint32_t q[3] = {0, 0, 0};
    for (int k = 0; k < DIM; ++k) {
        // floor(t) clamped to [0, qmax] (negative and NaN give 0, +inf gives
        // qmax), read from t's bits: the conversion instruction would run on
        // the FP64 units, which the subtraction and the product already keep busy
        const double t = __dmul_rn(__dsub_rn(xs[k][i], g->lo[k]), inv);
        q[k] = floor_clamped(t, qmax);
    }
    keys[i] = ((uint64_t)sim << (DIM * mbits)) | morton<DIM>(q);
    vals[i] = (uint32_t)i;
}

// ---- LSD radix sort, 8-bit digits ----------------------------------------

__global__ void k_rs_upsweep(int64_t n, const uint64_t* __restrict__ keys, int shift,
                             uint32_t* __restrict__ counts, int64_t nblocks)
{
    __shared__ uint32_t h[RS_BINS];
    h[threadIdx.x] = 0;
    h[threadIdx.x + RS_THREADS] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & RS_MASK], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
    counts[(int64_t)(threadIdx.x + RS_THREADS) * nblocks + blockIdx.x] = h[threadIdx.x + RS_THREADS];
}

// Per digit d (one block each): exclusive scan of the block counts
// counts[d * nblocks + b] along b, in place, and the digit's total in totals[d].
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* counts, int64_t nblocks, uint32_t* totals)
{
    __shared__ uint32_t wsum[32];
    uint32_t* row = counts + (int64_t)blockIdx.x * nblocks;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < nblocks; b0 += 1024) {
        const int64_t b = b0 + t;
        const uint32_t v = b < nblocks ? row[b] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t z = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            wsum[lane] = z;                    // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = (w ? wsum[w - 1] : 0u) + x - v;
        if (b < nblocks) row[b] = carry + before;
        carry += wsum[31];
        __syncthreads();
    }
    if (t == 0) totals[blockIdx.x] = carry;
}

// Scatter of one tile of RS_TILE keys: each warp ranks its 512 consecutive keys
// round by round (match on the digit), the warps' digit counts are scanned
// once per tile, and every key goes to digit base + block offset + rank.
__global__ void __launch_bounds__(RS_THREADS)
k_rs_downsweep(int64_t n, const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
               uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int shift,
               const uint32_t* __restrict__ counts, const uint32_t* __restrict__ totals, int64_t nblocks)
{
    constexpr int NW = RS_THREADS / 32;
    __shared__ uint32_t wc[NW][RS_BINS];
    __shared__ uint32_t dbase[RS_BINS];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    // digit bases: exclusive scan of the digit totals, thread t owning digits
    // 2t and 2t + 1, plus this tile's offset within each digit
    {
        const uint32_t v0 = totals[2 * t], v1 = totals[2 * t + 1];
        const uint32_t v = v0 + v1;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wc[0][w] = x;
        __syncthreads();
        uint32_t add = 0;
        for (int ww = 0; ww < w; ++ww) add += wc[0][ww];
        const uint32_t b0 = add + x - v;
        dbase[2 * t] = b0 + counts[(int64_t)(2 * t) * nblocks + blockIdx.x];
        dbase[2 * t + 1] = b0 + v0 + counts[(int64_t)(2 * t + 1) * nblocks + blockIdx.x];
    }
    __syncthreads();
    for (int d = lane; d < RS_BINS; d += 32) wc[w][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_ITEMS);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t key[RS_ITEMS];
    uint32_t val[RS_ITEMS], loc[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : 0ull;
        val[r] = valid ? vin[i] : 0u;
        const uint32_t d = valid ? (uint32_t)((key[r] >> shift) & RS_MASK) : RS_BINS + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const bool leader = (__ffs(peers) - 1) == lane;
        loc[r] = valid ? wc[w][d] + __popc(peers & lt) : 0u;
        __syncwarp();
        if (valid && leader) wc[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps' runs in tile order
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int d = t + h * RS_THREADS;
        uint32_t run = dbase[d];
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) {
            const uint32_t c = wc[ww][d];
            wc[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)((key[r] >> shift) & RS_MASK);
            const uint32_t pos = wc[w][d] + loc[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// gather the state into key order and split it into float hi/lo pairs
template <int DIM>
__global__ void k_gather(int64_t n, const uint32_t* __restrict__ perm, lp_particles p, DevCfg c,
                         double* sx0, double* sx1, double* sx2, double* sV, double* su0, double* su1,
                         double* su2, double* sP, double* sm, uint32_t* sid, float4* rec, float4* pos4,
                         const uint32_t* __restrict__ sim_of, unsigned long long* ext)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    {
        const uint32_t jw = i < n ? perm[i] : 0u;
        block_w_extent(i < n, i < n ? __dmul_rn(p.m[jw], p.V[jw]) : 0.0, (i < n && sim_of) ? sim_of[jw] : 0u, ext);
    }
    if (i >= n) return;
    uint32_t j = perm[i];
    float r[4 * REC_F4];
#pragma unroll
    for (int q = 0; q < 4 * REC_F4; ++q) r[q] = 0.0f;
    double* sx[3] = {sx0, sx1, sx2};
    double* su[3] = {su0, su1, su2};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double v = p.x[k][j];
        sx[k][i] = v;
        split(v, r[REC_XH + k], r[REC_XL + k]);
    }
    double V = p.V[j], P = p.P[j];
    sV[i] = V;
    sP[i] = P;
    constexpr int F = DIM + 2;
    split(V, r[rec_fh(0, F)], r[rec_fl(0, F)]);
    split(P, r[rec_fh(F - 1, F)], r[rec_fl(F - 1, F)]);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double v = p.u[k][j];
        su[k][i] = v;
        split(v, r[rec_fh(1 + k, F)], r[rec_fl(1 + k, F)]);
    }
#pragma unroll
    for (int q = 0; q < REC_F4; ++q) rec[i * REC_F4 + q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    const double m = p.m[j];
    // (r[rec_fh(0, F)] is RN(V))
    pos4[2 * i] = make_float4(r[REC_XH], r[REC_XH + 1], r[REC_XH + 2],
                              query_radius_ff(c, DIM, to_float_rn(m), r[rec_fh(0, F)]));
    pos4[2 * i + 1] = make_float4(r[REC_XL], r[REC_XL + 1], r[REC_XL + 2], 0.0f);
    sm[i] = m;
    sid[i] = p.id[j];
}

// The same gather in two kernels, for the end-to-end path (lp_step_host),
// where the fields are still being copied from the host while the neighbour
// query runs: the geometry (positions, m, V, id, the query's float positions
// and radius, the m V extent) before the query, the fields (u, P and the packed
// fit record) after it.  Together they write what k_gather writes, bit for bit.
template <int DIM>
__global__ void k_gather_geom(int64_t n, const uint32_t* __restrict__ perm, lp_particles p, DevCfg c,
                              double* sx0, double* sx1, double* sx2, double* sV, double* sm, uint32_t* sid,
                              float4* pos4, const uint32_t* __restrict__ sim_of, unsigned long long* ext)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    {
        const uint32_t jw = i < n ? perm[i] : 0u;
        block_w_extent(i < n, i < n ? __dmul_rn(p.m[jw], p.V[jw]) : 0.0, (i < n && sim_of) ? sim_of[jw] : 0u, ext);
    }
    if (i >= n) return;
    const uint32_t j = perm[i];
    double* sx[3] = {sx0, sx1, sx2};
    float xh[3] = {0.0f, 0.0f, 0.0f}, xl[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const double v = p.x[k][j];
        sx[k][i] = v;
        split(v, xh[k], xl[k]);
    }
    const double V = p.V[j], m = p.m[j];
    sV[i] = V;
    sm[i] = m;
    sid[i] = p.id[j];
    pos4[2 * i] = make_float4(xh[0], xh[1], xh[2], query_radius_ff(c, DIM, to_float_rn(m), to_float_rn(V)));
    pos4[2 * i + 1] = make_float4(xl[0], xl[1], xl[2], 0.0f);
}

template <int DIM>
__global__ void k_gather_fields(int64_t n, const uint32_t* __restrict__ perm, lp_particles p,
                                const double* sx0, const double* sx1, const double* sx2, const double* sV,
                                double* su0, double* su1, double* su2, double* sP, float4* rec)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    float r[4 * REC_F4];
#pragma unroll
    for (int q = 0; q < 4 * REC_F4; ++q) r[q] = 0.0f;
    const double* sx[3] = {sx0, sx1, sx2};
    double* su[3] = {su0, su1, su2};
#pragma unroll
    for (int k = 0; k < DIM; ++k) split(sx[k][i], r[REC_XH + k], r[REC_XL + k]);
    constexpr int F = DIM + 2;
    const double P = p.P[j];
    sP[i] = P;
    split(sV[i], r[rec_fh(0, F)], r[rec_fl(0, F)]);
    split(P, r[rec_fh(F - 1, F)], r[rec_fl(F - 1, F)]);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const double v = p.u[k][j];
        su[k][i] = v;
        split(v, r[rec_fh(1 + k, F)], r[rec_fl(1 + k, F)]);
    }
#pragma unroll
    for (int q = 0; q < REC_F4; ++q) rec[i * REC_F4 + q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
}

// cell tables: entry = start | end << 32 of the key-sorted particles in the cell
__global__ void k_tables(int dim, int mbits, int64_t n, const uint64_t* __restrict__ keys,
                         const int* __restrict__ grange, const int64_t* __restrict__ level_off,
                         unsigned long long* cells, int clear)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = keys[i];
    uint64_t kp = i > 0 ? keys[i - 1] : 0;
    uint64_t kn = i + 1 < n ? keys[i + 1] : 0;
    uint32_t* half = reinterpret_cast<uint32_t*>(cells);
    for (int l = grange[0]; l <= grange[1]; ++l) {
        int sh = dim * (mbits - l);
        uint64_t c = k >> sh;
        bool first = i == 0 || (kp >> sh) != c;
        bool last = i + 1 == n || (kn >> sh) != c;
        int64_t e = level_off[l] + (int64_t)c;
        if (clear) {
            if (first) cells[e] = 0ull;
        } else {
            if (first) half[2 * e] = (uint32_t)i;
            if (last) half[2 * e + 1] = (uint32_t)(i + 1);
        }
    }
}

__global__ void k_scatter_back(int dim, int64_t n, lp_particles p, const double* sx0, const double* sx1,
                               const double* sx2, const double* sV, const double* su0, const double* su1,
                               const double* su2, const double* sP, const double* sm, const uint32_t* sid)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* sx[3] = {sx0, sx1, sx2};
    const double* su[3] = {su0, su1, su2};
    for (int k = 0; k < dim; ++k) {
        p.x[k][i] = sx[k][i];
        p.u[k][i] = su[k][i];
    }
    p.V[i] = sV[i];
    p.P[i] = sP[i];
    p.m[i] = sm[i];
    p.id[i] = sid[i];
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

__global__ void k_sim_of(int64_t n, const int64_t* __restrict__ offsets, int nsim, uint32_t* __restrict__ sim_of)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nsim - 1;          // last simulation whose offset is <= i
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
    }
    sim_of[i] = (uint32_t)lo;
}

}  // namespace

cudaError_t build_grid(lp_ctx* c, const lp_particles* p, cudaStream_t s)
{
    int64_t n = p->n;
    int nsim = c->nsim;
    const uint32_t* sim_of = nullptr;
    if (nsim > 1) {
        k_sim_of<<<grid_for(n, 256), 256, 0, s>>>(n, c->offsets, nsim, c->sim_of);
        sim_of = c->sim_of;
    }
    k_init_extent<<<(unsigned)((8 * nsim + 255) / 256), 256, 0, s>>>(c->ext, nsim);
    int64_t nb_ = grid_for(n, 256);
    unsigned blocks = nsim > 1 ? (unsigned)((n + 256 * EXT_ITEMS - 1) / (256 * EXT_ITEMS))
                               : (unsigned)(nb_ < 152 * 8 ? nb_ : 152 * 8);
    if (blocks == 0) blocks = 1;
    const double* x1 = p->x[1] ? p->x[1] : p->x[0];
    const double* x2 = p->x[2] ? p->x[2] : p->x[0];
    if (c->dc.dim == 3) k_reduce_extent<3><<<blocks, 256, 0, s>>>(n, p->x[0], x1, x2, sim_of, c->ext);
    else if (c->dc.dim == 2) k_reduce_extent<2><<<blocks, 256, 0, s>>>(n, p->x[0], x1, x2, sim_of, c->ext);
    else k_reduce_extent<1><<<blocks, 256, 0, s>>>(n, p->x[0], x1, x2, sim_of, c->ext);
    k_finalize_cube<<<(unsigned)((nsim + 127) / 128), 128, 0, s>>>(c->dc, nsim, c->ext, c->grid);
    return cudaGetLastError();
}

cudaError_t make_keys(lp_ctx* c, const lp_particles* p, cudaStream_t s)
{
    int64_t n = p->n;
    int dim = c->dc.dim;
    const double* x1 = p->x[1] ? p->x[1] : p->x[0];
    const double* x2 = p->x[2] ? p->x[2] : p->x[0];
    const uint32_t* sim_of = c->nsim > 1 ? c->sim_of : nullptr;
    int mb = c->dc.mbits;
    unsigned gb = grid_for(n, 256);
    if (dim == 3) k_keys<3><<<gb, 256, 0, s>>>(n, p->x[0], x1, x2, c->grid, sim_of, mb, c->keys[0], c->vals[0]);
    else if (dim == 2) k_keys<2><<<gb, 256, 0, s>>>(n, p->x[0], x1, x2, c->grid, sim_of, mb, c->keys[0], c->vals[0]);
    else k_keys<1><<<gb, 256, 0, s>>>(n, p->x[0], x1, x2, c->grid, sim_of, mb, c->keys[0], c->vals[0]);
    return cudaGetLastError();
}

int radix_passes(const lp_ctx* c) { return (c->sort_hi_bit - c->sort_lo_bit + RS_BITS - 1) / RS_BITS; }

cudaError_t radix_sort(lp_ctx* c, int64_t n, cudaStream_t s)
{
    int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
    int cur = 0;
    for (int sh = c->sort_lo_bit; sh < c->sort_hi_bit; sh += RS_BITS) {
        uint32_t* totals = c->hist + RS_BINS * nblocks;
        k_rs_upsweep<<<(unsigned)nblocks, RS_THREADS, 0, s>>>(n, c->keys[cur], sh, c->hist, nblocks);
        k_rs_scan<<<RS_BINS, 1024, 0, s>>>(c->hist, nblocks, totals);
        k_rs_downsweep<<<(unsigned)nblocks, RS_THREADS, 0, s>>>(n, c->keys[cur], c->vals[cur], c->keys[cur ^ 1],
                                                                c->vals[cur ^ 1], sh, c->hist, totals, nblocks);
        cur ^= 1;
    }
    c->keys_sorted = c->keys[cur];
    c->perm_sorted = c->vals[cur];
    return cudaGetLastError();
}

cudaError_t gather(lp_ctx* c, const lp_particles* p, cudaStream_t s)
{
    int64_t n = p->n;
    int dim = c->dc.dim;
    unsigned gb = grid_for(n, 256);
    const uint32_t* perm = c->perm_sorted;
    lp_particles q = *p;
    for (int k = dim; k < 3; ++k) { q.x[k] = p->x[0]; q.u[k] = p->u[0]; }
    const uint32_t* sim_of = c->nsim > 1 ? c->sim_of : nullptr;
#define LP_GATHER_ARGS n, perm, q, c->dc, c->sx[0], c->sx[1], c->sx[2], c->sV, c->su[0], c->su[1], c->su[2], \
        c->sP, c->sm, c->sid, c->rec, c->pos4, sim_of, c->ext
    if (dim == 3) k_gather<3><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
    else if (dim == 2) k_gather<2><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
    else k_gather<1><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
#undef LP_GATHER_ARGS
    // the cell levels need the m V extent the gather took
    k_finalize_levels<<<1, LEVEL_THREADS, 0, s>>>(c->dc, c->lmax_cap, c->nsim, c->ext, c->grid, c->grange);
    return cudaGetLastError();
}

cudaError_t gather_geometry(lp_ctx* c, const lp_particles* p, cudaStream_t s)
{
    int64_t n = p->n;
    int dim = c->dc.dim;
    unsigned gb = grid_for(n, 256);
    const uint32_t* perm = c->perm_sorted;
    lp_particles q = *p;
    for (int k = dim; k < 3; ++k) q.x[k] = p->x[0];
    const uint32_t* sim_of = c->nsim > 1 ? c->sim_of : nullptr;
#define LP_GATHER_ARGS n, perm, q, c->dc, c->sx[0], c->sx[1], c->sx[2], c->sV, c->sm, c->sid, c->pos4, sim_of, c->ext
    if (dim == 3) k_gather_geom<3><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
    else if (dim == 2) k_gather_geom<2><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
    else k_gather_geom<1><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
#undef LP_GATHER_ARGS
    k_finalize_levels<<<1, LEVEL_THREADS, 0, s>>>(c->dc, c->lmax_cap, c->nsim, c->ext, c->grid, c->grange);
    return cudaGetLastError();
}

cudaError_t gather_fields(lp_ctx* c, const lp_particles* p, cudaStream_t s)
{
    int64_t n = p->n;
    int dim = c->dc.dim;
    unsigned gb = grid_for(n, 256);
    const uint32_t* perm = c->perm_sorted;
    lp_particles q = *p;
    for (int k = dim; k < 3; ++k) q.u[k] = p->u[0];
    const double* sx1 = c->sx[dim > 1 ? 1 : 0];
    const double* sx2 = c->sx[dim > 2 ? 2 : 0];
    double* su1 = c->su[dim > 1 ? 1 : 0];
    double* su2 = c->su[dim > 2 ? 2 : 0];
#define LP_GATHER_ARGS n, perm, q, c->sx[0], sx1, sx2, c->sV, c->su[0], su1, su2, c->sP, c->rec
    if (dim == 3) k_gather_fields<3><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
    else if (dim == 2) k_gather_fields<2><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
    else k_gather_fields<1><<<gb, 256, 0, s>>>(LP_GATHER_ARGS);
#undef LP_GATHER_ARGS
    return cudaGetLastError();
}

cudaError_t fill_tables(lp_ctx* c, int64_t n, bool clear, cudaStream_t s)
{
    if (c->dc.dim == 1 || n == 0) return cudaSuccess;
    k_tables<<<grid_for(n, 256), 256, 0, s>>>(c->dc.dim, c->dc.mbits, n, c->keys_sorted, c->grange,
                                               c->level_off_dev, c->cells, clear ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t scatter_back(lp_ctx* c, lp_particles* p, cudaStream_t s)
{
    int64_t n = p->n;
    if (n == 0) return cudaSuccess;
    lp_particles q = *p;
    for (int k = c->dc.dim; k < 3; ++k) { q.x[k] = p->x[0]; q.u[k] = p->u[0]; }
    k_scatter_back<<<grid_for(n, 256), 256, 0, s>>>(c->dc.dim, n, q, c->sx[0], c->sx[1], c->sx[2], c->sV, c->su[0],
                                                     c->su[1], c->su[2], c->sP, c->sm, c->sid);
    return cudaGetLastError();
}

}  // namespace lp

// ---------------------------------------------------------------------------
// Morton keys and sort order without any device allocation.
//
// Some callers cannot allocate device memory when they need the key order: a
// host application that owns every byte of device memory through its own pool
// and forbids other allocations, or a latency-critical loop where cudaMalloc's
// implicit device-wide synchronisation is not acceptable.  This entry point
// serves them: its scratch (key and index ping-pong buffers, digit histograms,
// the extent words and the cube) lives in one fixed file-scope device array,
// NOALLOC_MAX_N particles large, which every GPU that loads this library holds
// until the process exits.  It reuses the sort kernels above; nothing else in
// the library uses this array.
// ---------------------------------------------------------------------------
namespace lp {
namespace {

constexpr int64_t NOALLOC_MAX_N = LP_NOALLOC_MAX_N;
constexpr int64_t NA_BLOCKS = (NOALLOC_MAX_N + RS_TILE - 1) / RS_TILE;
// byte offsets inside the array (each 256-byte aligned)
constexpr size_t NA_KEYS0 = 0;
constexpr size_t NA_KEYS1 = NA_KEYS0 + 8 * NOALLOC_MAX_N;
constexpr size_t NA_VALS0 = NA_KEYS1 + 8 * NOALLOC_MAX_N;
constexpr size_t NA_VALS1 = NA_VALS0 + 4 * NOALLOC_MAX_N;
constexpr size_t NA_HIST = NA_VALS1 + 4 * NOALLOC_MAX_N;
constexpr size_t NA_EXT = NA_HIST + ((RS_BINS * (NA_BLOCKS + 1) * 4 + 255) / 256) * 256;   // counts + digit totals
constexpr size_t NA_GRID = NA_EXT + 256;
constexpr size_t NA_BYTES = NA_GRID + 256;

static __device__ __align__(256) unsigned char noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
unsigned char* na_ptr[NA_MAX_DEVICES] = {};

// The device address of the array on the current device.  Outside stream
// capture it is looked up again on every call, so an address cached before a
// cudaDeviceReset (after which the runtime loads the module again, possibly at
// another address) is never used.  While `s` is capturing, no runtime call that
// could load the module is made: the address cached by the last call on this
// device outside capture is used, and a device never set up that way is an
// error.
cudaError_t noalloc_setup(cudaStream_t s, unsigned char** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(na_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, noalloc_scratch);
        if (e != cudaSuccess) return e;
        na_ptr[dev] = static_cast<unsigned char*>(p);
    } else if (!na_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = na_ptr[dev];
    return cudaSuccess;
}

__global__ void k_copy_sorted(int64_t n, const uint64_t* __restrict__ ks, const uint32_t* __restrict__ vs,
                              uint64_t* __restrict__ ko, uint32_t* __restrict__ vo)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) { ko[i] = ks[i]; vo[i] = vs[i]; }
}

}  // namespace
}  // namespace lp

extern "C" lp_status lp_sort_keys_noalloc(int32_t dim, int64_t n, const double* x0, const double* x1,
                                          const double* x2, uint64_t* keys_out, uint32_t* perm_out,
                                          lp_stream stream)
{
    using namespace lp;
    if (dim < 1 || dim > 3 || n < 0 || !keys_out || !perm_out) return LP_ERR_ARG;
    if (n > NOALLOC_MAX_N) return LP_ERR_CAPACITY;
    if (n == 0) return LP_OK;
    if (!x0 || (dim > 1 && !x1) || (dim > 2 && !x2)) return LP_ERR_ARG;
    unsigned char* base = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (noalloc_setup(s, &base) != cudaSuccess) return LP_ERR_CUDA;
    uint64_t* keys[2] = {reinterpret_cast<uint64_t*>(base + NA_KEYS0), reinterpret_cast<uint64_t*>(base + NA_KEYS1)};
    uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(base + NA_VALS0), reinterpret_cast<uint32_t*>(base + NA_VALS1)};
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + NA_HIST);
    unsigned long long* ext = reinterpret_cast<unsigned long long*>(base + NA_EXT);
    Grid* grid = reinterpret_cast<Grid*>(base + NA_GRID);
    const double* p1 = x1 ? x1 : x0;
    const double* p2 = x2 ? x2 : x0;
    // the cube: same kernels and parameters as a default context (fixed radius 1,
    // finest table level 9 in 3D, 13 in 2D); the radius only sets the level range
    DevCfg dc;
    memset(&dc, 0, sizeof(dc));
    dc.dim = dim;
    dc.radius_mode = LP_RADIUS_FIXED;
    dc.radius = 1.0;
    dc.mbits = MORTON_BITS;
    dc.nsim_max = 1;
    int lmax_cap = dim == 3 ? 9 : (dim == 2 ? 13 : 0);
    int lo_bit = 0, hi_bit = 64;
    sort_bit_range(dim, MORTON_BITS, lmax_cap, 0, lo_bit, hi_bit);
    unsigned gb = grid_for(n, 256);
    int64_t nb_ = gb;
    unsigned rblocks = (unsigned)(nb_ < 152 * 8 ? nb_ : 152 * 8);
    k_init_extent<<<1, 32, 0, s>>>(ext, 1);
    if (dim == 3) k_reduce_extent<3><<<rblocks, 256, 0, s>>>(n, x0, p1, p2, nullptr, ext);
    else if (dim == 2) k_reduce_extent<2><<<rblocks, 256, 0, s>>>(n, x0, p1, p2, nullptr, ext);
    else k_reduce_extent<1><<<rblocks, 256, 0, s>>>(n, x0, p1, p2, nullptr, ext);
    k_finalize_cube<<<1, 1, 0, s>>>(dc, 1, ext, grid);
    if (dim == 3) k_keys<3><<<gb, 256, 0, s>>>(n, x0, p1, p2, grid, nullptr, MORTON_BITS, keys[0], vals[0]);
    else if (dim == 2) k_keys<2><<<gb, 256, 0, s>>>(n, x0, p1, p2, grid, nullptr, MORTON_BITS, keys[0], vals[0]);
    else k_keys<1><<<gb, 256, 0, s>>>(n, x0, p1, p2, grid, nullptr, MORTON_BITS, keys[0], vals[0]);
    int64_t nblocks = (n + RS_TILE - 1) / RS_TILE;
    int cur = 0;
    for (int sh = lo_bit; sh < hi_bit; sh += RS_BITS) {
        k_rs_upsweep<<<(unsigned)nblocks, RS_THREADS, 0, s>>>(n, keys[cur], sh, hist, nblocks);
        k_rs_scan<<<RS_BINS, 1024, 0, s>>>(hist, nblocks, hist + RS_BINS * nblocks);
        k_rs_downsweep<<<(unsigned)nblocks, RS_THREADS, 0, s>>>(n, keys[cur], vals[cur], keys[cur ^ 1],
                                                                vals[cur ^ 1], sh, hist, hist + RS_BINS * nblocks, nblocks);
        cur ^= 1;
    }
    k_copy_sorted<<<gb, 256, 0, s>>>(n, keys[cur], vals[cur], keys_out, perm_out);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}
