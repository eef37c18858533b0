// lp_ghosts.cu -- free-surface ghost particles (Sec. 2.2 step 3: where the
// free boundary condition applies and a particle's neighbours are incomplete
// in some of the six axis directions, ghost particles complete them).  The
// paper defers their placement and state; this build's reading: a direction
// (k, side) of a fluid particle is incomplete when fewer than min_per_side
// members of its list lie strictly on that side along axis k; its ghost sits
// one nearest-neighbour distance away along that axis with the particle's
// mass, specific volume and velocity and a given pressure (0: vacuum).
#include <string.h>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int GH_BLOCK = 256;

struct GhostArgs {
    int64_t n;
    int dim, k_max, min_per_side;
    int64_t n_fluid;
    const uint32_t* count;
    const uint32_t* idx;
    const double* d2min;
    DevCfg c;
    double p_ghost;
    uint32_t ghost_base;
};

// bit 2k + side: direction (axis k, side - or +) of particle i is incomplete
__device__ inline uint32_t incomplete_dirs(const GhostArgs& g, const lp_particles& p, int64_t i)
{
    if ((int64_t)p.id[i] >= g.n_fluid) return 0u;
    const uint32_t cnt = g.count[i];
    if (cnt == 0) return 0u;                     // no neighbour: no stencil to complete
    uint32_t dirs = 0u;
    for (int k = 0; k < g.dim; ++k) {
        int neg = 0, pos = 0;
        for (uint32_t t = 0; t < cnt; ++t) {
            const int64_t j = g.idx[i * (int64_t)g.k_max + t];
            const double dx = offset64(g.c, k, p.x[k][i], p.x[k][j]);
            neg += dx < 0.0 ? 1 : 0;
            pos += dx > 0.0 ? 1 : 0;
        }
        if (neg < g.min_per_side) dirs |= 1u << (2 * k);
        if (pos < g.min_per_side) dirs |= 1u << (2 * k + 1);
    }
    return dirs;
}

// the directions of every particle (to dirs) and the ghosts of each block
__global__ void k_ghost_count(GhostArgs g, lp_particles p, uint32_t* dirs, uint32_t* bc)
{
    __shared__ uint32_t s[GH_BLOCK / 32];
    const int64_t i = blockIdx.x * (int64_t)GH_BLOCK + threadIdx.x;
    uint32_t d = 0;
    if (i < g.n) {
        d = incomplete_dirs(g, p, i);
        dirs[i] = d;
    }
    uint32_t c = (uint32_t)__popc(d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31u) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < GH_BLOCK / 32; ++w) t += s[w];
        bc[blockIdx.x] = t;
    }
}

// exclusive prefix of the block counts, in order (one thread)
__global__ void k_ghost_scan(int64_t nb, uint32_t* bc, unsigned long long* total)
{
    if (threadIdx.x != 0) return;
    unsigned long long run = 0;
    for (int64_t q = 0; q < nb; ++q) {
        const uint32_t c = bc[q];
        bc[q] = (uint32_t)run;
        run += c;
    }
    *total = run;
}

// the ghosts, after the n particles, in (particle, axis, side) order
__global__ void k_ghost_write(GhostArgs g, lp_particles p, const uint32_t* dirs, const uint32_t* bc)
{
    __shared__ uint32_t s[GH_BLOCK / 32];
    const int64_t i = blockIdx.x * (int64_t)GH_BLOCK + threadIdx.x;
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t d = i < g.n ? dirs[i] : 0u;
    const uint32_t c = (uint32_t)__popc(d);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += v;
    }
    if (lane == 31u) s[w] = incl;
    __syncthreads();
    if (d == 0u) return;
    uint32_t off = bc[blockIdx.x] + incl - c;
    for (unsigned q = 0; q < w; ++q) off += s[q];
    const double ell = __dsqrt_rn(g.d2min[i]);
    int64_t o = g.n + (int64_t)off;
    for (int k = 0; k < g.dim; ++k)
        for (int side = 0; side < 2; ++side) {
            if (!((d >> (2 * k + side)) & 1u)) continue;
            for (int a = 0; a < g.dim; ++a) {
                p.x[a][o] = p.x[a][i];
                p.u[a][o] = p.u[a][i];
            }
            p.x[k][o] = side ? __dadd_rn(p.x[k][i], ell) : __dsub_rn(p.x[k][i], ell);
            p.V[o] = p.V[i];
            p.P[o] = g.p_ghost;
            p.m[o] = p.m[i];
            p.id[o] = g.ghost_base + (uint32_t)(2 * g.dim) * p.id[i] + (uint32_t)(2 * k + side);
            ++o;
        }
}

}  // namespace
}  // namespace lp

using namespace lp;

extern "C" lp_status lp_free_surface_ghosts(lp_ctx* c, lp_particles* p, int64_t capacity, int32_t min_per_side,
                                            double p_ghost, uint32_t ghost_base, int64_t* n_out, lp_stream stream)
{
    if (!c || !p || !n_out || c->dc.nsim_max > 1) return LP_ERR_ARG;
    const int dim = c->dc.dim;
    for (int k = 0; k < dim; ++k)
        if (c->dc.periodic[k]) return LP_ERR_ARG;               // no free surface in a periodic box
    if (min_per_side < 1 || min_per_side > c->dc.k_max || !(p_ghost >= 0.0) || !isfinite(p_ghost)) return LP_ERR_ARG;
    // ghosts must be frozen (ids >= n_fluid) and their ids must fit in 32 bits
    if ((int64_t)ghost_base < c->dc.n_fluid ||
        (uint64_t)ghost_base + (uint64_t)(2 * dim) * (uint64_t)c->dc.n_fluid > 0x100000000ull)
        return LP_ERR_ARG;
    if (p->n < 0 || capacity < p->n || capacity > c->cap) return LP_ERR_CAPACITY;
    *n_out = p->n;
    lp_neighbors nb;
    lp_status st = lp_build_neighbors(c, p, &nb, stream);      // p is now in key order, with its lists
    if (st != LP_OK) return st;
    if (p->n == 0) return LP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    GhostArgs g;
    g.n = p->n;
    g.dim = dim;
    g.k_max = c->dc.k_max;
    g.min_per_side = min_per_side;
    g.n_fluid = c->dc.n_fluid;
    g.count = c->nb_count;
    g.idx = c->nb_idx;
    g.d2min = c->nb_d2min;
    g.c = c->dc;
    g.p_ghost = p_ghost;
    g.ghost_base = ghost_base;
    // scratch: directions in the redo list, block offsets in the plain list
    uint32_t* dirs = c->redo_list;
    uint32_t* bc = c->plain_list;
    unsigned long long* total = c->counters + C_REDO_LEN;
    const int64_t nb_ = (p->n + GH_BLOCK - 1) / GH_BLOCK;
    k_ghost_count<<<(unsigned)nb_, GH_BLOCK, 0, s>>>(g, *p, dirs, bc);
    k_ghost_scan<<<1, 32, 0, s>>>(nb_, bc, total);
    unsigned long long ng = 0;
    if (cudaMemcpyAsync(&ng, total, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LP_ERR_CUDA;
    c->launches += 2;
    if (p->n + (int64_t)ng > capacity) return LP_ERR_CAPACITY;   // nothing appended
    if (ng > 0) {
        k_ghost_write<<<(unsigned)nb_, GH_BLOCK, 0, s>>>(g, *p, dirs, bc);
        c->launches += 1;
    }
    if (cudaGetLastError() != cudaSuccess) return LP_ERR_CUDA;
    c->lists_stale = 1;          // the lists do not include the ghosts
    *n_out = p->n + (int64_t)ng;
    return LP_OK;
}
