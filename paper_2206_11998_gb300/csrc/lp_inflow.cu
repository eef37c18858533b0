// lp_inflow.cu -- reservoir inflow through a nozzle inlet (Sec. 4, the nozzle
// inlet boundary condition of the supersonic-jet simulations): the inflow
// state from the mean pressure near the inlet, the reservoir's entropy and
// the enthalpy balance, and the insertion of whole lattice layers of
// particles (Sec. 2.2 step 1: inflow boundaries generate particles).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int IN_BLOCKS = 304;        // sampling blocks: the partial sums are reduced in this order
constexpr int IN_THREADS = 256;
constexpr int IN_LMAX = 64;           // layers one call may append
// device state: committed [0, 8), next [8, 16)
enum { S_TRAVEL = 0, S_LAYERS, S_STARTED, S_P, S_RHO, S_U, S_HZ, S_L, S_NEXT = 8, S_SAMPLED = 16, S_WORDS = 17 };

struct InGeom {
    double c[3];
    int ax, e1, e2;
    double R2, depth;
};

__device__ inline double axial(const InGeom& g, const double (&x)[3]) { return x[g.ax] - g.c[g.ax]; }

// per block: sum of P and count of the fluid particles near the inlet
__global__ void k_inflow_sample(int64_t n, InGeom g, int64_t n_fluid, const double* x0, const double* x1,
                                const double* x2, const double* P, const uint32_t* id, double* part)
{
    __shared__ double ss[IN_THREADS], sc[IN_THREADS];
    double s = 0.0, cnt = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if ((int64_t)id[i] >= n_fluid) continue;
        const double x[3] = {x0[i], x1[i], x2[i]};
        const double a = axial(g, x);
        if (!(a >= 0.0 && a <= g.depth)) continue;
        const double d1 = x[g.e1] - g.c[g.e1], d2 = x[g.e2] - g.c[g.e2];
        if (d1 * d1 + d2 * d2 > g.R2) continue;
        s += P[i];
        cnt += 1.0;
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = cnt;
    __syncthreads();
    for (int h = IN_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            ss[threadIdx.x] += ss[threadIdx.x + h];
            sc[threadIdx.x] += sc[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ss[0];
        part[2 * blockIdx.x + 1] = sc[0];
    }
}

// one thread: P_inf, the reservoir's isentrope and enthalpy balance, the
// layers this call appends -- into the "next" half of the state
__global__ void k_inflow_state(const double* part, lp_inlet in, double gamma, const double* dt_dev, double* st)
{
    double S = 0.0, C = 0.0;
    for (int b = 0; b < IN_BLOCKS; ++b) { S += part[2 * b]; C += part[2 * b + 1]; }
    const bool started = st[S_STARTED] != 0.0;
    const double P = (started && C > 0.0) ? S / C : in.P_res;       // first call: the reservoir pressure
    const double rho = in.rho_res * pow(P / in.P_res, 1.0 / gamma);  // P_res / rho_res^g = P / rho^g
    const double c2 = gamma * P / rho, c2r = gamma * in.P_res / in.rho_res;
    const double w = 2.0 / (gamma - 1.0) * (c2r - c2);               // u^2 from the enthalpy balance
    const double u = w > 0.0 ? sqrt(w) : 0.0;
    const double hz = in.mass / (rho * in.spacing * in.spacing);
    const double dt = started ? dt_dev[0] : 0.0;
    double travel = st[S_TRAVEL] + u * dt;
    double L = floor(travel / hz);
    if (!(L >= 0.0)) L = 0.0;
    if (L > (double)IN_LMAX) L = (double)IN_LMAX;
    travel -= L * hz;
    if (travel < 0.0) travel = 0.0;
    st[S_NEXT + S_TRAVEL] = travel;
    st[S_NEXT + S_LAYERS] = st[S_LAYERS] + L;
    st[S_NEXT + S_STARTED] = 1.0;
    st[S_NEXT + S_P] = P;
    st[S_NEXT + S_RHO] = rho;
    st[S_NEXT + S_U] = u;
    st[S_NEXT + S_HZ] = hz;
    st[S_NEXT + S_L] = L;
    st[S_SAMPLED] = C;
}

__global__ void k_inflow_commit(double* st)
{
    const int q = threadIdx.x;
    if (q < 8) st[q] = st[S_NEXT + q];
}

// in-plane shift of global layer gl: a Weyl sequence, in (-spacing/2, spacing/2]
__device__ inline void layer_shift(double gl, double h, double& s1, double& s2)
{
    const double a = gl * 0.6180339887498949, b = gl * 0.7548776662466927;
    s1 = (a - floor(a) - 0.5) * h;
    s2 = (b - floor(b) - 0.5) * h;
}

// a particle of layer gl at axial offset d (negative behind the inlet)
__device__ inline void place(const InGeom& g, const double* pat, int64_t k, double gl, double d, double h,
                             double (&x)[3])
{
    double s1, s2;
    layer_shift(gl, h, s1, s2);
    x[g.ax] = g.c[g.ax] + d;
    x[g.e1] = g.c[g.e1] + pat[2 * k] + s1;
    x[g.e2] = g.c[g.e2] + pat[2 * k + 1] + s2;
}

// appends the fluid layers of this call (the layer that entered first is the
// farthest from the inlet) and, on the first call, the reservoir ghosts
__global__ void k_inflow_insert(lp_particles p, int64_t n0, InGeom g, lp_inlet in, const double* pat, int64_t npat,
                                int64_t nfl, int64_t nghost, const double* st)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nfl + nghost) return;
    const double* nx = st + S_NEXT;
    const double L = nx[S_L], travel = nx[S_TRAVEL], hz = nx[S_HZ], layers_new = nx[S_LAYERS];
    double x[3];
    uint32_t id;
    if (q < nfl) {
        const int64_t l = q / npat, k = q % npat;           // l = 0: nearest the inlet
        const double gl = layers_new - 1.0 - (double)l;
        place(g, pat, k, gl, travel + (double)l * hz, in.spacing, x);
        id = in.first_id + (uint32_t)((int64_t)gl * npat + k);
    } else {
        const int64_t r = q - nfl, gg = r / npat, k = r % npat;
        place(g, pat, k, layers_new + (double)gg, travel - (double)(gg + 1) * hz, in.spacing, x);
        id = in.ghost_id + (uint32_t)(gg * npat + k);
    }
    (void)L;
    const int64_t i = n0 + q;
    p.x[0][i] = x[0];
    p.x[1][i] = x[1];
    p.x[2][i] = x[2];
    p.V[i] = 1.0 / nx[S_RHO];
    p.u[g.ax][i] = nx[S_U];
    p.u[g.e1][i] = 0.0;
    p.u[g.e2][i] = 0.0;
    p.P[i] = nx[S_P];
    p.m[i] = in.mass;
    p.id[i] = id;
}

// rewrites the reservoir ghosts already in the arrays (found by id) with this
// call's inflow state, behind the inlet
__global__ void k_inflow_ghosts(lp_particles p, InGeom g, lp_inlet in, const double* pat, int64_t npat, int64_t nghost,
                                const double* st)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const uint32_t id = p.id[i];
    if (id < in.ghost_id || (int64_t)(id - in.ghost_id) >= nghost) return;
    const double* nx = st + S_NEXT;
    const int64_t r = (int64_t)(id - in.ghost_id), gg = r / npat, k = r % npat;
    double x[3];
    place(g, pat, k, nx[S_LAYERS] + (double)gg, nx[S_TRAVEL] - (double)(gg + 1) * nx[S_HZ], in.spacing, x);
    p.x[0][i] = x[0];
    p.x[1][i] = x[1];
    p.x[2][i] = x[2];
    p.V[i] = 1.0 / nx[S_RHO];
    p.u[g.ax][i] = nx[S_U];
    p.u[g.e1][i] = 0.0;
    p.u[g.e2][i] = 0.0;
    p.P[i] = nx[S_P];
}

bool same_inlet(const lp_inlet& a, const lp_inlet& b) { return memcmp(&a, &b, sizeof(lp_inlet)) == 0; }

constexpr int RM_BLOCK = 1024;          // particles per block of the outflow compaction

// what stays: inside the box (when `box`), and with id < id_end
struct Box { double lo[3], hi[3]; int dim; int box; uint32_t id_end; };

__device__ inline bool keeps(const Box& b, const lp_particles& p, int64_t i)
{
    if (p.id[i] >= b.id_end) return false;
    if (!b.box) return true;
    for (int k = 0; k < b.dim; ++k) {
        const double x = p.x[k][i];
        if (!(x >= b.lo[k] && x <= b.hi[k])) return false;     // also drops NaN
    }
    return true;
}

// per block of RM_BLOCK particles: how many stay
__global__ void k_rm_count(lp_particles p, Box b, uint32_t* bc)
{
    __shared__ uint32_t s[RM_BLOCK / 32];
    const int64_t i = blockIdx.x * (int64_t)RM_BLOCK + threadIdx.x;
    const bool k = i < p.n && keeps(b, p, i);
    const unsigned m = __ballot_sync(0xffffffffu, k);
    if ((threadIdx.x & 31u) == 0) s[threadIdx.x >> 5] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < RM_BLOCK / 32; ++w) t += s[w];
        bc[blockIdx.x] = t;
    }
}

// exclusive prefix of the block counts, in order (one block)
__global__ void k_rm_scan(int64_t nb, uint32_t* bc, unsigned long long* total)
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

// the particles that stay, to the scratch copies in their order
__global__ void k_rm_scatter(lp_particles p, Box b, const uint32_t* bc, lp_particles out)
{
    __shared__ uint32_t s[RM_BLOCK / 32];
    const int64_t i = blockIdx.x * (int64_t)RM_BLOCK + threadIdx.x;
    const bool k = i < p.n && keeps(b, p, i);
    const unsigned m = __ballot_sync(0xffffffffu, k);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s[w] = __popc(m);
    __syncthreads();
    if (!k) return;
    uint32_t off = bc[blockIdx.x];
    for (int q = 0; q < w; ++q) off += s[q];
    const int64_t o = off + __popc(m & ((1u << lane) - 1u));
    for (int d = 0; d < b.dim; ++d) { out.x[d][o] = p.x[d][i]; out.u[d][o] = p.u[d][i]; }
    out.V[o] = p.V[i];
    out.P[o] = p.P[i];
    out.m[o] = p.m[i];
    out.id[o] = p.id[i];
}

__global__ void k_rm_copyback(int64_t n, int dim, lp_particles from, lp_particles p)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int d = 0; d < dim; ++d) { p.x[d][i] = from.x[d][i]; p.u[d][i] = from.u[d][i]; }
    p.V[i] = from.V[i];
    p.P[i] = from.P[i];
    p.m[i] = from.m[i];
    p.id[i] = from.id[i];
}

}  // namespace
}  // namespace lp

using namespace lp;

extern "C" lp_status lp_inflow(lp_ctx* c, lp_particles* p, int64_t capacity, const lp_inlet* in, int64_t* n_out,
                               lp_inflow_info* info, lp_stream stream)
{
    if (!c || !p || !in || !n_out || c->dc.dim != 3 || c->dc.nsim_max > 1) return LP_ERR_ARG;
    if (in->axis < 0 || in->axis > 2 || in->ghost_layers < 0 || !(in->radius > 0.0) || !(in->spacing > 0.0) ||
        !(in->mass > 0.0) || !(in->P_res > 0.0) || !(in->rho_res > 0.0) || !(in->sample_depth >= 0.0))
        return LP_ERR_ARG;
    if ((int64_t)in->ghost_id < c->dc.n_fluid && in->ghost_layers > 0) return LP_ERR_ARG;
    if (p->n < 0 || capacity < p->n) return LP_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        if (!p->x[k] || !p->u[k]) return LP_ERR_ARG;
    if (!p->V || !p->P || !p->m || !p->id) return LP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->in_pattern) {
        // the layer's lattice: cell centres of a square lattice within the disk
        const int h = (int)ceil(in->radius / in->spacing);
        double* pat = (double*)malloc(sizeof(double) * 2 * (size_t)(2 * h + 1) * (size_t)(2 * h + 1));
        if (!pat) return LP_ERR_CUDA;
        int64_t np = 0;
        for (int a = -h; a < h; ++a)
            for (int b = -h; b < h; ++b) {
                const double u = (a + 0.5) * in->spacing, v = (b + 0.5) * in->spacing;
                if (u * u + v * v <= in->radius * in->radius) { pat[2 * np] = u; pat[2 * np + 1] = v; ++np; }
            }
        if (np == 0) { free(pat); return LP_ERR_ARG; }
        cudaError_t e = cudaMalloc(&c->in_pattern, sizeof(double) * 2 * np);
        if (e == cudaSuccess) e = cudaMemcpy(c->in_pattern, pat, sizeof(double) * 2 * np, cudaMemcpyHostToDevice);
        free(pat);
        if (e == cudaSuccess) e = cudaMalloc(&c->in_state, sizeof(double) * S_WORDS);
        if (e == cudaSuccess) e = cudaMemset(c->in_state, 0, sizeof(double) * S_WORDS);
        if (e == cudaSuccess) e = cudaMalloc(&c->in_part, sizeof(double) * 2 * IN_BLOCKS);
        if (e != cudaSuccess) return LP_ERR_CUDA;
        c->in_npat = np;
        c->in_cfg = *in;
    } else if (!same_inlet(c->in_cfg, *in)) {
        return LP_ERR_ARG;
    }
    InGeom g;
    for (int k = 0; k < 3; ++k) g.c[k] = in->center[k];
    g.ax = in->axis;
    g.e1 = (in->axis + 1) % 3;
    g.e2 = (in->axis + 2) % 3;
    g.R2 = in->radius * in->radius;
    g.depth = in->sample_depth;
    k_inflow_sample<<<IN_BLOCKS, IN_THREADS, 0, s>>>(p->n, g, c->dc.n_fluid, p->x[0], p->x[1], p->x[2], p->P, p->id,
                                                    c->in_part);
    k_inflow_state<<<1, 1, 0, s>>>(c->in_part, *in, c->dc.gamma, c->dt_dev, c->in_state);
    double hs[S_WORDS];
    if (cudaMemcpyAsync(hs, c->in_state, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LP_ERR_CUDA;
    c->launches += 2;
    const int64_t np = c->in_npat;
    const int64_t L = (int64_t)hs[S_NEXT + S_L];
    const int64_t nghost = (int64_t)in->ghost_layers * np;
    const int64_t nfl = L * np, nadd = nfl + (c->in_ghosts ? 0 : nghost);
    if (info) {
        info->P_inf = hs[S_NEXT + S_P];
        info->rho_inf = hs[S_NEXT + S_RHO];
        info->u_inf = hs[S_NEXT + S_U];
        info->c_inf = sqrt(c->dc.gamma * info->P_inf / info->rho_inf);
        info->h_z = hs[S_NEXT + S_HZ];
        info->travel = hs[S_NEXT + S_TRAVEL];
        info->layers = L;
        info->layers_total = (int64_t)hs[S_NEXT + S_LAYERS];
        info->npat = np;
        info->sampled = (int64_t)hs[S_SAMPLED];
    }
    if (p->n + nadd > capacity) return LP_ERR_CAPACITY;       // nothing appended, the state not advanced
    if (c->in_ghosts && nghost > 0 && p->n > 0) {
        k_inflow_ghosts<<<(unsigned)((p->n + 255) / 256), 256, 0, s>>>(*p, g, *in, c->in_pattern, np, nghost,
                                                                       c->in_state);
        c->launches += 1;
    }
    if (nadd > 0) {
        k_inflow_insert<<<(unsigned)((nadd + 255) / 256), 256, 0, s>>>(*p, p->n, g, *in, c->in_pattern, np, nfl,
                                                                       c->in_ghosts ? 0 : nghost, c->in_state);
        c->launches += 1;
    }
    k_inflow_commit<<<1, 32, 0, s>>>(c->in_state);
    c->launches += 1;
    if (cudaGetLastError() != cudaSuccess) return LP_ERR_CUDA;
    c->in_ghosts = 1;
    *n_out = p->n + nadd;
    return LP_OK;
}

namespace {

// delete the particles b does not keep, keeping the order of the others
lp_status remove_where(lp_ctx* c, lp_particles* p, const Box& b, int64_t* n_out, cudaStream_t s)
{
    const int dim = c->dc.dim;
    const int64_t nb = (p->n + RM_BLOCK - 1) / RM_BLOCK;
    // scratch: block offsets in the redo list, the copies in the sorted state
    uint32_t* bc = c->redo_list;
    unsigned long long* total = c->counters + C_REDO_LEN;
    lp_particles tmp;
    memset(&tmp, 0, sizeof(tmp));
    for (int k = 0; k < dim; ++k) { tmp.x[k] = c->sx[k]; tmp.u[k] = c->su[k]; }
    tmp.V = c->sV; tmp.P = c->sP; tmp.m = c->sm; tmp.id = c->sid;
    k_rm_count<<<(unsigned)nb, RM_BLOCK, 0, s>>>(*p, b, bc);
    k_rm_scan<<<1, 32, 0, s>>>(nb, bc, total);
    k_rm_scatter<<<(unsigned)nb, RM_BLOCK, 0, s>>>(*p, b, bc, tmp);
    unsigned long long kept = 0;
    if (cudaMemcpyAsync(&kept, total, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return LP_ERR_CUDA;
    if (kept > 0)
        k_rm_copyback<<<(unsigned)((kept + 255) / 256), 256, 0, s>>>((int64_t)kept, dim, tmp, *p);
    c->launches += kept > 0 ? 4 : 3;
    if (cudaGetLastError() != cudaSuccess) return LP_ERR_CUDA;
    c->lists_stale = 1;          // the lists and sorted copies no longer describe p
    *n_out = (int64_t)kept;
    return LP_OK;
}

lp_status check_removal_args(const lp_ctx* c, const lp_particles* p)
{
    if (p->n > c->cap) return LP_ERR_CAPACITY;
    for (int k = 0; k < c->dc.dim; ++k)
        if (!p->x[k] || !p->u[k]) return LP_ERR_ARG;
    if (!p->V || !p->P || !p->m || !p->id) return LP_ERR_ARG;
    return LP_OK;
}

}  // namespace

extern "C" lp_status lp_remove_ghosts(lp_ctx* c, lp_particles* p, uint32_t first_id, int64_t* n_out, lp_stream stream)
{
    if (!c || !p || !n_out || p->n < 0 || c->dc.nsim_max > 1) return LP_ERR_ARG;
    lp_status st = check_removal_args(c, p);
    if (st != LP_OK) return st;
    *n_out = p->n;
    if (p->n == 0) return LP_OK;
    Box b;
    memset(&b, 0, sizeof(b));
    b.dim = c->dc.dim;
    b.box = 0;
    b.id_end = first_id;
    return remove_where(c, p, b, n_out, (cudaStream_t)stream);
}

extern "C" lp_status lp_remove_outside(lp_ctx* c, lp_particles* p, const double* lo, const double* hi, int64_t* n_out,
                                       lp_stream stream)
{
    if (!c || !p || !lo || !hi || !n_out || p->n < 0 || c->dc.nsim_max > 1) return LP_ERR_ARG;
    lp_status st = check_removal_args(c, p);
    if (st != LP_OK) return st;
    *n_out = p->n;
    if (p->n == 0) return LP_OK;
    Box b;
    memset(&b, 0, sizeof(b));
    b.dim = c->dc.dim;
    b.box = 1;
    b.id_end = 0xffffffffu;
    for (int k = 0; k < 3; ++k) { b.lo[k] = lo[k]; b.hi[k] = hi[k]; }
    return remove_where(c, p, b, n_out, (cudaStream_t)stream);
}
