// lp_fit.cuh -- GFD least-squares fits and the LP update (Sec. 2.1), as
// templates instantiated for FP32 (lp_fit_f32.cu, lp_fit_f32_refine.cu) and
// FP64 (lp_fit_f64.cu).
//
// Schedule: one thread per particle; no stencil is staged and no lane idles.
// The overdetermined GFD system of Sec. 2.1 (and its 1D/3D analogues) is
// solved in one of two forms, both with the factor, the right-hand sides of
// all fields and the running row in registers:
//  * FP32 central fit: the normal equations A^T [A | B], accumulated row by row
//    as the neighbours stream in (paired products in packed FP32 FMAs), factored
//    as U^T D U (square-root-free Cholesky).  Their error grows as cond(A)^2, so
//    where the factor's diagonal ratio is below refine_ratio one correction step
//    (semi-normal equations on the residual) follows, and below 0.02 the rows are
//    streamed again through the rotations below instead.
//  * FP64 fits, the FP32 fallback and every one-sided fit: square-root-free
//    Givens rotations applied row by row, which leave the same U^T D U form.
// Offsets are scaled by a power of two (exact) so the factor is well scaled;
// min|R_kk|/max|R_kk| decides the FP64 redo (FP32) or the first-order fallback
// (FP64).  The FP32 path forms offsets and field differences from split
// (hi, lo) floats, accurate to a few ulp of the offset itself.
#pragma once

#include "lp_internal.cuh"
#include "lp_mlp.cuh"

namespace lp {

template <int DIM> struct NU { static constexpr int v = DIM == 1 ? 2 : (DIM == 2 ? 5 : 9); };

// threads per block of every fit kernel (the FP32 correction pass keeps one
// shared-memory column per thread)
constexpr int FIT_THREADS = 128;

// Explicit round-to-nearest operations.  The fit and rate arithmetic is inlined
// into more than one kernel (fused and split schedules, the FP64 redo); with
// explicit operations the compiler cannot contract a*b + c into an FMA in one
// kernel and not in another, so every schedule produces the same bits.
template <typename T> struct RN;
template <> struct RN<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    // the hardware reciprocal (a few ulp), as fast as the square root it replaces
    static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.0f, a); }
};
template <> struct RN<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
};


// ---------------------------------------------------------------------------
// row-by-row Givens least squares:  min || A x - B ||, A: rows x N, B: rows x F
// ---------------------------------------------------------------------------
template <typename T, int N, int F>
struct Givens {
    // Square-root-free Givens rotations (Gentleman's form): R = D^{1/2} U with U
    // unit upper triangular and Q^T B = D^{1/2} Z.  A row (a, b) of weight w,
    // starting at 1, enters column k as
    //   d' = d_k + w a_k^2,  c = d_k / d',  s = w a_k / d',  w' = w c,
    //   t = a_l - a_k U_kl,  U_kl' = c U_kl + s a_l,  a_l' = t    (l > k; b likewise)
    // -- no square root.  U_kl' is the weighted mean of U_kl and a_l / a_k, not
    // U_kl + s t: that shorter form cancels catastrophically when a row much
    // larger than the column's previous rows meets a column built from tiny
    // ones (c near 0, U_kl huge), which drifted lattices produce (offsets of
    // 1e-17 where the lattice had exact zeros).  The row's remaining weight w
    // times its leftover b^2 is its share of the residual sum of squares.
    T d[N];
    T U[N * (N - 1) / 2 + 1];   // strict upper part of U, row by row
    T Z[N][F];

    __device__ static constexpr int id(int k, int l) { return k * (N - 1) - (k * (k - 1)) / 2 + (l - k - 1); }

    __device__ void zero()
    {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = T(0);
#pragma unroll
        for (int q = 0; q < N * (N - 1) / 2 + 1; ++q) U[q] = T(0);
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
            for (int f = 0; f < F; ++f) Z[k][f] = T(0);
    }

    // rotates the row in; returns its remaining weight
    __device__ T add(T (&a)[N], T (&b)[F])
    {
        using O = RN<T>;
        T w = T(1);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T ak = a[k];
            const T wa = O::mul(w, ak);
            const T dn = O::fma(wa, ak, d[k]);
            // a row absorbed by an empty column keeps weight 0 (live = false: no change)
            const bool live = wa != T(0) && dn > T(0);
            const T inv = live ? O::rcp(dn) : T(0);
            const T sk = O::mul(wa, inv);                     // 0 when not live
            const T ck = live ? O::mul(d[k], inv) : T(1);     // 1 when not live: U, Z unchanged
            w = O::mul(w, ck);
            d[k] = live ? dn : d[k];
#pragma unroll
            for (int l = k + 1; l < N; ++l) {
                const T t = O::fma(-ak, U[id(k, l)], a[l]);
                U[id(k, l)] = O::fma(ck, U[id(k, l)], O::mul(sk, a[l]));
                a[l] = t;
            }
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const T t = O::fma(-ak, Z[k][f], b[f]);
                Z[k][f] = O::fma(ck, Z[k][f], O::mul(sk, b[f]));
                b[f] = t;
            }
        }
        return w;
    }

    // min |R_kk| / max |R_kk| = sqrt(min d_k / max d_k)
    __device__ T ratio() const
    {
        T lo = d[0], hi = d[0];
#pragma unroll
        for (int k = 1; k < N; ++k) {
            lo = d[k] < lo ? d[k] : lo;
            hi = d[k] > hi ? d[k] : hi;
        }
        return hi > T(0) ? sqrt(RN<T>::div(lo, hi)) : T(0);
    }

    // x = R^{-1} Q^T B = U^{-1} Z
    __device__ void solve(T (&x)[N][F]) const
    {
        using O = RN<T>;
#pragma unroll
        for (int k = N - 1; k >= 0; --k) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                T s = Z[k][f];
#pragma unroll
                for (int l = k + 1; l < N; ++l) s = O::fma(-U[id(k, l)], x[l][f], s);
                x[k][f] = s;
            }
        }
    }

    // g <- (R^T R)^{-1} g = U^{-1} D^{-1} U^{-T} g  (one correction step of the
    // semi-normal equations)
    __device__ void solve_normal(T (&g)[N][F]) const
    {
        using O = RN<T>;
#pragma unroll
        for (int k = 0; k < N; ++k)           // U^T y = g (unit lower triangular)
#pragma unroll
            for (int f = 0; f < F; ++f) {
                T s = g[k][f];
#pragma unroll
                for (int l = 0; l < k; ++l) s = O::fma(-U[id(l, k)], g[l][f], s);
                g[k][f] = s;
            }
#pragma unroll
        for (int k = 0; k < N; ++k) {         // y <- D^{-1} y
            const T inv = O::rcp(d[k]);
#pragma unroll
            for (int f = 0; f < F; ++f) g[k][f] = O::mul(g[k][f], inv);
        }
#pragma unroll
        for (int k = N - 1; k >= 0; --k)      // U x = y
#pragma unroll
            for (int f = 0; f < F; ++f) {
                T s = g[k][f];
#pragma unroll
                for (int l = k + 1; l < N; ++l) s = O::fma(-U[id(k, l)], g[l][f], s);
                g[k][f] = s;
            }
    }
};

// Normal equations of the same least-squares problem, accumulated row by row:
// the Gram matrix A^T A (upper triangle) and A^T B -- one FMA per element and
// row, against two for a rotation.  factor() turns the Gram matrix into the
// form the Givens factor has (A^T A = U^T D U, U unit upper triangular), so
// the ratio, the semi-normal solves and the correction pass are shared; the
// factor it gives is R^T R of the same R up to rounding, accurate to about
// cond(A)^2 u relative, which the correction pass then removes.
template <typename T, int N, int F>
struct NormalEq {
    T Gm[N * (N + 1) / 2];      // upper triangle of A^T A, row by row
    T c[N][F];                  // A^T B

    __device__ static constexpr int id(int k, int l) { return k * N - (k * (k - 1)) / 2 + (l - k); }

    __device__ void zero()
    {
#pragma unroll
        for (int q = 0; q < N * (N + 1) / 2; ++q) Gm[q] = T(0);
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
            for (int f = 0; f < F; ++f) c[k][f] = T(0);
    }

    __device__ void add(const T (&a)[N], const T (&b)[F])
    {
        using O = RN<T>;
#pragma unroll
        for (int k = 0; k < N; ++k) {
#pragma unroll
            for (int l = k; l < N; ++l) Gm[id(k, l)] = O::fma(a[k], a[l], Gm[id(k, l)]);
#pragma unroll
            for (int f = 0; f < F; ++f) c[k][f] = O::fma(a[k], b[f], c[k][f]);
        }
    }

    // A^T A = U^T D U by rows (square-root-free Cholesky); a pivot that is not
    // positive leaves d_k = 0, which the ratio test then rejects
    template <int NF>
    __device__ void factor(Givens<T, N, NF>& G)
    {
        using O = RN<T>;
        T inv[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            // row k of D U: Gm[k][l] - sum_{j<k} U_jk (D U)_jl, with U_jk = (D U)_jk / d_j
#pragma unroll
            for (int j = 0; j < k; ++j) {
                const T ujk = O::mul(Gm[id(j, k)], inv[j]);
#pragma unroll
                for (int l = k; l < N; ++l) Gm[id(k, l)] = O::fma(-ujk, Gm[id(j, l)], Gm[id(k, l)]);
            }
            const T dk = Gm[id(k, k)];
            const bool pos = dk > T(0);
            G.d[k] = pos ? dk : T(0);
            inv[k] = pos ? O::rcp(dk) : T(0);
        }
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
            for (int l = k + 1; l < N; ++l) G.U[Givens<T, N, NF>::id(k, l)] = O::mul(Gm[id(k, l)], inv[k]);
    }
};

// The FP32 normal equations of NormalEq, accumulated two values per packed
// FP32 instruction (__ffma2_rn: per component the same rounding as __fmaf_rn,
// so the sums are bit for bit those of NormalEq::add).  Row k of A^T [A | B]
// is a[k] times v = (a_0 .. a_{N-1}, b_0 .. b_{F-1}) from v_k on; v is held
// in VP aligned pairs, and row k accumulates the pairs from k / 2 on, so an
// odd row also sums the product with v_{k-1}, which is not used.
template <int N, int F>
struct NormalEqPacked {
    static constexpr int L = N + F;                  // values of v
    static constexpr int VP = (L + 1) / 2;           // pairs (the last one padded when L is odd)
    static constexpr int off(int k)                  // first pair of row k in P
    {
        int o = 0;
        for (int r = 0; r < k; ++r) o += VP - r / 2;
        return o;
    }
    static constexpr int NP = off(N);
    float2 P[NP];

    __device__ void zero()
    {
#pragma unroll
        for (int q = 0; q < NP; ++q) P[q] = make_float2(0.0f, 0.0f);
    }

    __device__ void add(const float (&a)[N], const float (&b)[F])
    {
        float2 v[VP];
#pragma unroll
        for (int p = 0; p < VP; ++p) {
            const int j0 = 2 * p, j1 = 2 * p + 1;
            const float x = j0 < N ? a[j0 < N ? j0 : 0] : b[j0 < N ? 0 : (j0 - N < F ? j0 - N : 0)];
            const float y = j1 < N ? a[j1 < N ? j1 : 0] : (j1 - N < F ? b[j1 < N ? 0 : (j1 - N < F ? j1 - N : 0)] : 0.0f);
            v[p] = make_float2(x, y);
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float2 ak = make_float2(a[k], a[k]);
#pragma unroll
            for (int p = k / 2; p < VP; ++p) P[off(k) + p - k / 2] = __ffma2_rn(ak, v[p], P[off(k) + p - k / 2]);
        }
    }

    // value j (>= k) of row k
    __device__ float at(int k, int j) const
    {
        const float2 q = P[off(k) + j / 2 - k / 2];
        return (j & 1) ? q.y : q.x;
    }

    // the sums in NormalEq's layout
    __device__ void store(NormalEq<float, N, F>& E) const
    {
#pragma unroll
        for (int k = 0; k < N; ++k) {
#pragma unroll
            for (int l = k; l < N; ++l) E.Gm[NormalEq<float, N, F>::id(k, l)] = at(k, l);
#pragma unroll
            for (int f = 0; f < F; ++f) E.c[k][f] = at(k, N + f);
        }
    }
};

// GFD row for scaled offset e (Eq. linear_system_axb order, 1D/3D analogues)
template <typename T, int DIM>
__device__ inline void gfd_row(const T (&e)[DIM], T (&a)[NU<DIM>::v])
{
    if (DIM == 1) {
        a[0] = e[0];
        a[1] = T(0.5) * e[0] * e[0];
    } else if (DIM == 2) {
        a[0] = e[0]; a[1] = e[1];
        a[2] = T(0.5) * e[0] * e[0]; a[3] = T(0.5) * e[1] * e[1];
        a[4] = e[0] * e[1];
    } else {
        a[0] = e[0]; a[1] = e[1]; a[2] = e[DIM > 2 ? 2 : 0];
        a[3] = T(0.5) * e[0] * e[0]; a[4] = T(0.5) * e[1] * e[1];
        a[5] = T(0.5) * e[DIM > 2 ? 2 : 0] * e[DIM > 2 ? 2 : 0];
        a[6] = e[0] * e[1]; a[7] = e[0] * e[DIM > 2 ? 2 : 0]; a[8] = e[1] * e[DIM > 2 ? 2 : 0];
    }
}

// ---------------------------------------------------------------------------
// neighbour data sources
// ---------------------------------------------------------------------------
struct FitArgs {
    DevCfg c;
    int64_t n;
    int nf;
    const uint32_t* count;
    const uint32_t* idx;
    const double* d2min;
    const double* sx[3];
    const double* fd[5];      // field values (FP64)
    const float4* rec;        // packed fit records (positions and fields, hi/lo)
    const uint32_t* sid;
    const double* sm;
    unsigned long long* counters;
    uint32_t* redo_list;      // FP32 pass: particles to redo in FP64
    const uint32_t* list;     // FP64 pass over a list (null: all particles)
    const unsigned long long* list_len;
    const __nv_bfloat16* mlp_w;   // learned-estimator weights (BF16)
    const uint64_t* keys;         // key-sorted keys (simulation above bit key_shift)
    int key_shift;
    // split schedule: compacted list of particles that need the plain stage,
    // its length, and the intermediate record (component-major, mid_cap slots).
    // plain_ident (no learned gate: every fitted particle takes the plain
    // stage): slot t is particle t, plain_list[t] = t or all ones where the
    // particle has no plain stage, and the plain kernel runs over [0, n) in
    // key order
    uint32_t* plain_list;
    unsigned long long* plain_len;
    void* mid;
    int64_t mid_cap;
    int plain_ident;
    // split schedule, FP32: the central fits that need the correction pass,
    // listed by the first kernel for a kernel of their own
    uint32_t* refine_list;
    unsigned long long* refine_len;
    unsigned long long* queue;        // [2] work counters of the persistent split kernels
};

// statistics of the last field's differences b_j = s_j - s_i over the central
// stencil: extremes, sum of squares, and the least-squares residual (the
// learned estimator's inputs)
template <typename T>
struct FitStats {
    T bmin, bmax, ssb, ssr;
};

template <typename T, int DIM, int F> struct Src;

// FP32: offsets and differences from the packed hi/lo record of each neighbour
template <int DIM, int F>
struct Src<float, DIM, F> {
    const FitArgs& a;
    int64_t i;
    float ri[4 * REC_F4];
    __device__ Src(const FitArgs& a_, int64_t i_) : a(a_), i(i_) { load(i, ri); }
    __device__ void load(int64_t j, float (&r)[4 * REC_F4]) const
    {
        const float4* p = a.rec + j * REC_F4;
#pragma unroll
        for (int q = 0; q < REC_F4; q += 2) {
            float4 v, w;
            ldg256(p + q, v, w);
            r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
            r[4 * q + 4] = w.x; r[4 * q + 5] = w.y; r[4 * q + 6] = w.z; r[4 * q + 7] = w.w;
        }
    }
    __device__ void off_rec(const float (&r)[4 * REC_F4], float (&d)[DIM]) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            float dh = r[REC_XH + k] - ri[REC_XH + k];
            float dl = r[REC_XL + k] - ri[REC_XL + k];
            if (a.c.periodic[k]) {
                if (dh > 0.5f * a.c.Lper_h[k]) { dh -= a.c.Lper_h[k]; dl -= a.c.Lper_l[k]; }
                else if (dh < -0.5f * a.c.Lper_h[k]) { dh += a.c.Lper_h[k]; dl += a.c.Lper_l[k]; }
            }
            d[k] = dh + dl;
        }
    }
    __device__ void fetch(uint32_t j, float (&d)[DIM], float (&b)[F]) const
    {
        float r[4 * REC_F4];
        load(j, r);
        off_rec(r, d);
#pragma unroll
        for (int f = 0; f < F; ++f)
            b[f] = (r[rec_fh(f, F)] - ri[rec_fh(f, F)]) + (r[rec_fl(f, F)] - ri[rec_fl(f, F)]);
    }
    __device__ void off(uint32_t j, float (&d)[DIM]) const
    {
        float r[4 * REC_F4];
        load(j, r);
        off_rec(r, d);
    }
    // exact sign of the offset x_jk - x_ik (the oracle's definition), with the
    // record of j already loaded
    __device__ int side_rec(const float (&r)[4 * REC_F4], uint32_t j, int k) const
    {
        if (!a.c.periodic[k]) {
            float hj = r[REC_XH + k], hi = ri[REC_XH + k];
            if (hj != hi) return hj > hi ? 1 : -1;
            float lj = r[REC_XL + k], li = ri[REC_XL + k];
            if (lj != li) return lj > li ? 1 : -1;
        }
        double d = offset64(a.c, k, a.sx[k][i], a.sx[k][j]);
        return d > 0.0 ? 1 : (d < 0.0 ? -1 : 0);
    }
    // a neighbour's record as loaded (the pipelined loops load one ahead)
    struct Rec { float v[4 * REC_F4]; };
    __device__ void load_rec(uint32_t j, Rec& r) const { load(j, r.v); }
    // the first 32 bytes only: positions and the last field
    __device__ void load_half(uint32_t j, Rec& r) const
    {
        float4 v, w;
        ldg256(a.rec + (int64_t)j * REC_F4, v, w);
        r.v[0] = v.x; r.v[1] = v.y; r.v[2] = v.z; r.v[3] = v.w;
        r.v[4] = w.x; r.v[5] = w.y; r.v[6] = w.z; r.v[7] = w.w;
    }
    // offsets and the last field's difference from a half record
    __device__ void unpack_last(const Rec& r, float (&d)[DIM], float& bl) const
    {
        off_rec(r.v, d);
        bl = (r.v[rec_fh(F - 1, F)] - ri[rec_fh(F - 1, F)]) + (r.v[rec_fl(F - 1, F)] - ri[rec_fl(F - 1, F)]);
    }
    __device__ void unpack(const Rec& r, float (&d)[DIM], float (&b)[F]) const
    {
        off_rec(r.v, d);
#pragma unroll
        for (int f = 0; f < F; ++f)
            b[f] = (r.v[rec_fh(f, F)] - ri[rec_fh(f, F)]) + (r.v[rec_fl(f, F)] - ri[rec_fl(f, F)]);
    }
    __device__ int side(const Rec& r, uint32_t j, int k) const { return side_rec(r.v, j, k); }
    // side of j along axis k; when non-zero, also its offsets and differences
    __device__ int unpack_side(const Rec& r, uint32_t j, int k, float (&d)[DIM], float (&b)[F]) const
    {
        int sg = side_rec(r.v, j, k);
        if (sg != 0) unpack(r, d, b);
        return sg;
    }
};

// FP64: offsets and differences in FP64 (the oracle's operation order)
template <int DIM, int F>
struct Src<double, DIM, F> {
    const FitArgs& a;
    int64_t i;
    double xi[DIM], fi[F];
    __device__ Src(const FitArgs& a_, int64_t i_) : a(a_), i(i_)
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) xi[k] = a.sx[k][i];
#pragma unroll
        for (int f = 0; f < F; ++f) fi[f] = a.fd[f][i];
    }
    __device__ void off(uint32_t j, double (&d)[DIM]) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) d[k] = offset64(a.c, k, xi[k], a.sx[k][j]);
    }
    __device__ void diff(uint32_t j, double (&b)[F]) const
    {
#pragma unroll
        for (int f = 0; f < F; ++f) b[f] = a.fd[f][j] - fi[f];
    }
    __device__ void fetch(uint32_t j, double (&d)[DIM], double (&b)[F]) const
    {
        off(j, d);
        diff(j, b);
    }
    struct Rec { double x[DIM]; double f[F]; };
    __device__ void load_rec(uint32_t j, Rec& r) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) r.x[k] = a.sx[k][j];
#pragma unroll
        for (int f = 0; f < F; ++f) r.f[f] = a.fd[f][j];
    }
    __device__ void unpack(const Rec& r, double (&d)[DIM], double (&b)[F]) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) d[k] = offset64(a.c, k, xi[k], r.x[k]);
#pragma unroll
        for (int f = 0; f < F; ++f) b[f] = r.f[f] - fi[f];
    }
    __device__ void load_half(uint32_t j, Rec& r) const { load_rec(j, r); }
    __device__ void unpack_last(const Rec& r, double (&d)[DIM], double& bl) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) d[k] = offset64(a.c, k, xi[k], r.x[k]);
        bl = r.f[F - 1] - fi[F - 1];
    }
    __device__ int side(const Rec& r, uint32_t, int k) const
    {
        const double dk = offset64(a.c, k, xi[k], r.x[k]);
        return dk > 0.0 ? 1 : (dk < 0.0 ? -1 : 0);
    }
    __device__ int unpack_side(const Rec& r, uint32_t, int k, double (&d)[DIM], double (&b)[F]) const
    {
        double dk = offset64(a.c, k, xi[k], r.x[k]);
        int sg = dk > 0.0 ? 1 : (dk < 0.0 ? -1 : 0);
        if (sg != 0) unpack(r, d, b);
        return sg;
    }
};

// A particle's neighbour list entries, read one at a time by its thread.
// NbGlobal reads the list row in global memory: each lane of a warp on a line
// of its own, one L1 wavefront per lane and entry, as many as the record loads
// the entry leads to.  NbStaged<D> reads the first D entries from a
// shared-memory copy of the warp's 32 list rows, staged with coalesced loads
// (stage_rows), where a warp's read of one entry per lane is one wavefront.
struct NbGlobal {
    const uint32_t* p;
    __device__ __forceinline__ uint32_t operator[](int r) const { return __ldg(p + r); }
};
constexpr int NB_PITCH = FIT_THREADS + 1;   // entry-major, a column per thread (conflict-free both ways)
template <int D>
struct NbStaged {
    const uint32_t* p;        // the list row in global memory
    const uint32_t* s;        // this thread's column of the staged copy
    __device__ __forceinline__ uint32_t operator[](int r) const { return r < D ? s[r * NB_PITCH] : __ldg(p + r); }
};

// The warp's staging of the first D (32 or 64) entries of the list rows of its
// lanes' particles (particle i of each lane, none where i < 0) into
// stage[entry][threadIdx.x]: coalesced reads of 32 entries per instruction.
// All 32 lanes take part.
template <int D>
__device__ __forceinline__ void stage_rows(uint32_t (*stage)[NB_PITCH], const uint32_t* idx, int k_max, int64_t i)
{
    static_assert(D == 32 || D == 64, "stage depth");
    const unsigned lane = threadIdx.x & 31u;
    const int w0 = (int)(threadIdx.x & ~31u);
    const int nr = k_max < D ? k_max : D;
    // the 32 rows' loads all issued before their stores (one at a time, each
    // waiting for its load, the staging cost more than it saved)
    uint32_t v[32][D / 32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const long long ip = __shfl_sync(0xffffffffu, (long long)i, u);
#pragma unroll
        for (int h = 0; h < D / 32; ++h) {
            const int e = (int)lane + 32 * h;
            v[u][h] = (ip >= 0 && e < nr) ? __ldg(idx + ip * (int64_t)k_max + e) : 0u;
        }
    }
#pragma unroll
    for (int u = 0; u < 32; ++u)
#pragma unroll
        for (int h = 0; h < D / 32; ++h) {
            const int e = (int)lane + 32 * h;
            if (e < nr) stage[e][w0 + u] = v[u][h];
        }
    __syncwarp();
}

// Visit the neighbour list in order with the next record (and the index after
// it) already in flight: body(j, rec) returns false to stop early.
template <bool HALF = false, class S, class NB, class Body>
__device__ __forceinline__ void for_neighbors(const S& src, const NB& nb, int cnt, Body&& body)
{
    if (cnt <= 0) return;
    typename S::Rec nxt;
    uint32_t jn = nb[0];
    if (HALF) src.load_half(jn, nxt); else src.load_rec(jn, nxt);
    uint32_t jn2 = cnt > 1 ? nb[1] : 0u;
    for (int r = 0; r < cnt; ++r) {
        const typename S::Rec cur = nxt;
        const uint32_t j = jn;
        if (r + 1 < cnt) {
            jn = jn2;
            if (HALF) src.load_half(jn, nxt); else src.load_rec(jn, nxt);
            if (r + 2 < cnt) jn2 = nb[r + 2];
        }
        if (!body(j, cur)) break;
    }
}

// power-of-two 1/S with S >= sqrt(d2)
__device__ inline float inv_scale(float d2)
{
    if (!(d2 > 0.0f) || !isfinite(d2)) return 1.0f;
    int e = (int)ceilf(0.5f * log2f(d2));
    return ldexpf(1.0f, -e);
}

// Below this ratio the FP32 fit factors the rows by rotations instead of
// through the normal equations: there cond(A)^2 u is no longer small enough
// for one correction pass to remove the error of the Gram matrix.
constexpr float NE_RATIO_MIN = 0.02f;

// Central second-order fit.  x[u][f] unscaled derivatives.  Returns 0 ok,
// 1 ill-conditioned (ratio below tau), with x untouched.
//
// FP32: the normal equations, factored as U^T D U, then one correction pass
// (semi-normal equations with the residual of the first solution); when the
// factor's ratio is below NE_RATIO_MIN, the rows again through square-root-
// free Givens rotations (the FP64 path's only form).  The correction pass runs
// in the modes that ask for it, and for the gate's residual sum when the
// rotations did not give it.
// DEFER: return 2, with x untouched, where the correction pass would run
// (the caller lists the particle for a kernel that runs it in full warps).
template <typename T, int DIM, int F, bool STATS = false, bool DEFER = false, class NB>
__device__ int central_fit(const Src<T, DIM, F>& src, const NB& nb, int cnt, T invS, T tau,
                           const DevCfg& cf, T (&x)[NU<DIM>::v][F], FitStats<T>* st = nullptr,
                           bool* refined = nullptr)
{
    constexpr int N = NU<DIM>::v;
    constexpr bool NE = sizeof(T) == 4;
    Givens<T, N, F> G;
    T bmin = T(0), bmax = T(0), ssb = T(0), ssr = T(0);
    bool have_ssr = false;            // ssr already holds the residual sum
    bool solved = false;
    T ratio = T(0);
    using Rec = typename Src<T, DIM, F>::Rec;
    if constexpr (NE) {
        NormalEqPacked<N, F> EP;
        EP.zero();
        for_neighbors(src, nb, cnt, [&](uint32_t, const Rec& rec) {
            T d[DIM], a[N], b[F];
            src.unpack(rec, d, b);
#pragma unroll
            for (int k = 0; k < DIM; ++k) d[k] *= invS;
            gfd_row<T, DIM>(d, a);
            if (STATS) {
                T bl = b[F - 1];
                bmin = bl < bmin ? bl : bmin;
                bmax = bl > bmax ? bl : bmax;
                ssb = RN<T>::fma(bl, bl, ssb);
            }
            EP.add(a, b);
            return true;
        });
        NormalEq<T, N, F> E;
        EP.store(E);
        E.factor(G);
        ratio = G.ratio();
        if (ratio >= T(NE_RATIO_MIN)) {
            if (!(ratio >= tau) || cnt < N) {
                if (STATS && st) { st->bmin = bmin; st->bmax = bmax; st->ssb = ssb; st->ssr = T(0); }
                return 1;
            }
#pragma unroll
            for (int u = 0; u < N; ++u)
#pragma unroll
                for (int f = 0; f < F; ++f) x[u][f] = E.c[u][f];
            G.solve_normal(x);
            solved = true;
        }
    }
    if (!solved) {
        G.zero();
        bmin = bmax = ssb = T(0);
        for_neighbors(src, nb, cnt, [&](uint32_t, const Rec& rec) {
            T d[DIM], a[N], b[F];
            src.unpack(rec, d, b);
#pragma unroll
            for (int k = 0; k < DIM; ++k) d[k] *= invS;
            gfd_row<T, DIM>(d, a);
            if (STATS) {
                T bl = b[F - 1];
                bmin = bl < bmin ? bl : bmin;
                bmax = bl > bmax ? bl : bmax;
                ssb = RN<T>::fma(bl, bl, ssb);
            }
            const T w = G.add(a, b);
            if (STATS) ssr = RN<T>::fma(RN<T>::mul(w, b[F - 1]), b[F - 1], ssr);   // the row's weighted leftover
            return true;
        });
        have_ssr = true;
        ratio = G.ratio();
        if (!(ratio >= tau) || cnt < N) {
            if (STATS && st) { st->bmin = bmin; st->bmax = bmax; st->ssb = ssb; st->ssr = ssr; }
            return 1;
        }
        G.solve(x);
    }
    const bool refine = cf.refine == LP_REFINE_ALWAYS || (cf.refine == LP_REFINE_AUTO && ratio < (T)cf.refine_ratio);
    if (DEFER && refine) return 2;
    if (refined) *refined = refine;
    if (STATS && !have_ssr && !refine) {
        // only the gate's residual sum of the last field: half of each record
        for_neighbors<true>(src, nb, cnt, [&](uint32_t, const Rec& rec) {
            T d[DIM], a[N], bl;
            src.unpack_last(rec, d, bl);
#pragma unroll
            for (int k = 0; k < DIM; ++k) d[k] *= invS;
            gfd_row<T, DIM>(d, a);
            T res = bl;
#pragma unroll
            for (int u = 0; u < N; ++u) res = RN<T>::fma(-a[u], x[u][F - 1], res);
            ssr = RN<T>::fma(res, res, ssr);
            return true;
        });
        have_ssr = true;
    }
    if (!DEFER && (refine || (STATS && !have_ssr))) {
        // The FP32 3D factor (d and U, 45 values) waits in shared memory during
        // the correction pass, which holds the solution and the correction sums:
        // without that the pass spills.
        constexpr bool STASH = sizeof(T) == 4 && DIM == 3;
        constexpr int NS = N + N * (N - 1) / 2;
        __shared__ T stash[STASH ? NS : 1][FIT_THREADS];
        if (STASH) {
#pragma unroll
            for (int k = 0; k < N; ++k) stash[k][threadIdx.x] = G.d[k];
#pragma unroll
            for (int q = 0; q < N * (N - 1) / 2; ++q) stash[N + q][threadIdx.x] = G.U[q];
        }
        T g[N][F];
#pragma unroll
        for (int u = 0; u < N; ++u)
#pragma unroll
            for (int f = 0; f < F; ++f) g[u][f] = T(0);
        const bool sum_res = STATS && !have_ssr;
        for_neighbors(src, nb, cnt, [&](uint32_t, const Rec& rec) {
            T d[DIM], a[N], b[F];
            src.unpack(rec, d, b);
#pragma unroll
            for (int k = 0; k < DIM; ++k) d[k] *= invS;
            gfd_row<T, DIM>(d, a);
#pragma unroll
            for (int f = 0; f < F; ++f) {
                T res = b[f];
#pragma unroll
                for (int u = 0; u < N; ++u) res = RN<T>::fma(-a[u], x[u][f], res);
                if (STATS && f == F - 1 && sum_res) ssr = RN<T>::fma(res, res, ssr);
#pragma unroll
                for (int u = 0; u < N; ++u) g[u][f] = RN<T>::fma(a[u], res, g[u][f]);
            }
            return true;
        });
        if (refine) {
            if (STASH) {
                volatile T* sv = &stash[0][0];      // volatile: reloaded, not kept live
#pragma unroll
                for (int k = 0; k < N; ++k) G.d[k] = sv[k * FIT_THREADS + threadIdx.x];
#pragma unroll
                for (int q = 0; q < N * (N - 1) / 2; ++q) G.U[q] = sv[(N + q) * FIT_THREADS + threadIdx.x];
            }
            G.solve_normal(g);
#pragma unroll
            for (int u = 0; u < N; ++u)
#pragma unroll
                for (int f = 0; f < F; ++f) x[u][f] += g[u][f];
        }
    }
    if (STATS && st) { st->bmin = bmin; st->bmax = bmax; st->ssb = ssb; st->ssr = ssr; }
    T s2 = invS * invS;
#pragma unroll
    for (int u = 0; u < N; ++u)
#pragma unroll
        for (int f = 0; f < F; ++f) x[u][f] *= (u < DIM ? invS : s2);
    return 0;
}

// First-order fit on the whole list (fallback).  Returns 0 ok, 1 rank deficient.
template <typename T, int DIM, int F, class NB>
__device__ int linear_fit(const Src<T, DIM, F>& src, const NB& nb, int cnt, T invS, T tau, T (&x)[DIM][F])
{
    Givens<T, DIM, F> G;
    G.zero();
    for (int r = 0; r < cnt; ++r) {
        uint32_t j = nb[r];
        T d[DIM], b[F];
        src.fetch(j, d, b);
#pragma unroll
        for (int k = 0; k < DIM; ++k) d[k] *= invS;
        G.add(d, b);
    }
    if (!(G.ratio() >= tau) || cnt < DIM) return 1;
    G.solve(x);
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int f = 0; f < F; ++f) x[k][f] *= invS;
    return 0;
}

// One-sided first derivatives (Sec. 2.1 left/right derivatives): along each
// axis k and on each side, the first k_side list members whose offset along k
// has that sign; first-order fit; component k.  One pass over the list marks
// the members of all 2 DIM stencils (bit r of m[k][s]: list position r < 64),
// then each fit takes exactly its rows in list order.  A stencil that still
// takes members past position 63 (lists of k_max > 64) keeps their number in
// tailn and finds them by a scan of the list's tail.  ok[k][s] = false where
// fewer than DIM members or rank deficient.  ill = true when a system with
// enough members is below tau (FP32: redo in FP64).
template <typename T, int DIM, int F, class NB>
__device__ __forceinline__ void onesided_all(const Src<T, DIM, F>& src, const NB& nb, int cnt, int ks, T invS, T tau,
                             T tau_rank, T (&out)[DIM][2][F], bool (&ok)[DIM][2], bool& ill)
{
    uint64_t m[DIM][2];
    int c[DIM][2];
#pragma unroll
    for (int k = 0; k < DIM; ++k) { m[k][0] = m[k][1] = 0ull; c[k][0] = c[k][1] = 0; }
    using Rec = typename Src<T, DIM, F>::Rec;
    int r = 0;                      // list positions the marking pass visited
    if (ks > 0) {
        for_neighbors(src, nb, cnt, [&](uint32_t j, const Rec& rec) {
            bool more = false;
            const uint64_t bit = r < 64 ? 1ull << (r & 63) : 0ull;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const int sg = src.side(rec, j, k);
                if (sg > 0) {
                    if (c[k][1] < ks) { m[k][1] |= bit; ++c[k][1]; }
                } else if (sg < 0) {
                    if (c[k][0] < ks) { m[k][0] |= bit; ++c[k][0]; }
                }
                more = more || c[k][0] < ks || c[k][1] < ks;
            }
            ++r;
            return more;
        });
    }
    // members past position 63, 5 bits per stencil (k_side <= 16)
    unsigned tailn = 0u;
    if (r > 64) {
#pragma unroll
        for (int k = 0; k < DIM; ++k)
#pragma unroll
            for (int s = 0; s < 2; ++s) tailn |= (unsigned)(c[k][s] - __popcll(m[k][s])) << (5 * (2 * k + s));
    }
    // the 2 DIM fits in one rolled loop (one copy of its code); fit q = 2k + s
    // leaves its k-component in shared memory and a bit in okb
    __shared__ T osm[2 * DIM * F][FIT_THREADS];
    unsigned okb = 0;
#pragma unroll 1
    for (int q = 0; q < 2 * DIM; ++q) {
        const int k = q >> 1;
        uint64_t mm = m[0][0];
#pragma unroll
        for (int qq = 1; qq < 2 * DIM; ++qq) mm = q == qq ? m[qq >> 1][qq & 1] : mm;
        const int ntail = (int)((tailn >> (5 * q)) & 31u);
        if (__popcll(mm) + ntail < DIM) continue;
        Givens<T, DIM, F> G;
        G.zero();
        // rows in list order, the next record in flight
        // (with no member before position 64 the first load reads entry 0, unused)
        Rec nxt;
        uint32_t jn = nb[mm ? __ffsll((long long)mm) - 1 : 0];
        src.load_rec(jn, nxt);
        while (mm) {
            mm &= mm - 1;
            const Rec cur = nxt;
            if (mm) {
                jn = nb[__ffsll((long long)mm) - 1];
                src.load_rec(jn, nxt);
            }
            T d[DIM], b[F];
            src.unpack(cur, d, b);
#pragma unroll
            for (int u = 0; u < DIM; ++u) d[u] *= invS;
            G.add(d, b);
        }
        if (ntail > 0) {
            // the members past position 63, found again by their side
            int need = ntail;
            const int want = (q & 1) ? 1 : -1;
            for (int r = 64; r < cnt && need > 0; ++r) {
                const uint32_t j = nb[r];
                Rec rec;
                src.load_rec(j, rec);
                int sg = 0;                 // (k is not a compile-time index here)
#pragma unroll
                for (int kk = 0; kk < DIM; ++kk)
                    if (kk == k) sg = src.side(rec, j, kk);
                if (sg != want) continue;
                T d[DIM], b[F];
                src.unpack(rec, d, b);
#pragma unroll
                for (int u = 0; u < DIM; ++u) d[u] *= invS;
                G.add(d, b);
                --need;
            }
        }
        const T rt = G.ratio();
        if (!(rt >= tau_rank)) continue;              // rank deficient: central derivative
        if (!(rt >= tau)) ill = true;                 // usable only in higher precision
        T x[DIM][F];
        G.solve(x);
#pragma unroll
        for (int f = 0; f < F; ++f) {
            T v = x[0][f];
#pragma unroll
            for (int u = 1; u < DIM; ++u) v = k == u ? x[u][f] : v;
            osm[q * F + f][threadIdx.x] = v * invS;
        }
        okb |= 1u << q;
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            ok[k][s] = (okb >> (2 * k + s)) & 1u;
#pragma unroll
            for (int f = 0; f < F; ++f) out[k][s][f] = ok[k][s] ? osm[(2 * k + s) * F + f][threadIdx.x] : T(0);
        }
}

// ---------------------------------------------------------------------------
// estimator, limiter, rates (Sec. 2.1)
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline T phi_limiter(T r)
{
    if (isinf(r)) return T(0);
    T sr = sqrt(r);
    if (r <= T(1.5)) return T(1.25) * exp(T(1) - sr);
    T q = sr - T(1);
    return T(1.25) * exp(T(-4.5) * q * q);
}

template <typename T, int DIM>
__device__ inline T estimator_r(const T (&sl)[DIM], const T (&sr)[DIM], T ell, T s_i, T s_ref, T flat_eps,
                                T active_frac)
{
    T G = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        T g = fmax(fabs(sl[k]), fabs(sr[k]));
        G = g > G ? g : G;
    }
    T S = fmax(fabs(s_i), s_ref);
    if (G * ell <= flat_eps * S) return T(1);
    T r = T(1);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        T g = fmax(fabs(sl[k]), fabs(sr[k]));
        if (g < active_frac * G) continue;
        T rk;
        if (sl[k] * sr[k] <= T(0)) rk = T(INFINITY);
        else rk = T(0.5) * (sr[k] / sl[k] + sl[k] / sr[k]);
        r = rk > r ? rk : r;
    }
    return r;
}

// slot of d_c d_a in the second-order unknown ordering
template <int DIM>
__device__ constexpr int hess_slot(int c, int a)
{
    return c == a ? DIM + a : (DIM == 2 ? 4 : ((c < a ? c : a) == 0 ? ((c < a ? a : c) == 1 ? 6 : 7) : 8));
}

// Lax-Wendroff rates LW_s = s_t + dt/2 s_tt for an ideal gas (see the oracle
// for the derivation from V_t = V div u, u_t = -V grad P, P_t = -gamma P div u).
// cd[u][f] central derivatives, fields V, u_1..u_d, P.
template <typename T, int DIM>
__device__ inline void lw_rates(T gamma, T dt, T V, T P, const T (&cd)[NU<DIM>::v][DIM + 2], T (&lw)[DIM + 2])
{
    using O = RN<T>;
    constexpr int FP = DIM + 1;
    T divu = T(0), S2 = T(0), gVgP = T(0), lapP = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) divu = O::add(divu, cd[a][1 + a]);
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) S2 = O::fma(cd[b][1 + a], cd[a][1 + b], S2);
#pragma unroll
    for (int k = 0; k < DIM; ++k) gVgP = O::fma(cd[k][0], cd[k][FP], gVgP);
#pragma unroll
    for (int k = 0; k < DIM; ++k) lapP = O::add(lapP, cd[DIM + k][FP]);
    const T hdt = O::mul(T(0.5), dt);
    const T Vd = O::mul(V, divu);
    // V_tt = V (div u)^2 - V S2 - V grad V . grad P - V^2 lap P
    T Vtt = O::sub(O::sub(O::sub(O::mul(Vd, divu), O::mul(V, S2)), O::mul(V, gVgP)), O::mul(O::mul(V, V), lapP));
    lw[0] = O::fma(hdt, Vtt, Vd);
    const T c1 = O::mul(O::sub(gamma, T(1)), Vd);        // (gamma - 1) V div u
    const T gVP = O::mul(O::mul(gamma, V), P);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        T uPt = T(0), gdiv = T(0);
#pragma unroll
        for (int m = 0; m < DIM; ++m) uPt = O::fma(cd[i][1 + m], cd[m][FP], uPt);
#pragma unroll
        for (int a = 0; a < DIM; ++a) gdiv = O::add(gdiv, cd[hess_slot<DIM>(i, a)][1 + a]);
        T ut = O::mul(-V, cd[i][FP]);
        // u_i,tt = (gamma - 1) V div u d_i P + V sum_m d_i u_m d_m P + gamma V P d_i div u
        T utt = O::add(O::add(O::mul(c1, cd[i][FP]), O::mul(V, uPt)), O::mul(gVP, gdiv));
        lw[1 + i] = O::fma(hdt, utt, ut);
    }
    const T gP = O::mul(gamma, P);
    T Pt = O::mul(-gP, divu);
    // P_tt = gamma^2 P (div u)^2 + gamma P S2 + gamma P (grad V . grad P + V lap P)
    T Ptt = O::add(O::add(O::mul(O::mul(O::mul(gamma, gP), divu), divu), O::mul(gP, S2)),
                   O::mul(gP, O::fma(V, lapP, gVgP)));
    lw[FP] = O::fma(hdt, Ptt, Pt);
}

}  // namespace lp
