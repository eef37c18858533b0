// lp_fit_kern.cuh -- kernels of the fit phases and of the LP update, included
// by lp_fit_f32.cu and lp_fit_f64.cu with T = float / double.
#pragma once

#include "lp_fit.cuh"

namespace lp {

struct StepOut {
    double* x[3];
    double* V;
    double* u[3];
    double* P;
    double* m;
    uint32_t* id;
    uint8_t* flag;
    float* phi;
    float* r;
    float* features;
    const double* dt;
};

template <typename T> struct IsF32 { static constexpr bool v = false; };
template <> struct IsF32<float> { static constexpr bool v = true; };

__device__ inline void push_redo(const FitArgs& a, int64_t i)
{
    unsigned long long pos = atomicAdd(const_cast<unsigned long long*>(a.list_len), 1ull);
    a.redo_list[pos] = (uint32_t)i;
    atomicAdd(a.counters + C_FP64, 1ull);
}

template <typename T, int DIM, int F>
__device__ inline float last_d2(const Src<T, DIM, F>& src, const uint32_t* nb, int cnt)
{
    if (cnt <= 0) return 0.0f;
    T d[DIM];
    src.off(nb[cnt - 1], d);
    T s = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) s += d[k] * d[k];
    return (float)s;
}

// the eight inputs of the learned estimator (see lp_mlp_* in lp.h)
template <typename T, int DIM>
__device__ inline T curvature_ratio(const T (&cd)[NU<DIM>::v][DIM + 2], int f, T ell)
{
    // max over active axes (|d_k s| >= 1/2 of the largest) of
    // ell |d_kk s| / (|d_k s| + ell |d_kk s|), in [0, 1]; 1 at an extremum
    T gmax = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) gmax = fmax(gmax, fabs(cd[k][f]));
    T best = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        T g = fabs(cd[k][f]);
        if (g < T(0.5) * gmax) continue;
        T h = ell * fabs(cd[DIM + k][f]);
        T r = (g + h) > T(0) ? h / (g + h) : T(0);
        best = fmax(best, r);
    }
    return best;
}

template <typename T, int DIM>
__device__ inline void mlp_features(const T (&cd)[NU<DIM>::v][DIM + 2], const FitStats<T>& st, T ell, T V, T P,
                                    T gamma, float (&x)[MLP_IN])
{
    constexpr int FP = DIM + 1;
    T gP = T(0), gV = T(0), divu = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        gP += cd[k][FP] * cd[k][FP];
        gV += cd[k][0] * cd[k][0];
        divu += cd[k][1 + k];
    }
    T cs = sqrt(gamma * P * V);
    x[0] = feat_t((float)(ell * sqrt(gP) / P));
    x[1] = feat_t((float)(ell * sqrt(gV) / V));
    x[2] = feat_t((float)curvature_ratio<T, DIM>(cd, FP, ell));
    x[3] = feat_t((float)curvature_ratio<T, DIM>(cd, 0, ell));
    x[4] = feat_ts((float)(ell * divu / cs));
    x[5] = feat_t((float)(st.bmax / P));
    x[6] = feat_t((float)(-st.bmin / P));
    x[7] = feat_t((float)(st.ssb > T(0) ? sqrt(st.ssr / st.ssb) : T(0)));
}

// ---------------------------------------------------------------------------
// one LP step for particle i (sorted index)
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__device__ void step_one(const FitArgs& a, const StepOut& o, int64_t i)
{
    constexpr int F = DIM + 2;
    constexpr int N = NU<DIM>::v;
    const DevCfg& c = a.c;
    const double dt = o.dt[c.nsim_max > 1 ? (a.keys[i] >> a.key_shift) : 0];
    // frozen boundary particles are copied through
    double s0[F];
    s0[0] = a.fd[0][i];
#pragma unroll
    for (int k = 0; k < DIM; ++k) s0[1 + k] = a.fd[1 + k][i];
    s0[F - 1] = a.fd[F - 1][i];
    double x0[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) x0[k] = a.sx[k][i];
    uint32_t idi = a.sid[i];
    if ((int64_t)idi >= c.n_fluid) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) { o.x[k][i] = x0[k]; o.u[k][i] = s0[1 + k]; }
        o.V[i] = s0[0];
        o.P[i] = s0[F - 1];
        o.m[i] = a.sm[i];
        o.id[i] = idi;
        if (o.flag) o.flag[i] = 0;
        if (o.phi) for (int f = 0; f < F; ++f) o.phi[i * F + f] = 1.0f;
        if (o.r) for (int f = 0; f < F; ++f) o.r[i * F + f] = 1.0f;
        return;
    }
    Src<T, DIM, F> src(a, i);
    const int cnt = (int)a.count[i];
    const uint32_t* nb = a.idx + i * (int64_t)c.k_max;
    const T invS = (T)inv_scale(last_d2(src, nb, cnt));
    const T tau = IsF32<T>::v ? (T)c.tau32 : (T)c.tau64;
    const T tau_rank = (T)c.tau64;

    T cd[N][F];
    FitStats<T> fst = {T(0), T(0), T(0), T(0)};
    if (central_fit<T, DIM, F, true>(src, nb, cnt, invS, tau, c.refine != 0, cd, &fst)) {
        if (IsF32<T>::v) { push_redo(a, i); return; }
        T lin[DIM][F];
#pragma unroll
        for (int u = 0; u < N; ++u)
#pragma unroll
            for (int f = 0; f < F; ++f) cd[u][f] = T(0);
        atomicAdd(a.counters + C_LINEAR, 1ull);
        if (linear_fit<T, DIM, F>(src, nb, cnt, invS, tau_rank, lin) == 0) {
#pragma unroll
            for (int u = 0; u < DIM; ++u)
#pragma unroll
                for (int f = 0; f < F; ++f) cd[u][f] = lin[u][f];
        } else {
            atomicAdd(a.counters + C_NOFIT, 1ull);
        }
    }
    // learned estimator: below mlp_tau_lo the particle is unflagged and its
    // one-sided fits are skipped (unless auditing against the plain estimator)
    bool mlp_skip = false;
    if (o.features || c.estimator == LP_EST_MLP) {
        float xf[MLP_IN];
        mlp_features<T, DIM>(cd, fst, (T)sqrt(a.d2min[i]), (T)s0[0], (T)s0[F - 1], (T)c.gamma, xf);
        if (o.features)
#pragma unroll
            for (int k = 0; k < MLP_IN; ++k) o.features[i * MLP_IN + k] = xf[k];
        if (c.estimator == LP_EST_MLP) {
            mlp_skip = mlp_prob(xf, a.mlp_w) < c.mlp_tau_lo;
            warp_count(a.counters, C_MLP_SKIP, mlp_skip);
            warp_count(a.counters, C_MLP_UNCERTAIN, !mlp_skip);
        }
    }
    const bool plain = !mlp_skip || c.mlp_audit;
    // one-sided derivatives os[k][s][f]
    T os[DIM][2][F];
    bool ill = false;
    if (plain) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            T out[2][F];
            bool ok[2];
            onesided_axis<T, DIM, F>(src, nb, cnt, k, c.k_side, invS, tau, tau_rank, out, ok, ill);
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int f = 0; f < F; ++f) os[k][s][f] = ok[s] ? out[s][f] : cd[k][f];
        }
    } else {
#pragma unroll
        for (int k = 0; k < DIM; ++k)
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int f = 0; f < F; ++f) os[k][s][f] = cd[k][f];
    }
    if (IsF32<T>::v && ill) { push_redo(a, i); return; }

    // rates
    const T g = (T)c.gamma;
    const T V = (T)s0[0], P = (T)s0[F - 1];
    T lw[F], uw[F];
    lw_rates<T, DIM>(g, (T)dt, V, P, cd, lw);
    {
        T K = g * P / V;
        T sK = sqrt(K);
        T Vt = T(0), Pt = T(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            T ul = os[k][0][1 + k], ur = os[k][1][1 + k];
            T Pl = os[k][0][F - 1], Pr = os[k][1][F - 1];
            Vt += T(0.5) * V * (ur + ul) - V / (T(2) * sK) * (Pr - Pl);
            uw[1 + k] = T(0.5) * V * sK * (ur - ul) - T(0.5) * V * (Pr + Pl);
            Pt += T(-0.5) * V * K * (ur + ul) + T(0.5) * V * sK * (Pr - Pl);
        }
        uw[0] = Vt;
        uw[F - 1] = Pt;
    }
    // estimator
    const T ell = (T)sqrt(a.d2min[i]);
    T rs[F];
    bool any = false;
#pragma unroll
    for (int f = 0; f < F; ++f) {
        T sl[DIM], sr[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) { sl[k] = os[k][0][f]; sr[k] = os[k][1][f]; }
        rs[f] = plain ? estimator_r<T, DIM>(sl, sr, ell, (T)s0[f], (T)c.s_ref[f], (T)c.flat_eps, (T)c.active_frac)
                      : T(1);
        any = any || rs[f] > T(1.5);
    }
    warp_count(a.counters, C_MLP_MISS, mlp_skip && any);
    if (mlp_skip) {               // the learned call stands; the audit counts misses
        any = false;
#pragma unroll
        for (int f = 0; f < F; ++f) rs[f] = T(1);
    }
    double s1[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
        T p;
        switch (c.limiter) {
        case LP_LIM_PAPER: p = phi_limiter<T>(rs[f]); break;
        case LP_LIM_LW: p = T(1); break;
        case LP_LIM_UW: p = T(0); break;
        default: p = any ? phi_limiter<T>(rs[f]) : T(1); break;
        }
        T rate = uw[f] - p * (uw[f] - lw[f]);
        s1[f] = __dadd_rn(s0[f], __dmul_rn(dt, (double)rate));   // no contraction: the oracle's rounding
        if (o.phi) o.phi[i * F + f] = (float)p;
        if (o.r) o.r[i * F + f] = (float)rs[f];
    }
    // safeguard: an update that leaves V or P non-positive or any field non-finite
    // is not applied; the particle keeps its state and is counted
    bool admissible = s1[0] > 0.0 && s1[F - 1] > 0.0;
#pragma unroll
    for (int f = 0; f < F; ++f) admissible = admissible && isfinite(s1[f]);
    if (!admissible) {
#pragma unroll
        for (int f = 0; f < F; ++f) s1[f] = s0[f];
        atomicAdd(a.counters + C_NONFINITE, 1ull);
        atomicOr(reinterpret_cast<unsigned int*>(a.counters + C_STATUS), ST_NONFINITE);
    }
    // mover, Eq. timeIntegrate
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double xk = __dadd_rn(x0[k], __dmul_rn(__dmul_rn(0.5, dt), __dadd_rn(s0[1 + k], s1[1 + k])));
        if (c.periodic[k]) {
            if (xk >= c.box_hi[k]) xk = __dsub_rn(xk, c.Lper[k]);
            else if (xk < c.box_lo[k]) xk = __dadd_rn(xk, c.Lper[k]);
        }
        o.x[k][i] = xk;
        o.u[k][i] = s1[1 + k];
    }
    o.V[i] = s1[0];
    o.P[i] = s1[F - 1];
    o.m[i] = a.sm[i];
    o.id[i] = idi;
    if (o.flag) o.flag[i] = any ? 1 : 0;
    warp_count(a.counters, C_FLAGGED, any);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_step(FitArgs a, StepOut o)
{
    if (a.list) {
        unsigned long long len = *a.list_len;
        for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < len;
             t += (unsigned long long)gridDim.x * blockDim.x)
            step_one<T, DIM>(a, o, a.list[t]);
    } else {
        int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (i < a.n) step_one<T, DIM>(a, o, i);
    }
}

// ---------------------------------------------------------------------------
// central derivatives of F fields (lp_gfd_derivs)
// ---------------------------------------------------------------------------
struct DerivOut {
    void* out;
    int out_f64;
    int f_first;      // global index of field 0 of this chunk
    int f_real;       // fields of this chunk that exist (<= F)
    uint32_t* status;
};

template <typename T, int DIM, int F>
__device__ void derivs_one(const FitArgs& a, const DerivOut& o, int64_t i)
{
    constexpr int N = NU<DIM>::v;
    const DevCfg& c = a.c;
    Src<T, DIM, F> src(a, i);
    const int cnt = (int)a.count[i];
    const uint32_t* nb = a.idx + i * (int64_t)c.k_max;
    const T invS = (T)inv_scale(last_d2(src, nb, cnt));
    const T tau = IsF32<T>::v ? (T)c.tau32 : (T)c.tau64;
    T cd[N][F];
    uint32_t st = IsF32<T>::v ? 0u : (a.list ? FIT_FP64 : 0u);
    if (central_fit<T, DIM, F>(src, nb, cnt, invS, tau, c.refine != 0, cd)) {
        if (IsF32<T>::v) { push_redo(a, i); return; }
        st |= FIT_LINEAR;
#pragma unroll
        for (int u = 0; u < N; ++u)
#pragma unroll
            for (int f = 0; f < F; ++f) cd[u][f] = T(0);
        T lin[DIM][F];
        if (linear_fit<T, DIM, F>(src, nb, cnt, invS, (T)c.tau64, lin) == 0) {
#pragma unroll
            for (int u = 0; u < DIM; ++u)
#pragma unroll
                for (int f = 0; f < F; ++f) cd[u][f] = lin[u][f];
        } else {
            st |= FIT_NONE;
        }
        atomicAdd(a.counters + (st & FIT_NONE ? C_NOFIT : C_LINEAR), 1ull);
    }
#pragma unroll
    for (int f = 0; f < F; ++f) {
        if (f >= o.f_real) break;
        int64_t base = ((int64_t)(o.f_first + f) * a.n + i) * N;
#pragma unroll
        for (int u = 0; u < N; ++u) {
            if (o.out_f64) static_cast<double*>(o.out)[base + u] = (double)cd[u][f];
            else static_cast<float*>(o.out)[base + u] = (float)cd[u][f];
        }
    }
    if (o.status && o.f_first == 0) o.status[i] = st;
}

template <typename T, int DIM, int F>
__global__ void __launch_bounds__(128) k_derivs(FitArgs a, DerivOut o)
{
    if (a.list) {
        unsigned long long len = *a.list_len;
        for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < len;
             t += (unsigned long long)gridDim.x * blockDim.x)
            derivs_one<T, DIM, F>(a, o, a.list[t]);
    } else {
        int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (i < a.n) derivs_one<T, DIM, F>(a, o, i);
    }
}

// ---------------------------------------------------------------------------
// one-sided derivatives (lp_onesided_derivs), out[i][k][s][f] float64
// ---------------------------------------------------------------------------
template <typename T, int DIM, int F>
__device__ void onesided_one(const FitArgs& a, double* out, int f_real, int64_t i)
{
    constexpr int N = NU<DIM>::v;
    const DevCfg& c = a.c;
    Src<T, DIM, F> src(a, i);
    const int cnt = (int)a.count[i];
    const uint32_t* nb = a.idx + i * (int64_t)c.k_max;
    const T invS = (T)inv_scale(last_d2(src, nb, cnt));
    const T tau = IsF32<T>::v ? (T)c.tau32 : (T)c.tau64;
    T cd[N][F];
    if (central_fit<T, DIM, F>(src, nb, cnt, invS, tau, c.refine != 0, cd)) {
        if (IsF32<T>::v) { push_redo(a, i); return; }
#pragma unroll
        for (int u = 0; u < N; ++u)
#pragma unroll
            for (int f = 0; f < F; ++f) cd[u][f] = T(0);
        T lin[DIM][F];
        if (linear_fit<T, DIM, F>(src, nb, cnt, invS, (T)c.tau64, lin) == 0) {
#pragma unroll
            for (int u = 0; u < DIM; ++u)
#pragma unroll
                for (int f = 0; f < F; ++f) cd[u][f] = lin[u][f];
        }
    }
    bool ill = false;
    T os[DIM][2][F];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        T o2[2][F];
        bool ok[2];
        onesided_axis<T, DIM, F>(src, nb, cnt, k, c.k_side, invS, tau, (T)c.tau64, o2, ok, ill);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int f = 0; f < F; ++f) os[k][s][f] = ok[s] ? o2[s][f] : cd[k][f];
    }
    if (IsF32<T>::v && ill) { push_redo(a, i); return; }
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int f = 0; f < F; ++f)
                if (f < f_real) out[((i * DIM + k) * 2 + s) * f_real + f] = (double)os[k][s][f];
}

template <typename T, int DIM, int F>
__global__ void __launch_bounds__(128) k_onesided(FitArgs a, double* out, int f_real)
{
    if (a.list) {
        unsigned long long len = *a.list_len;
        for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < len;
             t += (unsigned long long)gridDim.x * blockDim.x)
            onesided_one<T, DIM, F>(a, out, f_real, a.list[t]);
    } else {
        int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (i < a.n) onesided_one<T, DIM, F>(a, out, f_real, i);
    }
}

// launchers, defined once per precision in lp_fit_f32.cu / lp_fit_f64.cu
cudaError_t launch_step_f32(int dim, const FitArgs& a, const StepOut& o, cudaStream_t s);
cudaError_t launch_step_f64(int dim, const FitArgs& a, const StepOut& o, cudaStream_t s);
cudaError_t launch_derivs_f32(int dim, int F, const FitArgs& a, const DerivOut& o, cudaStream_t s);
cudaError_t launch_derivs_f64(int dim, int F, const FitArgs& a, const DerivOut& o, cudaStream_t s);
cudaError_t launch_onesided_f32(int dim, const FitArgs& a, double* out, int f_real, cudaStream_t s);
cudaError_t launch_onesided_f64(int dim, const FitArgs& a, double* out, int f_real, cudaStream_t s);

inline unsigned fit_blocks(const FitArgs& a)
{
    return a.list ? 152u * 4u : (unsigned)((a.n + 127) / 128);
}

#define LP_DEFINE_FIT_LAUNCHERS(T, SUF)                                                         \
    cudaError_t launch_step_##SUF(int dim, const FitArgs& a, const StepOut& o, cudaStream_t s)  \
    {                                                                                           \
        unsigned b = fit_blocks(a);                                                             \
        if (b == 0) return cudaSuccess;                                                         \
        if (dim == 3) k_step<T, 3><<<b, 128, 0, s>>>(a, o);                                     \
        else if (dim == 2) k_step<T, 2><<<b, 128, 0, s>>>(a, o);                                \
        else k_step<T, 1><<<b, 128, 0, s>>>(a, o);                                              \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_derivs_##SUF(int dim, int F, const FitArgs& a, const DerivOut& o,        \
                                    cudaStream_t s)                                             \
    {                                                                                           \
        unsigned b = fit_blocks(a);                                                             \
        if (b == 0) return cudaSuccess;                                                         \
        if (dim == 3 && F == 1) k_derivs<T, 3, 1><<<b, 128, 0, s>>>(a, o);                     \
        else if (dim == 3) k_derivs<T, 3, 5><<<b, 128, 0, s>>>(a, o);                          \
        else if (dim == 2) k_derivs<T, 2, 5><<<b, 128, 0, s>>>(a, o);                          \
        else k_derivs<T, 1, 5><<<b, 128, 0, s>>>(a, o);                                        \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_onesided_##SUF(int dim, const FitArgs& a, double* out, int f_real,       \
                                      cudaStream_t s)                                           \
    {                                                                                           \
        unsigned b = fit_blocks(a);                                                             \
        if (b == 0) return cudaSuccess;                                                         \
        if (dim == 3) k_onesided<T, 3, 5><<<b, 128, 0, s>>>(a, out, f_real);                   \
        else if (dim == 2) k_onesided<T, 2, 5><<<b, 128, 0, s>>>(a, out, f_real);              \
        else k_onesided<T, 1, 5><<<b, 128, 0, s>>>(a, out, f_real);                            \
        return cudaGetLastError();                                                              \
    }

}  // namespace lp
