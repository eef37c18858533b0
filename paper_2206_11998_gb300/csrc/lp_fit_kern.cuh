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
    float* gate_p;
    const double* dt;
};

template <typename T> struct IsF32 { static constexpr bool v = false; };
template <> struct IsF32<float> { static constexpr bool v = true; };

// resident blocks per SM the FP32 step kernels are compiled for (measured on
// the 2M-particle cloud: the central kernel at 3 blocks, 168 registers, runs 5%
// faster than at 2 and 30% faster than at 4, where it spills; the plain kernel
// at 5 blocks, a few registers spilled, edges out 4 and 3); the FP64 kernels
// keep the default
template <typename T> struct FitOcc { static constexpr int fused = 1, central = 1, plain = 1; };
template <> struct FitOcc<float> { static constexpr int fused = 3, central = 3, plain = 5; };

__device__ inline void push_redo(const FitArgs& a, int64_t i)
{
    unsigned long long pos = atomicAdd(const_cast<unsigned long long*>(a.list_len), 1ull);
    a.redo_list[pos] = (uint32_t)i;
    atomicAdd(a.counters + C_FP64, 1ull);
}

template <typename T, int DIM, int F, class NB>
__device__ inline float last_d2(const Src<T, DIM, F>& src, const NB& nb, int cnt)
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
        T h = RN<T>::mul(ell, fabs(cd[DIM + k][f]));
        T gh = RN<T>::add(g, h);
        T r = gh > T(0) ? h / gh : T(0);
        best = fmax(best, r);
    }
    return best;
}

template <typename T, int DIM>
__device__ inline void mlp_features(const T (&cd)[NU<DIM>::v][DIM + 2], const FitStats<T>& st, T ell, T V, T P,
                                    T gamma, float (&x)[MLP_IN])
{
    constexpr int FP = DIM + 1;
    using O = RN<T>;
    T gP = T(0), gV = T(0), divu = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        gP = O::fma(cd[k][FP], cd[k][FP], gP);
        gV = O::fma(cd[k][0], cd[k][0], gV);
        divu = O::add(divu, cd[k][1 + k]);
    }
    T cs = sqrt(O::mul(O::mul(gamma, P), V));
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
// one LP step for particle i (sorted index), in stages
//
//   load     state of i; frozen boundary particles are copied through
//   central  central fit, LW rates (Sec. 2.3), learned gate (features + MLP)
//   plain    one-sided fits per axis (Sec. 2.4), falling back to the central
//            first derivatives where a side has too few points
//   finish   UW rates, estimator r and limiter phi, blend (Eq. 14), safeguard,
//            mover (Sec. 2.5)
//
// The fused schedule runs all stages in one thread.  The split schedule runs
// load + central in one kernel, which finishes particles the learned gate
// clears and appends the rest to a compacted list with a small intermediate
// record (central first derivatives, LW rates, gate bit); a second kernel
// runs plain + finish over that list with full warps.  Both schedules execute
// the same arithmetic on the same values, so their results are identical.
// ---------------------------------------------------------------------------
template <int DIM>
struct Loaded {
    double s0[DIM + 2];
    double x0[DIM];
    double dt;
    uint32_t id;
};

template <typename T, int DIM>
__device__ __forceinline__ bool step_load(const FitArgs& a, const StepOut& o, int64_t i, Loaded<DIM>& L)
{
    constexpr int F = DIM + 2;
    const DevCfg& c = a.c;
    L.dt = o.dt[c.nsim_max > 1 ? (a.keys[i] >> a.key_shift) : 0];
    L.s0[0] = a.fd[0][i];
#pragma unroll
    for (int k = 0; k < DIM; ++k) L.s0[1 + k] = a.fd[1 + k][i];
    L.s0[F - 1] = a.fd[F - 1][i];
#pragma unroll
    for (int k = 0; k < DIM; ++k) L.x0[k] = a.sx[k][i];
    L.id = a.sid[i];
    if ((int64_t)L.id < c.n_fluid) return false;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { o.x[k][i] = L.x0[k]; o.u[k][i] = L.s0[1 + k]; }
    o.V[i] = L.s0[0];
    o.P[i] = L.s0[F - 1];
    o.m[i] = a.sm[i];
    o.id[i] = L.id;
    if (o.flag) o.flag[i] = 0;
    if (o.gate_p && c.estimator == LP_EST_MLP) o.gate_p[i] = 0.0f;
    if (o.phi) for (int f = 0; f < F; ++f) o.phi[i * F + f] = 1.0f;
    if (o.r) for (int f = 0; f < F; ++f) o.r[i * F + f] = 1.0f;
    return true;
}

// central stage; false when i went to the FP64 redo list (or, DEFER, to the
// correction kernel's list).  GATE: the learned estimator or the feature
// output is in use (its inputs and code are compiled out otherwise)
template <typename T, int DIM, bool GATE, bool DEFER = false, class NB>
__device__ inline bool step_central(const FitArgs& a, const StepOut& o, int64_t i, const Loaded<DIM>& L,
                                    const Src<T, DIM, DIM + 2>& src, const NB& nb, int cnt, T invS,
                                    T (&cdf)[DIM][DIM + 2], T (&lw)[DIM + 2], bool& mlp_skip)
{
    constexpr int F = DIM + 2;
    constexpr int N = NU<DIM>::v;
    const DevCfg& c = a.c;
    const T tau = IsF32<T>::v ? (T)c.tau32 : (T)c.tau64;
    T cd[N][F];
    FitStats<T> fst = {T(0), T(0), T(0), T(0)};
    bool refined = false;
    const int ill = central_fit<T, DIM, F, GATE, DEFER>(src, nb, cnt, invS, tau, c, cd, &fst, &refined);
    if (IsF32<T>::v) warp_count(a.counters, C_REFINED, refined);
    if (DEFER && ill == 2) {
        const unsigned long long pos = atomicAdd(a.refine_len, 1ull);
        a.refine_list[pos] = (uint32_t)i;
        return false;
    }
    if (ill) {
        if (IsF32<T>::v) { push_redo(a, i); return false; }
        T lin[DIM][F];
#pragma unroll
        for (int u = 0; u < N; ++u)
#pragma unroll
            for (int f = 0; f < F; ++f) cd[u][f] = T(0);
        atomicAdd(a.counters + C_LINEAR, 1ull);
        if (linear_fit<T, DIM, F>(src, nb, cnt, invS, (T)c.tau64, lin) == 0) {
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
    mlp_skip = false;
    if (GATE && (o.features || c.estimator == LP_EST_MLP)) {
        float xf[MLP_IN];
        mlp_features<T, DIM>(cd, fst, (T)sqrt(a.d2min[i]), (T)L.s0[0], (T)L.s0[F - 1], (T)c.gamma, xf);
        if (o.features)
#pragma unroll
            for (int k = 0; k < MLP_IN; ++k) o.features[i * MLP_IN + k] = xf[k];
        if (c.estimator == LP_EST_MLP) {
            const float pg = mlp_prob(xf, a.mlp_w);
            if (o.gate_p) o.gate_p[i] = pg;
            mlp_skip = pg < c.mlp_tau_lo;
            warp_count(a.counters, C_MLP_SKIP, mlp_skip);
            warp_count(a.counters, C_MLP_UNCERTAIN, !mlp_skip);
        }
    }
    lw_rates<T, DIM>((T)c.gamma, (T)L.dt, (T)L.s0[0], (T)L.s0[F - 1], cd, lw);
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int f = 0; f < F; ++f) cdf[k][f] = cd[k][f];
    return true;
}

// plain stage; false when i went to the FP64 redo list
template <typename T, int DIM, class NB>
__device__ __forceinline__ bool step_plain(const FitArgs& a, int64_t i, const Src<T, DIM, DIM + 2>& src, const NB& nb,
                                  int cnt, T invS, const T (&cdf)[DIM][DIM + 2], T (&os)[DIM][2][DIM + 2])
{
    constexpr int F = DIM + 2;
    const DevCfg& c = a.c;
    const T tau = IsF32<T>::v ? (T)c.tau32 : (T)c.tau64;
    bool ill = false;
    T out[DIM][2][F];
    bool ok[DIM][2];
    onesided_all<T, DIM, F>(src, nb, cnt, c.k_side, invS, tau, (T)c.tau64, out, ok, ill);
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int f = 0; f < F; ++f) os[k][s][f] = ok[k][s] ? out[k][s][f] : cdf[k][f];
    if (IsF32<T>::v && ill) { push_redo(a, i); return false; }
    return true;
}

template <typename T, int DIM>
__device__ __forceinline__ void step_finish(const FitArgs& a, const StepOut& o, int64_t i, const Loaded<DIM>& L,
                                   const T (&os)[DIM][2][DIM + 2], const T (&lw)[DIM + 2], bool plain, bool mlp_skip)
{
    constexpr int F = DIM + 2;
    const DevCfg& c = a.c;
    const double dt = L.dt;
    using O = RN<T>;
    const T g = (T)c.gamma;
    const T V = (T)L.s0[0], P = (T)L.s0[F - 1];
    T uw[F];
    {
        // upwind rates, the 1D operator along each axis (the axis-sum reading)
        const T K = O::div(O::mul(g, P), V);
        const T sK = sqrt(K);
        const T hV = O::mul(T(0.5), V);
        const T hVsK = O::mul(hV, sK);
        const T hVK = O::mul(hV, K);
        const T VsK2 = O::div(V, O::mul(T(2), sK));
        T Vt = T(0), Pt = T(0);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            T ul = os[k][0][1 + k], ur = os[k][1][1 + k];
            T Pl = os[k][0][F - 1], Pr = os[k][1][F - 1];
            T su = O::add(ur, ul), du = O::sub(ur, ul), sP = O::add(Pr, Pl), dP = O::sub(Pr, Pl);
            Vt = O::add(Vt, O::sub(O::mul(hV, su), O::mul(VsK2, dP)));
            uw[1 + k] = O::sub(O::mul(hVsK, du), O::mul(hV, sP));
            Pt = O::add(Pt, O::sub(O::mul(hVsK, dP), O::mul(hVK, su)));
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
        rs[f] = plain ? estimator_r<T, DIM>(sl, sr, ell, (T)L.s0[f], (T)c.s_ref[f], (T)c.flat_eps, (T)c.active_frac)
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
        T rate = O::sub(uw[f], O::mul(p, O::sub(uw[f], lw[f])));
        s1[f] = __dadd_rn(L.s0[f], __dmul_rn(dt, (double)rate));   // no contraction: the oracle's rounding
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
        for (int f = 0; f < F; ++f) s1[f] = L.s0[f];
        atomicAdd(a.counters + C_NONFINITE, 1ull);
        atomicOr(reinterpret_cast<unsigned int*>(a.counters + C_STATUS), ST_NONFINITE);
    }
    // mover, Sec. 2.5: x += dt (u^n + u^{n+1}) / 2
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        double xk = __dadd_rn(L.x0[k], __dmul_rn(__dmul_rn(0.5, dt), __dadd_rn(L.s0[1 + k], s1[1 + k])));
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
    o.id[i] = L.id;
    if (o.flag) o.flag[i] = any ? 1 : 0;
    warp_count(a.counters, C_FLAGGED, any);
}

template <typename T, int DIM>
__device__ inline void skip_plain(const T (&cdf)[DIM][DIM + 2], T (&os)[DIM][2][DIM + 2])
{
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int f = 0; f < DIM + 2; ++f) os[k][s][f] = cdf[k][f];
}

// fused schedule: all stages in one thread
template <typename T, int DIM, bool GATE>
__device__ void step_one(const FitArgs& a, const StepOut& o, int64_t i)
{
    constexpr int F = DIM + 2;
    Loaded<DIM> L;
    if (step_load<T, DIM>(a, o, i, L)) return;
    Src<T, DIM, F> src(a, i);
    const int cnt = (int)a.count[i];
    const NbGlobal nb{a.idx + i * (int64_t)a.c.k_max};
    const T invS = (T)inv_scale(last_d2(src, nb, cnt));
    T cdf[DIM][F], lw[F];
    bool mlp_skip;
    if (!step_central<T, DIM, GATE>(a, o, i, L, src, nb, cnt, invS, cdf, lw, mlp_skip)) return;
    const bool plain = !mlp_skip || a.c.mlp_audit;
    T os[DIM][2][F];
    if (plain) {
        if (!step_plain<T, DIM>(a, i, src, nb, cnt, invS, cdf, os)) return;
    } else {
        skip_plain<T, DIM>(cdf, os);
    }
    step_finish<T, DIM>(a, o, i, L, os, lw, plain, mlp_skip);
}

template <typename T, int DIM, bool GATE>
__global__ void __launch_bounds__(FIT_THREADS, FitOcc<T>::fused) k_step(FitArgs a, StepOut o)
{
    if (a.list) {
        unsigned long long len = *a.list_len;
        for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < len;
             t += (unsigned long long)gridDim.x * blockDim.x)
            step_one<T, DIM, GATE>(a, o, a.list[t]);
    } else {
        int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (i < a.n) step_one<T, DIM, GATE>(a, o, i);
    }
}

// intermediate record of the split schedule, component-major over list slots:
// mid[q * cap + t], q < DIM*F central first derivatives, then F LW rates, then
// the gate bit
template <int DIM> struct MidN { static constexpr int v = DIM * (DIM + 2) + (DIM + 2) + 1; };

__device__ inline unsigned long long warp_append(unsigned long long* len, bool pred)
{
    unsigned m = __activemask();
    unsigned b = __ballot_sync(m, pred);
    int lane = (int)(threadIdx.x & 31u);
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader && b) base = atomicAdd(len, (unsigned long long)__popc(b));
    base = __shfl_sync(m, base, leader);
    return base + (unsigned long long)__popc(b & ((1u << lane) - 1u));
}

// the end of the split schedule's first stage: a particle the learned gate
// cleared is finished here; the others are appended to the plain-stage list
// with their central first derivatives and LW rates
template <typename T, int DIM>
__device__ __forceinline__ void central_append_or_finish(const FitArgs& a, const StepOut& o, int64_t i,
                                                         const Loaded<DIM>& L, const T (&cdf)[DIM][DIM + 2],
                                                         const T (&lw)[DIM + 2], bool mlp_skip)
{
    constexpr int F = DIM + 2;
    const bool plain = !mlp_skip || a.c.mlp_audit;
    const unsigned long long t = a.plain_ident ? (unsigned long long)i : warp_append(a.plain_len, plain);
    if (plain) {
        T* mid = static_cast<T*>(a.mid);
        const int64_t cap = a.mid_cap;
        a.plain_list[t] = (uint32_t)i;
        int q = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k)
#pragma unroll
            for (int f = 0; f < F; ++f) mid[(q++) * cap + t] = cdf[k][f];
#pragma unroll
        for (int f = 0; f < F; ++f) mid[(q++) * cap + t] = lw[f];
        mid[q * cap + t] = mlp_skip ? T(1) : T(0);
        return;
    }
    T os[DIM][2][F];
    skip_plain<T, DIM>(cdf, os);
    step_finish<T, DIM>(a, o, i, L, os, lw, false, true);
}

// the central stage of particle i as the split schedule's first kernel runs
// it, its list entries read through nb (NbGlobal, NbStaged)
template <typename T, int DIM, bool GATE, bool DEFER, class NB>
__device__ __forceinline__ void central_one(const FitArgs& a, const StepOut& o, int64_t i, const NB& nb)
{
    constexpr int F = DIM + 2;
    Loaded<DIM> L;
    if (step_load<T, DIM>(a, o, i, L)) return;
    Src<T, DIM, F> src(a, i);
    const int cnt = (int)a.count[i];
    const T invS = (T)inv_scale(last_d2(src, nb, cnt));
    T cdf[DIM][F], lw[F];
    bool mlp_skip;
    if (!step_central<T, DIM, GATE, DEFER>(a, o, i, L, src, nb, cnt, invS, cdf, lw, mlp_skip)) return;
    central_append_or_finish<T, DIM>(a, o, i, L, cdf, lw, mlp_skip);
}

// First kernel of the split schedule.  DEFER (FP32, correction pass where the
// ratio asks for it): a central fit that needs the correction pass is listed
// for k_step_central_refine instead, so that this kernel's warps do not run
// the pass for the few lanes that need it (2-3% of the gas cloud's stencils,
// in about half of the warps).
template <typename T, int DIM, bool GATE, bool DEFER>
__global__ void __launch_bounds__(FIT_THREADS, FitOcc<T>::central) k_step_central(FitArgs a, StepOut o)
{
    // the warp's list rows staged in shared memory (their index reads then
    // cost the L1 one wavefront per warp instead of one per lane); without
    // DEFER the correction pass's stash takes 23 KB, and 32 staged entries
    // keep the block below 48 KB of static shared memory
    constexpr int SD = DEFER ? 64 : 32;
    __shared__ uint32_t stage[SD][NB_PITCH];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    stage_rows<SD>(stage, a.idx, a.c.k_max, i < a.n ? i : -1);
    if (i >= a.n) return;
    central_one<T, DIM, GATE, DEFER>(a, o, i, NbStaged<SD>{a.idx + i * (int64_t)a.c.k_max, &stage[0][threadIdx.x]});
}

// The central fits k_step_central deferred, in full warps, with the correction
// pass on (the caller passes a configuration with refine = LP_REFINE_ALWAYS):
// the same arithmetic as an inline correction, so the same results.
template <typename T, int DIM, bool GATE>
__global__ void __launch_bounds__(FIT_THREADS, FitOcc<T>::central) k_step_central_refine(FitArgs a, StepOut o)
{
    const unsigned long long len = *a.refine_len;
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < len;
         t += (unsigned long long)gridDim.x * blockDim.x)
        central_one<T, DIM, GATE, false>(a, o, a.refine_list[t],
                                         NbGlobal{a.idx + (int64_t)a.refine_list[t] * (int64_t)a.c.k_max});
}

// the second stage of list entry t of the split schedule
template <typename T, int DIM>
__device__ __forceinline__ void plain_one(const FitArgs& a, const StepOut& o, unsigned long long t,
                                          const uint32_t* stage_col)
{
    constexpr int F = DIM + 2;
    const uint32_t iu = a.plain_list[t];
    if (iu == 0xffffffffu) return;          // (plain_ident) no plain stage for this slot
    const int64_t i = iu;
    Src<T, DIM, F> src(a, i);
    const int cnt = (int)a.count[i];
    const NbStaged<32> nb{a.idx + i * (int64_t)a.c.k_max, stage_col};
    const T invS = (T)inv_scale(last_d2(src, nb, cnt));
    // the one-sided fits first: the central stage's record and the particle's
    // state are read after them, so they hold no registers during the fits
    const DevCfg& c = a.c;
    bool ill = false;
    T out[DIM][2][F];
    bool ok[DIM][2];
    onesided_all<T, DIM, F>(src, nb, cnt, c.k_side, invS, IsF32<T>::v ? (T)c.tau32 : (T)c.tau64, (T)c.tau64,
                            out, ok, ill);
    if (IsF32<T>::v && ill) { push_redo(a, i); return; }
    const T* mid = static_cast<const T*>(a.mid);
    const int64_t cap = a.mid_cap;
    T os[DIM][2][F], lw[F];
    int q = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const T cd = mid[(q++) * cap + t];          // central derivative: where a side has no fit
            os[k][0][f] = ok[k][0] ? out[k][0][f] : cd;
            os[k][1][f] = ok[k][1] ? out[k][1][f] : cd;
        }
#pragma unroll
    for (int f = 0; f < F; ++f) lw[f] = mid[(q++) * cap + t];
    const bool mlp_skip = mid[q * cap + t] != T(0);
    Loaded<DIM> L;
    step_load<T, DIM>(a, o, i, L);          // never frozen: frozen particles are not listed
    step_finish<T, DIM>(a, o, i, L, os, lw, true, mlp_skip);
}

// the particle of plain-stage slot t (or -1: none)
__device__ __forceinline__ int64_t plain_particle(const FitArgs& a, unsigned long long t, unsigned long long len)
{
    if (t >= len) return -1;
    const uint32_t iu = a.plain_list[t];
    return iu == 0xffffffffu ? -1 : (int64_t)iu;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(FIT_THREADS, FitOcc<T>::plain) k_step_plain(FitArgs a, StepOut o)
{
    __shared__ uint32_t stage[32][NB_PITCH];
    const unsigned long long len = a.plain_ident ? (unsigned long long)a.n : *a.plain_len;
    const unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    stage_rows<32>(stage, a.idx, a.c.k_max, plain_particle(a, t, len));
    if (t < len) plain_one<T, DIM>(a, o, t, &stage[0][threadIdx.x]);
}

// Persistent forms of the split schedule's two kernels (LP_SCHED_QUEUE_FIT):
// a grid of resident blocks whose warps take their next 32 particles (list
// entries) from a work counter until none are left.  A warp whose particles
// had short stencils takes more work at once instead of holding its slot
// until the slowest warp of its block ends.  Every particle is computed by
// the same code as in the one-thread-per-particle kernels, so the results are
// identical.
__device__ __forceinline__ unsigned long long warp_take(unsigned long long* q)
{
    unsigned long long base = 0;
    if ((threadIdx.x & 31u) == 0u) base = atomicAdd(q, 32ull);
    return __shfl_sync(0xffffffffu, base, 0);
}

template <typename T, int DIM, bool GATE, bool DEFER>
__global__ void __launch_bounds__(FIT_THREADS, FitOcc<T>::central) k_step_central_q(FitArgs a, StepOut o)
{
    constexpr int SD = DEFER ? 64 : 32;               // (as in k_step_central)
    __shared__ uint32_t stage[SD][NB_PITCH];
    for (;;) {
        const unsigned long long base = warp_take(a.queue);
        if (base >= (unsigned long long)a.n) return;
        const int64_t i = (int64_t)base + (int64_t)(threadIdx.x & 31u);
        stage_rows<SD>(stage, a.idx, a.c.k_max, i < a.n ? i : -1);
        if (i < a.n)
            central_one<T, DIM, GATE, DEFER>(a, o, i,
                                             NbStaged<SD>{a.idx + i * (int64_t)a.c.k_max, &stage[0][threadIdx.x]});
        __syncwarp();                               // the staged rows are reused by the next batch
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(FIT_THREADS, FitOcc<T>::plain) k_step_plain_q(FitArgs a, StepOut o)
{
    __shared__ uint32_t stage[32][NB_PITCH];
    const unsigned long long len = a.plain_ident ? (unsigned long long)a.n : *a.plain_len;
    for (;;) {
        const unsigned long long base = warp_take(a.queue + 1);
        if (base >= len) return;
        const unsigned long long t = base + (threadIdx.x & 31u);
        stage_rows<32>(stage, a.idx, a.c.k_max, plain_particle(a, t, len));
        if (t < len) plain_one<T, DIM>(a, o, t, &stage[0][threadIdx.x]);
        __syncwarp();                               // the staged rows are reused by the next batch
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
    const NbGlobal nb{a.idx + i * (int64_t)c.k_max};
    const T invS = (T)inv_scale(last_d2(src, nb, cnt));
    const T tau = IsF32<T>::v ? (T)c.tau32 : (T)c.tau64;
    T cd[N][F];
    uint32_t st = IsF32<T>::v ? 0u : (a.list ? FIT_FP64 : 0u);
    if (central_fit<T, DIM, F>(src, nb, cnt, invS, tau, c, cd)) {
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
__global__ void __launch_bounds__(FIT_THREADS) k_derivs(FitArgs a, DerivOut o)
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
    const NbGlobal nb{a.idx + i * (int64_t)c.k_max};
    const T invS = (T)inv_scale(last_d2(src, nb, cnt));
    const T tau = IsF32<T>::v ? (T)c.tau32 : (T)c.tau64;
    T cd[N][F];
    if (central_fit<T, DIM, F>(src, nb, cnt, invS, tau, c, cd)) {
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
    {
        T o2[DIM][2][F];
        bool ok[DIM][2];
        onesided_all<T, DIM, F>(src, nb, cnt, c.k_side, invS, tau, (T)c.tau64, o2, ok, ill);
#pragma unroll
        for (int k = 0; k < DIM; ++k)
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int f = 0; f < F; ++f) os[k][s][f] = ok[k][s] ? o2[k][s][f] : cd[k][f];
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
__global__ void __launch_bounds__(FIT_THREADS) k_onesided(FitArgs a, double* out, int f_real)
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
cudaError_t launch_step_split_f32(int dim, const FitArgs& a, const StepOut& o, cudaStream_t s);
cudaError_t launch_step_split_f64(int dim, const FitArgs& a, const StepOut& o, cudaStream_t s);
cudaError_t launch_derivs_f32(int dim, int F, const FitArgs& a, const DerivOut& o, cudaStream_t s);
cudaError_t launch_derivs_f64(int dim, int F, const FitArgs& a, const DerivOut& o, cudaStream_t s);
cudaError_t launch_onesided_f32(int dim, const FitArgs& a, double* out, int f_real, cudaStream_t s);
cudaError_t launch_onesided_f64(int dim, const FitArgs& a, double* out, int f_real, cudaStream_t s);

// k_step_central_refine over the deferred list (FP32; its own translation
// unit, lp_fit_f32_refine.cu, so that its instantiation does not change how the
// other fit kernels are compiled)
template <typename T>
cudaError_t launch_central_refine(int dim, bool gate, const FitArgs& r, const StepOut& o, cudaStream_t s);
template <>
cudaError_t launch_central_refine<float>(int dim, bool gate, const FitArgs& r, const StepOut& o, cudaStream_t s);
template <>
inline cudaError_t launch_central_refine<double>(int, bool, const FitArgs&, const StepOut&, cudaStream_t)
{
    return cudaErrorNotSupported;
}

// the split schedule with its two kernels persistent over work counters
// (FP32; its own translation unit, lp_fit_f32_queue.cu).  The counters
// a.queue[0..1] must be zero.
cudaError_t launch_step_split_queue_f32(int dim, const FitArgs& a, const StepOut& o, cudaStream_t s);

// the split schedule lists the FP32 central fits that need the correction
// pass for a kernel of their own (where the correction runs only below the
// ratio; where it always runs, listing every particle would only repeat work)
template <typename T>
inline bool split_defers_t(const FitArgs& a)
{
    return IsF32<T>::v && a.refine_list && a.c.refine == LP_REFINE_AUTO;
}

inline unsigned fit_blocks(const FitArgs& a)
{
    return a.list ? 152u * 4u : (unsigned)((a.n + FIT_THREADS - 1) / FIT_THREADS);
}

#define LP_DEFINE_FIT_LAUNCHERS(T, SUF)                                                         \
    cudaError_t launch_step_##SUF(int dim, const FitArgs& a, const StepOut& o, cudaStream_t s)  \
    {                                                                                           \
        unsigned b = fit_blocks(a);                                                             \
        if (b == 0) return cudaSuccess;                                                         \
        const bool gate = o.features || a.c.estimator == LP_EST_MLP;                           \
        if (dim == 3) {                                                                         \
            if (gate) k_step<T, 3, true><<<b, FIT_THREADS, 0, s>>>(a, o);                               \
            else k_step<T, 3, false><<<b, FIT_THREADS, 0, s>>>(a, o);                                   \
        } else if (dim == 2) {                                                                  \
            if (gate) k_step<T, 2, true><<<b, FIT_THREADS, 0, s>>>(a, o);                               \
            else k_step<T, 2, false><<<b, FIT_THREADS, 0, s>>>(a, o);                                   \
        } else {                                                                                \
            if (gate) k_step<T, 1, true><<<b, FIT_THREADS, 0, s>>>(a, o);                               \
            else k_step<T, 1, false><<<b, FIT_THREADS, 0, s>>>(a, o);                                   \
        }                                                                                       \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_step_split_##SUF(int dim, const FitArgs& a, const StepOut& o,            \
                                        cudaStream_t s)                                         \
    {                                                                                           \
        auto split_defers = [](const FitArgs& x) { return split_defers_t<T>(x); };              \
        unsigned b = (unsigned)((a.n + FIT_THREADS - 1) / FIT_THREADS);                                             \
        if (b == 0) return cudaSuccess;                                                         \
        const bool gate = o.features || a.c.estimator == LP_EST_MLP;                           \
        if (split_defers(a)) {                                                                  \
            FitArgs r = a;                                                                      \
            r.c.refine = LP_REFINE_ALWAYS;                                                      \
            if (dim == 3) {                                                                     \
                if (gate) k_step_central<T, 3, true, true><<<b, FIT_THREADS, 0, s>>>(a, o);    \
                else k_step_central<T, 3, false, true><<<b, FIT_THREADS, 0, s>>>(a, o);        \
                launch_central_refine<T>(3, gate, r, o, s);                             \
                k_step_plain<T, 3><<<b, FIT_THREADS, 0, s>>>(a, o);                             \
            } else if (dim == 2) {                                                              \
                if (gate) k_step_central<T, 2, true, true><<<b, FIT_THREADS, 0, s>>>(a, o);    \
                else k_step_central<T, 2, false, true><<<b, FIT_THREADS, 0, s>>>(a, o);        \
                launch_central_refine<T>(2, gate, r, o, s);                             \
                k_step_plain<T, 2><<<b, FIT_THREADS, 0, s>>>(a, o);                             \
            } else {                                                                            \
                if (gate) k_step_central<T, 1, true, true><<<b, FIT_THREADS, 0, s>>>(a, o);    \
                else k_step_central<T, 1, false, true><<<b, FIT_THREADS, 0, s>>>(a, o);        \
                launch_central_refine<T>(1, gate, r, o, s);                             \
                k_step_plain<T, 1><<<b, FIT_THREADS, 0, s>>>(a, o);                             \
            }                                                                                   \
            return cudaGetLastError();                                                          \
        }                                                                                       \
        if (dim == 3) {                                                                         \
            if (gate) k_step_central<T, 3, true, false><<<b, FIT_THREADS, 0, s>>>(a, o);               \
            else k_step_central<T, 3, false, false><<<b, FIT_THREADS, 0, s>>>(a, o);                   \
            k_step_plain<T, 3><<<b, FIT_THREADS, 0, s>>>(a, o);                                         \
        } else if (dim == 2) {                                                                  \
            if (gate) k_step_central<T, 2, true, false><<<b, FIT_THREADS, 0, s>>>(a, o);               \
            else k_step_central<T, 2, false, false><<<b, FIT_THREADS, 0, s>>>(a, o);                   \
            k_step_plain<T, 2><<<b, FIT_THREADS, 0, s>>>(a, o);                                         \
        } else {                                                                                \
            if (gate) k_step_central<T, 1, true, false><<<b, FIT_THREADS, 0, s>>>(a, o);               \
            else k_step_central<T, 1, false, false><<<b, FIT_THREADS, 0, s>>>(a, o);                   \
            k_step_plain<T, 1><<<b, FIT_THREADS, 0, s>>>(a, o);                                         \
        }                                                                                       \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_derivs_##SUF(int dim, int F, const FitArgs& a, const DerivOut& o,        \
                                    cudaStream_t s)                                             \
    {                                                                                           \
        unsigned b = fit_blocks(a);                                                             \
        if (b == 0) return cudaSuccess;                                                         \
        if (dim == 3 && F == 1) k_derivs<T, 3, 1><<<b, FIT_THREADS, 0, s>>>(a, o);                     \
        else if (dim == 3) k_derivs<T, 3, 5><<<b, FIT_THREADS, 0, s>>>(a, o);                          \
        else if (dim == 2) k_derivs<T, 2, 5><<<b, FIT_THREADS, 0, s>>>(a, o);                          \
        else k_derivs<T, 1, 5><<<b, FIT_THREADS, 0, s>>>(a, o);                                        \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_onesided_##SUF(int dim, const FitArgs& a, double* out, int f_real,       \
                                      cudaStream_t s)                                           \
    {                                                                                           \
        unsigned b = fit_blocks(a);                                                             \
        if (b == 0) return cudaSuccess;                                                         \
        if (dim == 3) k_onesided<T, 3, 5><<<b, FIT_THREADS, 0, s>>>(a, out, f_real);                   \
        else if (dim == 2) k_onesided<T, 2, 5><<<b, FIT_THREADS, 0, s>>>(a, out, f_real);              \
        else k_onesided<T, 1, 5><<<b, FIT_THREADS, 0, s>>>(a, out, f_real);                            \
        return cudaGetLastError();                                                              \
    }

}  // namespace lp
