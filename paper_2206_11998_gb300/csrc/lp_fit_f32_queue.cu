// lp_fit_f32_queue.cu -- the split schedule's persistent kernels (FP32,
// LP_SCHED_QUEUE_FIT): grids of resident blocks whose warps take work from
// counters.  A translation unit of its own, so that these instantiations do
// not change how the other fit kernels are compiled.
#include "lp_fit_kern.cuh"

namespace lp {

namespace {

// blocks of `kernel` that fit on the device at once (0 if unknown)
template <typename K>
unsigned resident_grid(K kernel, int threads)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess || per < 1)
        return 0;
    return (unsigned)(sms * per);
}

template <int DIM, bool GATE, bool DEFER>
cudaError_t split_queue(const FitArgs& a, const StepOut& o, cudaStream_t s)
{
    const unsigned bc = resident_grid(k_step_central_q<float, DIM, GATE, DEFER>, FIT_THREADS);
    const unsigned bp = resident_grid(k_step_plain_q<float, DIM>, FIT_THREADS);
    if (bc == 0 || bp == 0) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaMemsetAsync(a.queue, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_step_central_q<float, DIM, GATE, DEFER><<<bc, FIT_THREADS, 0, s>>>(a, o);
    if (DEFER) {
        FitArgs r = a;
        r.c.refine = LP_REFINE_ALWAYS;
        if ((e = launch_central_refine<float>(DIM, GATE, r, o, s)) != cudaSuccess) return e;
    }
    k_step_plain_q<float, DIM><<<bp, FIT_THREADS, 0, s>>>(a, o);
    return cudaGetLastError();
}

template <int DIM>
cudaError_t split_queue_dim(bool gate, bool defer, const FitArgs& a, const StepOut& o, cudaStream_t s)
{
    if (gate) return defer ? split_queue<DIM, true, true>(a, o, s) : split_queue<DIM, true, false>(a, o, s);
    return defer ? split_queue<DIM, false, true>(a, o, s) : split_queue<DIM, false, false>(a, o, s);
}

}  // namespace

cudaError_t launch_step_split_queue_f32(int dim, const FitArgs& a, const StepOut& o, cudaStream_t s)
{
    if (a.n == 0) return cudaSuccess;
    const bool gate = o.features || a.c.estimator == LP_EST_MLP;
    const bool defer = split_defers_t<float>(a);
    if (dim == 3) return split_queue_dim<3>(gate, defer, a, o, s);
    if (dim == 2) return split_queue_dim<2>(gate, defer, a, o, s);
    return split_queue_dim<1>(gate, defer, a, o, s);
}

}  // namespace lp
