// lp_fit_f32_refine.cu -- the split schedule's correction kernel (FP32):
// the central fits the first kernel deferred, in full warps.
#include "lp_fit_kern.cuh"

namespace lp {

template <>
cudaError_t launch_central_refine<float>(int dim, bool gate, const FitArgs& r, const StepOut& o, cudaStream_t s)
{
    const unsigned b = 152u * 4u;
    if (dim == 3) {
        if (gate) k_step_central_refine<float, 3, true><<<b, FIT_THREADS, 0, s>>>(r, o);
        else k_step_central_refine<float, 3, false><<<b, FIT_THREADS, 0, s>>>(r, o);
    } else if (dim == 2) {
        if (gate) k_step_central_refine<float, 2, true><<<b, FIT_THREADS, 0, s>>>(r, o);
        else k_step_central_refine<float, 2, false><<<b, FIT_THREADS, 0, s>>>(r, o);
    } else {
        if (gate) k_step_central_refine<float, 1, true><<<b, FIT_THREADS, 0, s>>>(r, o);
        else k_step_central_refine<float, 1, false><<<b, FIT_THREADS, 0, s>>>(r, o);
    }
    return cudaGetLastError();
}

}  // namespace lp
