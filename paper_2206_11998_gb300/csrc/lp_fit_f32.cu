// lp_fit_f32.cu -- FP32 instantiations of the fit and step kernels.
#include "lp_fit_kern.cuh"

namespace lp {
LP_DEFINE_FIT_LAUNCHERS(float, f32)
}  // namespace lp
