// lp_fit_f64.cu -- FP64 instantiations of the fit and step kernels (the FP64
// path, and the FP64 redo of stencils the FP32 pass found ill-conditioned).
#include "lp_fit_kern.cuh"

namespace lp {
LP_DEFINE_FIT_LAUNCHERS(double, f64)
}  // namespace lp
