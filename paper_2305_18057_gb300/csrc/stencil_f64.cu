// stencil_f64.cu -- FP64 instantiations of the fused stencil kernel.
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_f64(const StencilParams<double> &p, int limiter, bool two_d, cudaStream_t s)
{
    return launch_stencil_t<double, double>(p, limiter, two_d, s);
}
}  // namespace sensei
