// stencil_f64.cu -- FP64 instantiations of the fused stencil kernel.
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_f64(const BatchParams<double> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    return StencilLauncher<double, double>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm(int precision_kind, int limiter, bool two_d)
{
    if (precision_kind == 0) return StencilLauncher<double, double>::ctas_per_sm(limiter, two_d);
    return stencil_ctas_per_sm_f32(precision_kind, limiter, two_d);
}
}  // namespace sensei
