// stencil_f64p.cu -- FP64 instantiations of the fused stencil kernel with the
// norm partials (the first stage of a step, residual evaluations).
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_f64_part(const BatchParams<double> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    return StencilLauncher<double, double, true>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm_f64_part(int limiter, bool two_d)
{
    return StencilLauncher<double, double, true>::ctas_per_sm(limiter, two_d);
}
}  // namespace sensei
