// stencil_df64p.cu -- double-float instantiations of the fused stencil kernel
// with the norm partials (the first stage of a step, residual evaluations).
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_df64_part(const BatchParams<df64> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    return StencilLauncher<df64, double, true>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm_df64_part(int limiter, bool two_d)
{
    return StencilLauncher<df64, double, true>::ctas_per_sm(limiter, two_d);
}
}  // namespace sensei
