// stencil_df64.cu -- the fused stencil kernel in double-float arithmetic on
// an FP64 state (FP64-class accuracy computed on the FP32 pipe; the update
// and every reduction FP64), with and without the norm partials.
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_df64(const BatchParams<df64> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    if (p.partials) return StencilLauncher<df64, double, true>::launch(p, limiter, two_d, grid, s);
    return StencilLauncher<df64, double, false>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm_df64(int limiter, bool two_d)
{
    const int a = StencilLauncher<df64, double, false>::ctas_per_sm(limiter, two_d);
    const int b = StencilLauncher<df64, double, true>::ctas_per_sm(limiter, two_d);
    return a < b ? a : b;
}
}  // namespace sensei
