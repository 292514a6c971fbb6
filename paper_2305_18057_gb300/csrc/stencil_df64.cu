// stencil_df64.cu -- the fused stencil kernel in double-float arithmetic on
// an FP64 state (FP64-class accuracy computed on the FP32 pipe; the update
// and every reduction FP64) without the norm partials, and the double-float
// dispatch; the instantiations with the partials are in stencil_df64p.cu
// (two translation units that compile in parallel).
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_df64_part(const BatchParams<df64> &p, int limiter, bool two_d, int grid, cudaStream_t s);
int stencil_ctas_per_sm_df64_part(int limiter, bool two_d);

cudaError_t launch_stencil_df64(const BatchParams<df64> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    if (p.partials) return launch_stencil_df64_part(p, limiter, two_d, grid, s);
    return StencilLauncher<df64, double, false>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm_df64(int limiter, bool two_d)
{
    const int a = StencilLauncher<df64, double, false>::ctas_per_sm(limiter, two_d);
    const int b = stencil_ctas_per_sm_df64_part(limiter, two_d);
    return a < b ? a : b;
}
}  // namespace sensei
