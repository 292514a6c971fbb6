// stencil_f32.cu -- FP32-arithmetic instantiations of the fused stencil
// kernel on an FP64 state (reconstruction and flux in FP32; the update and
// every reduction FP64).
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_f32(const BatchParams<float> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    return StencilLauncher<float, double>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm_f32(int precision_kind, int limiter, bool two_d)
{
    if (precision_kind == 1) return StencilLauncher<float, double>::ctas_per_sm(limiter, two_d);
    return stencil_ctas_per_sm_f32s(limiter, two_d);
}
}  // namespace sensei
