// stencil_f32.cu -- FP32-arithmetic instantiations of the fused stencil
// kernel on an FP64 state (reconstruction and flux in FP32; the update and
// every reduction FP64).
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_f32(const StencilParams<float> &p, int limiter, bool two_d, cudaStream_t s)
{
    return launch_stencil_t<float, double>(p, limiter, two_d, s);
}
}  // namespace sensei
