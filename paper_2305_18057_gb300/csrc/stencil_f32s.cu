// stencil_f32s.cu -- FP32-arithmetic instantiations of the fused stencil
// kernel on an FP32 stage state (the stages after the first of the
// FP32-storage mode).
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_f32s(const StencilParams<float> &p, int limiter, bool two_d, cudaStream_t s)
{
    return launch_stencil_t<float, float>(p, limiter, two_d, s);
}
}  // namespace sensei
