// stencil_f32s.cu -- the FP32-arithmetic stencil kernel on an FP32 stage
// state (the stages after the first of the FP32-storage mode), 2D; 3D
// launches go to the paired-flux kernel of stencil_f32p.cu.
#include "stencil32.cuh"

namespace sensei {
cudaError_t launch_stencil_f32s(const BatchParams<float> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    if (!two_d) return launch_stencil32p(p, limiter, true, grid, s);
    return Stencil32Launcher<float>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm_f32s(int limiter, bool two_d)
{
    return two_d ? Stencil32Launcher<float>::ctas_per_sm(limiter, two_d) : stencil32p_ctas_per_sm(limiter, true);
}
}  // namespace sensei
