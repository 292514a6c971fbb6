// stencil_f32.cu -- the FP32-arithmetic stencil kernel on an FP64 stage
// input (FP32 flux on the FP64 state; the first FP32-storage stage;
// residuals), instantiated for every limiter in 2D; 3D launches go to the
// paired-flux kernel of stencil_f32p.cu.
#include "stencil32.cuh"

namespace sensei {
cudaError_t launch_stencil_f32(const BatchParams<float> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    if (!two_d) return launch_stencil32p(p, limiter, false, grid, s);
    return Stencil32Launcher<double>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm_f32(int precision_kind, int limiter, bool two_d)
{
    if (precision_kind == 1)
        return two_d ? Stencil32Launcher<double>::ctas_per_sm(limiter, two_d) : stencil32p_ctas_per_sm(limiter, false);
    return stencil_ctas_per_sm_f32s(limiter, two_d);
}
}  // namespace sensei
