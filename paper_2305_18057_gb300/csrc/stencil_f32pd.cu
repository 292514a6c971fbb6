// stencil_f32pd.cu -- the 3D FP32-arithmetic stencil kernel with paired
// face fluxes (stencil32p.cuh) on an FP64 stage input: FP32 flux on the FP64
// state, the first FP32-storage stage and residuals, each update mode with
// and without the norm partials, for every limiter.
#include "stencil32p.cuh"

namespace sensei {
cudaError_t launch_stencil32p_f64in(const BatchParams<float> &p, int limiter, int grid, cudaStream_t s)
{
    return Stencil32PLauncher<double>::launch(p, limiter, grid, s);
}

int stencil32p_ctas_per_sm_f64in(int limiter) { return Stencil32PLauncher<double>::ctas_per_sm(limiter); }
}  // namespace sensei
