// stencil_f32pe.cu -- the 3D FP32-arithmetic stencil kernel with paired
// face fluxes (stencil32p.cuh) on an FP64 stage input with the FP32-storage
// update (the first stage: FP32 increment and stage state from U^n), with
// and without the norm partials and local time steps, for every limiter.
#include "stencil32p.cuh"

namespace sensei {
cudaError_t launch_stencil32p_f64in_incr(const BatchParams<float> &p, int limiter, int grid, cudaStream_t s)
{
    return Stencil32PLauncher<double, MODE_INCR>::launch(p, limiter, grid, s);
}

int stencil32p_ctas_per_sm_f64in_incr(int limiter) { return Stencil32PLauncher<double, MODE_INCR>::ctas_per_sm(limiter); }
}  // namespace sensei
