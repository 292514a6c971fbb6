// stencil_f32pd.cu -- the 3D FP32-arithmetic stencil kernel with paired
// face fluxes (stencil32p.cuh) on an FP64 stage input, the accumulating
// (FP32 flux on the FP64 state) and residual updates, with and without the
// norm partials and local time steps, for every limiter.  The FP32-storage
// first stages are in stencil_f32pe.cu.
#include "stencil32p.cuh"

namespace sensei {
cudaError_t launch_stencil32p_f64in_accum(const BatchParams<float> &p, int limiter, int grid, cudaStream_t s)
{
    return Stencil32PLauncher<double, MODE_ACCUM>::launch(p, limiter, grid, s);
}

cudaError_t launch_stencil32p_f64in_residual(const BatchParams<float> &p, int limiter, int grid, cudaStream_t s)
{
    return Stencil32PLauncher<double, MODE_RESIDUAL>::launch(p, limiter, grid, s);
}

int stencil32p_ctas_per_sm_f64in(int limiter, int mode)
{
    if (mode == MODE_INCR) return stencil32p_ctas_per_sm_f64in_incr(limiter);
    return mode == MODE_ACCUM ? Stencil32PLauncher<double, MODE_ACCUM>::ctas_per_sm(limiter)
                              : Stencil32PLauncher<double, MODE_RESIDUAL>::ctas_per_sm(limiter);
}
}  // namespace sensei
