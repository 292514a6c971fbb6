// stencil_f64.cu -- FP64 instantiations of the fused stencil kernel without
// the norm partials (the stages after the first), and the FP64 dispatch.
#include "stencil.cuh"

namespace sensei {
cudaError_t launch_stencil_f64_part(const BatchParams<double> &p, int limiter, bool two_d, int grid, cudaStream_t s);
int stencil_ctas_per_sm_f64_part(int limiter, bool two_d);

cudaError_t launch_stencil_f64(const BatchParams<double> &p, int limiter, bool two_d, int grid, cudaStream_t s)
{
    if (p.partials) return launch_stencil_f64_part(p, limiter, two_d, grid, s);
    return StencilLauncher<double, double, false>::launch(p, limiter, two_d, grid, s);
}

int stencil_ctas_per_sm(int precision_kind, int limiter, bool two_d)
{
    if (precision_kind == 0) {
        const int a = StencilLauncher<double, double, false>::ctas_per_sm(limiter, two_d);
        const int b = stencil_ctas_per_sm_f64_part(limiter, two_d);
        return a < b ? a : b;
    }
    if (precision_kind == 3) return stencil_ctas_per_sm_df64(limiter, two_d);
    return stencil_ctas_per_sm_f32(precision_kind, limiter, two_d);
}
}  // namespace sensei
