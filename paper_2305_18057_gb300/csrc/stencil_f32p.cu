// stencil_f32p.cu -- the 3D FP32-arithmetic stencil kernel with paired face
// fluxes (stencil32p.cuh) on an FP32 stage state (the later FP32-storage
// stages), for every limiter; the tensor maps of the state slots; the
// dispatch between this and the FP64-input kernel (stencil_f32pd.cu).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "stencil32p.cuh"

namespace sensei {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

}  // namespace

// The ghosted state array of a slot as a 4D tensor: (padded row of sj
// elements, nj + 4 rows, nk + 2 gk planes, NV variables) with the slot's
// strides; element (0, 0, 0, 0) is the corner ghost cell (-2, -2, -gk) of
// variable 0.  The box is one stencil tile of one plane, all variables:
// (TW, TH, 1, NV), which lands in shared memory as [NV][TH][TW].  Boxes
// start at x = i0 (cell i0 - 2), a multiple of 32 elements, so every copy
// starts on a 16-byte boundary; columns and rows beyond the array read as 0.
bool encode_state_map(void *out, const void *base, const BlockDev &B, bool f32)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || !base) return false;
    const cuuint64_t es = f32 ? 4 : 8;
    const cuuint64_t dims[4] = {(cuuint64_t)B.L.sj, (cuuint64_t)(B.nj + 2 * NG), (cuuint64_t)(B.nk + 2 * B.L.gk),
                                (cuuint64_t)NV};
    const cuuint64_t strides[3] = {(cuuint64_t)B.L.sj * es, (cuuint64_t)B.L.sk * es, (cuuint64_t)B.L.sv * es};
    const cuuint32_t box[4] = {(cuuint32_t)TW, (cuuint32_t)TH, 1u, (cuuint32_t)NV};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUresult r = fn(reinterpret_cast<CUtensorMap *>(out), f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                    4, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// the FP32-stage-state instantiations here, the FP64-input ones in
// stencil_f32pd.cu (accumulating and residual updates) and stencil_f32pe.cu
// (FP32-storage first stages): translation units that compile in parallel
cudaError_t launch_stencil32p(const BatchParams<float> &p, int limiter, bool in_f32, int grid, cudaStream_t s)
{
    if (in_f32) return Stencil32PLauncher<float, MODE_INCR>::launch(p, limiter, grid, s);
    switch (p.mode) {
    case MODE_ACCUM: return launch_stencil32p_f64in_accum(p, limiter, grid, s);
    case MODE_RESIDUAL: return launch_stencil32p_f64in_residual(p, limiter, grid, s);
    case MODE_INCR: return launch_stencil32p_f64in_incr(p, limiter, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

int stencil32p_ctas_per_sm(int limiter, bool in_f32)
{
    if (in_f32) return Stencil32PLauncher<float, MODE_INCR>::ctas_per_sm(limiter);
    int best = 1 << 30;
    for (int m : {MODE_ACCUM, MODE_RESIDUAL, MODE_INCR}) {
        const int n = stencil32p_ctas_per_sm_f64in(limiter, m);
        if (n <= 0) return 0;
        best = n < best ? n : best;
    }
    return best;
}
}  // namespace sensei
