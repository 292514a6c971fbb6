// dtbound.cuh -- the CFL time-step bound of one cell in FP32 arithmetic,
// the rule of the mixed-precision forms (Eq. runge_kutta with the reading
// dt = cfl * min over cells of |Omega| / sum_d (|u . Sbar_d| + c |Sbar_d|)).
// One definition serves the time-step kernel and the last stage of the 3D
// FP32 stencil, which forms the next step's bound from the state it has
// just written, so that both give the same bits.
#pragma once

#include "blocks.cuh"

namespace sensei {

__device__ __forceinline__ float dtb_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float dtb_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Cell m (metric index) of block B with the FP64 conserved state q0..q4:
// false for a non-physical state (rho or p not positive and finite); else
// isum = 1 / sum_d (|u . Sbar_d| + c |Sbar_d|) over the ndir directions and
// bound = |Omega| isum, on the FP32 metric copies.  gam and gm1 are
// (float)gamma and (float)(gamma - 1).
__device__ __forceinline__ bool dt_cell_f32(const BlockDev &B, long long m, int ndir, double q0, double q1, double q2,
                                            double q3, double q4, float gam, float gm1, float &isum, float &bound)
{
    const float rho = __double2float_rn(q0), mx = __double2float_rn(q1), my = __double2float_rn(q2),
                mz = __double2float_rn(q3), E = __double2float_rn(q4);
    const float ir = dtb_rcp(rho);
    const float u = mx * ir, v = my * ir, w = mz * ir;
    const float p = gm1 * (E - 0.5f * (mx * u + my * v + mz * w));
    if (!(rho > 0.0f && p > 0.0f && rho < INFINITY && p < INFINITY)) return false;
    const float a2 = gam * p * ir;
    const float a = a2 * dtb_rsqrt(a2);
    const long long mv = B.ml.mvolume;
    float sum = 0.0f;
    for (int d = 0; d < ndir; ++d) {
        const long long q = (long long)(d * 4) * mv + m;
        const float un = u * B.sbar32[q] + v * B.sbar32[mv + q] + w * B.sbar32[2 * mv + q];
        sum += fabsf(un) + a * B.sbar32[3 * mv + q];
    }
    isum = dtb_rcp(sum);
    bound = B.vol32[m] * isum;
    return true;
}

}  // namespace sensei
