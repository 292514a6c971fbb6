// reduce.cu -- the time-step reduction and the residual-norm finalisation.
//
// dt = cfl * min over cells of |Omega| / sum_d (|u . Sbar_d| + c |Sbar_d|)
// (the paper states no time-step rule; this spectral-radius bound is the
// reading used).  The minimum of positive doubles is taken with an integer
// atomicMin on their bit patterns, which order like the values, so the
// result is exact and independent of the order.
//
// Norms ("residual print", Sec. 4): the stencil kernel leaves per-CTA FP64
// partials; one CTA sums them in a fixed order (deterministic).
#include <math.h>

#include "sensei_internal.cuh"

namespace sensei {
namespace {

// Reciprocal and reciprocal square root of a positive normal double: the
// hardware approximations (20 bits on sm_103a) refined by two Newton steps,
// r' = r + r (1 - d r) and y' = y + (y/2) (1 - x y^2), to within an ulp.
__device__ __forceinline__ double rcp_exact(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    for (int n = 0; n < 2; ++n) r = fma(r, fma(-d, r, 1.0), r);
    return r;
}

__device__ __forceinline__ double rsqrt_exact(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    for (int n = 0; n < 2; ++n) y = fma(0.5 * y, fma(-(x * y), y, 1.0), y);
    return y;
}

__global__ void dt_kernel(int ni, int nj, int nk, StateLayout L, const double *__restrict__ U, CellMetrics cm,
                          MetricLayout ml, double gamma, unsigned long long *dt_bits, unsigned *err)
{
    const long long total = (long long)ni * nj * nk;
    const int ndir = nk == 1 ? 2 : 3;
    double best = INFINITY;
    bool bad = false;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % ni);
        int j = (int)((t / ni) % nj);
        int k = (int)(t / ((long long)ni * nj));
        const double *c = U + L.off + (long long)k * L.sk + (long long)j * L.sj + i;
        double rho = c[0], mx = c[L.sv], my = c[2 * L.sv], mz = c[3 * L.sv], E = c[4 * L.sv];
        double ir = rcp_exact(rho);
        double u = mx * ir, v = my * ir, w = mz * ir;
        double p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v + mz * w));
        if (!(rho > 0.0 && p > 0.0 && rho < INFINITY && p < INFINITY)) {
            bad = true;
            continue;
        }
        const double a2 = gamma * p * ir;
        double a = a2 * rsqrt_exact(a2);
        long long m = k * ml.mplane + j * ml.mpitch + i;
        double sum = 0.0;
        for (int d = 0; d < ndir; ++d) {
            double un = u * cm.sbar[d][0][m] + v * cm.sbar[d][1][m] + w * cm.sbar[d][2][m];
            sum += fabs(un) + a * cm.sbar[d][3][m];
        }
        double loc = cm.vol[m] * rcp_exact(sum);
        best = fmin(best, loc);
    }
    if (bad) atomicOr(err, ERR_NONPHYSICAL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_down_sync(0xffffffffu, best, o));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = fmin(best, red[w]);
        if (best < INFINITY) atomicMin(dt_bits, (unsigned long long)__double_as_longlong(best));
    }
}

__global__ void set_scalar_kernel(double *slot, double v) { *slot = v; }

__global__ void scale_copy_kernel(double *dst, const double *src, double scale) { *dst = scale * *src; }

// partials: 15 doubles per CTA (sum R^2 x5, max |R| x5, sum |Omega| U x5).
// Warp q sums quantity q: lane l takes parts l, l+32, ... in order, then a
// fixed shuffle tree.
__global__ void norms_finalize_kernel(const double *__restrict__ partials, int nparts, long long ncells,
                                      double *out15)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= 3 * NV) return;
    const bool is_max = q >= NV && q < 2 * NV;
    double acc = 0.0;
    for (int n = lane; n < nparts; n += 32) {
        double x = partials[(long long)n * 3 * NV + q];
        acc = is_max ? fmax(acc, x) : acc + x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double y = __shfl_down_sync(0xffffffffu, acc, o);
        acc = is_max ? fmax(acc, y) : acc + y;
    }
    if (lane == 0) out15[q] = q < NV ? sqrt(acc / (double)ncells) : acc;
}

}  // namespace

cudaError_t launch_dt(int ni, int nj, int nk, const StateLayout &L, const double *U, const CellMetrics &cm,
                      const MetricLayout &ml, double gamma, unsigned long long *dt_bits, unsigned *err,
                      cudaStream_t s)
{
    long long total = (long long)ni * nj * nk;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    dt_kernel<<<(unsigned)blocks, 256, 0, s>>>(ni, nj, nk, L, U, cm, ml, gamma, dt_bits, err);
    return cudaGetLastError();
}

cudaError_t launch_set_scalar(double *slot, double v, cudaStream_t s)
{
    set_scalar_kernel<<<1, 1, 0, s>>>(slot, v);
    return cudaGetLastError();
}

cudaError_t launch_scale_copy(double *dst, const double *src, double scale, cudaStream_t s)
{
    scale_copy_kernel<<<1, 1, 0, s>>>(dst, src, scale);
    return cudaGetLastError();
}

cudaError_t launch_norms_finalize(const double *partials, int nparts, long long ncells, double *out15, cudaStream_t s)
{
    norms_finalize_kernel<<<1, 32 * 3 * NV, 0, s>>>(partials, nparts, ncells, out15);
    return cudaGetLastError();
}

}  // namespace sensei
