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

#include "blocks.cuh"

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

struct DtUser {
    double *u[MAX_BLOCKS];
};

// One CTA per work item (tile column x k-chunk of one block), grid-stride
// over the items; each thread walks its column.
__global__ void __launch_bounds__(NTHREADS) dt_kernel(const BlockDev *blocks, int nblocks, long long nitems,
                                                      const __grid_constant__ DtUser user, double gamma,
                                                      int local, double cfl, unsigned long long *dt_bits,
                                                      unsigned *err)
{
    const int t = threadIdx.x;
    const int ti = t % TI, tj = t / TI;
    double best = INFINITY;
    bool bad = false;
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int b = find_block_item(blocks, nblocks, item);
        const BlockDev &B = blocks[b];
        long long rest = item - B.item0;
        const int tile_i = (int)(rest % B.tiles_i);
        rest /= B.tiles_i;
        const int tile_j = (int)(rest % B.tiles_j);
        const int chunk = (int)(rest / B.tiles_j);
        const int i = tile_i * TI + ti, j = tile_j * TJ + tj;
        if (i >= B.ni || j >= B.nj) continue;
        const int k0 = chunk * B.kchunk, k1 = min(k0 + B.kchunk, B.nk);
        const int ndir = B.nk == 1 ? 2 : 3;
        const double *U = user.u[b];
        const long long mv = B.ml.mvolume;
        for (int k = k0; k < k1; ++k) {
            const double *c = U + cell_index(B.L, i, j, k);
            double rho = c[0], mx = c[B.L.sv], my = c[2 * B.L.sv], mz = c[3 * B.L.sv], E = c[4 * B.L.sv];
            double ir = rcp_exact(rho);
            double u = mx * ir, v = my * ir, w = mz * ir;
            double p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v + mz * w));
            if (!(rho > 0.0 && p > 0.0 && rho < INFINITY && p < INFINITY)) {
                bad = true;
                continue;
            }
            const double a2 = gamma * p * ir;
            const double a = a2 * rsqrt_exact(a2);
            const long long m = k * B.ml.mplane + j * B.ml.mpitch + i;
            double sum = 0.0;
            for (int d = 0; d < ndir; ++d) {
                const double *sb = B.sbar + (long long)(d * 4) * mv;
                double un = u * sb[m] + v * sb[mv + m] + w * sb[2 * mv + m];
                sum += fabs(un) + a * sb[3 * mv + m];
            }
            const double isum = rcp_exact(sum);
            if (local) B.dtv[m] = cfl * isum;
            best = fmin(best, B.vol[m] * isum);
        }
    }
    if (bad) atomicOr(err, ERR_NONPHYSICAL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_down_sync(0xffffffffu, best, o));
    __shared__ double red[NTHREADS / 32];
    if ((t & 31) == 0) red[t >> 5] = best;
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < NTHREADS / 32; ++w) best = fmin(best, red[w]);
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

cudaError_t launch_dt(const BlockDev *blocks, int nblocks, long long nitems, double *const *user, double gamma,
                      int local, double cfl, unsigned long long *dt_bits, unsigned *err, int grid, cudaStream_t s)
{
    DtUser u;
    for (int b = 0; b < nblocks; ++b) u.u[b] = user[b];
    dt_kernel<<<grid, NTHREADS, 0, s>>>(blocks, nblocks, nitems, u, gamma, local, cfl, dt_bits, err);
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
