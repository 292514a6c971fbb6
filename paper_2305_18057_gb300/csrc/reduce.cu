// reduce.cu -- the time-step reduction and the residual-norm finalisation.
//
// dt = cfl * min over cells of |Omega| / sum_d (|u . Sbar_d| + c |Sbar_d|)
// (the paper states no time-step rule; this spectral-radius bound is the
// reading used), in FP64, or for the mixed-precision modes in FP32 (a time
// step within a few FP32 ulps of the FP64 one: any such dt is as stable).  The minimum of positive doubles is taken with an integer
// atomicMin on their bit patterns, which order like the values, so the
// result is exact and independent of the order.
//
// Norms ("residual print", Sec. 4): the stencil kernel leaves per-CTA FP64
// partials; one CTA sums them in a fixed order (deterministic).
#include <math.h>

#include "blocks.cuh"
#include "dtbound.cuh"

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

// Per-cell spectral radius sum_d (|u . Sbar_d| + c |Sbar_d|) and |Omega| in
// the arithmetic type R: FP64 on the FP64 metrics, or FP32 (the
// mixed-precision modes) on their FP32 copies.
template <typename R>
struct DtMath;
template <>
struct DtMath<double> {
    static __device__ __forceinline__ double cv(double x) { return x; }
    static __device__ __forceinline__ double rcp(double x) { return rcp_exact(x); }
    static __device__ __forceinline__ double rsqrt(double x) { return rsqrt_exact(x); }
    static __device__ __forceinline__ double sb(const BlockDev &B, long long q) { return B.sbar[q]; }
    static __device__ __forceinline__ double vol(const BlockDev &B, long long m) { return B.vol[m]; }
};
template <>
struct DtMath<float> {
    static __device__ __forceinline__ float cv(double x) { return __double2float_rn(x); }
    static __device__ __forceinline__ float rcp(float x)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float rsqrt(float x)
    {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float sb(const BlockDev &B, long long q) { return B.sbar32[q]; }
    static __device__ __forceinline__ float vol(const BlockDev &B, long long m) { return B.vol32[m]; }
};

// The stencil's work items (tile column x k-chunk of one block), grid-stride
// in x, each item's k-chunk split into pieces of DT_SUB planes along y, so
// that no thread walks a long column alone; each thread walks its piece.
constexpr int DT_SUB = 16;
template <typename R>
__global__ void __launch_bounds__(NTHREADS) dt_kernel(const BlockDev *blocks, int nblocks, long long nitems,
                                                      const __grid_constant__ DtUser user, double gamma,
                                                      int local, double cfl, unsigned long long *dt_bits,
                                                      unsigned *err, double vfac)
{
    using M = DtMath<R>;
    const int t = threadIdx.x;
    const int ti = t % TI, tj = t / TI;
    const R gam = (R)gamma, gm1 = (R)(gamma - 1.0);
    R best = R(INFINITY);
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
        const int k0 = chunk * B.kchunk + (int)blockIdx.y * DT_SUB;
        const int k1 = min(min(k0 + DT_SUB, chunk * B.kchunk + B.kchunk), B.nk);
        const int ndir = B.nk == 1 ? 2 : 3;
        const double *U = user.u[b];
        const long long mv = B.ml.mvolume;
        for (int k = k0; k < k1; ++k) {
            const double *c = U + cell_index(B.L, i, j, k);
            if constexpr (sizeof(R) == 4) {
                // the FP32 rule (no viscous term in the FP32 forms), shared
                // with the FP32 stencil's fused bound
                const long long m = k * B.ml.mplane + j * B.ml.mpitch + i;
                float isum, bound;
                if (!dt_cell_f32(B, m, ndir, c[0], c[B.L.sv], c[2 * B.L.sv], c[3 * B.L.sv], c[4 * B.L.sv], gam, gm1,
                                 isum, bound)) {
                    bad = true;
                    continue;
                }
                if (local) B.dtv[m] = cfl * (double)isum;
                best = fminf(best, bound);
                continue;
            }
            const R rho = M::cv(c[0]), mx = M::cv(c[B.L.sv]), my = M::cv(c[2 * B.L.sv]), mz = M::cv(c[3 * B.L.sv]),
                    E = M::cv(c[4 * B.L.sv]);
            const R ir = M::rcp(rho);
            const R u = mx * ir, v = my * ir, w = mz * ir;
            const R p = gm1 * (E - R(0.5) * (mx * u + my * v + mz * w));
            if (!(rho > R(0) && p > R(0) && rho < R(INFINITY) && p < R(INFINITY))) {
                bad = true;
                continue;
            }
            const R a2 = gam * p * ir;
            const R a = a2 * M::rsqrt(a2);
            const long long m = k * B.ml.mplane + j * B.ml.mpitch + i;
            R sum = R(0);
            // viscous bound per direction: vfac / rho |Sbar_d|^2 / |Omega| (the FP64 time step of the FP64 and double-float forms)
            const double vr = vfac > 0.0 ? vfac * (double)ir * B.ivol[m] : 0.0;
            for (int d = 0; d < ndir; ++d) {
                const long long q = (long long)(d * 4) * mv + m;
                const R un = u * M::sb(B, q) + v * M::sb(B, mv + q) + w * M::sb(B, 2 * mv + q);
                sum += fabs(un) + a * M::sb(B, 3 * mv + q);
                if (vfac > 0.0) {
                    const double s3 = (double)M::sb(B, 3 * mv + q);
                    sum += (R)(vr * (s3 * s3));
                }
            }
            const R isum = M::rcp(sum);
            if (local) B.dtv[m] = cfl * (double)isum;
            best = fmin(best, M::vol(B, m) * isum);
        }
    }
    if (bad) atomicOr(err, ERR_NONPHYSICAL);
    double bestd = (double)best;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bestd = fmin(bestd, __shfl_down_sync(0xffffffffu, bestd, o));
    __shared__ double red[NTHREADS / 32];
    if ((t & 31) == 0) red[t >> 5] = bestd;
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < NTHREADS / 32; ++w) bestd = fmin(bestd, red[w]);
        if (bestd < INFINITY) atomicMin(dt_bits, (unsigned long long)__double_as_longlong(bestd));
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
                      int local, double cfl, unsigned long long *dt_bits, unsigned *err, int grid_x, int kchunk,
                      bool fp32, double vfac, cudaStream_t s)
{
    DtUser u;
    for (int b = 0; b < nblocks; ++b) u.u[b] = user[b];
    const dim3 grid((unsigned)grid_x, (unsigned)((kchunk + DT_SUB - 1) / DT_SUB));
    if (fp32)
        dt_kernel<float><<<grid, NTHREADS, 0, s>>>(blocks, nblocks, nitems, u, gamma, local, cfl, dt_bits, err, 0.0);
    else
        dt_kernel<double><<<grid, NTHREADS, 0, s>>>(blocks, nblocks, nitems, u, gamma, local, cfl, dt_bits, err,
                                                    vfac);
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
