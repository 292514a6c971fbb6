// noalloc.cu -- residual norms for callers that cannot allocate device memory.
//
// Every other call of this library takes its scratch from a workspace the
// caller allocates.  Some callers cannot do that: a solver embedded in a host
// application whose memory pool has already reserved the device (a
// cudaMalloc there fails, or bypasses the application's accounting), or a
// monitoring hook inside a time-critical loop that must never pay for, or
// risk the failure of, an allocation.  For them this file offers one entry
// point, sensei_residual_norms_noalloc, whose scratch is a fixed array in the
// library's own device memory.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (164 KB) until the process exits.  In host code its name
// is only a stand-in, not a device address, so the address is looked up once
// per device with cudaGetSymbolAddress, with that device current, the first
// time the entry point runs on it.  The cached address belongs to the
// device's context at that time: after a cudaDeviceReset of that device the
// entry point must not be called again in the same process.
//
// A non-finite residual entry is not hidden: the sums of squares carry it
// into L2, and the maxima propagate NaN (fmax alone would drop it), so a NaN
// anywhere in R_q makes both norms of variable q NaN.
#include <mutex>

#include "sensei_internal.cuh"

namespace sensei {
namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr int kMaxParts = 2048;   // CTA partial slots in the scratch array
constexpr long long kMaxCells = (long long)kMaxParts * kThreads * kCellsPerThread;   // 8,388,608
constexpr int kQ = 2 * NV;        // per slot: sum R^2 x5, max |R| x5
constexpr int kMaxDevices = 64;

// slots [0, kMaxParts*kQ): CTA partials; the 2*NV doubles after them: results
static __device__ __align__(256) double g_norm_scratch[kMaxParts * kQ + 2 * NV];

std::mutex g_setup_mutex;

// max(a, b) that returns NaN when either operand is NaN
__device__ __forceinline__ double nan_max(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }
double *g_scratch_addr[kMaxDevices] = {};

// CTA b reduces the cells [b*chunk, (b+1)*chunk) of every variable of the
// dense residual R[5][n] and writes its 10 partials to slot b.  Every slot
// the finaliser reads is written by the same call, so nothing has to be
// cleared between calls.
__global__ void noalloc_partials(const double *__restrict__ R, long long n, long long chunk, double *scratch)
{
    const long long lo = blockIdx.x * chunk;
    const long long hi = min(lo + chunk, n);
    __shared__ double red[kQ][kThreads / 32];
    for (int v = 0; v < NV; ++v) {
        double s2 = 0.0, mx = 0.0;
        for (long long c = lo + threadIdx.x; c < hi; c += kThreads) {
            double r = R[v * n + c];
            s2 += r * r;
            mx = nan_max(mx, fabs(r));
        }
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
            mx = nan_max(mx, __shfl_down_sync(0xffffffffu, mx, o));
        }
        if ((threadIdx.x & 31) == 0) {
            red[v][threadIdx.x >> 5] = s2;
            red[NV + v][threadIdx.x >> 5] = mx;
        }
    }
    __syncthreads();
    if (threadIdx.x < kQ) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w)
            acc = threadIdx.x < NV ? acc + red[threadIdx.x][w] : nan_max(acc, red[threadIdx.x][w]);
        scratch[(long long)blockIdx.x * kQ + threadIdx.x] = acc;
    }
}

// one warp per quantity, fixed order: deterministic
__global__ void noalloc_finalize(double *scratch, int nparts, long long n)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= kQ) return;
    double acc = 0.0;
    for (int p = lane; p < nparts; p += 32) {
        double x = scratch[(long long)p * kQ + q];
        acc = q < NV ? acc + x : nan_max(acc, x);
    }
    for (int o = 16; o > 0; o >>= 1) {
        double y = __shfl_down_sync(0xffffffffu, acc, o);
        acc = q < NV ? acc + y : nan_max(acc, y);
    }
    if (lane == 0) scratch[kMaxParts * kQ + q] = q < NV ? sqrt(acc / (double)n) : acc;
}

}  // namespace
}  // namespace sensei

using namespace sensei;

extern "C" sensei_status sensei_residual_norms_noalloc(const double *R, int ni, int nj, int nk, double *l2,
                                                       double *linf, sensei_stream stream)
{
    if (!R) return fail_status(SENSEI_ERR_INVALID_ARG, "R is NULL");
    if (ni < 1 || nj < 1 || nk < 1) return fail_status(SENSEI_ERR_INVALID_ARG, "need ni, nj, nk >= 1");
    const long long n = (long long)ni * nj * nk;
    if (n > kMaxCells)
        return fail_status(SENSEI_ERR_INVALID_ARG,
                           "sensei_residual_norms_noalloc handles at most 8388608 cells (its fixed scratch "
                           "holds 2048 partials); got %lld",
                           n);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_status(SENSEI_ERR_UNSUPPORTED, "device index %d too large", dev);
    double *scratch;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            // set-up, once per device, with that device current
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_norm_scratch);
            if (e != cudaSuccess)
                return fail_status(SENSEI_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_scratch_addr[dev] = (double *)p;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long chunk = (long long)kThreads * kCellsPerThread;
    const int nparts = (int)((n + chunk - 1) / chunk);
    noalloc_partials<<<nparts, kThreads, 0, s>>>(R, n, chunk, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "partials kernel: %s", cudaGetErrorString(e));
    noalloc_finalize<<<1, 32 * kQ, 0, s>>>(scratch, nparts, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "finalize kernel: %s", cudaGetErrorString(e));
    double host[kQ];
    e = cudaMemcpyAsync(host, scratch + (long long)kMaxParts * kQ, sizeof host, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "reading the norms: %s", cudaGetErrorString(e));
    for (int q = 0; q < NV; ++q) {
        if (l2) l2[q] = host[q];
        if (linf) linf[q] = host[NV + q];
    }
    return SENSEI_OK;
}
