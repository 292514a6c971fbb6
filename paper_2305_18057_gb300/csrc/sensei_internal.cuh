// sensei_internal.cuh -- device-side data layouts and launch parameters of
// the GB300 library.  Internal to csrc/; the public ABI is include/sensei.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sensei.h"

namespace sensei {

constexpr int NV = 5;   // rho, rho u, rho v, rho w, rho e_t (Eq. governing)
constexpr int NG = 2;   // ghost layers: the MUSCL stencil (Eq. flux) reaches i-1..i+2

// Stencil tile: a CTA owns TI x TJ cells of an (i, j) column and marches in k.
constexpr int TI = 32;
constexpr int TJ = 8;
constexpr int NTHREADS = TI * TJ;

// Error bits OR-ed into the device error word.
constexpr unsigned ERR_NONPHYSICAL = 1u;

// ------------------------------------------------------------------------
// One block's state array: element  base[off + v*sv + k*sk + j*sj + i].
// ------------------------------------------------------------------------
struct StateLayout {
    long long sj, sk, sv;   // strides (elements)
    long long off;          // element offset of interior cell (0,0,0), variable 0
    long long elems;        // elements of the whole array
    int gk;                 // ghost layers in k (0 for a 2D block)
};

// ------------------------------------------------------------------------
// Metrics of one block, "node-grid" layout: entry (i, j, k) at
// k*mplane + j*mpitch + i for 0 <= i <= ni, 0 <= j <= nj, 0 <= k <= nk.
// Face family d (0 = i, 1 = j, 2 = k) stores the unit normal (nx, ny, nz)
// and the area |S| of the face with lowest corner node (i, j, k).  Cell
// arrays use the entries with i < ni, j < nj, k < nk.
// ------------------------------------------------------------------------
template <typename R>
struct FaceMetrics {
    const R *n[3][4];       // [family][nx, ny, nz, area]
};

struct CellMetrics {
    const double *vol;      // |Omega|
    const double *ivol;     // 1 / |Omega|
    const float *ivol32;    // 1 / |Omega| rounded to FP32 (FP32-storage stages)
    const double *sbar[3][4];   // per direction d: mean area vector of the two d-faces (3), its length
};

struct MetricLayout {
    long long mpitch, mplane, mvolume;
};

// Mutable pointers for the metrics kernel.
struct MetricsOut {
    double *n[3][4];
    float *n32[3][4];       // FP32 copies for the FP32-flux stencil (may be null)
    double *vol, *ivol;
    float *ivol32;          // may be null
    double *sbar[3][4];
};

// ------------------------------------------------------------------------
// Stencil launch modes:
//   MODE_RESIDUAL  write R
//   MODE_ACCUM     Runge-Kutta stage with an FP64 stage state:
//                    out = alpha * Un + beta * in - gdt * dt * ivol * R
//   MODE_INCR      Runge-Kutta stage with FP32 stage storage: the FP32
//                  increment D = U^(s) - U^n,
//                    D = beta * Dprev - gdt * dt * ivol * R,
//                  stored with the FP32 stage state X = float(U^n) + D
//                  (dout, xout), or on the last stage accumulated in FP64,
//                    out = Un + D.
// The stage input `in` is FP64 (TS = double) or FP32 (TS = float) with the
// element strides of StateLayout.
// ------------------------------------------------------------------------
enum { MODE_RESIDUAL = 0, MODE_ACCUM = 1, MODE_INCR = 2 };

template <typename R>
struct StencilParams {
    int ni, nj, nk;
    int tiles_i, tiles_j, kchunk, nchunks;
    StateLayout L;
    int mode;
    const void *in;         // stage input (ghosts filled), double or float
    const double *un;       // U^n (null when not needed)
    double *out;            // FP64 stage output
    const float *dprev;     // MODE_INCR: previous increment (null on the first stage)
    float *dout, *xout;     // MODE_INCR: increment and FP32 stage state (null on the last stage)
    double *Rout;           // residual R[5][nk][nj][ni] (residual mode)
    const double *src;      // |Omega| S_h, same layout as Rout (may be null)
    FaceMetrics<R> fm;
    CellMetrics cm;
    MetricLayout ml;
    R gamma, kappa, eps, fix;
    int cons;               // reconstruct conserved variables
    double alpha, beta, gdt;
    const double *dt_slot;  // dt = dt_scale * *dt_slot
    double dt_scale;
    double *partials;       // 15 doubles per CTA (null: no norms)
    unsigned *err;
};

// Boundary fill of one block: 6 faces; T = double (state) or float (FP32
// stage state).
template <typename T>
struct FaceBC {
    int type;
    double prim[NV];
    const T *nbr;           // neighbour block state (INTERFACE)
    StateLayout nL;
    int nni, nnj, nnk;      // neighbour dims
    int nbr_face;
};

template <typename T>
struct BCParamsT {
    int ni, nj, nk;
    StateLayout L;
    T *U;
    FaceBC<T> f[6];
    int nfaces;             // 4 in 2D, 6 in 3D
    long long count[6];     // work items per face (positions x layers)
    double gamma;
    FaceMetrics<double> fm;
    MetricLayout ml;
};
using BCParams = BCParamsT<double>;

// ------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ------------------------------------------------------------------------
cudaError_t launch_metrics(int ni, int nj, int nk, const double *X, const MetricsOut &mo,
                           const MetricLayout &ml, cudaStream_t s);
cudaError_t launch_bc(const BCParamsT<double> &p, cudaStream_t s);
cudaError_t launch_bc(const BCParamsT<float> &p, cudaStream_t s);
// FP64 arithmetic on an FP64 state
cudaError_t launch_stencil_f64(const StencilParams<double> &p, int limiter, bool two_d, cudaStream_t s);
// FP32 arithmetic on an FP64 state (FP32 flux; first FP32-storage stage; residuals)
cudaError_t launch_stencil_f32(const StencilParams<float> &p, int limiter, bool two_d, cudaStream_t s);
// FP32 arithmetic on an FP32 stage state
cudaError_t launch_stencil_f32s(const StencilParams<float> &p, int limiter, bool two_d, cudaStream_t s);
cudaError_t launch_dt(int ni, int nj, int nk, const StateLayout &L, const double *U, const CellMetrics &cm,
                      const MetricLayout &ml, double gamma, unsigned long long *dt_bits, unsigned *err,
                      cudaStream_t s);
cudaError_t launch_set_scalar(double *slot, double v, cudaStream_t s);
cudaError_t launch_scale_copy(double *dst, const double *src, double scale, cudaStream_t s);
// Record the thread-local message returned by sensei_last_error (api.cu).
sensei_status fail_status(sensei_status st, const char *fmt, ...);

cudaError_t launch_norms_finalize(const double *partials, int nparts, long long ncells, double *out15,
                                  cudaStream_t s);

}  // namespace sensei
