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
    double *sbar[3][4];
};

// ------------------------------------------------------------------------
// Stencil launch: residual mode (write R) or Runge-Kutta stage mode
//   out = alpha * Un + beta * in - gdt * dt * ivol * R
// ------------------------------------------------------------------------
template <typename R>
struct StencilParams {
    int ni, nj, nk;
    int tiles_i, tiles_j, kchunk, nchunks;
    StateLayout L;
    const double *in;       // stage input (ghosts filled)
    const double *un;       // U^n (null when alpha == 0)
    double *out;            // stage output (null in residual mode)
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

// Boundary fill of one block: 6 faces.
struct FaceBC {
    int type;
    double prim[NV];
    const double *nbr;      // neighbour block state (INTERFACE)
    StateLayout nL;
    int nni, nnj, nnk;      // neighbour dims
    int nbr_face;
};

struct BCParams {
    int ni, nj, nk;
    StateLayout L;
    double *U;
    FaceBC f[6];
    int nfaces;             // 4 in 2D, 6 in 3D
    long long count[6];     // work items per face (positions x layers)
    double gamma;
    FaceMetrics<double> fm;
    MetricLayout ml;
};

// ------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ------------------------------------------------------------------------
cudaError_t launch_metrics(int ni, int nj, int nk, const double *X, const MetricsOut &mo,
                           const MetricLayout &ml, cudaStream_t s);
cudaError_t launch_bc(const BCParams &p, cudaStream_t s);
cudaError_t launch_stencil_f64(const StencilParams<double> &p, int limiter, bool two_d, cudaStream_t s);
cudaError_t launch_stencil_f32(const StencilParams<float> &p, int limiter, bool two_d, cudaStream_t s);
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
