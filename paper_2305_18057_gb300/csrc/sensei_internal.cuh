// sensei_internal.cuh -- device-side data layouts and launch parameters of
// the GB300 library.  Internal to csrc/; the public ABI is include/sensei.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sensei.h"
#include "df64.cuh"

namespace sensei {

constexpr int NV = 5;   // rho, rho u, rho v, rho w, rho e_t (Eq. governing)
constexpr int NG = 2;   // ghost layers: the MUSCL stencil (Eq. flux) reaches i-1..i+2

// Stencil tile: a CTA owns TI x TJ cells of an (i, j) column and marches in k.
constexpr int TI = 32;
constexpr int TJ = 8;
constexpr int NTHREADS = TI * TJ;

// Error bits OR-ed into the device error word.
constexpr unsigned ERR_NONPHYSICAL = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;     // a bounded wait on an asynchronous copy gave up

// The FP32 stencil's face-metric record of one (tile, k-plane): the unit
// normal and area (4 components, component-major) of the tile's i-faces
// (TJ rows x TI+1), j-faces (TJ+1 rows x TI) and upper k-faces (TJ x TI),
// then 1/|Omega| of its cells (TJ x TI); entries outside the block are 0.
// Records are stored k-plane-major: ((k * tiles_j + tile_j) * tiles_i + tile_i).
constexpr int REC_I = 4 * TJ * (TI + 1);
constexpr int REC_J = 4 * (TJ + 1) * TI;
constexpr int REC_K = 4 * TJ * TI;
constexpr int REC_V = TJ * TI;
constexpr int REC = REC_I + REC_J + REC_K + REC_V;
static_assert((REC * 4) % 16 == 0, "a record is one 16-byte-multiple bulk copy");

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
struct MetricLayout {
    long long mpitch, mplane, mvolume;
};

// Mutable pointers for the metrics kernel.
struct MetricsOut {
    double *n[3][4];
    double *vol, *ivol;
    double *sbar[3][4];
    float *sbar32[3][4], *vol32;   // may be null
};

// ------------------------------------------------------------------------
// Batched launches.  Every kernel of a step covers all blocks of the grid in
// one launch.  A block's static description lives in the workspace
// (BlockDev); work items are (block, tile_i, tile_j, k-chunk) numbered
// block-major, block b owning items [item0, item0 + tiles_i*tiles_j*nchunks).
// ------------------------------------------------------------------------
constexpr int MAX_BLOCKS = 256;

// state buffer slots a launch reads or writes
enum { SLOT_USER = 0, SLOT_ST0 = 1, SLOT_ST1 = 2, SLOT_X0 = 3, SLOT_X1 = 4 };

// arrays of face-gradient metrics per face family (viscous mode): grad xi_a
// (9), the area vector (3), grad xi_a . S (3)
constexpr int GVIS = 15;

struct BlockDev {
    int ni, nj, nk;
    StateLayout L;
    MetricLayout ml;
    const double *fn;       // face metrics: 12 arrays of mvolume, index (family*4 + q)
    const float2 *fdf;      // double-float grids: fn as (hi, lo) float pairs, same index (else null)
    const float *rec32;     // FP32 face-metric records of the FP32 stencil (null in FP64 mode)
    const double *vol, *ivol;
    const double *sbar;     // spectral metrics: 12 arrays of mvolume, index (direction*4 + q)
    const float *sbar32, *vol32;   // their FP32 copies and |Omega| in FP32 (null in FP64 mode)
    double *dtv;            // local time stepping: dt_c / |Omega| per cell (mvolume)
    double *wv;             // viscous: (u, v, w, p / rho) of the stage input, state layout, 4 variables
    double *rvis;           // viscous: R_nu = sum over the faces of F_nu . S_out, dense interior [5][nk][nj][ni]
    double *fvis;           // viscous: F_nu . S of every face, [family * 5 + q][mvolume]
    double *gvis;           // viscous: face-gradient metrics, [family * GVIS + n][mvolume] (viscous.cu)
    double *st64[2];        // FP64 stage states
    float *xs[2], *ds[2];   // FP32 stage states and increments
    // 3D FP32-arithmetic grids: one 128-byte tensor map per state slot
    // (SLOT_USER .. SLOT_X1) describing the slot's ghosted array as a 4D
    // tensor (padded row, rows, planes, variables) for the bulk tensor copy
    // of a stencil tile; null otherwise
    const unsigned char *tmaps;
    int tiles_i, tiles_j, kchunk, nchunks;
    long long item0;        // first work item
    long long bc0;          // first ghost-fill work unit
    int bc_type[6], nbr[6], nbr_face[6];
    double bc_prim[6][NV];
};

// ------------------------------------------------------------------------
// Stencil launch modes:
//   MODE_RESIDUAL  write R
//   MODE_ACCUM     Runge-Kutta stage with an FP64 stage state:
//                    out = alpha * Un + beta * in - gdt * dt * ivol * R
//   MODE_INCR      Runge-Kutta stage with FP32 stage storage: the FP32
//                  increment D = U^(s) - U^n,
//                    D = beta * Dprev - gdt * dt * ivol * R,
//                  stored with the FP32 stage state X = float(U^n) + D, or on
//                  the last stage accumulated in FP64, out = Un + D.
// The stage input is FP64 (TS = double: the caller's U or an FP64 stage
// state) or FP32 (TS = float: an FP32 stage state).  With push set, every
// new cell value is also written into the ghost layers it feeds (the
// neighbour's interface ghosts, the opposite periodic ghosts, the mirrored
// wall ghosts, the extrapolation ghosts) of the same output slot, so the
// next stage needs no separate ghost fill.
// ------------------------------------------------------------------------
enum { MODE_RESIDUAL = 0, MODE_ACCUM = 1, MODE_INCR = 2 };

template <typename R>
struct BatchParams {
    const BlockDev *blocks;
    int nblocks;
    long long nitems;
    int mode;
    int in_slot, out_slot;  // out_slot: SLOT_USER / SLOT_ST* (FP64) or SLOT_X* (FP32)
    int dprev, dout;        // MODE_INCR: increment slots (0 or 1), -1 for none
    int push;
    int local;              // local time stepping: the stage step is dtv[cell], not dt / |Omega|
    R gamma, kappa, eps, fix;
    R ifix;                 // 1 / fix (0 when fix is 0: the entropy fix never applies)
    R gm1, kg, c1, c2, half_eps;   // gamma - 1, gamma / (gamma - 1), eps (1 -+ kappa) / 4, eps / 2 in R
    int cons;
    int vis;                // subtract the viscous residual B.rvis
    long long wait_limit;   // bounded mbarrier waits: clock cycles before giving up
    unsigned tx_extra;      // test hook: bytes added to every tile phase's expected count
    double alpha, beta, gdt;
    const double *dt_slot;  // dt = dt_scale * *dt_slot
    double dt_scale;
    double *partials;       // 15 doubles per item (null: no norms)
    const int *order;       // launch position -> work item (null: block-major); item costs descending
    unsigned long long *dt_next;   // 3D FP32 last stage: the next step's time-step bound (bits), or null
    double gamma_d;         // gamma in FP64 (the time-step rule's constants)
    unsigned *err;
    double *user[MAX_BLOCKS];        // the caller's U, per block
    double *rout[MAX_BLOCKS];        // MODE_RESIDUAL: R[5][nk][nj][ni]
    const double *src[MAX_BLOCKS];   // MODE_RESIDUAL: |Omega| S_h (or null)
};

// The viscous residual of every block's stage input (FP64 slots).
struct VisBatch {
    const BlockDev *blocks;
    int nblocks;
    int slot;               // SLOT_USER or SLOT_ST*
    double gamma, mu;
    double kcond;           // mu gamma / ((gamma - 1) Pr)
    double *user[MAX_BLOCKS];
};

// Ghost fill of every boundary face of every block of one buffer slot.
struct BCBatch {
    const BlockDev *blocks;
    int nblocks;
    long long total;        // work units (positions x 2 layers over all faces)
    int slot;               // SLOT_USER, SLOT_ST*, SLOT_X*
    double gamma;
    double *user[MAX_BLOCKS];
};

// ------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ------------------------------------------------------------------------
cudaError_t launch_metrics(int ni, int nj, int nk, const double *X, const MetricsOut &mo,
                           const MetricLayout &ml, cudaStream_t s);
cudaError_t launch_bc(const BCBatch &p, cudaStream_t s);
// the two cell layers next to face f of state u: pack (interior) or unpack (ghosts)
cudaError_t launch_face_exchange(const BlockDev &B, double *u, int f, double *buf, int unpack, cudaStream_t s);
// the block-edge ghosts of every block of one slot (after launch_bc of the
// slot); max_units: the largest per-block count, 16 (ni + nj + nk)
cudaError_t launch_edges(const BCBatch &p, int max_units, cudaStream_t s);
// pack block B's FP64 face metrics and 1/|Omega| into its FP32 records B.rec32
cudaError_t launch_pack_records(const BlockDev &B, cudaStream_t s);
cudaError_t launch_split_df64(const BlockDev &B, cudaStream_t s);
// FP64 arithmetic on an FP64 state
cudaError_t launch_stencil_f64(const BatchParams<double> &p, int limiter, bool two_d, int grid, cudaStream_t s);
// FP32 arithmetic on an FP64 state (FP32 flux; first FP32-storage stage; residuals)
cudaError_t launch_stencil_f32(const BatchParams<float> &p, int limiter, bool two_d, int grid, cudaStream_t s);
// FP32 arithmetic on an FP32 stage state
cudaError_t launch_stencil_f32s(const BatchParams<float> &p, int limiter, bool two_d, int grid, cudaStream_t s);
// the 3D FP32-arithmetic kernel with paired face fluxes (in_f32: on an FP32 stage state)
cudaError_t launch_stencil32p(const BatchParams<float> &p, int limiter, bool in_f32, int grid, cudaStream_t s);
int stencil32p_ctas_per_sm(int limiter, bool in_f32);
cudaError_t launch_stencil32p_f64in_accum(const BatchParams<float> &p, int limiter, int grid, cudaStream_t s);
cudaError_t launch_stencil32p_f64in_residual(const BatchParams<float> &p, int limiter, int grid, cudaStream_t s);
cudaError_t launch_stencil32p_f64in_incr(const BatchParams<float> &p, int limiter, int grid, cudaStream_t s);
int stencil32p_ctas_per_sm_f64in(int limiter, int mode);
int stencil32p_ctas_per_sm_f64in_incr(int limiter);
// double-float arithmetic on an FP64 state
cudaError_t launch_stencil_df64(const BatchParams<df64> &p, int limiter, bool two_d, int grid, cudaStream_t s);
int stencil_ctas_per_sm_df64(int limiter, bool two_d);
// resident CTAs per SM of a stencil variant (0 on error); precision_kind
// 0 = FP64, 1 = FP32 arithmetic on an FP64 state, 2 = on an FP32 state
int stencil_ctas_per_sm(int precision_kind, int limiter, bool two_d);
int stencil_ctas_per_sm_f32(int precision_kind, int limiter, bool two_d);
int stencil_ctas_per_sm_f32s(int limiter, bool two_d);
// min over cells of |Omega| / sum_d (|u.Sbar_d| + c |Sbar_d|) into dt_bits; with local set,
// also dtv = cfl / sum_d (...) = dt_c / |Omega| per cell
// fp32: FP32 arithmetic on the FP32 metric copies (the mixed-precision modes);
// vfac = 4 max(4/3, gamma) mu / Pr adds the viscous bound vfac |Sbar_d|^2 / (rho |Omega|)
cudaError_t launch_dt(const BlockDev *blocks, int nblocks, long long nitems, double *const *user, double gamma,
                      int local, double cfl, unsigned long long *dt_bits, unsigned *err, int grid_x, int kchunk,
                      bool fp32, double vfac, cudaStream_t s);
// the face gradient metrics B.gvis of every block (after the descriptors
// with the boundary rules are on the device); max_faces: the largest mvolume
cudaError_t launch_vis_metrics(const BlockDev *blocks, int nblocks, long long max_faces, cudaStream_t s);
// the viscous residual B.rvis of the slot's states (after the slot's face
// and edge ghosts); max_state, max_faces, max_cells: the largest block's
// state entries per variable, mvolume and interior cells
cudaError_t launch_viscous(const VisBatch &p, long long max_state, long long max_faces, long long max_cells,
                           cudaStream_t s);
cudaError_t launch_set_scalar(double *slot, double v, cudaStream_t s);
cudaError_t launch_scale_copy(double *dst, const double *src, double scale, cudaStream_t s);
// Record the thread-local message returned by sensei_last_error (api.cu).
sensei_status fail_status(sensei_status st, const char *fmt, ...);

// Encode the tensor map of one state slot of block B (base: the slot's
// array; f32: FP32 elements, else FP64) into out (128 bytes); false if the
// driver rejects it
bool encode_state_map(void *out, const void *base, const BlockDev &B, bool f32);
constexpr int TMAP_BYTES = 128;

// The grid's CFL minimum (without the cfl factor) into host memory min_out,
// asynchronously on stream s (api.cu; the co-execution driver overlaps it
// with the host worker's minimum)
sensei_status dt_min_launch(sensei_grid *grid, double *const *U, double *min_out, cudaStream_t s);

cudaError_t launch_norms_finalize(const double *partials, int nparts, long long ncells, double *out15,
                                  cudaStream_t s);

}  // namespace sensei
