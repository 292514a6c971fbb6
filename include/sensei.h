/*
 * sensei.h -- C ABI of the GB300 (sm_103a) library for the explicit
 * finite-volume Euler residual and Runge-Kutta stage update on structured
 * (multi)block grids: the data-parallel hot path of the SENSEI solver,
 * arXiv 2305.18057.
 *
 * The problem statement the calls follow (citations are to the paper):
 *   - the conserved variables Q = (rho, rho u, rho v, rho w, rho e_t) and the
 *     inviscid normal flux F_{i,n} of Eq. governing (Sec. 2);
 *   - the multi-block structured grid of Sec. 2;
 *   - the semi-discrete form |Omega_i| dU/dt + R_h = 0 (Eq. spatial_residual)
 *     with R_h = sum over the f cell faces of F_{i,n} Delta s - |Omega| S_h
 *     (Eq. residual; f = 4 in 2D, 6 in 3D);
 *   - MUSCL extrapolation with a limiter (Eq. flux, Sec. 5);
 *   - explicit Runge-Kutta marching (Eq. runge_kutta, Sec. 3.2);
 *   - ghost-cell boundary enforcement kept on the GPU (Sec. 5, "Ghost cell
 *     extrapolation on the GPU") and a per-iteration residual print (Sec. 4).
 *
 * Readings of what the paper leaves open (the flux function, reconstructed
 * variables, limiter, RK coefficients, time-step rule, ghost rules) are the
 * documented defaults of each call below.
 *
 * Conventions for every call:
 *   - All state, residual, node and source arrays are CALLER-OWNED device
 *     memory.  The library never allocates device memory: its scratch
 *     (metrics, Runge-Kutta stage buffers, reduction partials) lives in a
 *     caller-allocated workspace handed to sensei_create_grid.  The one
 *     exception is sensei_residual_norms_noalloc, whose scratch is a static
 *     164 KB array in the library's own device memory (below).
 *   - Pointer arrays ("one per block") are HOST arrays of DEVICE pointers.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) except sensei_norms, which synchronises it.
 *   - Errors: a call returns a sensei_status; nothing throws or aborts
 *     across the ABI.  Argument errors are detected on the host before any
 *     launch and leave device memory untouched.  sensei_last_error() gives a
 *     thread-local message for the last failing call of the calling thread.
 *   - Threading: a grid may be used by one host thread at a time.
 *   - Device: the grid belongs to the device that was current when it was
 *     created; later calls make that device current.
 *   - Batching: a grid holds up to 256 blocks, all 2D or all 3D; every kernel
 *     of a call covers all blocks in one launch.  Calls after sensei_set_bc
 *     (or sensei_autotune) first upload the block table, which synchronises
 *     the stream once.
 */
#ifndef SENSEI_H
#define SENSEI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sensei_grid sensei_grid;   /* opaque, library-owned host object */
typedef void *sensei_stream;              /* a cudaStream_t */

typedef enum {
    SENSEI_OK = 0,
    SENSEI_ERR_INVALID_ARG = 1,   /* bad pointer, size, enum, block/face index or layout */
    SENSEI_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has the CUDA error) */
    SENSEI_ERR_NONPHYSICAL = 3,   /* a kernel met rho <= 0, p <= 0 or a non-finite value */
    SENSEI_ERR_TIMEOUT = 4,       /* a bounded device wait gave up (the FP32 stencil's tile copies; reported by sensei_norms) */
    SENSEI_ERR_UNSUPPORTED = 5,   /* valid request this build does not implement */
    SENSEI_ERR_STATE = 6          /* call out of order (e.g. a boundary face left unset) */
} sensei_status;

/* Arithmetic of the stencil (reconstruction + flux).  The Runge-Kutta
 * accumulation, the conservation sums and the residual norms are FP64 in
 * every mode. */
typedef enum {
    SENSEI_FP64 = 0,        /* FP64 state, FP64 flux */
    SENSEI_FP32_FLUX = 1,   /* FP64 state; reconstruction and flux in FP32 */
    SENSEI_FP32_STORE = 2,  /* FP64 master state U^n; FP32 stage states and FP32 flux */
    SENSEI_DF64 = 3         /* FP64 state; reconstruction and flux in double-float arithmetic
                             * (pairs of FP32 numbers, about 48 significant bits, computed on
                             * the FP32 pipe); not in the paper: an FP64-class alternative for
                             * GPUs whose FP64 pipe is narrow.  The workspace then also holds
                             * the face metrics split into float pairs (96 B per cell) */
} sensei_precision;

/* Ghost-cell rules, 2 ghost layers per boundary face. */
typedef enum {
    SENSEI_BC_PERIODIC = 0,     /* copy of the opposite face's interior layers */
    SENSEI_BC_INFLOW = 1,       /* fixed freestream state (supersonic inflow / farfield) */
    SENSEI_BC_EXTRAPOLATE = 2,  /* zeroth-order extrapolation (supersonic outflow) */
    SENSEI_BC_SLIP_WALL = 3,    /* mirror: rho, rho e_t copied, momentum m - 2 (m.n) n */
    SENSEI_BC_INTERFACE = 4,    /* copy of a neighbour block's interior layers */
    SENSEI_BC_EXTERNAL = 5      /* ghost layers written by the caller (sensei_face_exchange): the
                                 * face borders cells another worker advances (heterogeneous
                                 * co-execution, Sec. 4); no kernel of the library writes them.
                                 * Euler only (SENSEI_ERR_UNSUPPORTED with mu > 0) */
} sensei_bc_type;

/* Explicit RK schemes, the optimal strong-stability-preserving ones: the
 * paper's second-order 2-stage and 4-stage schemes, and the 3-stage scheme. */
typedef enum {
    SENSEI_RK2_SSP = 0,     /* SSPRK(2,2) */
    SENSEI_RK3_SSP = 1,     /* SSPRK(3,3) */
    SENSEI_RK4_SSP2 = 2     /* SSPRK(4,2): second order, 4 stages */
} sensei_rk;

typedef enum {
    SENSEI_LIM_NONE = 0,    /* unlimited kappa scheme */
    SENSEI_LIM_MINMOD = 1,
    SENSEI_LIM_VANLEER = 2
} sensei_limiter;

/* Cells of one block; nk == 1 makes the block two-dimensional (one cell
 * deep, no k-faces, rho w carried but left unchanged).  Every other extent
 * is at least 2, the ghost depth (the ghost rules read up to two cells
 * inside a face); SENSEI_ERR_INVALID_ARG otherwise. */
typedef struct {
    int ni, nj, nk;
} sensei_block_desc;

typedef struct {
    double gamma;           /* ratio of specific heats, e.g. 1.4 */
    int limiter;            /* sensei_limiter */
    double kappa;           /* MUSCL kappa of Eq. flux (only matters for SENSEI_LIM_NONE) */
    double eps;             /* MUSCL epsilon of Eq. flux: 1 second order, 0 first order */
    double entropy_fix;     /* Harten's fix width delta = entropy_fix * (Roe sound speed); 0 = off */
    int precision;          /* sensei_precision */
    int reconstruct_conserved; /* 0: reconstruct primitive (rho, u, v, w, p); 1: conserved Q */
    /* Viscous flux F_nu,n of Eq. governing (Stokes's hypothesis; Theta = work
     * of the viscous stresses + heat conduction).  mu = 0: the Euler
     * equations.  mu > 0: constant dynamic viscosity, heat conductivity
     * mu c_p / prandtl; face gradients by central differences in the index
     * directions and the metric identity grad xi_d = Sbar_d / |Omega| (the
     * paper fixes neither; these are this library's readings).  FP64
     * precision only (SENSEI_ERR_UNSUPPORTED otherwise). */
    double mu;
    double prandtl;         /* > 0 when mu > 0, e.g. 0.72 */
} sensei_scheme;

/* Where cell (i, j, k), variable v of a block's state lives: element
 *   offset + v * stride_var + k * stride_k + j * stride_j + i
 * of an array of `elems` doubles, for i in [-ghost_i, ni + ghost_i),
 * j in [-ghost_j, nj + ghost_j), k in [-ghost_k, nk + ghost_k).  Rows are
 * padded so that every row and every variable plane starts on a 32-byte
 * boundary.  State arrays are allocated by the caller with this layout. */
typedef struct {
    long long stride_j, stride_k, stride_var;
    long long offset;
    long long elems;
    int ghost_i, ghost_j, ghost_k;
    int elem_bytes;
} sensei_layout;

/* Bytes of device workspace a grid with these blocks and scheme needs. */
sensei_status sensei_workspace_size(const sensei_block_desc *blocks, int nblocks,
                                    const sensei_scheme *scheme, size_t *bytes);

/* Create a grid.  nodes[b] is a device array X[3][nk+1][nj+1][ni+1] (FP64,
 * x then y then z) of block b's node coordinates; a 2D block has two node
 * planes (z = 0 and z = 1, unit depth).  The face area vectors (half the
 * cross product of the face diagonals, oriented toward increasing index)
 * and the cell volumes (divergence theorem on the position vector) are
 * computed on the device into `workspace` (device memory, >= the size from
 * sensei_workspace_size, 256-byte aligned), which the caller keeps alive
 * and unchanged until sensei_destroy_grid.  The node arrays may be freed
 * once the stream has passed this call.  Boundary faces start unset. */
sensei_status sensei_create_grid(const sensei_block_desc *blocks, int nblocks,
                                 const double *const *nodes, const sensei_scheme *scheme,
                                 void *workspace, size_t workspace_bytes, sensei_stream stream,
                                 sensei_grid **out);

/* Free the host object (the workspace stays the caller's). */
sensei_status sensei_destroy_grid(sensei_grid *grid);

/* Layout of block `block`'s state arrays (see sensei_layout). */
sensei_status sensei_state_layout(const sensei_grid *grid, int block, sensei_layout *out);

/* Boundary rule of face `face` (0 imin, 1 imax, 2 jmin, 3 jmax, 4 kmin,
 * 5 kmax) of block `block`.  prim (host, 5 doubles rho, u, v, w, p) is
 * required for SENSEI_BC_INFLOW.  SENSEI_BC_INTERFACE connects to face
 * nbr_face of block nbr_block, which must be the opposite side of the same
 * index direction with the same tangential size; orientation must be 0
 * (tangential indices aligned).  Every face of every block (faces 0-3 in 2D)
 * must be set before the first fill/residual/step call. */
sensei_status sensei_set_bc(sensei_grid *grid, int block, int face, int type, const double *prim,
                            int nbr_block, int nbr_face, int orientation);

/* Fill the two ghost layers of every boundary face of every block of the
 * states U[b] (Sec. 5, ghost cells on the GPU).  Edge and corner ghosts are
 * never read by the dimension-by-dimension inviscid stencil and are left
 * alone; with mu > 0 the block-edge ghosts (two indices outside the block,
 * read by the viscous face gradients) are then filled by the rule of the
 * lower face family (an i-face's rule at j- and k-ghost positions, a
 * j-face's at k-ghost positions), which reads the other family's ghosts.
 * Corner ghosts are never read. */
sensei_status sensei_fill_ghosts(sensei_grid *grid, double *const *U, sensei_stream stream);

/* Fill the ghosts of U, then write the residual R_h of Eq. residual for
 * every interior cell to R[b], a dense device array R[5][nk][nj][ni] (FP64):
 *   R = sum over the faces of the cell of (F_hat - F_nu) . S_out  -  src
 * with F_hat the Roe flux (Harten entropy fix) of the MUSCL face states,
 * F_nu the viscous flux (zero for mu = 0) and S_out the outward area
 * vector.  src[b] (may be NULL, or src itself NULL)
 * is |Omega| S_h per interior cell in the same layout as R.  Also records
 * the norms of this R (read them with sensei_norms). */
sensei_status sensei_residual(sensei_grid *grid, double *const *U, double *const *R,
                              const double *const *src, sensei_stream stream);

/* One explicit Runge-Kutta step of all blocks, in place on U[b]
 * (Eq. runge_kutta with the 1/|Omega| of Eq. spatial_residual; evaluated in
 * the equivalent low-storage Shu-Osher form).  If cfl > 0 the step is
 * dt = cfl * min over cells of |Omega| / sum_d (|u . Sbar_d| + c |Sbar_d|
 *      + 4 max(4/3, gamma) mu / (Pr rho) |Sbar_d|^2 / |Omega|)
 * evaluated on the device from U^n (the viscous term only for mu > 0);
 * otherwise `dt` (> 0) is used.  If
 * dt_used is not NULL the step's dt is written there (device, 1 double).
 * The norms of R(U^n) and the sums of |Omega| U^n are recorded for
 * sensei_norms.  The ghost layers of U are refilled; on return they are
 * not those of the new state. */
sensei_status sensei_rk_step(sensei_grid *grid, double *const *U, int rk, double cfl, double dt,
                             double *dt_used, sensei_stream stream);

/* nsteps >= 1 consecutive sensei_rk_step calls on the same U, with the same
 * results bit for bit (Eq. runge_kutta; the time-step rule above).  The 3D
 * FP32-storage form (SENSEI_FP32_STORE) in CFL mode forms each step's CFL
 * bound in the last Runge-Kutta stage of the step before, from the state it
 * writes, by the same FP32 arithmetic as the time-step reduction, and skips
 * that reduction's pass over U (its first step still runs it); so U must
 * not be changed between the steps, which is what this call guarantees.  dt_used (device, nsteps
 * doubles, may be NULL) receives each step's dt.  The recorded norms are
 * those of the last step's first stage. */
sensei_status sensei_rk_steps(sensei_grid *grid, double *const *U, int nsteps, int rk, double cfl, double dt,
                              double *dt_used, sensei_stream stream);

/* One step with local time stepping, for marching to a steady state (the
 * paper's inlet case is steady): every cell advances by its own step
 * dt_c = cfl |Omega_c| / sum_d (|u . Sbar_d| + c |Sbar_d|), evaluated on U^n
 * and frozen over the stages (the spectral-radius bound of sensei_rk_step,
 * without the minimum over cells).  Not time-accurate; the steady state
 * R(U) = 0 is the same.  dt_min (device, 1 double, may be NULL) receives the
 * smallest dt_c.  Norms as for sensei_rk_step; watch their decay. */
sensei_status sensei_rk_step_local(sensei_grid *grid, double *const *U, int rk, double cfl, double *dt_min,
                                   sensei_stream stream);

/* Synchronise `stream` and copy out (host arrays of 5 doubles, any may be
 * NULL) the norms recorded by the last sensei_residual or sensei_rk_step:
 *   l2[q] = sqrt(sum_c R_q^2 / N), linf[q] = max_c |R_q|, cons[q] = sum_c |Omega_c| U_q
 * over all N interior cells of all blocks (Sec. 4 "residual print").  Sums
 * are taken in a fixed order, so results are deterministic.  Returns
 * SENSEI_ERR_NONPHYSICAL (and clears the flag) if a kernel met a
 * non-physical or non-finite state since the last call. */
sensei_status sensei_norms(sensei_grid *grid, double *l2, double *linf, double *cons, sensei_stream stream);

/* A CUDA graph of one sensei_rk_step (same arguments, fixed pointers),
 * replayed by sensei_step_graph_launch on any stream.  With a captured step a
 * whole SSPRK3 step of any number of blocks is one graph launch of six
 * kernels: ghost fill, dt reduction, three batched stencil launches,
 * norm finalisation.  Creation synchronises `stream` and captures on a
 * private stream (graph instantiation is done by the CUDA driver).  A graph
 * refuses to launch (SENSEI_ERR_STATE) once boundary rules or the schedule of
 * its grid have changed; make a new one then. */
typedef struct sensei_step_graph sensei_step_graph;
sensei_status sensei_step_graph_create(sensei_grid *grid, double *const *U, int rk, double cfl, double dt,
                                       double *dt_used, sensei_stream stream, sensei_step_graph **out);
/* The same for sensei_rk_steps: one graph of nsteps steps (dt_used: nsteps
 * doubles or NULL), replayed as a whole; where sensei_rk_steps fuses the
 * time-step bound, every replay's first step runs the time-step reduction
 * and the others take the bound of the step before. */
sensei_status sensei_steps_graph_create(sensei_grid *grid, double *const *U, int nsteps, int rk, double cfl,
                                        double dt, double *dt_used, sensei_stream stream, sensei_step_graph **out);
sensei_status sensei_step_graph_launch(sensei_step_graph *graph, sensei_stream stream);
sensei_status sensei_step_graph_destroy(sensei_step_graph *graph);

/* Pick the work schedule of the batched stencil launches by timing them
 * on this grid and the states U (the launches of a three-stage step with
 * dt = 0 -- a first stage from U and two later stages -- into the stage
 * buffers; U's ghosts are refilled, its interior untouched): the k-extent of
 * a work item (tile of 32 x 8 cells x kchunk planes) and persistent CTAs
 * (resident CTAs x SMs, items taken round-robin) versus one CTA per item.
 * Outputs (may be NULL) receive the choice.  Synchronises `stream`. */
sensei_status sensei_autotune(sensei_grid *grid, double *const *U, int *kchunk, int *persistent,
                              sensei_stream stream);

/* The schedule stencil launches use (sensei_autotune's choice, or the
 * default): the k-chunk of a work item, persistent (CTAs = resident CTAs
 * per SM x SMs, striding over the items) or one CTA per item, work items
 * in block-major order or by descending cost (longest first, tried by the
 * autotuner when the blocks differ in size), and the resident CTAs per SM
 * of the stencil variants measured so far (0 before any launch).  Any
 * pointer may be NULL. */
sensei_status sensei_schedule(const sensei_grid *grid, int *kchunk, int *persistent, int *order_by_cost,
                              int *ctas_per_sm);

/* Instrumentation (not part of the method).  While enabled (enable != 0),
 * every launch of the fused stencil kernel (the residual / Runge-Kutta stage
 * kernel) is bracketed by a CUDA event pair recorded on its own stream, and
 * every kernel launch the library issues is counted.  Events are created on
 * first use; do not enable it inside a CUDA-graph capture. */
sensei_status sensei_profile_enable(sensei_grid *grid, int enable);

/* Synchronise the recorded events and return, for the interval since the
 * last reset: the summed stencil-kernel time in milliseconds, the number of
 * stencil launches and the number of all kernel launches (any pointer may be
 * NULL).  reset != 0 starts a new interval. */
sensei_status sensei_profile_read(sensei_grid *grid, double *stencil_ms, long long *stencil_launches,
                                  long long *kernel_launches, int reset);

/* The durations in milliseconds of the individual stencil launches timed
 * since the last reset, in launch order (for a step: one per Runge-Kutta
 * stage): the first min(cap, *count) go to ms[] (caller-owned host array),
 * *count receives how many there are.  Synchronises those events; resets
 * nothing (sensei_profile_read does). */
sensei_status sensei_profile_launches(sensei_grid *grid, double *ms, int cap, int *count);

/* ---- Heterogeneous CPU + GPU co-execution (Sec. 4 workflow, Sec. 6 Eq.
 * hete, Sec. 7 workload ratio): the cells of one time step split between
 * the GPU and the host cores, the ghost layers of the cut exchanged every
 * Runge-Kutta stage.  FP64 Euler only (SENSEI_ERR_UNSUPPORTED otherwise).
 *
 * GPU side, stage by stage (the building blocks the co-execution driver
 * below uses; any caller may use them with SENSEI_BC_EXTERNAL faces): */

/* Stage `stage` (0-based) of one explicit step of RK scheme `rk` with the
 * time step dt (> 0, host value): stage 0 fills U's ghosts (every face but
 * the SENSEI_BC_EXTERNAL ones, which must already hold the neighbour's
 * layers), sets dt and records the norm partials of R(U^n); every stage
 * writes its output and pushes it into the ghosts it feeds (again not the
 * external ones); the last stage writes U^{n+1} into U and finalises the
 * norms (sensei_norms).  The stages of one step must be issued in order on
 * one stream.  Asynchronous on `stream`. */
sensei_status sensei_rk_stage(sensei_grid *grid, double *const *U, int rk, int stage, double dt,
                              sensei_stream stream);

/* The two cell layers next to face `face` of block `block` of the state
 * that stage `stage` reads (stage 0: the caller's U[block]; stage s > 0:
 * the internal output of stage s - 1): unpack = 0 copies the two interior
 * layers (the boundary cell layer first) into buf; unpack = 1 writes buf
 * into the two ghost layers (the one next to the face first).  buf is
 * device memory of 5 * 2 * n1 * n2 doubles, layout [v][layer][t2][t1]
 * with (t1, t2) = (j, k) on i-faces, (i, k) on j-faces, (i, j) on k-faces.
 * Asynchronous on `stream`. */
sensei_status sensei_face_exchange(sensei_grid *grid, double *const *U, int block, int stage, int face, double *buf,
                                   int unpack, sensei_stream stream);

/* The CFL time step of this grid's cells alone: cfl * min |Omega| /
 * sum_d (|u . Sbar_d| + c |Sbar_d|) over the cells of U (no ghosts read).
 * Synchronises `stream`; *dt_out is a host double. */
sensei_status sensei_dt_min(sensei_grid *grid, double *const *U, double cfl, double *dt_out, sensei_stream stream);

/* Host side: one block advanced by host threads (OpenMP) with the same
 * method in FP64 -- the library's own host implementation, not a fallback:
 * it runs only as the host share of a co-executed step.  The state is a
 * host array owned by the worker, layout from sensei_host_layout (2 ghost
 * layers per side, rows not padded).  Faces take the rules above except
 * SENSEI_BC_INTERFACE. */
typedef struct sensei_host_block sensei_host_block;

/* nodes: host (3, nk+1, nj+1, ni+1); scheme->precision must be SENSEI_FP64
 * and mu 0; threads >= 1. */
sensei_status sensei_host_create(int ni, int nj, int nk, const double *nodes, const sensei_scheme *scheme, int threads,
                                 sensei_host_block **out);
sensei_status sensei_host_destroy(sensei_host_block *h);
sensei_status sensei_host_set_bc(sensei_host_block *h, int face, int type, const double *prim);
sensei_status sensei_host_layout(const sensei_host_block *h, sensei_layout *out);
/* the worker's state U (host, read-write, sensei_host_layout) */
double *sensei_host_state(sensei_host_block *h);
/* ghost fill of U (every face but the external ones) */
sensei_status sensei_host_fill_ghosts(sensei_host_block *h);
/* R of U (ghosts filled first) into R (host, [5][nk][nj][ni]) */
sensei_status sensei_host_residual(sensei_host_block *h, double *R);
/* cfl * min over the worker's cells of |Omega| / sum_d (...) */
sensei_status sensei_host_dt_min(sensei_host_block *h, double cfl, double *dt_out);
/* stage `stage` of an explicit step with dt, as sensei_rk_stage */
sensei_status sensei_host_stage(sensei_host_block *h, int rk, int stage, double dt);
/* as sensei_face_exchange, on the worker's state; buf is host memory */
sensei_status sensei_host_face_exchange(sensei_host_block *h, int stage, int face, double *buf, int unpack);

/* The co-execution driver: one 3D block of ni x nj x nk cells, the planes
 * k < nk - nk_host on the GPU, the last nk_host planes on `threads` host
 * threads (2 <= nk_host <= nk - 2; the paper's 1D slab split).
 * bc_type[6] / bc_prim (6 x 5 primitive states, or NULL without inflow
 * faces) are the block's own rules; the cut faces become
 * SENSEI_BC_EXTERNAL on both sides, and with periodic k-faces the GPU
 * part's kmin face borders the host part's kmax face.  Per step: the two
 * time-step minima are combined on the host; then, per stage, the GPU stage
 * is launched, the host threads advance their part meanwhile, and the
 * cut's two layers travel both ways (device -> pinned host -> device)
 * before the next stage.  workspace: device memory of
 * sensei_hetero_workspace_size bytes, 256-byte aligned, caller-owned (the
 * GPU part's grid workspace, its state and the exchange buffers).  The
 * driver allocates pinned host buffers of its own. */
typedef struct sensei_hetero sensei_hetero;

sensei_status sensei_hetero_workspace_size(const sensei_block_desc *block, const sensei_scheme *scheme, int nk_host,
                                           size_t *bytes);
/* nodes: host (3, nk+1, nj+1, ni+1) of the whole block */
sensei_status sensei_hetero_create(const sensei_block_desc *block, const double *nodes, const sensei_scheme *scheme,
                                   const int *bc_type, const double *bc_prim, int nk_host, int threads,
                                   void *workspace, size_t workspace_bytes, sensei_stream stream,
                                   sensei_hetero **out);
sensei_status sensei_hetero_destroy(sensei_hetero *h);
/* the whole block's interior state, host (5, nk, nj, ni): in and out */
sensei_status sensei_hetero_upload(sensei_hetero *h, const double *U);
sensei_status sensei_hetero_download(sensei_hetero *h, double *U);
/* One step; cfl > 0: dt = cfl * min over both parts, else dt > 0 as given.
 * *dt_used (host, may be NULL) receives dt; times_ms (host, 4 doubles, may
 * be NULL) receives the step's wall time, the GPU stages' time (events),
 * the host stages' time and the exchange time (the part of the wall time
 * spent neither in a host stage nor waiting for the GPU). */
sensei_status sensei_hetero_step(sensei_hetero *h, int rk, double cfl, double dt, double *dt_used, double *times_ms);

/* Residual norms that allocate nothing.  The paper has no counterpart: this
 * exists for callers that cannot allocate device memory, e.g. a solver
 * embedded in an application whose memory pool already owns the device, or
 * a monitor inside a time-critical loop that must not risk an allocation.
 * It needs no grid and no workspace.  R is a dense device array
 * R[5][nk][nj][ni] (the layout sensei_residual writes); l2 and linf (host,
 * 5 doubles each, either may be NULL) receive sqrt(sum R_q^2 / N) and
 * max |R_q| over the N = ni*nj*nk cells; a NaN entry of R_q makes both
 * norms of q NaN (the maxima propagate it).  Synchronises `stream`: the
 * norms are read back to the host before the call returns.
 * Scratch: a fixed 164 KB array in the library's own device memory, held by
 * every GPU that loads the library until the process exits; N above
 * 8,388,608 cells is rejected with SENSEI_ERR_INVALID_ARG.  The first call on
 * a device does a one-time set-up: it looks up that array's address (with
 * the device current) and keeps it; make that first call before any stream
 * capture begins, and do not call the entry point again on a device after a
 * cudaDeviceReset of it (the kept address belongs to the old context).  All
 * calls share the array and it keeps the last call's contents (each call
 * overwrites every slot it reads), so calls that overlap on the GPU, from
 * different streams or threads, race: serialise them. */
sensei_status sensei_residual_norms_noalloc(const double *R, int ni, int nj, int nk, double *l2, double *linf,
                                            sensei_stream stream);

/* Test hooks of the bounded device waits (the paper has no counterpart;
 * they exist so that failure detection can be tested without a GPU fault).
 * The FP32 stencil waits on mbarriers for its bulk tile copies; every wait
 * gives up after a limit, sets the device error word, waits once more for
 * the copies in flight (bounded too) and leaves, and sensei_norms then
 * returns SENSEI_ERR_TIMEOUT.  If that second wait also gives up, the CTA
 * leaves with a copy into its shared memory still pending: after a genuine
 * timeout treat the run's later results as unsound.
 *   SENSEI_DEBUG_WAIT_LIMIT: the limit in SM clock cycles (0 = the default
 *     2^31, about a second).
 *   SENSEI_DEBUG_TX_EXTRA: bytes added to every tile phase's expected count
 *     (0 = none).  A positive value makes every such wait run out: the data
 *     arrives, the phase never completes.  For tests only.
 *   SENSEI_DEBUG_ITEM_ORDER: 0 block-major work items, 1 by descending cost
 *     (the autotuner's two orders; for tests that compare them).
 * Apply to the following launches of this grid.  SENSEI_ERR_INVALID_ARG for
 * an unknown key or a negative value. */
enum { SENSEI_DEBUG_WAIT_LIMIT = 1, SENSEI_DEBUG_TX_EXTRA = 2, SENSEI_DEBUG_ITEM_ORDER = 3 };
sensei_status sensei_debug_set(sensei_grid *grid, int key, long long value);

/* Message of the last failing call on this thread ("" if none). */
const char *sensei_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SENSEI_H */
