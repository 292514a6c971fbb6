// api.cu -- host side of the C ABI declared in include/sensei.h.
//
// The library allocates no device memory: every device array is either the
// caller's (states, residuals, nodes, sources) or a slice of the caller's
// workspace (block descriptors, metrics, Runge-Kutta stage buffers, reduction
// partials, the time-step slot, the norms and the error word).
//
// Every kernel of a step covers all blocks of the grid in one launch: the
// ghost fill, the time-step reduction, one persistent stencil launch per RK
// stage (which pushes the ghost layers of its output), the norm
// finalisation.  The blocks' static descriptions live in a device table in
// the workspace, refreshed from the host copy when boundary rules or the
// schedule change.
#include <nvtx3/nvToolsExt.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sensei_internal.cuh"

using namespace sensei;

namespace {

// NVTX range for the duration of a scope (tracing with Nsight tools; a no-op
// without an attached tool)
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};


thread_local char g_msg[512] = "";

sensei_status fail(sensei_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return st;
}

#define CUDA_TRY(expr)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess) return fail(SENSEI_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// smallest k-chunk the schedule may use: sizes the per-item partials
constexpr int KCHUNK_MIN = 4;
constexpr int KCHUNK_CANDIDATES[] = {4, 8, 16, 32, 64, 128};

struct HostBlock {
    BlockDev dev;   // the image uploaded to the device table
    bool two_d;
    bool bc_set[6];
};

// Byte offsets of every workspace slice, computed identically by
// sensei_workspace_size and sensei_create_grid.
struct Plan {
    std::vector<HostBlock> blocks;
    std::vector<size_t> off_fn, off_fdf, off_rec32, off_vol, off_ivol, off_sbar, off_sbar32, off_dtv, off_stage, off_wv,
        off_rvis, off_fvis, off_gvis, off_tmap;
    size_t off_desc = 0, off_partials = 0, off_dtbits = 0, off_dtnext = 0, off_dtslot = 0, off_norms = 0, off_order = 0;
    size_t bytes = 0;
    long long max_items = 0;   // partial slots (items at the smallest k-chunk)
    long long ncells = 0;
    long long bc_total = 0;
    bool two_d = false;
};

size_t take(size_t &cursor, size_t bytes)
{
    size_t at = (size_t)round_up((long long)cursor, 256);
    cursor = at + bytes;
    return at;
}

sensei_status check_scheme(const sensei_scheme *s)
{
    if (!s) return fail(SENSEI_ERR_INVALID_ARG, "scheme is NULL");
    if (!(s->gamma > 1.0)) return fail(SENSEI_ERR_INVALID_ARG, "gamma must be > 1 (got %g)", s->gamma);
    if (s->limiter < SENSEI_LIM_NONE || s->limiter > SENSEI_LIM_VANLEER)
        return fail(SENSEI_ERR_INVALID_ARG, "unknown limiter %d", s->limiter);
    if (s->precision < SENSEI_FP64 || s->precision > SENSEI_DF64)
        return fail(SENSEI_ERR_INVALID_ARG, "unknown precision %d", s->precision);
    if (!(s->entropy_fix >= 0.0)) return fail(SENSEI_ERR_INVALID_ARG, "entropy_fix must be >= 0");
    if (!(s->eps >= 0.0 && s->eps <= 1.0)) return fail(SENSEI_ERR_INVALID_ARG, "eps must lie in [0, 1]");
    if (!(s->kappa >= -1.0 && s->kappa <= 1.0)) return fail(SENSEI_ERR_INVALID_ARG, "kappa must lie in [-1, 1]");
    if (!(s->mu >= 0.0 && s->mu < INFINITY)) return fail(SENSEI_ERR_INVALID_ARG, "mu must be finite and >= 0");
    if (s->mu > 0.0 && !(s->prandtl > 0.0 && s->prandtl < INFINITY))
        return fail(SENSEI_ERR_INVALID_ARG, "prandtl must be finite and > 0 when mu > 0");
    if (s->mu > 0.0 && s->precision != SENSEI_FP64 && s->precision != SENSEI_DF64)
        return fail(SENSEI_ERR_UNSUPPORTED, "the viscous flux runs with the FP64 state update only (FP64, DF64)");
    return SENSEI_OK;
}

int chunks_for(int nk, bool two_d, int kchunk) { return two_d ? 1 : (nk + kchunk - 1) / kchunk; }

long long bc_units(const HostBlock &H)
{
    long long u = 0;
    const int nf = H.two_d ? 4 : 6;
    for (int f = 0; f < nf; ++f) {
        long long n1 = f < 2 ? H.dev.nj : H.dev.ni, n2 = f < 4 ? H.dev.nk : H.dev.nj;
        u += n1 * n2 * 2;
    }
    return u;
}

// Item numbering (block-major) and ghost-fill unit numbering for a k-chunk;
// returns the number of items.
long long assign_items(std::vector<HostBlock> &blocks, int kchunk)
{
    long long items = 0, bc = 0;
    for (HostBlock &H : blocks) {
        BlockDev &B = H.dev;
        B.kchunk = H.two_d ? 1 : std::min(kchunk, B.nk);
        B.nchunks = chunks_for(B.nk, H.two_d, B.kchunk);
        B.item0 = items;
        items += (long long)B.tiles_i * B.tiles_j * B.nchunks;
        B.bc0 = bc;
        bc += bc_units(H);
    }
    return items;
}

long long total_items(const std::vector<HostBlock> &blocks)
{
    const BlockDev &L = blocks.back().dev;
    return L.item0 + (long long)L.tiles_i * L.tiles_j * L.nchunks;
}

sensei_status make_plan(const sensei_block_desc *blocks, int nblocks, const sensei_scheme *scheme, Plan &P)
{
    if (!blocks || nblocks <= 0) return fail(SENSEI_ERR_INVALID_ARG, "need at least one block");
    if (nblocks > MAX_BLOCKS) return fail(SENSEI_ERR_UNSUPPORTED, "at most %d blocks per grid", MAX_BLOCKS);
    sensei_status st = check_scheme(scheme);
    if (st != SENSEI_OK) return st;
    size_t cur = 0;
    P.blocks.resize(nblocks);
    for (auto *v : {&P.off_fn, &P.off_fdf, &P.off_rec32, &P.off_vol, &P.off_ivol, &P.off_sbar, &P.off_sbar32, &P.off_dtv,
                    &P.off_wv, &P.off_rvis, &P.off_fvis, &P.off_gvis,
                    &P.off_stage, &P.off_tmap})
        v->resize(nblocks);
    const bool f32 = scheme->precision == SENSEI_FP32_FLUX || scheme->precision == SENSEI_FP32_STORE;
    P.two_d = blocks[0].nk == 1;
    long long tiles_total = 0;
    for (int b = 0; b < nblocks; ++b) {
        const sensei_block_desc &d = blocks[b];
        // every ghost rule reads up to NG cells inside a face (periodic,
        // wall, interface), so a 3D extent is at least NG; nk == 1 is 2D
        if (d.ni < NG || d.nj < NG || d.nk < 1 || (d.nk > 1 && d.nk < NG))
            return fail(SENSEI_ERR_INVALID_ARG,
                        "block %d: need ni, nj >= %d and nk >= %d or nk == 1 (got %d x %d x %d)", b, NG, NG, d.ni,
                        d.nj, d.nk);
        if ((long long)d.ni * d.nj * d.nk > (1LL << 34))
            return fail(SENSEI_ERR_INVALID_ARG, "block %d: too many cells", b);
        if ((d.nk == 1) != P.two_d)
            return fail(SENSEI_ERR_INVALID_ARG, "block %d: 2D (nk == 1) and 3D blocks cannot share a grid", b);
        HostBlock &H = P.blocks[b];
        memset(&H, 0, sizeof H);
        H.two_d = d.nk == 1;
        BlockDev &B = H.dev;
        B.ni = d.ni;
        B.nj = d.nj;
        B.nk = d.nk;
        const int gk = H.two_d ? 0 : NG;
        const long long pitch = round_up(d.ni + 2 * NG, 4);
        B.L.sj = pitch;
        B.L.sk = pitch * (d.nj + 2 * NG);
        B.L.sv = round_up(B.L.sk * (d.nk + 2 * gk), 32);
        B.L.elems = NV * B.L.sv;
        B.L.off = gk * B.L.sk + NG * B.L.sj + NG;
        B.L.gk = gk;
        B.ml.mpitch = round_up(d.ni + 1, 4);
        B.ml.mplane = B.ml.mpitch * (d.nj + 1);
        B.ml.mvolume = round_up(B.ml.mplane * (d.nk + 1), 32);
        B.tiles_i = (d.ni + TI - 1) / TI;
        B.tiles_j = (d.nj + TJ - 1) / TJ;
        for (int f = 0; f < 6; ++f) {
            B.bc_type[f] = -1;
            B.nbr[f] = -1;
            B.nbr_face[f] = -1;
        }
        tiles_total += (long long)B.tiles_i * B.tiles_j;
        P.ncells += (long long)d.ni * d.nj * d.nk;
        const size_t mv = (size_t)B.ml.mvolume;
        P.off_fn[b] = take(cur, 12 * mv * sizeof(double));
        // double-float: the face metrics split once into float pairs
        P.off_fdf[b] = scheme->precision == SENSEI_DF64 ? take(cur, 12 * mv * 2 * sizeof(float)) : 0;
        P.off_rec32[b] =
            f32 ? take(cur, (size_t)B.tiles_i * B.tiles_j * d.nk * REC * sizeof(float)) : 0;
        P.off_vol[b] = take(cur, mv * sizeof(double));
        P.off_ivol[b] = take(cur, mv * sizeof(double));
        P.off_sbar[b] = take(cur, 12 * mv * sizeof(double));
        // FP32 spectral metrics (12 arrays) and |Omega| (1) for the FP32 time step
        P.off_sbar32[b] = f32 ? take(cur, 13 * mv * sizeof(float)) : 0;
        P.off_dtv[b] = take(cur, mv * sizeof(double));
        // viscous: the stage input's (u, v, w, p / rho) and the viscous residual
        const bool vis = scheme->mu > 0.0;
        P.off_wv[b] = vis ? take(cur, 4 * (size_t)B.L.sv * sizeof(double)) : 0;
        P.off_rvis[b] = vis ? take(cur, (size_t)NV * d.ni * d.nj * d.nk * sizeof(double)) : 0;
        P.off_fvis[b] = vis ? take(cur, 3 * (size_t)NV * mv * sizeof(double)) : 0;
        P.off_gvis[b] = vis ? take(cur, 3 * GVIS * mv * sizeof(double)) : 0;
        // two FP64 stage states, or two FP32 stage states + two FP32 increments
        P.off_stage[b] = take(cur, 2 * (size_t)B.L.elems * sizeof(double));
        // the tensor maps of the state slots (3D FP32 arithmetic)
        P.off_tmap[b] = f32 && !H.two_d ? take(cur, 5 * (size_t)TMAP_BYTES) : 0;
    }
    // partial slots for the finest schedule
    P.max_items = assign_items(P.blocks, KCHUNK_MIN);
    P.bc_total = P.blocks.back().dev.bc0 + bc_units(P.blocks.back());
    if (P.max_items > (1LL << 31)) return fail(SENSEI_ERR_INVALID_ARG, "grid too large");
    // default schedule: about 8 items per SM of a 152-SM GB300
    int max_nk = 1;
    for (auto &H : P.blocks) max_nk = std::max(max_nk, H.dev.nk);
    const long long nch = std::max(1LL, (152LL * 8 + tiles_total - 1) / tiles_total);
    const int kchunk = (int)std::max<long long>(KCHUNK_MIN, (max_nk + nch - 1) / nch);
    assign_items(P.blocks, kchunk);
    P.off_desc = take(cur, (size_t)nblocks * sizeof(BlockDev));
    P.off_partials = take(cur, (size_t)P.max_items * 3 * NV * sizeof(double));
    P.off_order = take(cur, (size_t)P.max_items * sizeof(int));
    P.off_dtbits = take(cur, sizeof(unsigned long long));
    P.off_dtnext = take(cur, 2 * sizeof(unsigned long long));
    P.off_dtslot = take(cur, sizeof(double));
    P.off_norms = take(cur, 16 * sizeof(double));   // 15 norms + the error word
    P.bytes = round_up((long long)cur, 256);
    return SENSEI_OK;
}

struct Device {
    int saved = -1;
    cudaError_t set(int dev)
    {
        cudaError_t e = cudaGetDevice(&saved);
        if (e != cudaSuccess) return e;
        return saved == dev ? cudaSuccess : cudaSetDevice(dev);
    }
    ~Device()
    {
        int cur;
        if (saved >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != saved) cudaSetDevice(saved);
    }
};

}  // namespace

sensei_status sensei::fail_status(sensei_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return st;
}

struct sensei_grid {
    int device;
    int sms;
    sensei_scheme scheme;
    Plan plan;
    char *ws;
    BlockDev *desc;     // device table
    double *partials;
    unsigned long long *dt_bits;
    unsigned long long *dt_next;   // two slots: the fused next-step bounds of a multi-step run
    double *dt_slot;
    double *norms;      // 15 doubles, then the error word
    unsigned *err;
    bool dirty = true;          // descriptors changed since the last upload
    long long wait_limit = 1LL << 31;   // bounded device waits (sensei_debug_set)
    unsigned tx_extra = 0;
    bool stage_ghosts = false;  // fixed (inflow) ghosts of the stage buffers set
    // tensor maps of the state slots (3D FP32 grids): host copies, and the
    // caller's state pointer each block's SLOT_USER map was encoded for
    std::vector<unsigned char> tmaps_host;
    std::vector<const void *> tmap_user;
    int grid_mode = 0;          // 0: persistent (resident CTAs x SMs), 1: one CTA per item
    int order_mode = 0;         // 0: items block-major; 1: by descending cost (longest first)
    int *order = nullptr;       // device: launch position -> item (order_mode 1)
    int ctas_cache[4] = {0, 0, 0, 0};
    // instrumentation
    bool prof = false;
    std::vector<cudaEvent_t> ev;   // start/end pairs
    size_t ev_used = 0;
    long long stencil_launches = 0, kernel_launches = 0;
    ~sensei_grid()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

struct sensei_step_graph {
    sensei_grid *grid;
    cudaGraphExec_t exec;
};

namespace {

sensei_status check_grid(const sensei_grid *g)
{
    if (!g) return fail(SENSEI_ERR_INVALID_ARG, "grid is NULL");
    return SENSEI_OK;
}

sensei_status check_states(const sensei_grid *g, double *const *U, const char *what)
{
    if (!U) return fail(SENSEI_ERR_INVALID_ARG, "%s pointer array is NULL", what);
    for (size_t b = 0; b < g->plan.blocks.size(); ++b) {
        if (!U[b]) return fail(SENSEI_ERR_INVALID_ARG, "%s[%zu] is NULL", what, b);
        if (((uintptr_t)U[b]) % 16) return fail(SENSEI_ERR_INVALID_ARG, "%s[%zu] is not 16-byte aligned", what, b);
    }
    return SENSEI_OK;
}

sensei_status check_bcs(const sensei_grid *g)
{
    for (size_t b = 0; b < g->plan.blocks.size(); ++b) {
        const HostBlock &H = g->plan.blocks[b];
        for (int f = 0; f < (H.two_d ? 4 : 6); ++f)
            if (!H.bc_set[f]) return fail(SENSEI_ERR_STATE, "block %zu face %d has no boundary condition", b, f);
    }
    return SENSEI_OK;
}

// 0 FP64, 1 FP32 arithmetic on an FP64 input, 2 on an FP32 input, 3 double-float
int precision_kind(const sensei_grid *g, bool in_f32)
{
    if (g->scheme.precision == SENSEI_FP64) return 0;
    if (g->scheme.precision == SENSEI_DF64) return 3;
    return in_f32 ? 2 : 1;
}

// persistent grid size of a stencil variant
int stencil_grid(sensei_grid *g, int kind, long long nitems)
{
    if (g->grid_mode == 1) return (int)std::min<long long>(nitems, (1LL << 31) - 1);
    if (!g->ctas_cache[kind])
        g->ctas_cache[kind] = std::max(1, stencil_ctas_per_sm(kind, g->scheme.limiter, g->plan.two_d));
    return (int)std::min<long long>(nitems, (long long)g->ctas_cache[kind] * g->sms);
}

// The work items of the current assignment by descending cost, longest
// first (so that a launch's last wave holds the short ones): an item's cost
// is its k-planes plus the two warm-up planes of the FP32 stencil (a tile
// costs about the same whether its columns are all inside the block or
// not); ties keep block-major order.
std::vector<int> items_by_cost(const std::vector<HostBlock> &blocks)
{
    std::vector<std::pair<int, int>> cost;   // (-cost, item)
    for (const HostBlock &H : blocks) {
        const BlockDev &B = H.dev;
        const long long per_chunk = (long long)B.tiles_i * B.tiles_j;
        for (int ch = 0; ch < B.nchunks; ++ch) {
            const int planes = H.two_d ? 1 : std::min(B.kchunk, B.nk - ch * B.kchunk);
            for (long long t = 0; t < per_chunk; ++t)
                cost.push_back({-(planes + 2), (int)(B.item0 + ch * per_chunk + t)});
        }
    }
    std::stable_sort(cost.begin(), cost.end(),
                     [](const std::pair<int, int> &a, const std::pair<int, int> &b) { return a.first < b.first; });
    std::vector<int> order(cost.size());
    for (size_t n = 0; n < cost.size(); ++n) order[n] = cost[n].second;
    return order;
}

// Upload the descriptor table (and the item order) if boundary rules or the
// schedule changed.  Synchronises `s` (a pageable host-to-device copy);
// never inside a capture.
sensei_status sync_descriptors(sensei_grid *g, cudaStream_t s)
{
    if (!g->dirty) return SENSEI_OK;
    std::vector<BlockDev> tab(g->plan.blocks.size());
    for (size_t b = 0; b < tab.size(); ++b) tab[b] = g->plan.blocks[b].dev;
    CUDA_TRY(cudaMemcpyAsync(g->desc, tab.data(), tab.size() * sizeof(BlockDev), cudaMemcpyHostToDevice, s));
    std::vector<int> order;
    if (g->order_mode == 1) {
        order = items_by_cost(g->plan.blocks);
        CUDA_TRY(cudaMemcpyAsync(g->order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    if (g->scheme.mu > 0.0) {
        // the viscous face metrics follow the boundary rules (the geometry a
        // ghost cell carries)
        long long max_faces = 0;
        for (auto &H : g->plan.blocks) max_faces = std::max<long long>(max_faces, H.dev.ml.mvolume);
        CUDA_TRY(launch_vis_metrics(g->desc, (int)tab.size(), max_faces, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    g->dirty = false;
    return SENSEI_OK;
}

sensei_status fill_slot(sensei_grid *g, int slot, double *const *U, cudaStream_t s)
{
    BCBatch p;
    memset(&p, 0, sizeof p);
    p.blocks = g->desc;
    p.nblocks = (int)g->plan.blocks.size();
    p.total = g->plan.bc_total;
    p.slot = slot;
    p.gamma = g->scheme.gamma;
    if (U)
        for (int b = 0; b < p.nblocks; ++b) p.user[b] = U[b];
    CUDA_TRY(launch_bc(p, s));
    g->kernel_launches++;
    return SENSEI_OK;
}

bool viscous(const sensei_grid *g) { return g->scheme.mu > 0.0; }

// Grids whose last Runge-Kutta stage forms the next step's time-step bound
// itself: the 3D FP32-storage form with a global CFL step (its last stage
// writes U^n + D in FP64; the FP32 rule of the time-step kernel, the same
// function).  Not the FP32-flux form: there the added work in its FP64-input
// last stage cost as much as the time-step kernel it saved (measured).
bool fused_next_dt(const sensei_grid *g, double cfl)
{
    return cfl > 0.0 && !g->plan.two_d && !viscous(g) && g->scheme.precision == SENSEI_FP32_STORE;
}

// The block-edge ghosts of a slot's states (the face ghosts are in place).
sensei_status fill_edges(sensei_grid *g, int slot, double *const *U, cudaStream_t s)
{
    BCBatch p;
    memset(&p, 0, sizeof p);
    p.blocks = g->desc;
    p.nblocks = (int)g->plan.blocks.size();
    p.total = g->plan.bc_total;
    p.slot = slot;
    p.gamma = g->scheme.gamma;
    if (U)
        for (int b = 0; b < p.nblocks; ++b) p.user[b] = U[b];
    long long max_edges = 0;
    for (auto &H : g->plan.blocks)
        max_edges = std::max<long long>(max_edges, 16LL * (H.dev.ni + H.dev.nj + H.dev.nk));
    CUDA_TRY(launch_edges(p, (int)std::min<long long>(max_edges, 1 << 30), s));
    g->kernel_launches++;
    return SENSEI_OK;
}

// The viscous residual of a slot's states: the block-edge ghosts, then the
// primitives and R_nu of every block.
sensei_status viscous_residual(sensei_grid *g, int slot, double *const *U, cudaStream_t s)
{
    sensei_status st = fill_edges(g, slot, U, s);
    if (st != SENSEI_OK) return st;
    long long max_state = 0, max_faces = 0, max_cells = 0;
    for (auto &H : g->plan.blocks) {
        max_state = std::max<long long>(max_state, H.dev.L.sv);
        max_faces = std::max<long long>(max_faces, H.dev.ml.mvolume);
        max_cells = std::max<long long>(max_cells, (long long)H.dev.ni * H.dev.nj * H.dev.nk);
    }
    const int nb = (int)g->plan.blocks.size();
    VisBatch v;
    memset(&v, 0, sizeof v);
    v.blocks = g->desc;
    v.nblocks = nb;
    v.slot = slot;
    v.gamma = g->scheme.gamma;
    v.mu = g->scheme.mu;
    v.kcond = g->scheme.mu * g->scheme.gamma / ((g->scheme.gamma - 1.0) * g->scheme.prandtl);
    if (U)
        for (int b = 0; b < nb; ++b) v.user[b] = U[b];
    CUDA_TRY(launch_viscous(v, max_state, max_faces, max_cells, s));
    g->kernel_launches += 3;
    return SENSEI_OK;
}

// the viscous time-step factor 4 max(4/3, gamma) mu / Pr (0 without viscosity)
double viscous_dt_factor(const sensei_grid *g)
{
    if (!viscous(g)) return 0.0;
    return 4.0 * std::max(4.0 / 3.0, g->scheme.gamma) * g->scheme.mu / g->scheme.prandtl;
}

struct StencilCall {
    int mode;
    int in_slot, out_slot, dprev, dout;
    int push;
    int local;
    double alpha, beta, gdt;
    const double *dt_slot;
    double dt_scale;
    bool partials;
    bool vis;
    double *const *user;
    double *const *rout;
    const double *const *src;
    unsigned long long *dt_next;   // the 3D FP32 last stage's fused next-step bound (or null)
};

template <typename R>
void fill_params(BatchParams<R> &p, const sensei_grid *g, const StencilCall &c)
{
    memset(&p, 0, sizeof p);
    const int nb = (int)g->plan.blocks.size();
    p.blocks = g->desc;
    p.nblocks = nb;
    p.nitems = total_items(g->plan.blocks);
    p.mode = c.mode;
    p.in_slot = c.in_slot;
    p.out_slot = c.out_slot;
    p.dprev = c.dprev;
    p.dout = c.dout;
    p.push = c.push;
    p.local = c.local;
    p.gamma = (R)g->scheme.gamma;
    p.kappa = (R)g->scheme.kappa;
    p.eps = (R)g->scheme.eps;
    p.fix = (R)g->scheme.entropy_fix;
    p.ifix = (R)(g->scheme.entropy_fix > 0.0 ? 1.0 / g->scheme.entropy_fix : 0.0);
    // the derived constants, in R arithmetic as the kernels would form them
    p.gm1 = p.gamma - (R)1;
    p.kg = p.gamma / p.gm1;
    p.c1 = p.eps * ((R)1 - p.kappa) * (R)0.25;
    p.c2 = p.eps * ((R)1 + p.kappa) * (R)0.25;
    p.half_eps = (R)0.5 * p.eps;
    p.cons = g->scheme.reconstruct_conserved ? 1 : 0;
    p.vis = c.vis ? 1 : 0;
    p.wait_limit = g->wait_limit;
    p.tx_extra = g->tx_extra;
    p.alpha = c.alpha;
    p.beta = c.beta;
    p.gdt = c.gdt;
    p.dt_slot = c.dt_slot;
    p.dt_scale = c.dt_scale;
    p.partials = c.partials ? g->partials : nullptr;
    p.order = g->order_mode == 1 ? g->order : nullptr;
    p.dt_next = c.dt_next;
    p.gamma_d = g->scheme.gamma;
    p.err = g->err;
    for (int b = 0; b < nb; ++b) {
        p.user[b] = c.user ? c.user[b] : nullptr;
        p.rout[b] = c.rout ? c.rout[b] : nullptr;
        p.src[b] = c.src ? c.src[b] : nullptr;
    }
}

sensei_status ensure_user_maps(sensei_grid *g, double *const *U, cudaStream_t s);

sensei_status stencil_launch(sensei_grid *g, const StencilCall &c, cudaStream_t s)
{
    if (c.in_slot == SLOT_USER) {
        sensei_status st = ensure_user_maps(g, c.user, s);
        if (st != SENSEI_OK) return st;
    }
    const bool in_f32 = c.in_slot == SLOT_X0 || c.in_slot == SLOT_X1;
    const int kind = precision_kind(g, in_f32);
    const long long nitems = total_items(g->plan.blocks);
    const int grid = stencil_grid(g, kind, nitems);
    if (kind == 0) {
        BatchParams<double> p;
        fill_params(p, g, c);
        CUDA_TRY(launch_stencil_f64(p, g->scheme.limiter, g->plan.two_d, grid, s));
    } else if (kind == 3) {
        BatchParams<df64> p;
        fill_params(p, g, c);
        CUDA_TRY(launch_stencil_df64(p, g->scheme.limiter, g->plan.two_d, grid, s));
    } else {
        BatchParams<float> p;
        fill_params(p, g, c);
        if (kind == 2)
            CUDA_TRY(launch_stencil_f32s(p, g->scheme.limiter, g->plan.two_d, grid, s));
        else
            CUDA_TRY(launch_stencil_f32(p, g->scheme.limiter, g->plan.two_d, grid, s));
    }
    return SENSEI_OK;
}

sensei_status stencil(sensei_grid *g, const StencilCall &c, cudaStream_t s)
{
    if (!g->prof) {
        g->kernel_launches++;
        return stencil_launch(g, c, s);
    }
    if (g->ev_used + 2 > g->ev.size()) {
        for (int n = 0; n < 2; ++n) {
            cudaEvent_t e;
            CUDA_TRY(cudaEventCreate(&e));
            g->ev.push_back(e);
        }
    }
    cudaEvent_t e0 = g->ev[g->ev_used], e1 = g->ev[g->ev_used + 1];
    g->ev_used += 2;
    CUDA_TRY(cudaEventRecord(e0, s));
    sensei_status st = stencil_launch(g, c, s);
    if (st != SENSEI_OK) return st;
    CUDA_TRY(cudaEventRecord(e1, s));
    g->kernel_launches++;
    g->stencil_launches++;
    return SENSEI_OK;
}

const double RK_COEF[3][4][3] = {
    // alpha, beta, gdt of U^(s) = alpha U^n + beta U^(s-1) - gdt dt R/|Omega|
    {{0.0, 1.0, 1.0}, {0.5, 0.5, 0.5}},
    {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}},
    {{0.0, 1.0, 1.0 / 3.0}, {0.0, 1.0, 1.0 / 3.0}, {0.0, 1.0, 1.0 / 3.0}, {0.25, 0.75, 0.25}},
};
const int RK_STAGES[3] = {2, 3, 4};

bool incr_mode(const sensei_grid *g) { return g->scheme.precision == SENSEI_FP32_STORE; }

// The SLOT_USER tensor maps of the FP32 stencil for the caller's state
// pointers: re-encoded and uploaded (stream-ordered) when a pointer differs
// from the one a map was made for.  Not inside a stream capture: the
// capturing entry points run prepare_step, which calls this, first.
sensei_status ensure_user_maps(sensei_grid *g, double *const *U, cudaStream_t s)
{
    if (!U || g->tmap_user.empty()) return SENSEI_OK;
    for (size_t b = 0; b < g->plan.blocks.size(); ++b) {
        const BlockDev &B = g->plan.blocks[b].dev;
        if (!B.tmaps || g->tmap_user[b] == U[b]) continue;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CUDA_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return fail(SENSEI_ERR_STATE, "state pointers changed inside a stream capture");
        unsigned char *h = g->tmaps_host.data() + b * 5 * TMAP_BYTES;
        if (!encode_state_map(h, U[b], B, false))
            return fail(SENSEI_ERR_CUDA, "cuTensorMapEncodeTiled rejected the state of block %zu", b);
        CUDA_TRY(cudaMemcpyAsync((void *)B.tmaps, h, TMAP_BYTES, cudaMemcpyHostToDevice, s));
        g->tmap_user[b] = U[b];
    }
    return SENSEI_OK;
}

// Everything of a step that must not happen inside a stream capture: the
// descriptor upload, the tensor maps of the caller's states and the
// one-time ghost fill of the stage buffers (it sets their fixed inflow
// ghosts; all other ghosts are pushed every stage).
sensei_status prepare_step(sensei_grid *g, double *const *U, cudaStream_t s)
{
    sensei_status st = sync_descriptors(g, s);
    if (st != SENSEI_OK) return st;
    st = ensure_user_maps(g, U, s);
    if (st != SENSEI_OK) return st;
    if (!g->stage_ghosts) {
        const bool incr = incr_mode(g);
        for (int n = 0; n < 2; ++n) {
            st = fill_slot(g, incr ? SLOT_X0 + n : SLOT_ST0 + n, nullptr, s);
            if (st != SENSEI_OK) return st;
        }
        g->stage_ghosts = true;
    }
    return SENSEI_OK;
}

// One RK step, launches only (capturable once prepare_step has run).  With
// local set every cell advances by its own step cfl |Omega_c| / sum_d(...).
// dt_in (CFL mode): the bound the previous step's last stage left, which
// replaces the time-step kernel; dt_out: the slot this step's last stage
// fills with the next step's bound (both for fused_next_dt grids only).
sensei_status rk_step_launches(sensei_grid *grid, double *const *U, int rk, double cfl, double dt, double *dt_used,
                               cudaStream_t s, bool local = false, const unsigned long long *dt_in = nullptr,
                               unsigned long long *dt_out = nullptr)
{
    sensei_status st = fill_slot(grid, SLOT_USER, U, s);
    if (st != SENSEI_OK) return st;
    const double *dt_src;
    double dt_scale;
    const long long nitems = total_items(grid->plan.blocks);
    if (dt_out) CUDA_TRY(cudaMemsetAsync(dt_out, 0x7F, sizeof(unsigned long long), s));
    if (cfl > 0.0 && dt_in) {
        dt_src = (const double *)dt_in;
        dt_scale = cfl;
    } else if (cfl > 0.0) {
        CUDA_TRY(cudaMemsetAsync(grid->dt_bits, 0x7F, sizeof(unsigned long long), s));
        int kchunk = 1;
        for (const HostBlock &H : grid->plan.blocks) kchunk = std::max(kchunk, H.dev.kchunk);
        CUDA_TRY(launch_dt(grid->desc, (int)grid->plan.blocks.size(), nitems, U, grid->scheme.gamma, local ? 1 : 0,
                           cfl, grid->dt_bits, grid->err, (int)std::min<long long>(nitems, 8LL * grid->sms), kchunk,
                           grid->scheme.precision == SENSEI_FP32_FLUX || grid->scheme.precision == SENSEI_FP32_STORE,
                           viscous_dt_factor(grid), s));
        grid->kernel_launches++;
        dt_src = (const double *)grid->dt_bits;
        dt_scale = cfl;
    } else {
        CUDA_TRY(launch_set_scalar(grid->dt_slot, dt, s));
        grid->kernel_launches++;
        dt_src = grid->dt_slot;
        dt_scale = 1.0;
    }
    if (dt_used) {
        CUDA_TRY(launch_scale_copy(dt_used, dt_src, dt_scale, s));
        grid->kernel_launches++;
    }
    const int S = RK_STAGES[rk];
    const bool incr = incr_mode(grid);
    for (int stage = 0; stage < S; ++stage) {
        const double *co = RK_COEF[rk][stage];
        const bool last = stage == S - 1;
        StencilCall c;
        memset(&c, 0, sizeof c);
        c.alpha = co[0];
        c.beta = co[1];
        c.gdt = co[2];
        c.dt_slot = dt_src;
        c.dt_scale = dt_scale;
        c.partials = stage == 0;
        c.user = U;
        c.push = 1;
        c.local = local ? 1 : 0;
        c.dprev = -1;
        c.dout = -1;
        c.dt_next = last ? dt_out : nullptr;
        if (!incr) {
            // FP64 stage states: U -> ST0 -> ST1 -> ST0 ... -> U
            c.mode = MODE_ACCUM;
            c.in_slot = stage == 0 ? SLOT_USER : SLOT_ST0 + (stage - 1) % 2;
            c.out_slot = last ? SLOT_USER : SLOT_ST0 + stage % 2;
        } else {
            // FP32 storage: the first stage reads the FP64 master U, later
            // stages the FP32 stage state X^(s-1); every stage but the last
            // writes the FP32 increment D^(s) and X^(s); the last adds its
            // increment to U in FP64
            c.mode = MODE_INCR;
            c.in_slot = stage == 0 ? SLOT_USER : SLOT_X0 + (stage - 1) % 2;
            c.out_slot = last ? SLOT_USER : SLOT_X0 + stage % 2;
            c.dprev = stage == 0 ? -1 : (stage - 1) % 2;
            c.dout = last ? -1 : stage % 2;
        }
        TraceRange trace_stage(stage == 0 ? "rk stage 1" : stage == 1 ? "rk stage 2" : stage == 2 ? "rk stage 3"
                                                                                    : "rk stage 4");
        if (viscous(grid)) {
            // R_nu of the stage input (its face ghosts are in place: filled
            // for U, pushed by the previous stage otherwise)
            st = viscous_residual(grid, c.in_slot, U, s);
            if (st != SENSEI_OK) return st;
            c.vis = true;
        }
        st = stencil(grid, c, s);
        if (st != SENSEI_OK) return st;
    }
    CUDA_TRY(launch_norms_finalize(grid->partials, (int)nitems, grid->plan.ncells, grid->norms, s));
    grid->kernel_launches++;
    return SENSEI_OK;
}

sensei_status check_step_args(sensei_grid *grid, double *const *U, int rk, double cfl, double dt)
{
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st == SENSEI_OK) st = check_bcs(grid);
    if (st != SENSEI_OK) return st;
    if (rk < SENSEI_RK2_SSP || rk > SENSEI_RK4_SSP2) return fail(SENSEI_ERR_INVALID_ARG, "unknown RK scheme %d", rk);
    if (!(cfl > 0.0) && !(dt > 0.0 && dt < INFINITY))
        return fail(SENSEI_ERR_INVALID_ARG, "need cfl > 0 or a finite dt > 0");
    return SENSEI_OK;
}

}  // namespace

// The CFL minimum over the grid's cells, |Omega| / sum_d (...) without the
// cfl factor, copied to the host address min_out (pinned for the copy to
// stay asynchronous) on `stream`; the caller synchronises.  The first half of
// sensei_dt_min, for drivers that overlap it with host work.
sensei_status sensei::dt_min_launch(sensei_grid *grid, double *const *U, double *min_out, cudaStream_t s)
{
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st != SENSEI_OK) return st;
    if (!min_out) return fail(SENSEI_ERR_INVALID_ARG, "no output");
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    st = sync_descriptors(grid, s);
    if (st != SENSEI_OK) return st;
    const long long nitems = total_items(grid->plan.blocks);
    int kchunk = 1;
    for (const HostBlock &H : grid->plan.blocks) kchunk = std::max(kchunk, H.dev.kchunk);
    CUDA_TRY(cudaMemsetAsync(grid->dt_bits, 0x7F, sizeof(unsigned long long), s));
    CUDA_TRY(launch_dt(grid->desc, (int)grid->plan.blocks.size(), nitems, U, grid->scheme.gamma, 0, 1.0,
                       grid->dt_bits, grid->err, (int)std::min<long long>(nitems, 8LL * grid->sms), kchunk,
                       grid->scheme.precision == SENSEI_FP32_FLUX || grid->scheme.precision == SENSEI_FP32_STORE,
                       viscous_dt_factor(grid), s));
    grid->kernel_launches++;
    CUDA_TRY(cudaMemcpyAsync(min_out, grid->dt_bits, sizeof(double), cudaMemcpyDeviceToHost, s));
    return SENSEI_OK;
}

extern "C" {

const char *sensei_last_error(void) { return g_msg; }

sensei_status sensei_debug_set(sensei_grid *grid, int key, long long value)
{
    sensei_status st = check_grid(grid);
    if (st != SENSEI_OK) return st;
    if (value < 0) return fail(SENSEI_ERR_INVALID_ARG, "debug value must be >= 0");
    if (key == SENSEI_DEBUG_WAIT_LIMIT) {
        grid->wait_limit = value > 0 ? value : (1LL << 31);
    } else if (key == SENSEI_DEBUG_TX_EXTRA) {
        if (value > (1 << 16)) return fail(SENSEI_ERR_INVALID_ARG, "tx_extra above 65536 bytes");
        grid->tx_extra = (unsigned)value;
    } else if (key == SENSEI_DEBUG_ITEM_ORDER) {
        if (value > 1) return fail(SENSEI_ERR_INVALID_ARG, "item order 0 or 1");
        grid->order_mode = (int)value;
        grid->dirty = true;
    } else {
        return fail(SENSEI_ERR_INVALID_ARG, "unknown debug key %d", key);
    }
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_profile_enable(sensei_grid *grid, int enable)
{
    sensei_status st = check_grid(grid);
    if (st != SENSEI_OK) return st;
    grid->prof = enable != 0;
    return SENSEI_OK;
}

sensei_status sensei_profile_read(sensei_grid *grid, double *stencil_ms, long long *stencil_launches,
                                  long long *kernel_launches, int reset)
{
    sensei_status st = check_grid(grid);
    if (st != SENSEI_OK) return st;
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    double ms = 0.0;
    for (size_t n = 0; n + 1 < grid->ev_used; n += 2) {
        CUDA_TRY(cudaEventSynchronize(grid->ev[n + 1]));
        float t = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&t, grid->ev[n], grid->ev[n + 1]));
        ms += t;
    }
    if (stencil_ms) *stencil_ms = ms;
    if (stencil_launches) *stencil_launches = grid->stencil_launches;
    if (kernel_launches) *kernel_launches = grid->kernel_launches;
    if (reset) {
        grid->ev_used = 0;
        grid->stencil_launches = 0;
        grid->kernel_launches = 0;
    }
    return SENSEI_OK;
}

sensei_status sensei_profile_launches(sensei_grid *grid, double *ms, int cap, int *count)
{
    sensei_status st = check_grid(grid);
    if (st != SENSEI_OK) return st;
    if (!count) return fail(SENSEI_ERR_INVALID_ARG, "count is NULL");
    if (cap < 0 || (cap > 0 && !ms)) return fail(SENSEI_ERR_INVALID_ARG, "ms is NULL or cap < 0");
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    const int n = (int)(grid->ev_used / 2);
    for (int i = 0; i < n && i < cap; ++i) {
        CUDA_TRY(cudaEventSynchronize(grid->ev[2 * i + 1]));
        float t = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&t, grid->ev[2 * i], grid->ev[2 * i + 1]));
        ms[i] = t;
    }
    *count = n;
    return SENSEI_OK;
}

sensei_status sensei_workspace_size(const sensei_block_desc *blocks, int nblocks, const sensei_scheme *scheme,
                                    size_t *bytes)
{
    if (!bytes) return fail(SENSEI_ERR_INVALID_ARG, "bytes is NULL");
    Plan P;
    sensei_status st = make_plan(blocks, nblocks, scheme, P);
    if (st != SENSEI_OK) return st;
    *bytes = P.bytes;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_create_grid(const sensei_block_desc *blocks, int nblocks, const double *const *nodes,
                                 const sensei_scheme *scheme, void *workspace, size_t workspace_bytes,
                                 sensei_stream stream, sensei_grid **out)
{
    TraceRange trace("sensei_create_grid");
    if (!out) return fail(SENSEI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    Plan P;
    sensei_status st = make_plan(blocks, nblocks, scheme, P);
    if (st != SENSEI_OK) return st;
    if (!nodes) return fail(SENSEI_ERR_INVALID_ARG, "nodes is NULL");
    for (int b = 0; b < nblocks; ++b)
        if (!nodes[b]) return fail(SENSEI_ERR_INVALID_ARG, "nodes[%d] is NULL", b);
    if (!workspace) return fail(SENSEI_ERR_INVALID_ARG, "workspace is NULL");
    if (((uintptr_t)workspace) % 256) return fail(SENSEI_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (workspace_bytes < P.bytes)
        return fail(SENSEI_ERR_INVALID_ARG, "workspace too small: %zu bytes given, %zu needed", workspace_bytes,
                    P.bytes);
    cudaStream_t s = (cudaStream_t)stream;
    sensei_grid *g = new sensei_grid();
    if (cudaGetDevice(&g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
        delete g;
        return fail(SENSEI_ERR_CUDA, "cannot query the current device");
    }
    g->scheme = *scheme;
    g->plan = P;
    g->ws = (char *)workspace;
    g->desc = (BlockDev *)(g->ws + P.off_desc);
    g->partials = (double *)(g->ws + P.off_partials);
    g->dt_bits = (unsigned long long *)(g->ws + P.off_dtbits);
    g->dt_next = (unsigned long long *)(g->ws + P.off_dtnext);
    g->dt_slot = (double *)(g->ws + P.off_dtslot);
    g->norms = (double *)(g->ws + P.off_norms);
    g->order = (int *)(g->ws + P.off_order);
    g->err = (unsigned *)(g->norms + 15);
    for (int b = 0; b < nblocks; ++b) {
        BlockDev &B = g->plan.blocks[b].dev;
        const size_t mv = (size_t)B.ml.mvolume;
        B.fn = (const double *)(g->ws + P.off_fn[b]);
        B.fdf = P.off_fdf[b] ? (const float2 *)(g->ws + P.off_fdf[b]) : nullptr;
        B.rec32 = P.off_rec32[b] ? (const float *)(g->ws + P.off_rec32[b]) : nullptr;
        B.vol = (const double *)(g->ws + P.off_vol[b]);
        B.ivol = (const double *)(g->ws + P.off_ivol[b]);
        B.sbar = (const double *)(g->ws + P.off_sbar[b]);
        B.sbar32 = P.off_sbar32[b] ? (const float *)(g->ws + P.off_sbar32[b]) : nullptr;
        B.vol32 = B.sbar32 ? B.sbar32 + 12 * mv : nullptr;
        B.dtv = (double *)(g->ws + P.off_dtv[b]);
        B.wv = P.off_wv[b] ? (double *)(g->ws + P.off_wv[b]) : nullptr;
        B.rvis = P.off_rvis[b] ? (double *)(g->ws + P.off_rvis[b]) : nullptr;
        B.fvis = P.off_fvis[b] ? (double *)(g->ws + P.off_fvis[b]) : nullptr;
        B.gvis = P.off_gvis[b] ? (double *)(g->ws + P.off_gvis[b]) : nullptr;
        B.st64[0] = (double *)(g->ws + P.off_stage[b]);
        B.st64[1] = B.st64[0] + B.L.elems;
        // FP32 storage reuses the same bytes: X0, X1, D0, D1
        B.xs[0] = (float *)B.st64[0];
        B.xs[1] = B.xs[0] + B.L.elems;
        B.ds[0] = B.xs[1] + B.L.elems;
        B.ds[1] = B.ds[0] + B.L.elems;
        B.tmaps = P.off_tmap[b] ? (const unsigned char *)(g->ws + P.off_tmap[b]) : nullptr;
        MetricsOut mo;
        memset(&mo, 0, sizeof mo);
        for (int fam = 0; fam < 3; ++fam)
            for (int q = 0; q < 4; ++q) {
                mo.n[fam][q] = (double *)B.fn + (fam * 4 + q) * mv;
                mo.sbar[fam][q] = (double *)B.sbar + (fam * 4 + q) * mv;
                mo.sbar32[fam][q] = B.sbar32 ? (float *)B.sbar32 + (fam * 4 + q) * mv : nullptr;
            }
        mo.vol = (double *)B.vol;
        mo.ivol = (double *)B.ivol;
        mo.vol32 = (float *)B.vol32;
        cudaError_t e = launch_metrics(B.ni, B.nj, B.nk, nodes[b], mo, B.ml, s);
        if (e == cudaSuccess) e = launch_pack_records(B, s);
        if (e == cudaSuccess) e = launch_split_df64(B, s);
        if (e != cudaSuccess) {
            delete g;
            return fail(SENSEI_ERR_CUDA, "metrics kernel: %s", cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaMemsetAsync(g->norms, 0, 16 * sizeof(double), s);
    if (e != cudaSuccess) {
        delete g;
        return fail(SENSEI_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    // tensor maps of the internal state slots (fixed addresses); the
    // SLOT_USER maps follow the caller's pointers (ensure_user_maps)
    g->tmaps_host.assign((size_t)nblocks * 5 * TMAP_BYTES, 0);
    g->tmap_user.assign(nblocks, nullptr);
    for (int b = 0; b < nblocks; ++b) {
        const BlockDev &B = g->plan.blocks[b].dev;
        if (!B.tmaps) continue;
        unsigned char *h = g->tmaps_host.data() + (size_t)b * 5 * TMAP_BYTES;
        const void *bases[5] = {nullptr, B.st64[0], B.st64[1], B.xs[0], B.xs[1]};
        for (int slot = SLOT_ST0; slot <= SLOT_X1; ++slot)
            if (!encode_state_map(h + slot * TMAP_BYTES, bases[slot], B, slot >= SLOT_X0)) {
                delete g;
                return fail(SENSEI_ERR_CUDA, "cuTensorMapEncodeTiled rejected the state slot %d of block %d", slot, b);
            }
        e = cudaMemcpyAsync((void *)B.tmaps, h, 5 * TMAP_BYTES, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            delete g;
            return fail(SENSEI_ERR_CUDA, "uploading tensor maps: %s", cudaGetErrorString(e));
        }
    }
    *out = g;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_destroy_grid(sensei_grid *grid)
{
    if (!grid) return fail(SENSEI_ERR_INVALID_ARG, "grid is NULL");
    delete grid;
    return SENSEI_OK;
}

sensei_status sensei_state_layout(const sensei_grid *grid, int block, sensei_layout *out)
{
    sensei_status st = check_grid(grid);
    if (st != SENSEI_OK) return st;
    if (!out) return fail(SENSEI_ERR_INVALID_ARG, "out is NULL");
    if (block < 0 || block >= (int)grid->plan.blocks.size())
        return fail(SENSEI_ERR_INVALID_ARG, "block %d out of range", block);
    const BlockDev &B = grid->plan.blocks[block].dev;
    out->stride_j = B.L.sj;
    out->stride_k = B.L.sk;
    out->stride_var = B.L.sv;
    out->offset = B.L.off;
    out->elems = B.L.elems;
    out->ghost_i = NG;
    out->ghost_j = NG;
    out->ghost_k = B.L.gk;
    out->elem_bytes = (int)sizeof(double);
    return SENSEI_OK;
}

sensei_status sensei_set_bc(sensei_grid *grid, int block, int face, int type, const double *prim, int nbr_block,
                            int nbr_face, int orientation)
{
    sensei_status st = check_grid(grid);
    if (st != SENSEI_OK) return st;
    const int nb = (int)grid->plan.blocks.size();
    if (block < 0 || block >= nb) return fail(SENSEI_ERR_INVALID_ARG, "block %d out of range", block);
    HostBlock &H = grid->plan.blocks[block];
    BlockDev &B = H.dev;
    if (face < 0 || face >= (H.two_d ? 4 : 6))
        return fail(SENSEI_ERR_INVALID_ARG, "face %d out of range for a %s block", face, H.two_d ? "2D" : "3D");
    if (type < SENSEI_BC_PERIODIC || type > SENSEI_BC_EXTERNAL)
        return fail(SENSEI_ERR_INVALID_ARG, "unknown boundary type %d", type);
    if (type == SENSEI_BC_EXTERNAL && grid->scheme.mu > 0.0)
        return fail(SENSEI_ERR_UNSUPPORTED, "caller-written ghost layers with the viscous flux");
    const int axis = face >> 1;
    const int n_own = axis == 0 ? B.ni : axis == 1 ? B.nj : B.nk;
    // every rule reads or feeds the two cell layers next to a boundary
    if (n_own < NG)
        return fail(SENSEI_ERR_INVALID_ARG, "a block needs at least %d cells along a bounded direction (has %d)", NG,
                    n_own);
    if (type == SENSEI_BC_INFLOW) {
        if (!prim) return fail(SENSEI_ERR_INVALID_ARG, "inflow needs the primitive state");
        if (!(prim[0] > 0.0) || !(prim[4] > 0.0))
            return fail(SENSEI_ERR_INVALID_ARG, "inflow state needs rho > 0 and p > 0");
        memcpy(B.bc_prim[face], prim, sizeof B.bc_prim[face]);
    } else if (type == SENSEI_BC_INTERFACE) {
        if (orientation != 0) return fail(SENSEI_ERR_UNSUPPORTED, "only aligned interfaces (orientation 0)");
        if (nbr_block < 0 || nbr_block >= nb) return fail(SENSEI_ERR_INVALID_ARG, "neighbour block out of range");
        const HostBlock &NH = grid->plan.blocks[nbr_block];
        const BlockDev &N = NH.dev;
        if (nbr_face < 0 || nbr_face >= (NH.two_d ? 4 : 6) || (nbr_face >> 1) != axis || nbr_face == face)
            return fail(SENSEI_ERR_INVALID_ARG, "neighbour face must be the opposite side of the same direction");
        int a1 = face < 2 ? B.nj : B.ni, a2 = face < 4 ? B.nk : B.nj;
        int b1 = nbr_face < 2 ? N.nj : N.ni, b2 = nbr_face < 4 ? N.nk : N.nj;
        if (a1 != b1 || a2 != b2)
            return fail(SENSEI_ERR_INVALID_ARG, "interface faces differ in size (%d x %d vs %d x %d)", a1, a2, b1, b2);
        const int nb_n = axis == 0 ? N.ni : axis == 1 ? N.nj : N.nk;
        if (nb_n < NG) return fail(SENSEI_ERR_INVALID_ARG, "neighbour block too thin for two ghost layers");
        B.nbr[face] = nbr_block;
        B.nbr_face[face] = nbr_face;
    }
    B.bc_type[face] = type;
    H.bc_set[face] = true;
    grid->dirty = true;
    grid->stage_ghosts = false;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_fill_ghosts(sensei_grid *grid, double *const *U, sensei_stream stream)
{
    TraceRange trace("sensei_fill_ghosts");
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st == SENSEI_OK) st = check_bcs(grid);
    if (st != SENSEI_OK) return st;
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = sync_descriptors(grid, s);
    if (st == SENSEI_OK) st = fill_slot(grid, SLOT_USER, U, s);
    if (st == SENSEI_OK && viscous(grid)) st = fill_edges(grid, SLOT_USER, U, s);
    if (st == SENSEI_OK) g_msg[0] = 0;
    return st;
}

sensei_status sensei_residual(sensei_grid *grid, double *const *U, double *const *R, const double *const *src,
                              sensei_stream stream)
{
    TraceRange trace("sensei_residual");
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st == SENSEI_OK) st = check_states(grid, R, "R");
    if (st == SENSEI_OK) st = check_bcs(grid);
    if (st != SENSEI_OK) return st;
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = sync_descriptors(grid, s);
    if (st == SENSEI_OK) st = fill_slot(grid, SLOT_USER, U, s);
    if (st != SENSEI_OK) return st;
    StencilCall c;
    memset(&c, 0, sizeof c);
    c.mode = MODE_RESIDUAL;
    c.in_slot = SLOT_USER;
    c.out_slot = SLOT_USER;
    c.dprev = -1;
    c.dout = -1;
    c.partials = true;
    c.user = U;
    c.rout = R;
    c.src = src;
    if (viscous(grid)) {
        st = viscous_residual(grid, SLOT_USER, U, s);
        if (st != SENSEI_OK) return st;
        c.vis = true;
    }
    st = stencil(grid, c, s);
    if (st != SENSEI_OK) return st;
    CUDA_TRY(launch_norms_finalize(grid->partials, (int)total_items(grid->plan.blocks), grid->plan.ncells,
                                   grid->norms, s));
    grid->kernel_launches++;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_rk_step(sensei_grid *grid, double *const *U, int rk, double cfl, double dt, double *dt_used,
                             sensei_stream stream)
{
    TraceRange trace("sensei_rk_step");
    sensei_status st = check_step_args(grid, U, rk, cfl, dt);
    if (st != SENSEI_OK) return st;
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = prepare_step(grid, U, s);
    if (st == SENSEI_OK) st = rk_step_launches(grid, U, rk, cfl, dt, dt_used, s);
    if (st == SENSEI_OK) g_msg[0] = 0;
    return st;
}

// nsteps Runge-Kutta steps, launches only (after prepare_step).  On
// fused_next_dt grids every step but the last leaves the next step's bound
// in one of the two dt_next slots and the next step reads it instead of
// running the time-step kernel: the same dt, one pass over the state fewer.
sensei_status rk_steps_launches(sensei_grid *grid, double *const *U, int nsteps, int rk, double cfl, double dt,
                                double *dt_used, cudaStream_t s)
{
    const bool fused = fused_next_dt(grid, cfl);
    for (int n = 0; n < nsteps; ++n) {
        const unsigned long long *in = fused && n > 0 ? grid->dt_next + (n - 1) % 2 : nullptr;
        unsigned long long *out = fused && n + 1 < nsteps ? grid->dt_next + n % 2 : nullptr;
        sensei_status st = rk_step_launches(grid, U, rk, cfl, dt, dt_used ? dt_used + n : nullptr, s, false, in, out);
        if (st != SENSEI_OK) return st;
    }
    return SENSEI_OK;
}

sensei_status sensei_rk_steps(sensei_grid *grid, double *const *U, int nsteps, int rk, double cfl, double dt,
                              double *dt_used, sensei_stream stream)
{
    TraceRange trace("sensei_rk_steps");
    sensei_status st = check_step_args(grid, U, rk, cfl, dt);
    if (st != SENSEI_OK) return st;
    if (nsteps < 1) return fail(SENSEI_ERR_INVALID_ARG, "nsteps must be at least 1 (got %d)", nsteps);
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = prepare_step(grid, U, s);
    if (st == SENSEI_OK) st = rk_steps_launches(grid, U, nsteps, rk, cfl, dt, dt_used, s);
    if (st == SENSEI_OK) g_msg[0] = 0;
    return st;
}

sensei_status sensei_rk_stage(sensei_grid *grid, double *const *U, int rk, int stage, double dt,
                              sensei_stream stream)
{
    TraceRange trace("sensei_rk_stage");
    sensei_status st = check_step_args(grid, U, rk, 0.0, dt);
    if (st != SENSEI_OK) return st;
    if (grid->scheme.precision != SENSEI_FP64 || viscous(grid))
        return fail(SENSEI_ERR_UNSUPPORTED, "stage-by-stage stepping runs the FP64 Euler form");
    const int S = RK_STAGES[rk];
    if (stage < 0 || stage >= S) return fail(SENSEI_ERR_INVALID_ARG, "stage %d out of range (%d stages)", stage, S);
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (stage == 0) {
        st = prepare_step(grid, U, s);
        if (st == SENSEI_OK) st = fill_slot(grid, SLOT_USER, U, s);
        if (st != SENSEI_OK) return st;
        CUDA_TRY(launch_set_scalar(grid->dt_slot, dt, s));
        grid->kernel_launches++;
    }
    const double *co = RK_COEF[rk][stage];
    StencilCall c;
    memset(&c, 0, sizeof c);
    c.alpha = co[0];
    c.beta = co[1];
    c.gdt = co[2];
    c.dt_slot = grid->dt_slot;
    c.dt_scale = 1.0;
    c.partials = stage == 0;
    c.user = U;
    c.push = 1;
    c.dprev = -1;
    c.dout = -1;
    c.mode = MODE_ACCUM;
    c.in_slot = stage == 0 ? SLOT_USER : SLOT_ST0 + (stage - 1) % 2;
    c.out_slot = stage == S - 1 ? SLOT_USER : SLOT_ST0 + stage % 2;
    st = stencil(grid, c, s);
    if (st != SENSEI_OK) return st;
    if (stage == S - 1) {
        CUDA_TRY(launch_norms_finalize(grid->partials, (int)total_items(grid->plan.blocks), grid->plan.ncells,
                                       grid->norms, s));
        grid->kernel_launches++;
    }
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_face_exchange(sensei_grid *grid, double *const *U, int block, int stage, int face, double *buf,
                                   int unpack, sensei_stream stream)
{
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st != SENSEI_OK) return st;
    if (block < 0 || block >= (int)grid->plan.blocks.size())
        return fail(SENSEI_ERR_INVALID_ARG, "block %d out of range", block);
    const HostBlock &H = grid->plan.blocks[block];
    if (face < 0 || face >= (H.two_d ? 4 : 6)) return fail(SENSEI_ERR_INVALID_ARG, "face %d out of range", face);
    if (stage < 0 || stage > 3) return fail(SENSEI_ERR_INVALID_ARG, "stage %d out of range", stage);
    if (!buf) return fail(SENSEI_ERR_INVALID_ARG, "buf is NULL");
    if (grid->scheme.precision != SENSEI_FP64)
        return fail(SENSEI_ERR_UNSUPPORTED, "face exchange of the FP64 stage states only");
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    const BlockDev &B = H.dev;
    double *u = stage == 0 ? U[block] : B.st64[(stage - 1) % 2];
    CUDA_TRY(launch_face_exchange(B, u, face, buf, unpack ? 1 : 0, (cudaStream_t)stream));
    grid->kernel_launches++;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_dt_min(sensei_grid *grid, double *const *U, double cfl, double *dt_out, sensei_stream stream)
{
    if (!dt_out || !(cfl > 0.0)) return fail(SENSEI_ERR_INVALID_ARG, "need cfl > 0 and an output");
    double m = 0.0;
    sensei_status st = dt_min_launch(grid, U, &m, (cudaStream_t)stream);
    if (st != SENSEI_OK) return st;
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *dt_out = cfl * m;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_rk_step_local(sensei_grid *grid, double *const *U, int rk, double cfl, double *dt_min,
                                   sensei_stream stream)
{
    TraceRange trace("sensei_rk_step_local");
    sensei_status st = check_step_args(grid, U, rk, cfl, 0.0);
    if (st != SENSEI_OK) return st;
    if (!(cfl > 0.0)) return fail(SENSEI_ERR_INVALID_ARG, "local time stepping needs cfl > 0");
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = prepare_step(grid, U, s);
    if (st == SENSEI_OK) st = rk_step_launches(grid, U, rk, cfl, 0.0, dt_min, s, true);
    if (st == SENSEI_OK) g_msg[0] = 0;
    return st;
}

static sensei_status steps_graph_create(sensei_grid *grid, double *const *U, int nsteps, int rk, double cfl,
                                        double dt, double *dt_used, sensei_stream stream, sensei_step_graph **out)
{
    if (!out) return fail(SENSEI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    sensei_status st = check_step_args(grid, U, rk, cfl, dt);
    if (st != SENSEI_OK) return st;
    if (nsteps < 1) return fail(SENSEI_ERR_INVALID_ARG, "nsteps must be at least 1 (got %d)", nsteps);
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = prepare_step(grid, U, s);
    if (st != SENSEI_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(s));
    // capture on a private stream: the caller's may be the legacy stream
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const bool prof = grid->prof;
    grid->prof = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = rk_steps_launches(grid, U, nsteps, rk, cfl, dt, dt_used, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st == SENSEI_OK && e2 != cudaSuccess) st = fail(SENSEI_ERR_CUDA, "capture: %s", cudaGetErrorString(e2));
    } else {
        st = fail(SENSEI_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    grid->prof = prof;
    cudaStreamDestroy(cs);
    if (st != SENSEI_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(SENSEI_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    sensei_step_graph *gr = new sensei_step_graph();
    gr->grid = grid;
    gr->exec = exec;
    *out = gr;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_step_graph_create(sensei_grid *grid, double *const *U, int rk, double cfl, double dt,
                                       double *dt_used, sensei_stream stream, sensei_step_graph **out)
{
    return steps_graph_create(grid, U, 1, rk, cfl, dt, dt_used, stream, out);
}

sensei_status sensei_steps_graph_create(sensei_grid *grid, double *const *U, int nsteps, int rk, double cfl,
                                        double dt, double *dt_used, sensei_stream stream, sensei_step_graph **out)
{
    return steps_graph_create(grid, U, nsteps, rk, cfl, dt, dt_used, stream, out);
}

sensei_status sensei_step_graph_launch(sensei_step_graph *graph, sensei_stream stream)
{
    TraceRange trace("sensei_step_graph_launch");
    if (!graph) return fail(SENSEI_ERR_INVALID_ARG, "graph is NULL");
    if (graph->grid->dirty || !graph->grid->stage_ghosts)
        return fail(SENSEI_ERR_STATE, "the grid's boundary rules or schedule changed since the graph was made");
    Device dev;
    CUDA_TRY(dev.set(graph->grid->device));
    CUDA_TRY(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
    return SENSEI_OK;
}

sensei_status sensei_step_graph_destroy(sensei_step_graph *graph)
{
    if (!graph) return fail(SENSEI_ERR_INVALID_ARG, "graph is NULL");
    cudaGraphExecDestroy(graph->exec);
    delete graph;
    return SENSEI_OK;
}

sensei_status sensei_autotune(sensei_grid *grid, double *const *U, int *kchunk_out, int *persistent_out,
                              sensei_stream stream)
{
    TraceRange trace("sensei_autotune");
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st == SENSEI_OK) st = check_bcs(grid);
    if (st != SENSEI_OK) return st;
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = prepare_step(grid, U, s);
    if (st == SENSEI_OK) st = fill_slot(grid, SLOT_USER, U, s);
    if (st != SENSEI_OK) return st;
    // the stage launches of a three-stage step with dt = 0 into the stage
    // buffers: a first stage (the caller's state in, norm partials) and twice
    // a later stage (a stage state in, blended with U^n); the first and the
    // later stages are different kernels in the FP32-storage form and
    // different instantiations in the others, and their best schedules can
    // differ.  Nothing of the caller's state is written.
    CUDA_TRY(launch_set_scalar(grid->dt_slot, 0.0, s));
    const bool incr = incr_mode(grid);
    StencilCall c, c2;
    memset(&c, 0, sizeof c);
    c.mode = incr ? MODE_INCR : MODE_ACCUM;
    c.in_slot = SLOT_USER;
    c.out_slot = incr ? SLOT_X0 : SLOT_ST0;
    c.dprev = -1;
    c.dout = incr ? 0 : -1;
    c.beta = 1.0;
    c.gdt = 1.0;
    c.dt_slot = grid->dt_slot;
    c.dt_scale = 1.0;
    c.user = U;
    c.partials = true;
    c.push = 1;
    c2 = c;
    c2.partials = false;
    c2.in_slot = incr ? SLOT_X0 : SLOT_ST0;
    c2.out_slot = incr ? SLOT_X1 : SLOT_ST1;
    c2.alpha = 0.75;
    c2.beta = 0.25;
    c2.gdt = 0.25;
    c2.dprev = incr ? 0 : -1;
    c2.dout = incr ? 1 : -1;
    int max_nk = 1;
    for (auto &H : grid->plan.blocks) max_nk = std::max(max_nk, H.dev.nk);
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const bool prof = grid->prof;
    grid->prof = false;
    float best = 1e30f;
    int best_k = grid->plan.blocks[0].dev.kchunk, best_mode = grid->grid_mode, best_order = grid->order_mode;
    // item orders: block-major, and by cost when the blocks differ in size
    // (one block: every item but a last shorter chunk costs the same)
    const int orders = grid->plan.blocks.size() > 1 ? 2 : 1;
    for (int kc : KCHUNK_CANDIDATES) {
        if (grid->plan.two_d && kc != KCHUNK_CANDIDATES[0]) continue;
        if (kc > 2 * max_nk) continue;
        assign_items(grid->plan.blocks, kc);
        for (int om = 0; om < orders && st == SENSEI_OK; ++om) {
        grid->order_mode = om;
        grid->dirty = true;
        st = sync_descriptors(grid, s);
        if (st != SENSEI_OK) break;
        for (int mode = 0; mode < 2 && st == SENSEI_OK; ++mode) {
            grid->grid_mode = mode;
            float ms = 1e30f;
            for (int rep = 0; rep < 3 && st == SENSEI_OK; ++rep) {
                cudaEventRecord(e0, s);
                st = stencil_launch(grid, c, s);
                for (int later = 0; later < 2 && st == SENSEI_OK; ++later) st = stencil_launch(grid, c2, s);
                cudaEventRecord(e1, s);
                if (st == SENSEI_OK && cudaEventSynchronize(e1) != cudaSuccess)
                    st = fail(SENSEI_ERR_CUDA, "autotune timing failed");
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms = std::min(ms, t);   // the first launch warms up
            }
            if (st == SENSEI_OK && ms < best) {
                best = ms;
                best_k = kc;
                best_mode = mode;
                best_order = om;
            }
        }
        }
        if (st != SENSEI_OK) break;
    }
    grid->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    assign_items(grid->plan.blocks, best_k);
    grid->grid_mode = best_mode;
    grid->order_mode = best_order;
    grid->dirty = true;
    sensei_status st2 = sync_descriptors(grid, s);
    if (st == SENSEI_OK) st = st2;
    if (st != SENSEI_OK) return st;
    if (kchunk_out) *kchunk_out = best_k;
    if (persistent_out) *persistent_out = best_mode == 0;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_schedule(const sensei_grid *grid, int *kchunk, int *persistent, int *order_by_cost,
                              int *ctas_per_sm)
{
    sensei_status st = check_grid(grid);
    if (st != SENSEI_OK) return st;
    int kc = 1;
    for (const HostBlock &H : grid->plan.blocks) kc = std::max(kc, H.dev.kchunk);
    if (kchunk) *kchunk = kc;
    if (persistent) *persistent = grid->grid_mode == 0;
    if (order_by_cost) *order_by_cost = grid->order_mode == 1;
    if (ctas_per_sm) {
        int best = 0;
        for (int kind = 0; kind < 4; ++kind) best = std::max(best, grid->ctas_cache[kind]);
        *ctas_per_sm = best;
    }
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_norms(sensei_grid *grid, double *l2, double *linf, double *cons, sensei_stream stream)
{
    sensei_status st = check_grid(grid);
    if (st != SENSEI_OK) return st;
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    double host[16];
    CUDA_TRY(cudaMemcpyAsync(host, grid->norms, sizeof host, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int q = 0; q < NV; ++q) {
        if (l2) l2[q] = host[q];
        if (linf) linf[q] = host[NV + q];
        if (cons) cons[q] = host[2 * NV + q];
    }
    unsigned errw;
    memcpy(&errw, &host[15], sizeof errw);
    if (errw) {
        CUDA_TRY(cudaMemsetAsync(grid->err, 0, sizeof(unsigned), s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (errw & ERR_TIMEOUT)
            return fail(SENSEI_ERR_TIMEOUT, "a bounded wait on an asynchronous tile copy gave up (error word 0x%x)",
                        errw);
        return fail(SENSEI_ERR_NONPHYSICAL, "a kernel met rho <= 0, p <= 0 or a non-finite state (error word 0x%x)",
                    errw);
    }
    g_msg[0] = 0;
    return SENSEI_OK;
}

}  // extern "C"
