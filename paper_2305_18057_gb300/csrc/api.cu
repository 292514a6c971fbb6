// api.cu -- host side of the C ABI declared in include/sensei.h.
//
// The library allocates no device memory: every device array is either the
// caller's (states, residuals, nodes, sources) or a slice of the caller's
// workspace (metrics, Runge-Kutta stage buffers, reduction partials, the
// time-step slot, the norms and the error word).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "sensei_internal.cuh"

using namespace sensei;

namespace {

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

struct Block {
    int ni, nj, nk;
    bool two_d;
    StateLayout L;
    MetricLayout ml;
    double *fn[3][4];
    float *fn32[3][4];
    double *vol, *ivol;
    float *ivol32;
    double *sbar[3][4];
    double *stage[2];       // FP64 stage states (FP64, FP32-flux)
    float *xs[2], *ds[2];   // FP32 stage states and increments (FP32 storage)
    int tiles_i, tiles_j, kchunk, nchunks;
    long long part_off;   // first partial slot (CTA index) of this block
    int nparts;
    bool bc_set[6];
    int bc_type[6];
    double bc_prim[6][NV];
    int nbr[6], nbr_face[6];
};

// Byte offsets of every workspace slice, computed identically by
// sensei_workspace_size and sensei_create_grid.
struct Plan {
    std::vector<Block> blocks;
    size_t bytes = 0;
    size_t off_partials = 0, off_dtbits = 0, off_dtslot = 0, off_norms = 0;
    long long nparts = 0;
    long long ncells = 0;
    // per-block offsets (same order as the Block fields)
    std::vector<size_t> off_fn, off_fn32, off_vol, off_ivol, off_ivol32, off_sbar, off_stage;
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
    if (s->precision < SENSEI_FP64 || s->precision > SENSEI_FP32_STORE)
        return fail(SENSEI_ERR_INVALID_ARG, "unknown precision %d", s->precision);
    if (!(s->entropy_fix >= 0.0)) return fail(SENSEI_ERR_INVALID_ARG, "entropy_fix must be >= 0");
    if (!(s->eps >= 0.0 && s->eps <= 1.0)) return fail(SENSEI_ERR_INVALID_ARG, "eps must lie in [0, 1]");
    if (!(s->kappa >= -1.0 && s->kappa <= 1.0)) return fail(SENSEI_ERR_INVALID_ARG, "kappa must lie in [-1, 1]");
    return SENSEI_OK;
}

sensei_status make_plan(const sensei_block_desc *blocks, int nblocks, const sensei_scheme *scheme, Plan &P)
{
    if (!blocks || nblocks <= 0) return fail(SENSEI_ERR_INVALID_ARG, "need at least one block");
    sensei_status st = check_scheme(scheme);
    if (st != SENSEI_OK) return st;
    size_t cur = 0;
    P.blocks.resize(nblocks);
    P.off_fn.resize(nblocks);
    P.off_fn32.resize(nblocks);
    P.off_vol.resize(nblocks);
    P.off_ivol.resize(nblocks);
    P.off_ivol32.resize(nblocks);
    P.off_sbar.resize(nblocks);
    P.off_stage.resize(nblocks);
    const bool f32 = scheme->precision != SENSEI_FP64;
    for (int b = 0; b < nblocks; ++b) {
        const sensei_block_desc &d = blocks[b];
        if (d.ni < 1 || d.nj < 1 || d.nk < 1)
            return fail(SENSEI_ERR_INVALID_ARG, "block %d: need ni, nj, nk >= 1 (got %d x %d x %d)", b, d.ni, d.nj,
                        d.nk);
        if ((long long)d.ni * d.nj * d.nk > (1LL << 34))
            return fail(SENSEI_ERR_INVALID_ARG, "block %d: too many cells", b);
        Block &B = P.blocks[b];
        memset(&B, 0, sizeof B);
        B.ni = d.ni;
        B.nj = d.nj;
        B.nk = d.nk;
        B.two_d = d.nk == 1;
        const int gk = B.two_d ? 0 : NG;
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
        if (B.two_d) {
            B.nchunks = 1;
            B.kchunk = 1;
        } else {
            const long long target = 152LL * 8;
            long long tiles = (long long)B.tiles_i * B.tiles_j;
            long long nch = (target + tiles - 1) / tiles;
            if (nch < 1) nch = 1;
            if (nch > d.nk) nch = d.nk;
            B.kchunk = (int)((d.nk + nch - 1) / nch);
            B.nchunks = (d.nk + B.kchunk - 1) / B.kchunk;
        }
        B.nparts = B.tiles_i * B.tiles_j * B.nchunks;
        B.part_off = P.nparts;
        P.nparts += B.nparts;
        P.ncells += (long long)d.ni * d.nj * d.nk;
        const size_t mv = (size_t)B.ml.mvolume;
        P.off_fn[b] = take(cur, 12 * mv * sizeof(double));
        P.off_fn32[b] = f32 ? take(cur, 12 * mv * sizeof(float)) : 0;
        P.off_vol[b] = take(cur, mv * sizeof(double));
        P.off_ivol[b] = take(cur, mv * sizeof(double));
        P.off_ivol32[b] = f32 ? take(cur, mv * sizeof(float)) : 0;
        P.off_sbar[b] = take(cur, 12 * mv * sizeof(double));
        // two FP64 stage states, or two FP32 stage states + two FP32 increments
        P.off_stage[b] = take(cur, 2 * (size_t)B.L.elems * sizeof(double));
    }
    if (P.nparts > (1LL << 30)) return fail(SENSEI_ERR_INVALID_ARG, "grid too large");
    P.off_partials = take(cur, (size_t)P.nparts * 3 * NV * sizeof(double));
    P.off_dtbits = take(cur, sizeof(unsigned long long));
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
    sensei_scheme scheme;
    Plan plan;
    char *ws;
    double *partials;
    unsigned long long *dt_bits;
    double *dt_slot;
    double *norms;   // 15 doubles, then the error word
    unsigned *err;
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
        const Block &B = g->plan.blocks[b];
        for (int f = 0; f < (B.two_d ? 4 : 6); ++f)
            if (!B.bc_set[f]) return fail(SENSEI_ERR_STATE, "block %zu face %d has no boundary condition", b, f);
    }
    return SENSEI_OK;
}

CellMetrics cell_metrics(const Block &B)
{
    CellMetrics cm;
    cm.vol = B.vol;
    cm.ivol = B.ivol;
    cm.ivol32 = B.ivol32;
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 4; ++q) cm.sbar[d][q] = B.sbar[d][q];
    return cm;
}

template <typename T>
sensei_status fill_ghosts_impl(sensei_grid *g, T *const *U, cudaStream_t s)
{
    const auto &blocks = g->plan.blocks;
    for (size_t b = 0; b < blocks.size(); ++b) {
        const Block &B = blocks[b];
        BCParamsT<T> p;
        memset(&p, 0, sizeof p);
        p.ni = B.ni;
        p.nj = B.nj;
        p.nk = B.nk;
        p.L = B.L;
        p.U = U[b];
        p.nfaces = B.two_d ? 4 : 6;
        p.gamma = g->scheme.gamma;
        p.ml = B.ml;
        for (int fam = 0; fam < 3; ++fam)
            for (int q = 0; q < 4; ++q) p.fm.n[fam][q] = B.fn[fam][q];
        for (int f = 0; f < p.nfaces; ++f) {
            FaceBC<T> &fb = p.f[f];
            fb.type = B.bc_type[f];
            memcpy(fb.prim, B.bc_prim[f], sizeof fb.prim);
            long long n1 = f < 2 ? B.nj : B.ni;
            long long n2 = f < 4 ? B.nk : B.nj;
            p.count[f] = n1 * n2 * 2;
            if (fb.type == SENSEI_BC_INTERFACE) {
                const Block &N = blocks[B.nbr[f]];
                fb.nbr = U[B.nbr[f]];
                fb.nL = N.L;
                fb.nni = N.ni;
                fb.nnj = N.nj;
                fb.nnk = N.nk;
                fb.nbr_face = B.nbr_face[f];
            }
        }
        CUDA_TRY(launch_bc(p, s));
        g->kernel_launches++;
    }
    return SENSEI_OK;
}

const double RK_COEF[3][4][3] = {
    // alpha, beta, gdt of out = alpha U^n + beta U^(s-1) - gdt dt R/|Omega|
    {{0.0, 1.0, 1.0}, {0.5, 0.5, 0.5}},
    {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}},
    {{0.0, 1.0, 1.0 / 3.0}, {0.0, 1.0, 1.0 / 3.0}, {0.0, 1.0, 1.0 / 3.0}, {0.25, 0.75, 0.25}},
};
const int RK_STAGES[3] = {2, 3, 4};

template <typename R>
void fill_common(StencilParams<R> &p, const sensei_grid *g, const Block &B)
{
    p.ni = B.ni;
    p.nj = B.nj;
    p.nk = B.nk;
    p.tiles_i = B.tiles_i;
    p.tiles_j = B.tiles_j;
    p.kchunk = B.kchunk;
    p.nchunks = B.nchunks;
    p.L = B.L;
    p.cm = cell_metrics(B);
    p.ml = B.ml;
    p.gamma = (R)g->scheme.gamma;
    p.kappa = (R)g->scheme.kappa;
    p.eps = (R)g->scheme.eps;
    p.fix = (R)g->scheme.entropy_fix;
    p.cons = g->scheme.reconstruct_conserved ? 1 : 0;
    p.err = g->err;
}

struct StencilCall {
    int mode;
    const void *in;
    bool in_f32;            // the stage input is an FP32 stage state
    const double *un;
    double *out;
    const float *dprev;
    float *dout, *xout;
    double *Rout;
    const double *src;
    double alpha, beta, gdt;
    const double *dt_slot;
    double dt_scale;
    bool partials;
};

sensei_status stencil_launch(sensei_grid *g, const Block &B, const StencilCall &c, cudaStream_t s);

sensei_status stencil(sensei_grid *g, const Block &B, const StencilCall &c, cudaStream_t s)
{
    if (!g->prof) {
        g->kernel_launches++;
        return stencil_launch(g, B, c, s);
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
    sensei_status st = stencil_launch(g, B, c, s);
    if (st != SENSEI_OK) return st;
    CUDA_TRY(cudaEventRecord(e1, s));
    g->kernel_launches++;
    g->stencil_launches++;
    return SENSEI_OK;
}

sensei_status stencil_launch(sensei_grid *g, const Block &B, const StencilCall &c, cudaStream_t s)
{
    if (g->scheme.precision == SENSEI_FP64) {
        StencilParams<double> p;
        memset(&p, 0, sizeof p);
        fill_common(p, g, B);
        for (int fam = 0; fam < 3; ++fam)
            for (int q = 0; q < 4; ++q) p.fm.n[fam][q] = B.fn[fam][q];
        p.mode = c.mode;
        p.in = c.in;
        p.un = c.un;
        p.out = c.out;
        p.Rout = c.Rout;
        p.src = c.src;
        p.alpha = c.alpha;
        p.beta = c.beta;
        p.gdt = c.gdt;
        p.dt_slot = c.dt_slot;
        p.dt_scale = c.dt_scale;
        p.partials = c.partials ? g->partials + B.part_off * 3 * NV : nullptr;
        CUDA_TRY(launch_stencil_f64(p, g->scheme.limiter, B.two_d, s));
    } else {
        StencilParams<float> p;
        memset(&p, 0, sizeof p);
        fill_common(p, g, B);
        for (int fam = 0; fam < 3; ++fam)
            for (int q = 0; q < 4; ++q) p.fm.n[fam][q] = B.fn32[fam][q];
        p.mode = c.mode;
        p.in = c.in;
        p.un = c.un;
        p.out = c.out;
        p.dprev = c.dprev;
        p.dout = c.dout;
        p.xout = c.xout;
        p.Rout = c.Rout;
        p.src = c.src;
        p.alpha = c.alpha;
        p.beta = c.beta;
        p.gdt = c.gdt;
        p.dt_slot = c.dt_slot;
        p.dt_scale = c.dt_scale;
        p.partials = c.partials ? g->partials + B.part_off * 3 * NV : nullptr;
        if (c.in_f32)
            CUDA_TRY(launch_stencil_f32s(p, g->scheme.limiter, B.two_d, s));
        else
            CUDA_TRY(launch_stencil_f32(p, g->scheme.limiter, B.two_d, s));
    }
    return SENSEI_OK;
}

}  // namespace

extern "C" {

const char *sensei_last_error(void) { return g_msg; }

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
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return fail(SENSEI_ERR_CUDA, "cudaGetDevice failed");
    }
    g->scheme = *scheme;
    g->plan = P;
    g->ws = (char *)workspace;
    g->partials = (double *)(g->ws + P.off_partials);
    g->dt_bits = (unsigned long long *)(g->ws + P.off_dtbits);
    g->dt_slot = (double *)(g->ws + P.off_dtslot);
    g->norms = (double *)(g->ws + P.off_norms);
    g->err = (unsigned *)(g->norms + 15);
    for (int b = 0; b < nblocks; ++b) {
        Block &B = g->plan.blocks[b];
        const size_t mv = (size_t)B.ml.mvolume;
        double *fn = (double *)(g->ws + P.off_fn[b]);
        float *fn32 = P.off_fn32[b] ? (float *)(g->ws + P.off_fn32[b]) : nullptr;
        double *sb = (double *)(g->ws + P.off_sbar[b]);
        for (int fam = 0; fam < 3; ++fam)
            for (int q = 0; q < 4; ++q) {
                B.fn[fam][q] = fn + (fam * 4 + q) * mv;
                B.fn32[fam][q] = fn32 ? fn32 + (fam * 4 + q) * mv : nullptr;
                B.sbar[fam][q] = sb + (fam * 4 + q) * mv;
            }
        B.vol = (double *)(g->ws + P.off_vol[b]);
        B.ivol = (double *)(g->ws + P.off_ivol[b]);
        B.ivol32 = P.off_ivol32[b] ? (float *)(g->ws + P.off_ivol32[b]) : nullptr;
        B.stage[0] = (double *)(g->ws + P.off_stage[b]);
        B.stage[1] = B.stage[0] + B.L.elems;
        // FP32 storage reuses the same bytes: X0, X1, D0, D1
        B.xs[0] = (float *)B.stage[0];
        B.xs[1] = B.xs[0] + B.L.elems;
        B.ds[0] = B.xs[1] + B.L.elems;
        B.ds[1] = B.ds[0] + B.L.elems;
        for (int f = 0; f < 6; ++f) {
            B.bc_set[f] = false;
            B.nbr[f] = -1;
            B.nbr_face[f] = -1;
        }
        MetricsOut mo;
        memset(&mo, 0, sizeof mo);
        for (int fam = 0; fam < 3; ++fam)
            for (int q = 0; q < 4; ++q) {
                mo.n[fam][q] = B.fn[fam][q];
                mo.n32[fam][q] = B.fn32[fam][q];
                mo.sbar[fam][q] = B.sbar[fam][q];
            }
        mo.vol = B.vol;
        mo.ivol = B.ivol;
        mo.ivol32 = B.ivol32;
        cudaError_t e = launch_metrics(B.ni, B.nj, B.nk, nodes[b], mo, B.ml, s);
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
    const Block &B = grid->plan.blocks[block];
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
    Block &B = grid->plan.blocks[block];
    if (face < 0 || face >= (B.two_d ? 4 : 6))
        return fail(SENSEI_ERR_INVALID_ARG, "face %d out of range for a %s block", face, B.two_d ? "2D" : "3D");
    if (type < SENSEI_BC_PERIODIC || type > SENSEI_BC_INTERFACE)
        return fail(SENSEI_ERR_INVALID_ARG, "unknown boundary type %d", type);
    if (type == SENSEI_BC_INFLOW) {
        if (!prim) return fail(SENSEI_ERR_INVALID_ARG, "inflow needs the primitive state");
        if (!(prim[0] > 0.0) || !(prim[4] > 0.0))
            return fail(SENSEI_ERR_INVALID_ARG, "inflow state needs rho > 0 and p > 0");
        memcpy(B.bc_prim[face], prim, sizeof B.bc_prim[face]);
    }
    if (type == SENSEI_BC_INTERFACE) {
        if (orientation != 0) return fail(SENSEI_ERR_UNSUPPORTED, "only aligned interfaces (orientation 0)");
        if (nbr_block < 0 || nbr_block >= nb) return fail(SENSEI_ERR_INVALID_ARG, "neighbour block out of range");
        const Block &N = grid->plan.blocks[nbr_block];
        if (nbr_face < 0 || nbr_face >= (N.two_d ? 4 : 6) || (nbr_face >> 1) != (face >> 1) || nbr_face == face)
            return fail(SENSEI_ERR_INVALID_ARG, "neighbour face must be the opposite side of the same direction");
        if (N.two_d != B.two_d) return fail(SENSEI_ERR_INVALID_ARG, "cannot connect a 2D block to a 3D block");
        int a1 = face < 2 ? B.nj : B.ni, a2 = face < 4 ? B.nk : B.nj;
        int b1 = nbr_face < 2 ? N.nj : N.ni, b2 = nbr_face < 4 ? N.nk : N.nj;
        if (a1 != b1 || a2 != b2)
            return fail(SENSEI_ERR_INVALID_ARG, "interface faces differ in size (%d x %d vs %d x %d)", a1, a2, b1, b2);
        const int axis = face >> 1;
        const int nb_n = axis == 0 ? N.ni : axis == 1 ? N.nj : N.nk;
        if (nb_n < NG) return fail(SENSEI_ERR_INVALID_ARG, "neighbour block too thin for two ghost layers");
        B.nbr[face] = nbr_block;
        B.nbr_face[face] = nbr_face;
    } else if (type == SENSEI_BC_PERIODIC || type == SENSEI_BC_SLIP_WALL) {
        // both rules read the two cells next to a boundary
        const int axis = face >> 1;
        const int n = axis == 0 ? B.ni : axis == 1 ? B.nj : B.nk;
        if (n < NG) return fail(SENSEI_ERR_INVALID_ARG, "block too thin for this boundary rule (needs %d cells)", NG);
    }
    B.bc_type[face] = type;
    B.bc_set[face] = true;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_fill_ghosts(sensei_grid *grid, double *const *U, sensei_stream stream)
{
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st == SENSEI_OK) st = check_bcs(grid);
    if (st != SENSEI_OK) return st;
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    st = fill_ghosts_impl(grid, U, (cudaStream_t)stream);
    if (st == SENSEI_OK) g_msg[0] = 0;
    return st;
}

sensei_status sensei_residual(sensei_grid *grid, double *const *U, double *const *R, const double *const *src,
                              sensei_stream stream)
{
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st == SENSEI_OK) st = check_states(grid, R, "R");
    if (st == SENSEI_OK) st = check_bcs(grid);
    if (st != SENSEI_OK) return st;
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    st = fill_ghosts_impl(grid, U, s);
    if (st != SENSEI_OK) return st;
    const auto &blocks = grid->plan.blocks;
    for (size_t b = 0; b < blocks.size(); ++b) {
        StencilCall c;
        memset(&c, 0, sizeof c);
        c.mode = MODE_RESIDUAL;
        c.in = U[b];
        c.Rout = R[b];
        c.src = src ? src[b] : nullptr;
        c.partials = true;
        st = stencil(grid, blocks[b], c, s);
        if (st != SENSEI_OK) return st;
    }
    CUDA_TRY(launch_norms_finalize(grid->partials, (int)grid->plan.nparts, grid->plan.ncells, grid->norms, s));
    grid->kernel_launches++;
    g_msg[0] = 0;
    return SENSEI_OK;
}

sensei_status sensei_rk_step(sensei_grid *grid, double *const *U, int rk, double cfl, double dt, double *dt_used,
                             sensei_stream stream)
{
    sensei_status st = check_grid(grid);
    if (st == SENSEI_OK) st = check_states(grid, U, "U");
    if (st == SENSEI_OK) st = check_bcs(grid);
    if (st != SENSEI_OK) return st;
    if (rk < SENSEI_RK2_SSP || rk > SENSEI_RK4_SSP2) return fail(SENSEI_ERR_INVALID_ARG, "unknown RK scheme %d", rk);
    if (!(cfl > 0.0) && !(dt > 0.0 && dt < INFINITY))
        return fail(SENSEI_ERR_INVALID_ARG, "need cfl > 0 or a finite dt > 0");
    Device dev;
    CUDA_TRY(dev.set(grid->device));
    cudaStream_t s = (cudaStream_t)stream;
    const auto &blocks = grid->plan.blocks;
    const int nb = (int)blocks.size();

    st = fill_ghosts_impl(grid, U, s);
    if (st != SENSEI_OK) return st;
    const double *dt_src;
    double dt_scale;
    if (cfl > 0.0) {
        CUDA_TRY(cudaMemsetAsync(grid->dt_bits, 0x7F, sizeof(unsigned long long), s));
        for (int b = 0; b < nb; ++b) {
            const Block &B = blocks[b];
            CUDA_TRY(launch_dt(B.ni, B.nj, B.nk, B.L, U[b], cell_metrics(B), B.ml, grid->scheme.gamma, grid->dt_bits,
                               grid->err, s));
            grid->kernel_launches++;
        }
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
    const bool incr = grid->scheme.precision == SENSEI_FP32_STORE;
    std::vector<double *> in(nb), outp(nb);
    std::vector<float *> xin(nb);
    for (int stage = 0; stage < S; ++stage) {
        const double *co = RK_COEF[rk][stage];
        const bool last = stage == S - 1;
        if (!incr) {
            // FP64 stage states: U -> st0 -> st1 -> ... -> U
            for (int b = 0; b < nb; ++b) {
                in[b] = stage == 0 ? U[b] : blocks[b].stage[(stage - 1) % 2];
                outp[b] = last ? U[b] : blocks[b].stage[stage % 2];
            }
            if (stage > 0) {
                st = fill_ghosts_impl(grid, in.data(), s);
                if (st != SENSEI_OK) return st;
            }
            for (int b = 0; b < nb; ++b) {
                StencilCall c;
                memset(&c, 0, sizeof c);
                c.mode = MODE_ACCUM;
                c.in = in[b];
                c.un = co[0] != 0.0 ? U[b] : nullptr;
                c.out = outp[b];
                c.alpha = co[0];
                c.beta = co[1];
                c.gdt = co[2];
                c.dt_slot = dt_src;
                c.dt_scale = dt_scale;
                c.partials = stage == 0;
                st = stencil(grid, blocks[b], c, s);
                if (st != SENSEI_OK) return st;
            }
        } else {
            // FP32 storage: the first stage reads the FP64 master U, later
            // stages the FP32 stage state X^(s-1); every stage but the last
            // writes the FP32 increment D^(s) and X^(s); the last adds its
            // increment to U in FP64.
            if (stage > 0) {
                for (int b = 0; b < nb; ++b) xin[b] = blocks[b].xs[(stage - 1) % 2];
                st = fill_ghosts_impl(grid, xin.data(), s);
                if (st != SENSEI_OK) return st;
            }
            for (int b = 0; b < nb; ++b) {
                const Block &B = blocks[b];
                StencilCall c;
                memset(&c, 0, sizeof c);
                c.mode = MODE_INCR;
                c.in = stage == 0 ? (const void *)U[b] : (const void *)B.xs[(stage - 1) % 2];
                c.in_f32 = stage > 0;
                c.un = U[b];
                c.dprev = stage == 0 ? nullptr : B.ds[(stage - 1) % 2];
                c.out = last ? U[b] : nullptr;
                c.dout = last ? nullptr : B.ds[stage % 2];
                c.xout = last ? nullptr : B.xs[stage % 2];
                c.alpha = co[0];
                c.beta = co[1];
                c.gdt = co[2];
                c.dt_slot = dt_src;
                c.dt_scale = dt_scale;
                c.partials = stage == 0;
                st = stencil(grid, B, c, s);
                if (st != SENSEI_OK) return st;
            }
        }
    }
    CUDA_TRY(launch_norms_finalize(grid->partials, (int)grid->plan.nparts, grid->plan.ncells, grid->norms, s));
    grid->kernel_launches++;
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
        return fail(SENSEI_ERR_NONPHYSICAL, "a kernel met rho <= 0, p <= 0 or a non-finite state (error word 0x%x)",
                    errw);
    }
    g_msg[0] = 0;
    return SENSEI_OK;
}

}  // extern "C"
