// hetero.cu -- heterogeneous CPU + GPU co-execution of one block (Sec. 4:
// the cells of a time step split between the GPU and the host cores, the
// interface ghost layers exchanged through host memory every Runge-Kutta
// stage; Sec. 6, Eq. hete: the split that balances the two speeds).  The
// split is by k-planes (the paper's 1D slabs): the GPU part's cost then
// falls in proportion to its planes, where an i- or j-split would move in
// steps of a stencil tile.
//
// The GPU part is an ordinary grid of this library whose cut faces are
// SENSEI_BC_EXTERNAL; the host part is a host worker (host_worker.cpp).  A
// step: both time-step minima, combined on the host; then per stage the
// GPU stage is launched, the host threads advance their part while it runs,
// and the cut's two cell layers go device -> pinned host -> host worker and
// host worker -> pinned host -> device before the next stage.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "sensei_internal.cuh"

struct sensei_hetero {
    int ni, nj, nk, nk_host, nk_dev;
    bool periodic_k;
    sensei_grid *g = nullptr;
    sensei_host_block *h = nullptr;
    double *U_dev = nullptr;
    sensei_layout Ld{}, Lh{};
    int nx = 0;                     // exchanged faces: 1 (the cut) or 2 (and the periodic wrap)
    int gface[2] = {5, 4};          // GPU-part face of exchange n
    int hface[2] = {4, 5};          // the host-part face it borders
    size_t xcount = 0;              // doubles per exchanged face
    double *xdev[2] = {};           // device buffers
    double *pin_out[2] = {};        // GPU layers, pinned
    double *pin_in[2] = {};         // host layers, pinned
    double *pin_dt = nullptr;       // the GPU part's CFL minimum, pinned
    cudaStream_t s = nullptr;
    cudaEvent_t ev[4] = {};
    ~sensei_hetero()
    {
        if (g) sensei_destroy_grid(g);
        if (h) sensei_host_destroy(h);
        for (int n = 0; n < 2; ++n) {
            if (pin_out[n]) cudaFreeHost(pin_out[n]);
            if (pin_in[n]) cudaFreeHost(pin_in[n]);
        }
        if (pin_dt) cudaFreeHost(pin_dt);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

using sensei::fail_status;

constexpr int NV_ = 5;

struct WsPlan {
    size_t grid_bytes, off_state, state_bytes, off_x, x_bytes, total;
};

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

sensei_status ws_plan(const sensei_block_desc *block, const sensei_scheme *scheme, int nk_host, WsPlan &P)
{
    if (!block || !scheme) return fail_status(SENSEI_ERR_INVALID_ARG, "block or scheme is NULL");
    if (block->ni < 2 || block->nj < 2 || block->nk < 4) return fail_status(SENSEI_ERR_INVALID_ARG, "a 3D block is needed");
    if (nk_host < 2 || nk_host > block->nk - 2)
        return fail_status(SENSEI_ERR_INVALID_ARG, "nk_host must lie in [2, nk - 2] (got %d of %d)", nk_host,
                           block->nk);
    if (scheme->precision != SENSEI_FP64 || scheme->mu != 0.0)
        return fail_status(SENSEI_ERR_UNSUPPORTED, "co-execution runs the FP64 Euler form");
    sensei_block_desc d = *block;
    d.nk = block->nk - nk_host;
    size_t gb = 0;
    sensei_status st = sensei_workspace_size(&d, 1, scheme, &gb);
    if (st != SENSEI_OK) return st;
    // the GPU part's state: the library's layout (rows padded to 4 elements)
    const long long pitch = ((long long)d.ni + 4 + 3) / 4 * 4;
    const long long sk = pitch * (d.nj + 4);
    const long long sv = (sk * (d.nk + 4) + 31) / 32 * 32;
    P.grid_bytes = round256(gb);
    P.off_state = P.grid_bytes;
    P.state_bytes = round256((size_t)(NV_ * sv) * sizeof(double));
    P.off_x = P.off_state + P.state_bytes;
    P.x_bytes = round256((size_t)NV_ * 2 * d.ni * d.nj * sizeof(double));
    P.total = P.off_x + 2 * P.x_bytes;
    return SENSEI_OK;
}

// the interior of a ghosted array (layout L) <-> planes [k0, k0 + nk_part)
// of a dense (5, nk, nj, ni) array
void copy_interior(double *ghosted, const sensei_layout &L, double *dense, int ni, int nj, int nk, int k0, int nk_part,
                   bool to_ghosted)
{
    for (int v = 0; v < NV_; ++v)
        for (int k = 0; k < nk_part; ++k)
            for (int j = 0; j < nj; ++j) {
                double *g = ghosted + L.offset + v * L.stride_var + k * L.stride_k + j * L.stride_j;
                double *dn = dense + (((long long)v * nk + k0 + k) * nj + j) * ni;
                if (to_ghosted)
                    memcpy(g, dn, sizeof(double) * ni);
                else
                    memcpy(dn, g, sizeof(double) * ni);
            }
}

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// both directions of the cut layers of the state stage `stage` reads
sensei_status exchange(sensei_hetero *x, int stage)
{
    const size_t bytes = x->xcount * sizeof(double);
    sensei_status st = SENSEI_OK;
    for (int n = 0; n < x->nx && st == SENSEI_OK; ++n) {
        st = sensei_face_exchange(x->g, &x->U_dev, 0, stage, x->gface[n], x->xdev[n], 0, x->s);
        if (st == SENSEI_OK &&
            cudaMemcpyAsync(x->pin_out[n], x->xdev[n], bytes, cudaMemcpyDeviceToHost, x->s) != cudaSuccess)
            st = fail_status(SENSEI_ERR_CUDA, "cut layers to the host");
    }
    if (st != SENSEI_OK) return st;
    for (int n = 0; n < x->nx && st == SENSEI_OK; ++n)
        st = sensei_host_face_exchange(x->h, stage, x->hface[n], x->pin_in[n], 0);
    if (st != SENSEI_OK) return st;
    if (cudaStreamSynchronize(x->s) != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "waiting for the GPU part");
    for (int n = 0; n < x->nx && st == SENSEI_OK; ++n) {
        st = sensei_host_face_exchange(x->h, stage, x->hface[n], x->pin_out[n], 1);
        if (st == SENSEI_OK &&
            cudaMemcpyAsync(x->xdev[n], x->pin_in[n], bytes, cudaMemcpyHostToDevice, x->s) != cudaSuccess)
            st = fail_status(SENSEI_ERR_CUDA, "cut layers to the device");
        if (st == SENSEI_OK) st = sensei_face_exchange(x->g, &x->U_dev, 0, stage, x->gface[n], x->xdev[n], 1, x->s);
    }
    return st;
}

}  // namespace

extern "C" {

sensei_status sensei_hetero_workspace_size(const sensei_block_desc *block, const sensei_scheme *scheme, int nk_host,
                                           size_t *bytes)
{
    if (!bytes) return fail_status(SENSEI_ERR_INVALID_ARG, "bytes is NULL");
    WsPlan P;
    sensei_status st = ws_plan(block, scheme, nk_host, P);
    if (st == SENSEI_OK) *bytes = P.total;
    return st;
}

sensei_status sensei_hetero_create(const sensei_block_desc *block, const double *nodes, const sensei_scheme *scheme,
                                   const int *bc_type, const double *bc_prim, int nk_host, int threads,
                                   void *workspace, size_t workspace_bytes, sensei_stream stream, sensei_hetero **out)
{
    if (!out) return fail_status(SENSEI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    WsPlan P;
    sensei_status st = ws_plan(block, scheme, nk_host, P);
    if (st != SENSEI_OK) return st;
    if (!nodes || !bc_type) return fail_status(SENSEI_ERR_INVALID_ARG, "nodes or bc_type is NULL");
    if (threads < 1) return fail_status(SENSEI_ERR_INVALID_ARG, "threads must be >= 1");
    if (!workspace || ((uintptr_t)workspace) % 256)
        return fail_status(SENSEI_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
    if (workspace_bytes < P.total)
        return fail_status(SENSEI_ERR_INVALID_ARG, "workspace too small: %zu bytes given, %zu needed", workspace_bytes,
                           P.total);
    for (int f = 0; f < 6; ++f) {
        if (bc_type[f] == SENSEI_BC_INTERFACE || bc_type[f] == SENSEI_BC_EXTERNAL || bc_type[f] < 0 ||
            bc_type[f] > SENSEI_BC_EXTERNAL)
            return fail_status(SENSEI_ERR_INVALID_ARG, "face %d: the block's own rules only (no interfaces)", f);
        if (bc_type[f] == SENSEI_BC_INFLOW && !bc_prim)
            return fail_status(SENSEI_ERR_INVALID_ARG, "face %d: inflow needs bc_prim", f);
    }
    if ((bc_type[4] == SENSEI_BC_PERIODIC) != (bc_type[5] == SENSEI_BC_PERIODIC))
        return fail_status(SENSEI_ERR_INVALID_ARG, "periodic k-faces come in pairs");
    sensei_hetero *x = new (std::nothrow) sensei_hetero();
    if (!x) return fail_status(SENSEI_ERR_INVALID_ARG, "out of host memory");
    x->ni = block->ni;
    x->nj = block->nj;
    x->nk = block->nk;
    x->nk_host = nk_host;
    x->nk_dev = block->nk - nk_host;
    x->periodic_k = bc_type[4] == SENSEI_BC_PERIODIC;
    x->nx = x->periodic_k ? 2 : 1;
    x->s = (cudaStream_t)stream;
    x->xcount = (size_t)NV_ * 2 * block->ni * block->nj;
    const int ni = x->ni, nj = x->nj, nd = x->nk_dev, nh = nk_host;
    // node arrays of the two parts: node planes [0, nd] and [nd, nk] of the block's
    const size_t nplane = (size_t)(nj + 1) * (ni + 1);
    const size_t nnode = nplane * (x->nk + 1);
    std::vector<double> Xd(3 * nplane * (nd + 1)), Xh(3 * nplane * (nh + 1));
    for (int c = 0; c < 3; ++c) {
        memcpy(&Xd[c * nplane * (nd + 1)], nodes + c * nnode, sizeof(double) * nplane * (nd + 1));
        memcpy(&Xh[c * nplane * (nh + 1)], nodes + c * nnode + nplane * nd, sizeof(double) * nplane * (nh + 1));
    }
    char *ws = (char *)workspace;
    sensei_block_desc dd{ni, nj, nd};
    // the GPU part's node array passes through its (later) state bytes,
    // which are large enough: 3 (ni+1)(nj+1)(nd+1) <= 5 (ni+4)(nj+4)(nd+4)
    double *Xd_dev = (double *)(ws + P.off_state);
    x->U_dev = Xd_dev;
    cudaError_t e = cudaMemcpyAsync(Xd_dev, Xd.data(), Xd.size() * sizeof(double), cudaMemcpyHostToDevice, x->s);
    if (e != cudaSuccess) {
        delete x;
        return fail_status(SENSEI_ERR_CUDA, "uploading the GPU part's nodes: %s", cudaGetErrorString(e));
    }
    const double *node_ptrs[1] = {Xd_dev};
    st = sensei_create_grid(&dd, 1, node_ptrs, scheme, ws, P.grid_bytes, stream, &x->g);
    if (st == SENSEI_OK && cudaStreamSynchronize(x->s) != cudaSuccess)
        st = fail_status(SENSEI_ERR_CUDA, "grid set-up of the GPU part");
    if (st == SENSEI_OK) st = sensei_host_create(ni, nj, nh, Xh.data(), scheme, threads, &x->h);
    if (st != SENSEI_OK) {
        delete x;
        return st;
    }
    for (int f = 0; f < 6 && st == SENSEI_OK; ++f) {
        const double *pr = bc_type[f] == SENSEI_BC_INFLOW ? bc_prim + 5 * f : nullptr;
        int tg = bc_type[f], th = bc_type[f];
        if (f == 5) tg = SENSEI_BC_EXTERNAL;                       // the cut
        if (f == 4) th = SENSEI_BC_EXTERNAL;
        if (f == 4 && x->periodic_k) tg = SENSEI_BC_EXTERNAL;      // the wrap
        if (f == 5 && x->periodic_k) th = SENSEI_BC_EXTERNAL;
        st = sensei_set_bc(x->g, 0, f, tg, tg == SENSEI_BC_INFLOW ? pr : nullptr, -1, -1, 0);
        if (st == SENSEI_OK) st = sensei_host_set_bc(x->h, f, th, th == SENSEI_BC_INFLOW ? pr : nullptr);
    }
    if (st == SENSEI_OK) st = sensei_state_layout(x->g, 0, &x->Ld);
    if (st == SENSEI_OK) st = sensei_host_layout(x->h, &x->Lh);
    for (int n = 0; n < 2 && st == SENSEI_OK; ++n) {
        x->xdev[n] = (double *)(ws + P.off_x + n * P.x_bytes);
        if (cudaHostAlloc((void **)&x->pin_out[n], x->xcount * sizeof(double), cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&x->pin_in[n], x->xcount * sizeof(double), cudaHostAllocDefault) != cudaSuccess)
            st = fail_status(SENSEI_ERR_CUDA, "pinned exchange buffers");
    }
    if (st == SENSEI_OK && cudaHostAlloc((void **)&x->pin_dt, sizeof(double), cudaHostAllocDefault) != cudaSuccess)
        st = fail_status(SENSEI_ERR_CUDA, "pinned time-step slot");
    for (int n = 0; n < 4 && st == SENSEI_OK; ++n)
        if (cudaEventCreate(&x->ev[n]) != cudaSuccess) st = fail_status(SENSEI_ERR_CUDA, "events");
    if (st != SENSEI_OK) {
        delete x;
        return st;
    }
    *out = x;
    return SENSEI_OK;
}

sensei_status sensei_hetero_destroy(sensei_hetero *x)
{
    delete x;
    return SENSEI_OK;
}

sensei_status sensei_hetero_upload(sensei_hetero *x, const double *U)
{
    if (!x || !U) return fail_status(SENSEI_ERR_INVALID_ARG, "NULL argument");
    std::vector<double> stage((size_t)x->Ld.elems, 0.0);
    double *dense = const_cast<double *>(U);
    copy_interior(stage.data(), x->Ld, dense, x->ni, x->nj, x->nk, 0, x->nk_dev, true);
    copy_interior(sensei_host_state(x->h), x->Lh, dense, x->ni, x->nj, x->nk, x->nk_dev, x->nk_host, true);
    if (cudaMemcpyAsync(x->U_dev, stage.data(), stage.size() * sizeof(double), cudaMemcpyHostToDevice, x->s) !=
            cudaSuccess ||
        cudaStreamSynchronize(x->s) != cudaSuccess)
        return fail_status(SENSEI_ERR_CUDA, "uploading the GPU part's state");
    sensei_status st = sensei_fill_ghosts(x->g, &x->U_dev, x->s);
    if (st == SENSEI_OK) st = sensei_host_fill_ghosts(x->h);
    if (st == SENSEI_OK) st = exchange(x, 0);
    if (st == SENSEI_OK && cudaStreamSynchronize(x->s) != cudaSuccess)
        st = fail_status(SENSEI_ERR_CUDA, "initial exchange");
    return st;
}

sensei_status sensei_hetero_download(sensei_hetero *x, double *U)
{
    if (!x || !U) return fail_status(SENSEI_ERR_INVALID_ARG, "NULL argument");
    std::vector<double> stage((size_t)x->Ld.elems);
    if (cudaMemcpyAsync(stage.data(), x->U_dev, stage.size() * sizeof(double), cudaMemcpyDeviceToHost, x->s) !=
            cudaSuccess ||
        cudaStreamSynchronize(x->s) != cudaSuccess)
        return fail_status(SENSEI_ERR_CUDA, "downloading the GPU part's state");
    copy_interior(stage.data(), x->Ld, U, x->ni, x->nj, x->nk, 0, x->nk_dev, false);
    copy_interior(sensei_host_state(x->h), x->Lh, U, x->ni, x->nj, x->nk, x->nk_dev, x->nk_host, false);
    return SENSEI_OK;
}

sensei_status sensei_hetero_step(sensei_hetero *x, int rk, double cfl, double dt, double *dt_used, double *times_ms)
{
    if (!x) return fail_status(SENSEI_ERR_INVALID_ARG, "NULL driver");
    if (rk < SENSEI_RK2_SSP || rk > SENSEI_RK4_SSP2) return fail_status(SENSEI_ERR_INVALID_ARG, "unknown RK scheme");
    const auto t0 = std::chrono::steady_clock::now();
    sensei_status st = SENSEI_OK;
    if (cfl > 0.0) {
        // the GPU part's minimum in flight while the host cores take theirs
        double dh = 0.0;
        st = sensei::dt_min_launch(x->g, &x->U_dev, x->pin_dt, x->s);
        if (st == SENSEI_OK) st = sensei_host_dt_min(x->h, cfl, &dh);
        if (st != SENSEI_OK) return st;
        if (cudaStreamSynchronize(x->s) != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "GPU time-step minimum");
        const double dg = cfl * *x->pin_dt;
        dt = std::min(dg, dh);
    }
    if (!(dt > 0.0)) return fail_status(SENSEI_ERR_INVALID_ARG, "need cfl > 0 or dt > 0");
    const int S = rk == SENSEI_RK2_SSP ? 2 : rk == SENSEI_RK3_SSP ? 3 : 4;
    double host_ms = 0.0, gpu_ms = 0.0, wait_ms = 0.0;
    const size_t bytes = x->xcount * sizeof(double);
    for (int stage = 0; stage < S && st == SENSEI_OK; ++stage) {
        const int next = stage == S - 1 ? 0 : stage + 1;   // the state the next stage reads
        if (cudaEventRecord(x->ev[0], x->s) != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "event");
        st = sensei_rk_stage(x->g, &x->U_dev, rk, stage, dt, x->s);
        if (st != SENSEI_OK) return st;
        if (cudaEventRecord(x->ev[1], x->s) != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "event");
        for (int n = 0; n < x->nx && st == SENSEI_OK; ++n) {
            st = sensei_face_exchange(x->g, &x->U_dev, 0, next, x->gface[n], x->xdev[n], 0, x->s);
            if (st == SENSEI_OK &&
                cudaMemcpyAsync(x->pin_out[n], x->xdev[n], bytes, cudaMemcpyDeviceToHost, x->s) != cudaSuccess)
                st = fail_status(SENSEI_ERR_CUDA, "cut layers to the host");
        }
        if (st != SENSEI_OK) return st;
        if (cudaEventRecord(x->ev[2], x->s) != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "event");
        // the host part of the stage while the GPU runs its part
        auto th = std::chrono::steady_clock::now();
        st = sensei_host_stage(x->h, rk, stage, dt);
        for (int n = 0; n < x->nx && st == SENSEI_OK; ++n)
            st = sensei_host_face_exchange(x->h, next, x->hface[n], x->pin_in[n], 0);
        host_ms += ms_since(th);
        if (st != SENSEI_OK) return st;
        auto tw = std::chrono::steady_clock::now();
        if (cudaEventSynchronize(x->ev[2]) != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "waiting for the GPU");
        wait_ms += ms_since(tw);
        float g = 0.0f;
        if (cudaEventElapsedTime(&g, x->ev[0], x->ev[1]) == cudaSuccess) gpu_ms += g;
        // the host's layers to the device first (asynchronous), then the
        // GPU's into the host ghosts while that copy runs
        for (int n = 0; n < x->nx && st == SENSEI_OK; ++n) {
            if (cudaMemcpyAsync(x->xdev[n], x->pin_in[n], bytes, cudaMemcpyHostToDevice, x->s) != cudaSuccess)
                st = fail_status(SENSEI_ERR_CUDA, "cut layers to the device");
            if (st == SENSEI_OK) st = sensei_face_exchange(x->g, &x->U_dev, 0, next, x->gface[n], x->xdev[n], 1, x->s);
        }
        for (int n = 0; n < x->nx && st == SENSEI_OK; ++n)
            st = sensei_host_face_exchange(x->h, next, x->hface[n], x->pin_out[n], 1);
    }
    if (st != SENSEI_OK) return st;
    if (cudaStreamSynchronize(x->s) != cudaSuccess) return fail_status(SENSEI_ERR_CUDA, "end of step");
    if (dt_used) *dt_used = dt;
    if (times_ms) {
        times_ms[0] = ms_since(t0);
        times_ms[1] = gpu_ms;
        times_ms[2] = host_ms;
        times_ms[3] = std::max(0.0, times_ms[0] - host_ms - wait_ms);
    }
    return SENSEI_OK;
}

}  // extern "C"
