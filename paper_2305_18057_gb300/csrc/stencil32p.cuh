// stencil32p.cuh -- the 3D fused residual / Runge-Kutta stage kernel with
// FP32 reconstruction and flux arithmetic (the mixed-precision forms), built
// around paired face fluxes.
//
// Same work items (block, TI x TJ column tile, k-chunk), the same MUSCL /
// Roe / residual / stage arithmetic (Eq. flux, Eq. residual, Eq.
// runge_kutta) and the same launch modes as the FP64 kernel of stencil.cuh.
// Organisation, per k-plane of an item, one CTA barrier per plane:
//   * the stage input's (TI+4) x (TJ+4) tile of plane k+2 (state with its
//     two-cell halo, SoA, FP64 or FP32) and the FP32 face-metric record of
//     plane k have been staged into shared memory by bulk asynchronous
//     copies of the tensor memory accelerator (one cp.async.bulk.tensor of
//     the tile's 4D box -- all variables -- through the slot's tensor map,
//     one cp.async.bulk of the record; byte-counted completion on an
//     mbarrier), issued two planes ahead;
//   * every thread converts two cells of that tile to reconstruction
//     variables at once (its own column's cell and one halo cell) into a
//     three-plane ring of FP32 tiles; the tile of plane k was converted two
//     planes earlier;
//   * every thread then forms two pairs of face fluxes, each pair by one
//     copy of the MUSCL + Roe code in packed f32x2 arithmetic (pair32.cuh):
//     (the i-face left of its cell, the j-face below it) and (the k-face
//     above it, one of the tile's 40 right/top edge faces -- five lanes per
//     warp -- or a discarded duplicate).  Every warp does the same work;
//   * after the barrier: the residual of the own cell from its six faces
//     (the right i-face by a shuffle from the next lane, the top j-face from
//     shared memory, the lower k-face carried from the previous plane), the
//     stage update, the ghost push and the norm partials.
// The own column's planes k-1, k and k+1 are read from the tile ring (plane
// k-1 sits where plane k+2 goes; the thread writes its own cell of plane k+2
// there only after its k-face), so no k-window is held in registers.
// Every wait on an mbarrier is bounded (by default 2^31 clock cycles); on
// expiry the CTA sets ERR_TIMEOUT, waits (bounded) for the copies it has in
// flight and leaves.
#pragma once

#include "dtbound.cuh"
#include "pair32.cuh"
#include "stencil32.cuh"

namespace sensei {

constexpr int RING = 3;   // FP32 reconstruction-variable tiles: planes k, k+1, k+2

template <typename TS>
struct SmemP {
    // raw[2][NV][TH][TW] TS | met[2][REC] | W[RING][NV][TH][TW] | Fj[2][NV][TJ+1][TI]
    // (row TJ: the tile's top j-faces) | FiE[2][NV][TJ] (the tile's right
    // i-faces) | reduction scratch (FP64 input only) | two mbarriers
    // each raw tile on a 128-byte boundary (bulk tensor copy destination)
    static constexpr size_t raw_buf = ((size_t)NV * TPLANE * sizeof(TS) + 127) / 128 * 128;
    static constexpr size_t off_raw = 0;
    static constexpr size_t off_met = off_raw + 2 * raw_buf;
    static constexpr size_t off_w = off_met + 2 * (size_t)REC * sizeof(float);
    static constexpr size_t off_fj = off_w + (size_t)RING * NV * TPLANE * sizeof(float);
    static constexpr size_t fj_buf = (size_t)NV * (TJ + 1) * TI;
    static constexpr size_t off_fie = off_fj + 2 * fj_buf * sizeof(float);
    static constexpr size_t off_red = (off_fie + 2 * (size_t)NV * TJ * sizeof(float) + 15) / 16 * 16;
    static constexpr size_t red_bytes = sizeof(TS) == 8 ? 3 * NV * (NTHREADS / 32) * sizeof(double) : 0;
    static constexpr size_t off_bar = off_red + red_bytes;
    static constexpr size_t bytes = off_bar + 2 * sizeof(unsigned long long);
    static_assert(raw_buf % 16 == 0 && off_met % 16 == 0, "bulk-copy destinations are 16-byte aligned");
};

// Issue (thread 0) one copy group into a slot: the raw tile of plane `c`
// -- the tile's (TW x TH) cells with their halo, all NV variables, as one
// bulk tensor copy through the slot's tensor map (rows and columns beyond
// the array arrive as 0) -- and, if rec != null, one face-metric record.
// Called after the barrier that frees the slot.
template <typename TS>
__device__ __forceinline__ void issue_group(const unsigned char *tmap, int i0, int j0, int zc, const float *rec,
                                            TS *raw, float *met, uint32_t bar, unsigned tx_extra)
{
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, (uint32_t)(NV * TPLANE * (int)sizeof(TS) + (rec ? REC * (int)sizeof(float) : 0)) +
                                   tx_extra);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_addr(raw)),
        "l"(tmap), "r"(i0), "r"(j0), "r"(zc), "r"(0), "r"(bar)
        : "memory");
    if (rec) bulk_copy_g2s(smem_addr(met), rec, (uint32_t)(REC * sizeof(float)), bar);
}

// L2 prefetch of the rows of one of the update's per-cell operand arrays
// for a plane: `rows` (<= TJ) rows of `rowb` (<= 3 x 128) bytes from
// 16-byte aligned starts, `stride` bytes apart, `nv` variables `vstride`
// bytes apart; the CTA's threads take the rows' lines (start, +128, +256
// and the last byte of the row) in turn.
static_assert((TJ & (TJ - 1)) == 0, "the prefetch slots index rows with a mask");
__device__ __forceinline__ void prefetch_lines(const void *base, long long stride, int rows, long long vstride, int nv,
                                              int rowb, int t)
{
    for (int n = t; n < nv * TJ * 4; n += NTHREADS) {
        const int v = n / (TJ * 4), r = (n >> 2) & (TJ - 1), part = n & 3;
        const int off = part == 3 ? rowb - 1 : 128 * part;
        if (r < rows && off < rowb) {
            const char *a = reinterpret_cast<const char *>(base) + v * vstride + r * stride + off;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
        }
    }
}

// the halo cell (tile row r, column c) a thread t < NHALO converts
__device__ __forceinline__ int halo_cell(int t)
{
    int r, c;
    if (t < 2 * TW) {
        r = t / TW;
        c = t - r * TW;
    } else if (t < 4 * TW) {
        r = TJ + 2 + (t - 2 * TW) / TW;
        c = (t - 2 * TW) % TW;
    } else {
        const int g = t - 4 * TW;
        r = 2 + (g >> 2);
        c = (g & 3) < 2 ? (g & 3) : TI + (g & 3);
    }
    return r * TW + c;
}

// PART: the launch accumulates the norm partials (the first stage of a
// step, or a residual); a separate instantiation, so that the other stages
// do not hold the accumulators' registers.  MODE: the launch's update
// (MODE_ACCUM, MODE_INCR or MODE_RESIDUAL, the BatchParams field it
// replaces), and LOCAL: local time steps (the BatchParams flag), both
// fixed at compile time so that each instantiation carries only its own
// update code and operands.  DTN (the last FP32-storage stage of a step
// with a global CFL step): every cell's next-step time-step bound from the
// FP64 state just written (the rule of the FP32 time-step kernel, the same
// function), reduced into p.dt_next, so that the next step needs no
// time-step kernel.
template <typename TS, int LIM, bool PART, int MODE, bool LOCAL, bool DTN>
__global__ void __launch_bounds__(NTHREADS, 2) stencil32p_kernel(const __grid_constant__ BatchParams<float> p)
{
    using SM = SmemP<TS>;
    constexpr bool WIDE = sizeof(TS) == 8;   // FP64 stage input: the only case that computes norms
    constexpr bool NORMS = WIDE && PART;
    extern __shared__ __align__(128) unsigned char smem[];
    TS *sRaw = reinterpret_cast<TS *>(smem + SM::off_raw);
    auto rawbuf = [&](int n) { return reinterpret_cast<TS *>(smem + SM::off_raw + n * SM::raw_buf); };
    float *sMet = reinterpret_cast<float *>(smem + SM::off_met);
    float *sW = reinterpret_cast<float *>(smem + SM::off_w);
    float *sFj = reinterpret_cast<float *>(smem + SM::off_fj);
    float *sFiE = reinterpret_cast<float *>(smem + SM::off_fie);
    double *sRed = reinterpret_cast<double *>(smem + SM::off_red);
    const uint32_t bar0 = smem_addr(smem + SM::off_bar);
    __shared__ BlockDev sB;
    __shared__ PushFace sPush[6];   // the item's ghost push, face by face

    constexpr int FJV = (TJ + 1) * TI;   // sFj variable plane

    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int ti = lane, tj = warp;
    const int e_own = (tj + 2) * TW + ti + 2;   // own cell in a tile
    const int e_halo = t < NHALO ? halo_cell(t) : e_own;

    // the MUSCL scale: eps / 2, or eps for van Leer (which folds the 2 of its slope in)
    const P2 gm1 = sp2(p.gm1), kg = sp2(p.kg), c1 = sp2(p.c1), c2 = sp2(p.c2),
             he = sp2(LIM == SENSEI_LIM_VANLEER ? 2.0f * p.half_eps : p.half_eps);
    const P2 fix = sp2(p.fix), ifix = sp2(p.ifix);
    const int cons = p.cons;
    const bool update = MODE != MODE_RESIDUAL;
    const double dt = update ? p.dt_scale * *p.dt_slot : 0.0;
    const float gdt_dt32 = (float)(p.gdt * dt);
    const float gdt32 = (float)p.gdt;
    const float beta32 = (float)p.beta;
    // the next step's bound (DTN): this thread's minimum over its cells
    const float dgam = (float)p.gamma_d, dgm1 = (float)(p.gamma_d - 1.0);
    float dtn_best = INFINITY;
    bool dtn_bad = false;

    // the edge face of pair 2: lanes 0..4 of warp w own edge e = 5 w + lane
    // (e < TI: the top j-face of column e; else the right i-face of row
    // e - TI); the other lanes form a copy of some edge face and discard it,
    // so that every lane runs the same loads
    const int edge = (5 * warp + lane) % (TI + TJ);
    const bool edge_own = lane < 5;

    if (t == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t phase = 0;     // bit n: parity of slot n's next phase
    bool failed = false;

    for (long long pos = blockIdx.x; pos < p.nitems && !failed; pos += gridDim.x) {
        const long long item = p.order ? p.order[pos] : pos;
        const int b = find_block_item(p.blocks, p.nblocks, item);
        __syncthreads();   // the previous item is done with sB and every buffer
        {
            const int *src = reinterpret_cast<const int *>(&p.blocks[b]);
            int *dst = reinterpret_cast<int *>(&sB);
            for (int w = t; w < (int)(sizeof(BlockDev) / sizeof(int)); w += NTHREADS) dst[w] = src[w];
            if (t < 6 && p.push) push_face_setup(p, p.blocks[b], b, t, sPush[t]);
        }
        __syncthreads();
        const BlockDev &B = sB;
        long long local = item - B.item0;
        const int tile_i = (int)(local % B.tiles_i);
        local /= B.tiles_i;
        const int tile_j = (int)(local % B.tiles_j);
        const int chunk = (int)(local / B.tiles_j);
        const int i0 = tile_i * TI, j0 = tile_j * TJ;
        const int k0 = chunk * B.kchunk;
        const int k1 = min(k0 + B.kchunk, B.nk);
        const int ci = i0 + ti, cj = j0 + tj;
        const bool col_valid = ci < B.ni && cj < B.nj;
        const StateLayout L = B.L;
        const TS *in = (p.in_slot == SLOT_X0 || p.in_slot == SLOT_X1)
                           ? reinterpret_cast<const TS *>(slot32(B, p.in_slot))
                           : reinterpret_cast<const TS *>(slot64(B, p.user[b], p.in_slot));
        const bool out_wide = MODE != MODE_RESIDUAL && p.out_slot < SLOT_X0;
        const int len = min(TW, (int)L.sj - i0);
        const long long rec_stride = (long long)B.tiles_i * B.tiles_j * REC;
        const float *rec0 = B.rec32 + ((long long)tile_j * B.tiles_i + tile_i) * REC;
        const bool need_un = (MODE == MODE_ACCUM && p.alpha != 0.0) || (MODE == MODE_INCR && (out_wide || !WIDE));
        // the update's per-cell operands, prefetched into L2 two planes ahead
        // (rows of the tile's interior: FP64 from cell i0, FP32 from i0 - 2,
        // so that every row start is 16-byte aligned)
        const int nrow_in = min(TJ, B.nj - j0);
        const int row64 = ((min(TI, B.ni - i0) + 1) & ~1) * 8;
        const MetricLayout ml = B.ml;

        // copy groups G(c) = {raw tile of plane c, record of plane c - 2},
        // c = k0 .. k1 + 1, slot (c - k0) & 1; G(k0), G(k0+1) now
        const unsigned char *tmap = B.tmaps + p.in_slot * TMAP_BYTES;
        if (t == 0) {
            issue_group<TS>(tmap, i0, j0, k0 + L.gk, nullptr, sRaw, sMet, bar0, p.tx_extra);
            issue_group<TS>(tmap, i0, j0, k0 + 1 + L.gk, nullptr, rawbuf(1), sMet + REC, bar0 + 8, p.tx_extra);
        }

        // norm partials (FP64 stage input only): the sum of squares of the
        // FP32 residual in FP32 along the thread's column (at most a k-chunk
        // of 128 terms: relative error below 128 x 2^-24 = 7.6e-6, under the
        // FP32 residual's own), FP64 across threads and items; FP32 max;
        // FP64 conservation sums
        float nsq[NV], nmax[NV];
        double ncons[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            nsq[v] = nmax[v] = 0.0f;
            ncons[v] = 0.0;
        }

        // planes k0 - 2 and k0 - 1 of the own column, straight from the
        // stage input: plane k0 - 1 into the ring slot of plane k0 + 2
        // (where the k-window reads plane k - 1), plane k0 - 2 in registers
        // for the warm-up k-face
        float Wm2[NV];
        {
            TS q[NV];
            float qf[NV], w1[NV];
            load_cell<TS>(in, L, B.ni, B.nj, B.nk, ci, cj, k0 - 2, q);
#pragma unroll
            for (int v = 0; v < NV; ++v) qf[v] = tile_f32<TS>(q[v]);
            to_recon(qf, p.gm1, cons, false, p.err, Wm2);
            load_cell<TS>(in, L, B.ni, B.nj, B.nk, ci, cj, k0 - 1, q);
#pragma unroll
            for (int v = 0; v < NV; ++v) qf[v] = tile_f32<TS>(q[v]);
            to_recon(qf, p.gm1, cons, false, p.err, w1);
            float *dst = sW + ((k0 + 2) % RING) * NV * TPLANE + e_own;
#pragma unroll
            for (int v = 0; v < NV; ++v) dst[v * TPLANE] = w1[v];
        }

        float Fkm[NV];   // flux of the own cell's lower k-face
        // per-thread element index of the own column's cell at plane 0
        const long long cell0 = L.off + (long long)cj * L.sj + ci;

        for (int k = k0 - 2; k < k1; ++k) {
            const int c = k + 2;                  // the plane converted now
            const int s = (c - k0) & 1;           // its copy slot
            const bool warm = k < k0;
            const float *met = sMet + s * REC;    // record of plane k (G(c))
            float *wring_c = sW + (c % RING) * NV * TPLANE;
            const float *wring_k = sW + ((k + RING) % RING) * NV * TPLANE;   // k >= k0 - 2 >= -2
            const float *wk1 = sW + ((k + 1 + RING) % RING) * NV * TPLANE + e_own;

            // ---- wait for G(c); convert the own cell and one halo cell
            // (a thread whose wait gives up carries on with whatever the
            // buffers hold; the CTA leaves at the barrier after the fluxes)
            const bool ok = mbar_wait(bar0 + 8 * s, (phase >> s) & 1u, p.wait_limit);
            phase ^= 1u << s;
            float Wn[NV];   // own cell of plane c
            {
                const TS *raw = rawbuf(s);
                P2 q[NV], w[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    q[v] = mk2(tile_f32<TS>(raw[v * TPLANE + e_own]), tile_f32<TS>(raw[v * TPLANE + e_halo]));
                bool okx;
                to_prim2(q, gm1, w, okx);
                if (ok && col_valid && c < B.nk && !okx) atomicOr(p.err, ERR_NONPHYSICAL);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const P2 o = cons ? q[v] : w[v];
                    Wn[v] = o.v.x;
                    if (t < NHALO) wring_c[v * TPLANE + e_halo] = o.v.y;
                }
            }

            // ---- fluxes
            float Fi[NV], Fkp[NV], ivol = 0.0f;
            if (k == k0 - 2) {
                // nothing to form: the own cell of plane k0 goes straight
                // into the ring (no k-face reads it before the barrier)
#pragma unroll
                for (int v = 0; v < NV; ++v) wring_c[v * TPLANE + e_own] = Wn[v];
            } else {
                const int fb = k & 1;
                float *Fj = sFj + fb * SM::fj_buf;
                float *FiE = sFiE + fb * NV * TJ;
                // k-window of the own column: planes k-1 (in the slot of
                // plane c until this thread overwrites it), k, k+1, and c
#pragma unroll 1
                for (int job = warm ? 1 : 0; job < 2; ++job) {
                    P2 Ls[NV], Rs[NV], m[4];
                    if (job == 0) {
                        // x: the i-face left of the own cell; y: the j-face below it
                        const float *ax = wring_k + (tj + 2) * TW + ti;
                        const float *ay = wring_k + tj * TW + ti + 2;
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            const float *x = ax + v * TPLANE, *y = ay + v * TPLANE;
                            line_states2<LIM>(mk2(x[0], y[0]), mk2(x[1], y[TW]), mk2(x[2], y[2 * TW]),
                                              mk2(x[3], y[3 * TW]), c1, c2, he, Ls[v], Rs[v]);
                        }
                        const float *mx = met + tj * (TI + 1) + ti;
                        const float *my = met + REC_I + tj * TI + ti;
#pragma unroll
                        for (int q = 0; q < 4; ++q) m[q] = mk2(mx[q * TJ * (TI + 1)], my[q * (TJ + 1) * TI]);
                        ivol = met[REC - REC_V + tj * TI + ti];
                    } else {
                        // x: the own cell's upper k-face (planes k-1 .. k+2 of
                        // the own column; at the warm-up plane k0 - 1 the
                        // lower face of plane k0, from planes k0-2 .. k0+1);
                        // y: an edge face of the tile, or a duplicate of x
                        const float *km1 = wring_c + e_own;
                        const float *k00 = wring_k + e_own;
                        const float *ybase = nullptr;
                        int yst = 0;
                        if (!warm) {
                            if (edge < TI) {
                                ybase = wring_k + TJ * TW + edge + 2;
                                yst = TW;
                            } else {
                                ybase = wring_k + (edge - TI + 2) * TW + TI;
                                yst = 1;
                            }
                        }
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            const float x0 = warm ? Wm2[v] : km1[v * TPLANE];
                            const float x1 = k00[v * TPLANE];
                            const float x2 = wk1[v * TPLANE];
                            const float x3 = Wn[v];
                            P2 w0, w1, w2, w3;
                            if (ybase) {
                                const float *y = ybase + v * TPLANE;
                                w0 = mk2(x0, y[0]);
                                w1 = mk2(x1, y[yst]);
                                w2 = mk2(x2, y[2 * yst]);
                                w3 = mk2(x3, y[3 * yst]);
                            } else {
                                w0 = sp2(x0);
                                w1 = sp2(x1);
                                w2 = sp2(x2);
                                w3 = sp2(x3);
                            }
                            line_states2<LIM>(w0, w1, w2, w3, c1, c2, he, Ls[v], Rs[v]);
                        }
                        // the own cell of plane c may now replace plane k-1
#pragma unroll
                        for (int v = 0; v < NV; ++v) wring_c[v * TPLANE + e_own] = Wn[v];
                        float mxk[4], myk[4];
                        const float *mk = met + REC_I + REC_J + tj * TI + ti;
                        if (warm) {
                            // face k0 - 1/2: the FP64 metrics (no record yet)
                            const long long fk = (long long)k0 * ml.mplane + (long long)min(cj, B.nj - 1) * ml.mpitch +
                                                 min(ci, B.ni - 1);
                            const double *f2 = B.fn + 8 * ml.mvolume;
#pragma unroll
                            for (int q = 0; q < 4; ++q) mxk[q] = to_f32(f2[q * ml.mvolume + fk]);
                        } else {
#pragma unroll
                            for (int q = 0; q < 4; ++q) mxk[q] = mk[q * TJ * TI];
                        }
                        if (ybase) {
                            const float *my = edge < TI ? met + REC_I + TJ * TI + edge
                                                        : met + (edge - TI) * (TI + 1) + TI;
                            const int mst = edge < TI ? (TJ + 1) * TI : TJ * (TI + 1);
#pragma unroll
                            for (int q = 0; q < 4; ++q) myk[q] = my[q * mst];
                        } else {
#pragma unroll
                            for (int q = 0; q < 4; ++q) myk[q] = mxk[q];
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) m[q] = mk2(mxk[q], myk[q]);
                    }
                    P2 F[NV];
                    face_flux2(Ls, Rs, m[0], m[1], m[2], m[3], gm1, kg, fix, ifix, cons, F);
                    const bool store_edge = job == 1 && !warm && edge_own;
                    if (job == 0) {
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            Fi[v] = F[v].v.x;
                            Fj[v * FJV + tj * TI + ti] = F[v].v.y;
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < NV; ++v) Fkp[v] = F[v].v.x;
                        if (store_edge) {
                            if (edge < TI) {
#pragma unroll
                                for (int v = 0; v < NV; ++v) Fj[v * FJV + TJ * TI + edge] = F[v].v.y;
                            } else {
#pragma unroll
                                for (int v = 0; v < NV; ++v) FiE[v * TJ + edge - TI] = F[v].v.y;
                            }
                        }
                    }
                }
            }
            // the update's per-cell operands of plane k, loaded before the
            // barrier so that their latency overlaps the wait
            double uin[NV], unv[NV];
            float dpv[NV];
            double ivd = 0.0, dtvd = 0.0, vold = 0.0;
            const long long cell = cell0 + (long long)k * L.sk;
            const long long mc = (long long)k * ml.mplane + (long long)cj * ml.mpitch + ci;
            if (!warm && col_valid) {
                const bool want_in = WIDE && (MODE == MODE_ACCUM || NORMS || (MODE == MODE_INCR && !out_wide));
                const double *ind = reinterpret_cast<const double *>(in);
                const float *dprev = p.dprev >= 0 ? B.ds[p.dprev] : nullptr;
                const double *un = p.user[b];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    uin[v] = want_in ? ind[cell + v * L.sv] : 0.0;
                    unv[v] = need_un ? un[cell + v * L.sv] : 0.0;
                    dpv[v] = dprev ? dprev[cell + v * L.sv] : 0.0f;
                }
                if (LOCAL) dtvd = B.dtv[mc];
                else if (MODE == MODE_ACCUM) ivd = B.ivol[mc];
                if (NORMS) vold = B.vol[mc];
            }
            if (__syncthreads_or(!ok)) {
                // the copies this CTA has in flight (this slot's, if it is
                // still pending, and the other slot's group) once more,
                // bounded, before the CTA and its shared memory go away
                if (t == 0) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    mbar_wait(bar0 + 8 * s, ((phase >> s) & 1u) ^ 1u, p.wait_limit);
                    if (c + 1 <= k1 + 1) mbar_wait(bar0 + 8 * (s ^ 1), (phase >> (s ^ 1)) & 1u, p.wait_limit);
                }
                failed = true;
                break;
            }

            // the group two planes on into this slot (its raw tile and record
            // have been read by every thread)
            if (t == 0 && c + 2 <= k1 + 1)
                issue_group<TS>(tmap, i0, j0, c + 2 + L.gk, c < k1 ? rec0 + (long long)c * rec_stride : nullptr,
                                rawbuf(s), sMet + s * REC, bar0 + 8 * s, p.tx_extra);
            // the operands of plane c's update into L2, one line per thread
            if (c < k1 && nrow_in > 0) {
                const long long row0 = L.off + (long long)c * L.sk + (long long)j0 * L.sj + i0;
                const long long m0 = (long long)c * ml.mplane + (long long)j0 * ml.mpitch + i0;
                if (need_un) prefetch_lines(p.user[b] + row0, L.sj * 8, nrow_in, L.sv * 8, NV, row64, t);
                if (p.dprev >= 0) prefetch_lines(B.ds[p.dprev] + row0 - 2, L.sj * 4, nrow_in, L.sv * 4, NV, len * 4, t);
                if (MODE == MODE_ACCUM && !LOCAL)
                    prefetch_lines(B.ivol + m0, ml.mpitch * 8, nrow_in, 0, 1, row64, t);
                if (NORMS) prefetch_lines(B.vol + m0, ml.mpitch * 8, nrow_in, 0, 1, row64, t);
                if (DTN) {
                    // the next-step bound's metrics: 12 FP32 spectral arrays and |Omega|
                    const int row32 = min(TI, B.ni - i0) * 4;
                    prefetch_lines(B.sbar32 + m0, ml.mpitch * 4, nrow_in, ml.mvolume * 4, 12, row32, t);
                    prefetch_lines(B.vol32 + m0, ml.mpitch * 4, nrow_in, 0, 1, row32, t);
                }
            }

            if (warm) {
                if (k == k0 - 1)
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fkm[v] = Fkp[v];
                continue;
            }

            // ---- residual, update, ghost push, norm partials of plane k
            const int fb = k & 1;
            const float *Fj = sFj + fb * SM::fj_buf;
            const float *FiE = sFiE + fb * NV * TJ;
            float Fr[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Fr[v] = __shfl_down_sync(0xffffffffu, Fi[v], 1);
                if (lane == TI - 1) Fr[v] = FiE[v * TJ + tj];
            }
            float rres[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                rres[v] = ((Fr[v] - Fi[v]) + (Fj[v * FJV + (tj + 1) * TI + ti] - Fj[v * FJV + tj * TI + ti])) +
                          (Fkp[v] - Fkm[v]);
                Fkm[v] = Fkp[v];
            }
            if (col_valid) {
                const long long nint = (long long)B.ni * B.nj * B.nk;
                const long long rc = ((long long)k * B.nj + cj) * B.ni + ci;
                const bool boundary =
                    ci < 2 || ci >= B.ni - 2 || cj < 2 || cj >= B.nj - 2 || k < 2 || k >= B.nk - 2;
                if (MODE == MODE_INCR) {
                    // FP32 increment D = beta Dprev - gdt dt/|Omega| R; X = float(U^n) + D,
                    // or on the last stage U^n + D in FP64
                    const float c32 = LOCAL ? gdt32 * to_f32(dtvd) : gdt_dt32 * ivol;
                    const bool has_prev = p.dprev >= 0;
                    if (out_wide) {
                        double *out64 = slot64(B, p.user[b], p.out_slot);
                        double q64[NV];
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            float delta = -c32 * rres[v];
                            if (has_prev) delta = fmaf(beta32, dpv[v], delta);
                            q64[v] = unv[v] + to_f64(delta);
                            out64[cell + v * L.sv] = q64[v];
                        }
                        if (DTN) {
                            float isum, bound;
                            if (dt_cell_f32(B, mc, 3, q64[0], q64[1], q64[2], q64[3], q64[4], dgam, dgm1, isum, bound))
                                dtn_best = fminf(dtn_best, bound);
                            else
                                dtn_bad = true;
                        }
                        if (p.push && boundary) push_affine<double, 6>(sPush, B, ci, cj, k, q64);
                    } else {
                        float *xout = slot32(B, p.out_slot);
                        float *dout = B.ds[p.dout];
                        float q32[NV];
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            float delta = -c32 * rres[v];
                            if (has_prev) delta = fmaf(beta32, dpv[v], delta);
                            // float(U^n) by the hardware conversion (round to
                            // nearest even, off the integer pipe), from the
                            // stage input on the first stage, from U^n later
                            const float xc = __double2float_rn(WIDE ? uin[v] : unv[v]);
                            dout[cell + v * L.sv] = delta;
                            q32[v] = xc + delta;
                            xout[cell + v * L.sv] = q32[v];
                        }
                        if (p.push && boundary) push_affine<float, 6>(sPush, B, ci, cj, k, q32);
                    }
                } else {
                    // FP64 stage state: U^(s) = alpha U^n + beta U^(s-1) + coef R
                    // in FP64 with the FP64 1/|Omega| (the conservation sums
                    // hold to FP64 round-off)
                    const double coef = MODE != MODE_ACCUM ? 0.0 : LOCAL ? -p.gdt * dtvd : -p.gdt * dt * ivd;
                    double q64[NV];
                    double *out64 = out_wide ? slot64(B, p.user[b], p.out_slot) : nullptr;
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        if (MODE == MODE_ACCUM) {
                            double val = p.beta * uin[v] + coef * to_f64(rres[v]);
                            if (p.alpha != 0.0) val += p.alpha * unv[v];
                            out64[cell + v * L.sv] = val;
                            q64[v] = val;
                        } else {
                            double r = to_f64(rres[v]);
                            if (p.src[b]) r -= p.src[b][v * nint + rc];
                            p.rout[b][v * nint + rc] = r;
                        }
                    }
                    if (p.push && boundary && MODE != MODE_RESIDUAL) push_affine<double, 6>(sPush, B, ci, cj, k, q64);
                }
                if (NORMS) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        // r exactly as hi + lo: the FP32 residual, or with a
                        // source term its FP64 value split in two floats
                        float hi = rres[v], lo = 0.0f;
                        if (MODE == MODE_RESIDUAL && p.src[b]) {
                            const double r = to_f64(rres[v]) - p.src[b][v * nint + rc];
                            hi = to_f32(r);
                            lo = to_f32(r - to_f64(hi));
                        }
                        nsq[v] = fmaf(hi, fmaf(2.0f, lo, hi), nsq[v]);
                        nmax[v] = fmaxf(nmax[v], fabsf(hi + lo));
                        ncons[v] = fma(vold, uin[v], ncons[v]);
                    }
                }
            }
        }
        if (failed) break;

        // ---- norm partials of this item, fixed-order reduction in FP64
        if (NORMS) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double a = (double)nsq[v], bm = (double)nmax[v], cc = ncons[v];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_down_sync(0xffffffffu, a, o);
                    bm = fmax(bm, __shfl_down_sync(0xffffffffu, bm, o));
                    cc += __shfl_down_sync(0xffffffffu, cc, o);
                }
                if (lane == 0) {
                    sRed[(0 * NV + v) * (NTHREADS / 32) + warp] = a;
                    sRed[(1 * NV + v) * (NTHREADS / 32) + warp] = bm;
                    sRed[(2 * NV + v) * (NTHREADS / 32) + warp] = cc;
                }
            }
            __syncthreads();
            if (t < 3 * NV) {
                const int kind = t / NV;
                double acc = 0.0;
                for (int w = 0; w < NTHREADS / 32; ++w) {
                    const double x = sRed[t * (NTHREADS / 32) + w];
                    acc = kind == 1 ? fmax(acc, x) : acc + x;
                }
                p.partials[item * 3 * NV + t] = acc;
            }
        }
    }

    // ---- the next step's time-step bound: one atomic minimum per warp on
    // the bit patterns of the positive doubles (they order like the values)
    if (DTN) {
        if (dtn_bad) atomicOr(p.err, ERR_NONPHYSICAL);
        double bd = (double)dtn_best;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bd = fmin(bd, __shfl_down_sync(0xffffffffu, bd, o));
        if (lane == 0 && bd < INFINITY) atomicMin(p.dt_next, (unsigned long long)__double_as_longlong(bd));
    }
}

// Launch of one update mode's instantiations (TS: the stage input's
// element type); each translation unit instantiates the modes it serves.
template <typename TS, int MODE>
struct Stencil32PLauncher {
    using Fn = void (*)(const BatchParams<float>);
    // the fused next-step bound exists for the last FP32-storage stage (an
    // FP32 stage state in, U^n + D written in FP64, a global step); in the
    // FP32-flux form's last stage (FP64 input) it cost what it saved
    // (measured), so that form keeps the time-step kernel
    static constexpr bool HAS_DTN = MODE == MODE_INCR && sizeof(TS) == 4;
    template <int LIM, bool PART>
    static Fn pick_local(bool local, bool dtn)
    {
        if constexpr (MODE == MODE_RESIDUAL) {
            return dtn ? nullptr : stencil32p_kernel<TS, LIM, PART, MODE, false, false>;   // no time step
        } else if constexpr (HAS_DTN && !PART) {
            if (dtn) return local ? nullptr : stencil32p_kernel<TS, LIM, PART, MODE, false, true>;
            return local ? stencil32p_kernel<TS, LIM, PART, MODE, true, false>
                         : stencil32p_kernel<TS, LIM, PART, MODE, false, false>;
        } else {
            if (dtn) return nullptr;
            return local ? stencil32p_kernel<TS, LIM, PART, MODE, true, false>
                         : stencil32p_kernel<TS, LIM, PART, MODE, false, false>;
        }
    }
    template <int LIM>
    static Fn pick_lim(bool part, bool local, bool dtn)
    {
        // an FP32 stage input exists only in the later FP32-storage stages
        // (no norm partials); norm partials only from an FP64 stage input
        if constexpr (sizeof(TS) == 4)
            return part ? nullptr : pick_local<LIM, false>(local, dtn);
        else
            return part ? pick_local<LIM, true>(local, dtn) : pick_local<LIM, false>(local, dtn);
    }
    static Fn pick(int limiter, bool part, bool local, bool dtn = false)
    {
        switch (limiter) {
        case SENSEI_LIM_NONE: return pick_lim<SENSEI_LIM_NONE>(part, local, dtn);
        case SENSEI_LIM_MINMOD: return pick_lim<SENSEI_LIM_MINMOD>(part, local, dtn);
        default: return pick_lim<SENSEI_LIM_VANLEER>(part, local, dtn);
        }
    }
    static cudaError_t prepare(Fn fn)
    {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SmemP<TS>::bytes);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    static cudaError_t launch(const BatchParams<float> &p, int limiter, int grid, cudaStream_t s)
    {
        if (p.mode != MODE) return cudaErrorInvalidValue;
        Fn fn = pick(limiter, p.partials != nullptr, p.local != 0, p.dt_next != nullptr);
        if (!fn) return cudaErrorInvalidValue;
        cudaError_t e = prepare(fn);
        if (e != cudaSuccess) return e;
        fn<<<grid, NTHREADS, SmemP<TS>::bytes, s>>>(p);
        return cudaGetLastError();
    }
    // the smallest resident CTAs per SM over this mode's instantiations
    // (0 on error, 1 << 30 if it has none)
    static int ctas_per_sm(int limiter)
    {
        int best = 1 << 30;
        for (int part = 0; part < 2; ++part)
            for (int local = 0; local < 3; ++local) {
                // local: 0, 1 (local steps), 2 (the fused next-step bound)
                Fn fn = pick(limiter, part != 0, local == 1, local == 2);
                if (!fn) continue;
                if (prepare(fn) != cudaSuccess) return 0;
                int n = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NTHREADS, SmemP<TS>::bytes) != cudaSuccess)
                    return 0;
                best = n < best ? n : best;
            }
        return best;
    }
};

}  // namespace sensei
