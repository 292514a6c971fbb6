// stencil32.cuh -- the fused residual / Runge-Kutta stage kernel with FP32
// reconstruction and flux arithmetic (the mixed-precision forms).
//
// Same work items (block, TI x TJ column tile, k-chunk), the same MUSCL /
// Roe / residual / stage arithmetic (Eq. flux, Eq. residual, Eq.
// runge_kutta) and the same launch modes as the FP64 kernel of
// stencil.cuh.  The FP32 forms move 2-4x fewer bytes per cell than FP64
// arithmetic needs FP64 instructions, so this kernel is organised around
// its data movement instead:
//   * the (TI+4) x (TJ+4) state tile of each k-plane (the tile's cells with
//     their two-cell halo, SoA, FP64 or FP32) is staged into shared memory
//     by bulk asynchronous copies of the tensor memory accelerator
//     (cp.async.bulk global -> shared, one per tile row and variable,
//     completion counted in bytes on an mbarrier), one plane ahead of its
//     use, double buffered;
//   * with it, one bulk copy brings the plane's face-metric record (the
//     tile's i-, j- and upper k-face normals and areas and 1/|Omega|,
//     packed in FP32 at grid creation, 13.9 KB);
//   * the two MUSCL states of a face are formed from the four cells along
//     its direction and its Roe flux computed at once, once per face, so a
//     plane needs two CTA barriers: after the primitive tile, after the
//     fluxes;
//   * the own column's k-window (primitives of planes k..k+2, the plus
//     state of plane k, the flux of its lower k-face) stays in registers,
//     fed by a register prefetch of the raw state three planes ahead.
// Every wait on an mbarrier is bounded (by default 2^31 clock cycles);
// on expiry the CTA sets ERR_TIMEOUT, waits (bounded) for its copies in
// flight and leaves.
#pragma once

#include "stencil.cuh"

namespace sensei {

constexpr int TW = TI + 4;          // state-tile row: cells i0-2 .. i0+TI+1
constexpr int TH = TJ + 4;          // state-tile rows: j0-2 .. j0+TJ+1
constexpr int TPLANE = TW * TH;
constexpr int NHALO = TPLANE - TI * TJ;
static_assert(TI == 32, "one warp per tile row");

template <typename TS>
struct Smem32 {
    // raw[2][NV][TH][TW] TS | met[2][REC] | W[NV][TH][TW] | Fj[NV][TJ+1][TI] |
    // FiE[NV][TJ] (the tile's right i-faces) | K[3][NV][NTHREADS] (own column:
    // planes k+1 and k+2, the flux of the lower k-face) | reduction scratch
    // (FP64 input only) | two mbarriers
    static constexpr size_t raw_buf = (size_t)NV * TPLANE * sizeof(TS);
    static constexpr size_t off_raw = 0;
    static constexpr size_t off_met = off_raw + 2 * raw_buf;
    static constexpr size_t off_w = off_met + 2 * (size_t)REC * sizeof(float);
    static constexpr size_t off_fj = off_w + (size_t)NV * TPLANE * sizeof(float);
    static constexpr size_t off_fie = off_fj + (size_t)NV * (TJ + 1) * TI * sizeof(float);
    static constexpr size_t off_k = off_fie + (size_t)NV * TJ * sizeof(float);
    static constexpr size_t off_red = (off_k + 3 * (size_t)NV * NTHREADS * sizeof(float) + 15) / 16 * 16;
    static constexpr size_t red_bytes = sizeof(TS) == 8 ? 3 * NV * (NTHREADS / 32) * sizeof(double) : 0;
    static constexpr size_t off_bar = off_red + red_bytes;
    static constexpr size_t bytes = off_bar + 2 * sizeof(unsigned long long);
    static_assert(raw_buf % 16 == 0 && off_met % 16 == 0, "bulk-copy destinations are 16-byte aligned");
    static_assert((TW * sizeof(TS)) % 16 == 0, "tile rows are 16-byte aligned");
};

// ---- PTX wrappers: mbarrier and the bulk asynchronous copy ----------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// one arrival that also raises the phase's expected transaction bytes
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the phase of the given parity to complete; false after `limit`
// clock cycles (2^31 by default, about one second at 2 GHz)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// order this thread's earlier shared-memory accesses before later
// asynchronous-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// global -> shared bulk copy of `bytes` (multiple of 16; both addresses
// 16-byte aligned), completion counted on mbarrier `bar`
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Issue (warp 0) the copies of k-plane `k` of a tile: rows j0-2 .. j0-2+nrows-1
// of each variable, `len` cells from i0-2 (len a multiple of 4 and at most
// the padded row pitch minus i0, so no copy leaves the row's allocation),
// and the plane's face-metric record.
template <typename TS>
__device__ __forceinline__ void issue_plane(const TS *in, const StateLayout &L, int i0, int j0, int k, int nrows,
                                            int len, const float *rec, TS *raw, float *met, uint32_t bar, int lane,
                                            unsigned tx_extra)
{
    const uint32_t bytes = (uint32_t)(NV * nrows * len * (int)sizeof(TS) + REC * (int)sizeof(float)) + tx_extra;
    if (lane == 0) {
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, bytes);
    }
    __syncwarp();
    const TS *base = in + L.off + (long long)k * L.sk + (long long)(j0 - 2) * L.sj + (i0 - 2);
    for (int e = lane; e < NV * nrows; e += 32) {
        const int v = e / nrows, r = e - v * nrows;
        bulk_copy_g2s(smem_addr(raw + v * TPLANE + r * TW), base + v * L.sv + (long long)r * L.sj,
                      (uint32_t)(len * (int)sizeof(TS)), bar);
    }
    if (lane == 31) bulk_copy_g2s(smem_addr(met), rec, (uint32_t)(REC * sizeof(float)), bar);
}

// ---- FP32 helpers -----------------------------------------------------------

__device__ __forceinline__ void prefetch_l2(const void *ptr) { asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr)); }

// raw loads of one cell of the own column (no conversion: the value is
// consumed planes later, so the load latency stays hidden)
template <typename TS>
__device__ __forceinline__ void load_cell(const TS *in, const StateLayout &L, int ni, int nj, int nk, int i, int j,
                                          int k, TS q[NV])
{
    if (i >= -NG && i < ni + NG && j >= -NG && j < nj + NG && k >= -L.gk && k < nk + L.gk) {
        const TS *c = in + L.off + (long long)k * L.sk + (long long)j * L.sj + i;
#pragma unroll
        for (int v = 0; v < NV; ++v) q[v] = __ldg(c + v * L.sv);
    } else {
        q[0] = TS(1);
        q[1] = q[2] = q[3] = TS(0);
        q[4] = TS(2.5);
    }
}

// The Roe flux of the face between cells a and a+1 of a line of four
// primitive cells (a-1, a, a+1, a+2) in shared memory (variable planes
// TPLANE apart, neighbours `st` apart): left state the plus state of a,
// right state the minus state of a+1 (Eq. flux), metrics at met[q * mst].
template <int LIM>
__device__ __forceinline__ void line_flux(const float *w, int st, const float *met, int mst, float gm1, float kg,
                                          float fix, float ifix, float c1, float c2, float half_eps, int cons,
                                          float F[NV])
{
    float Lf[NV], Rf[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float *x = w + v * TPLANE;
        const float w0 = x[0], w1 = x[st], w2 = x[2 * st], w3 = x[3 * st];
        float unused;
        face_states<float, LIM>(w0, w1, w2, c1, c2, half_eps, Lf[v], unused);
        face_states<float, LIM>(w1, w2, w3, c1, c2, half_eps, unused, Rf[v]);
    }
    face_flux(Lf, Rf, met[0], met[mst], met[2 * mst], met[3 * mst], gm1, kg, fix, ifix, cons, F);
}

// s + (hi, lo) in double-single arithmetic (Knuth's two-sum, then a
// renormalising fast two-sum): the pair carries about 48 significant bits
__device__ __forceinline__ void ds_add(float &s_hi, float &s_lo, float hi, float lo)
{
    const float s = s_hi + hi;
    const float bv = s - s_hi;
    float e = (s_hi - (s - bv)) + (hi - bv);
    e += s_lo + lo;
    s_hi = s + e;
    s_lo = e - (s_hi - s);
}

template <typename TS, int LIM, bool TWO_D>
__global__ void __launch_bounds__(NTHREADS, sizeof(TS) == 4 ? 3 : 2) stencil32_kernel(const __grid_constant__ BatchParams<float> p)
{
    using SM = Smem32<TS>;
    constexpr bool WIDE = sizeof(TS) == 8;   // FP64 stage input: the only case that computes norms
    extern __shared__ __align__(128) unsigned char smem[];
    TS *sRaw = reinterpret_cast<TS *>(smem + SM::off_raw);
    float *sMet = reinterpret_cast<float *>(smem + SM::off_met);
    float *sW = reinterpret_cast<float *>(smem + SM::off_w);
    float *sFj = reinterpret_cast<float *>(smem + SM::off_fj);
    float *sFiE = reinterpret_cast<float *>(smem + SM::off_fie);
    float *sK = reinterpret_cast<float *>(smem + SM::off_k);
    double *sRed = reinterpret_cast<double *>(smem + SM::off_red);
    const uint32_t bar0 = smem_addr(smem + SM::off_bar);
    __shared__ BlockDev sB;
    __shared__ PushFace sPush[6];   // the item's ghost push, face by face

    constexpr int FJV = (TJ + 1) * TI;   // sFj variable plane
    constexpr int NFACES = TWO_D ? 4 : 6;

    const int t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int ti = lane, tj = warp;

    // scheme constants straight from the parameter bank (no registers held)
#define gm1 p.gm1
#define kg p.kg
#define c1 p.c1
#define c2 p.c2
#define half_eps p.half_eps
#define fix p.fix
#define ifix p.ifix
#define cons p.cons
    const bool update = p.mode != MODE_RESIDUAL;
    const double dt = update ? p.dt_scale * *p.dt_slot : 0.0;
    const float gdt_dt32 = (float)(p.gdt * dt);
    const float gdt32 = (float)p.gdt;
    const float beta32 = (float)p.beta;

    if (t == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t phase = 0;     // bit n: parity of buffer n's next phase
    bool failed = false;

    for (long long pos = blockIdx.x; pos < p.nitems && !failed; pos += gridDim.x) {
        const long long item = p.order ? p.order[pos] : pos;
        const int b = find_block_item(p.blocks, p.nblocks, item);
        __syncthreads();   // the previous item is done with sB and every tile buffer
        {
            const int *src = reinterpret_cast<const int *>(&p.blocks[b]);
            int *dst = reinterpret_cast<int *>(&sB);
            for (int w = t; w < (int)(sizeof(BlockDev) / sizeof(int)); w += NTHREADS) dst[w] = src[w];
            if (t < NFACES && p.push) push_face_setup(p, p.blocks[b], b, t, sPush[t]);
        }
        __syncthreads();
        const BlockDev &B = sB;
        long long local = item - B.item0;
        const int tile_i = (int)(local % B.tiles_i);
        local /= B.tiles_i;
        const int tile_j = (int)(local % B.tiles_j);
        const int chunk = (int)(local / B.tiles_j);
        const int i0 = tile_i * TI, j0 = tile_j * TJ;
        const int k0 = TWO_D ? 0 : chunk * B.kchunk;
        const int k1 = TWO_D ? 1 : min(k0 + B.kchunk, B.nk);
        const int ci = i0 + ti, cj = j0 + tj;
        const bool col_valid = ci < B.ni && cj < B.nj;
        const StateLayout L = B.L;
        const MetricLayout ml = B.ml;
        const TS *in = (p.in_slot == SLOT_X0 || p.in_slot == SLOT_X1)
                           ? reinterpret_cast<const TS *>(slot32(B, p.in_slot))
                           : reinterpret_cast<const TS *>(slot64(B, p.user[b], p.in_slot));
        // the update's pointers, formed from the descriptor in shared memory
        // where they are used (not held in registers through the fluxes)
        const bool out_wide = p.mode != MODE_RESIDUAL && p.out_slot < SLOT_X0;
        const int nrows = min(TH, B.nj + 4 - j0);
        const int len = min(TW, (int)L.sj - i0);
        const long long rec_stride = (long long)B.tiles_i * B.tiles_j * REC;
        const float *rec0 = B.rec32 + ((long long)tile_j * B.tiles_i + tile_i) * REC;

        // the first plane of the item into buffer 0 (every buffer is free:
        // each issued plane is waited for within its item)
        int cb = 0;
        if (warp == 0)
            issue_plane<TS>(in, L, i0, j0, k0, nrows, len, rec0 + k0 * rec_stride, sRaw, sMet, bar0, lane,
                            p.tx_extra);

        // FP64 norm partials: double-single sum of squares, FP32 max, FP64
        // conservation sums (FP64 stage input only)
        float nsq_hi[NV], nsq_lo[NV], nmax[NV];
        double ncons[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            nsq_hi[v] = nsq_lo[v] = nmax[v] = 0.0f;
            ncons[v] = 0.0;
        }

        // own-column k-window (3D)
        // sK[kb] holds plane k+1 of the own column, sK[kb ^ 1] plane k+2
        // (each thread touches only its own entries)
        int kb = 0;
        float *sFkm = sK + 2 * NV * NTHREADS;   // [NV][NTHREADS]: the own column's lower k-face flux
        float Wc[NV], Pp[NV];
        TS pre[NV];
        if (!TWO_D) {
            TS q[NV];
            float qf[NV], Wm2[NV], Wm1[NV];
            load_cell<TS>(in, L, B.ni, B.nj, B.nk, ci, cj, k0 - 2, q);
#pragma unroll
            for (int v = 0; v < NV; ++v) qf[v] = cvt<float, TS>(q[v]);
            to_recon(qf, gm1, cons, false, p.err, Wm2);
            load_cell<TS>(in, L, B.ni, B.nj, B.nk, ci, cj, k0 - 1, q);
#pragma unroll
            for (int v = 0; v < NV; ++v) qf[v] = cvt<float, TS>(q[v]);
            to_recon(qf, gm1, cons, false, p.err, Wm1);
            load_cell<TS>(in, L, B.ni, B.nj, B.nk, ci, cj, k0, q);
#pragma unroll
            for (int v = 0; v < NV; ++v) qf[v] = cvt<float, TS>(q[v]);
            to_recon(qf, gm1, cons, col_valid, p.err, Wc);
            load_cell<TS>(in, L, B.ni, B.nj, B.nk, ci, cj, k0 + 1, q);
#pragma unroll
            for (int v = 0; v < NV; ++v) qf[v] = cvt<float, TS>(q[v]);
            float W1[NV], W2[NV];
            to_recon(qf, gm1, cons, col_valid && k0 + 1 < B.nk, p.err, W1);
            load_cell<TS>(in, L, B.ni, B.nj, B.nk, ci, cj, k0 + 2, q);
#pragma unroll
            for (int v = 0; v < NV; ++v) qf[v] = cvt<float, TS>(q[v]);
            to_recon(qf, gm1, cons, col_valid && k0 + 2 < B.nk, p.err, W2);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                sK[(0 * NV + v) * NTHREADS + t] = W1[v];
                sK[(1 * NV + v) * NTHREADS + t] = W2[v];
            }
            float Lk[NV], Rk[NV], unused;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                face_states<float, LIM>(Wm2[v], Wm1[v], Wc[v], c1, c2, half_eps, Lk[v], unused);
                face_states<float, LIM>(Wm1[v], Wc[v], W1[v], c1, c2, half_eps, Pp[v], Rk[v]);
            }
            // the k0 - 1/2 face, from the FP64 metrics
            const long long fk = (long long)k0 * ml.mplane + (long long)min(cj, B.nj - 1) * ml.mpitch + min(ci, B.ni - 1);
            const double *f2 = B.fn + 8 * ml.mvolume;
            float Fkm[NV];
            face_flux(Lk, Rk, to_f32(f2[fk]), to_f32(f2[ml.mvolume + fk]), to_f32(f2[2 * ml.mvolume + fk]),
                      to_f32(f2[3 * ml.mvolume + fk]), gm1, kg, fix, ifix, cons, Fkm);
#pragma unroll
            for (int v = 0; v < NV; ++v) sFkm[v * NTHREADS + t] = Fkm[v];
        }

        for (int k = k0; k < k1; ++k) {
            if (!TWO_D) load_cell<TS>(in, L, B.ni, B.nj, B.nk, ci, cj, k + 3, pre);
            const bool need_un = (p.mode == MODE_ACCUM && p.alpha != 0.0) || (p.mode == MODE_INCR && (out_wide || !WIDE));
            if (col_valid) {
                // warm L2 with the update's per-cell operands; they are loaded
                // after the fluxes
                const long long cell = L.off + (long long)k * L.sk + (long long)cj * L.sj + ci;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (need_un) prefetch_l2(p.user[b] + cell + v * L.sv);
                    if (p.dprev >= 0) prefetch_l2(B.ds[p.dprev] + cell + v * L.sv);
                }
            }

            // ---- P0: wait for the plane's tile, primitives into sW
            const TS *raw = sRaw + cb * NV * TPLANE;
            const float *met = sMet + cb * REC;
            const bool ok = mbar_wait(bar0 + 8 * cb, (phase >> cb) & 1u, p.wait_limit);
            phase ^= 1u << cb;
            if (TWO_D) {
                for (int e = t; e < TPLANE; e += NTHREADS) {
                    const int r = e / TW, c = e - (e / TW) * TW;
                    float qf[NV], w[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) qf[v] = cvt<float, TS>(raw[v * TPLANE + e]);
                    const int gi = i0 + c - 2, gj = j0 + r - 2;
                    to_recon(qf, gm1, cons,
                             gi >= i0 && gi < min(i0 + TI, B.ni) && gj >= j0 && gj < min(j0 + TJ, B.nj), p.err, w);
#pragma unroll
                    for (int v = 0; v < NV; ++v) sW[v * TPLANE + e] = w[v];
                }
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) sW[v * TPLANE + (tj + 2) * TW + ti + 2] = Wc[v];
                if (t < NHALO) {
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
                    const int e = r * TW + c;
                    float qf[NV], w[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) qf[v] = cvt<float, TS>(raw[v * TPLANE + e]);
                    to_recon(qf, gm1, cons, false, p.err, w);
#pragma unroll
                    for (int v = 0; v < NV; ++v) sW[v * TPLANE + e] = w[v];
                }
            }
            if (__syncthreads_or(!ok)) {
                // the copies of this plane once more (bounded) before the CTA
                // and its shared memory go away; every other issued plane has
                // been waited for
                if (t == 0) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    mbar_wait(bar0 + 8 * cb, ((phase >> cb) & 1u) ^ 1u, p.wait_limit);
                }
                failed = true;
                break;
            }
            // the next plane into the other buffer (its last reader, the
            // previous plane's update, is behind the barrier above)
            if (k + 1 < k1) {
                const int nb = cb ^ 1;
                if (warp == 0)
                    issue_plane<TS>(in, L, i0, j0, k + 1, nrows, len, rec0 + (k + 1) * rec_stride,
                                    sRaw + nb * NV * TPLANE, sMet + nb * REC, bar0 + 8 * nb, lane, p.tx_extra);
            }

            // ---- P1: fluxes: the own column's upper k-face (registers);
            //      then, through one copy of the MUSCL + Roe code, the j-face
            //      below the own cell (to sFj), the tile's top j-faces (warp
            //      0) and right i-faces (warp 1) (to sFj, sFiE), and the
            //      i-face left of the own cell (registers)
            float Fkp[NV], Ppn[NV];
            if (!TWO_D) {
                float Rk[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    face_states<float, LIM>(sW[v * TPLANE + (tj + 2) * TW + ti + 2], sK[(kb * NV + v) * NTHREADS + t],
                                            sK[((kb ^ 1) * NV + v) * NTHREADS + t], c1, c2, half_eps, Ppn[v], Rk[v]);
                const float *mk = met + REC_I + REC_J + tj * TI + ti;
                face_flux(Pp, Rk, mk[0], mk[TJ * TI], mk[2 * TJ * TI], mk[3 * TJ * TI], gm1, kg, fix, ifix, cons,
                          Fkp);
            }
            float Fi[NV];
#pragma unroll 1
            for (int job = 0; job < 3; ++job) {
                const float *w;
                const float *mt;
                int st, mst;
                float *dst = nullptr;
                int dstv = 0;
                if (job == 0) {
                    w = sW + tj * TW + ti + 2;
                    st = TW;
                    mt = met + REC_I + tj * TI + ti;
                    mst = (TJ + 1) * TI;
                    dst = sFj + tj * TI + ti;
                    dstv = FJV;
                } else if (job == 1) {
                    if (warp > 1 || (warp == 1 && lane >= TJ)) continue;
                    if (warp == 0) {
                        w = sW + TJ * TW + lane + 2;
                        st = TW;
                        mt = met + REC_I + TJ * TI + lane;
                        mst = (TJ + 1) * TI;
                        dst = sFj + TJ * TI + lane;
                        dstv = FJV;
                    } else {
                        w = sW + (lane + 2) * TW + TI;
                        st = 1;
                        mt = met + lane * (TI + 1) + TI;
                        mst = TJ * (TI + 1);
                        dst = sFiE + lane;
                        dstv = TJ;
                    }
                } else {
                    w = sW + (tj + 2) * TW + ti;
                    st = 1;
                    mt = met + tj * (TI + 1) + ti;
                    mst = TJ * (TI + 1);
                }
                float F[NV];
                line_flux<LIM>(w, st, mt, mst, gm1, kg, fix, ifix, c1, c2, half_eps, cons, F);
                if (dst) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) dst[v * dstv] = F[v];
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fi[v] = F[v];
                }
            }
            __syncthreads();

            // ---- P2: residual, update, ghost push, norm partials
            // the i-face right of the own cell: the next lane's, or for lane
            // 31 the tile's right face (all lanes take part in the shuffle)
            float Fr[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Fr[v] = __shfl_down_sync(0xffffffffu, Fi[v], 1);
                if (lane == TI - 1) Fr[v] = sFiE[v * TJ + tj];
            }
            if (col_valid) {
                const long long cell = L.off + (long long)k * L.sk + (long long)cj * L.sj + ci;
                const long long mc = (long long)k * ml.mplane + (long long)cj * ml.mpitch + ci;
                const double *un = p.user[b];
                const float *dprev = p.dprev >= 0 ? B.ds[p.dprev] : nullptr;
                double unv[NV];
                float dpv[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    unv[v] = need_un ? un[cell + v * L.sv] : 0.0;
                    dpv[v] = dprev ? dprev[cell + v * L.sv] : 0.0f;
                }
                const double dtvd = p.local ? B.dtv[mc] : 0.0;
                const double ivd = (!p.local && p.mode == MODE_ACCUM) ? B.ivol[mc] : 0.0;
                const double vold = (WIDE && p.partials) ? B.vol[mc] : 0.0;
                double *out64 = out_wide ? slot64(B, p.user[b], p.out_slot) : nullptr;
                float *xout = (p.mode == MODE_INCR && p.out_slot >= SLOT_X0) ? slot32(B, p.out_slot) : nullptr;
                float *dout = p.dout >= 0 ? B.ds[p.dout] : nullptr;
                float rres[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    float rr = (Fr[v] - Fi[v]) + (sFj[v * FJV + (tj + 1) * TI + ti] - sFj[v * FJV + tj * TI + ti]);
                    if (!TWO_D) rr += Fkp[v] - sFkm[v * NTHREADS + t];
                    rres[v] = rr;
                }
                const int e_own = (tj + 2) * TW + ti + 2;
                const bool boundary = ci < 2 || ci >= B.ni - 2 || cj < 2 || cj >= B.nj - 2 ||
                                      (!TWO_D && (k < 2 || k >= B.nk - 2));
                if (p.mode == MODE_INCR) {
                    // FP32 increment D = beta Dprev - gdt dt/|Omega| R; X = float(U^n) + D,
                    // or on the last stage U^n + D in FP64
                    const float c32 = p.local ? gdt32 * to_f32(dtvd) : gdt_dt32 * met[REC - REC_V + tj * TI + ti];
                    double q64[NV];
                    float q32[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        float delta = -c32 * rres[v];
                        if (dprev) delta = fmaf(beta32, dpv[v], delta);
                        if (out64) {
                            q64[v] = unv[v] + to_f64(delta);
                            out64[cell + v * L.sv] = q64[v];
                        } else {
                            const float xc = WIDE ? cvt<float, TS>(raw[v * TPLANE + e_own]) : to_f32(unv[v]);
                            dout[cell + v * L.sv] = delta;
                            q32[v] = xc + delta;
                            xout[cell + v * L.sv] = q32[v];
                        }
                    }
                    if (p.push && boundary) {
                        if (out64)
                            push_affine<double, NFACES>(sPush, B, ci, cj, k, q64);
                        else
                            push_affine<float, NFACES>(sPush, B, ci, cj, k, q32);
                    }
                } else {
                    const double coef = p.local ? -p.gdt * dtvd : -p.gdt * dt * ivd;
                    const long long rc = ((long long)k * B.nj + cj) * B.ni + ci;
                    const long long nint = (long long)B.ni * B.nj * B.nk;
                    double q64[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        double r = to_f64(rres[v]);
                        if (p.mode == MODE_RESIDUAL && p.src[b]) r -= p.src[b][v * nint + rc];
                        const double uin = cvt<double, TS>(raw[v * TPLANE + e_own]);
                        if (p.mode == MODE_ACCUM) {
                            double val = p.beta * uin + coef * r;
                            if (p.alpha != 0.0) val += p.alpha * unv[v];
                            out64[cell + v * L.sv] = val;
                            q64[v] = val;
                        } else {
                            p.rout[b][v * nint + rc] = r;
                        }
                    }
                    if (p.push && boundary && p.mode != MODE_RESIDUAL) push_affine<double, NFACES>(sPush, B, ci, cj, k, q64);
                }
                if (WIDE && p.partials) {
                    const double vol = vold;
                    const long long rc = ((long long)k * B.nj + cj) * B.ni + ci;
                    const long long nint = (long long)B.ni * B.nj * B.nk;
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        // r exactly as hi + lo: the FP32 residual, or with a
                        // source term its FP64 value split in two floats
                        float hi = rres[v], lo = 0.0f;
                        if (p.mode == MODE_RESIDUAL && p.src[b]) {
                            const double r = to_f64(rres[v]) - p.src[b][v * nint + rc];
                            hi = to_f32(r);
                            lo = to_f32(r - to_f64(hi));
                        }
                        const float sq = hi * hi;
                        ds_add(nsq_hi[v], nsq_lo[v], sq, fmaf(hi, hi, -sq) + 2.0f * hi * lo);
                        nmax[v] = fmaxf(nmax[v], fabsf(hi + lo));
                        ncons[v] = fma(vol, cvt<double, TS>(raw[v * TPLANE + e_own]), ncons[v]);
                    }
                }
            }
            if (!TWO_D) {
                float qf[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    sFkm[v * NTHREADS + t] = Fkp[v];
                    Pp[v] = Ppn[v];
                    Wc[v] = sK[(kb * NV + v) * NTHREADS + t];
                    qf[v] = cvt<float, TS>(pre[v]);
                }
                float w3[NV];
                to_recon(qf, gm1, cons, col_valid && k + 3 < B.nk, p.err, w3);
#pragma unroll
                for (int v = 0; v < NV; ++v) sK[(kb * NV + v) * NTHREADS + t] = w3[v];
                kb ^= 1;
            }
            cb ^= 1;
        }
        if (failed) break;

        // ---- norm partials of this item, fixed-order reduction in FP64
        if (WIDE && p.partials) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double a = (double)nsq_hi[v] + (double)nsq_lo[v], bm = (double)nmax[v], c = ncons[v];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_down_sync(0xffffffffu, a, o);
                    bm = fmax(bm, __shfl_down_sync(0xffffffffu, bm, o));
                    c += __shfl_down_sync(0xffffffffu, c, o);
                }
                if (lane == 0) {
                    sRed[(0 * NV + v) * (NTHREADS / 32) + warp] = a;
                    sRed[(1 * NV + v) * (NTHREADS / 32) + warp] = bm;
                    sRed[(2 * NV + v) * (NTHREADS / 32) + warp] = c;
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
#undef gm1
#undef kg
#undef c1
#undef c2
#undef half_eps
#undef fix
#undef ifix
#undef cons
}

template <typename TS>
struct Stencil32Launcher {
    using Fn = void (*)(const BatchParams<float>);
    static Fn pick(int limiter, bool two_d)
    {
        switch (limiter) {
        case SENSEI_LIM_NONE: return two_d ? stencil32_kernel<TS, SENSEI_LIM_NONE, true>
                                           : stencil32_kernel<TS, SENSEI_LIM_NONE, false>;
        case SENSEI_LIM_MINMOD: return two_d ? stencil32_kernel<TS, SENSEI_LIM_MINMOD, true>
                                             : stencil32_kernel<TS, SENSEI_LIM_MINMOD, false>;
        default: return two_d ? stencil32_kernel<TS, SENSEI_LIM_VANLEER, true>
                              : stencil32_kernel<TS, SENSEI_LIM_VANLEER, false>;
        }
    }
    static cudaError_t prepare(Fn fn)
    {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Smem32<TS>::bytes);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    static cudaError_t launch(const BatchParams<float> &p, int limiter, bool two_d, int grid, cudaStream_t s)
    {
        Fn fn = pick(limiter, two_d);
        cudaError_t e = prepare(fn);
        if (e != cudaSuccess) return e;
        fn<<<grid, NTHREADS, Smem32<TS>::bytes, s>>>(p);
        return cudaGetLastError();
    }
    static int ctas_per_sm(int limiter, bool two_d)
    {
        Fn fn = pick(limiter, two_d);
        if (prepare(fn) != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NTHREADS, Smem32<TS>::bytes) != cudaSuccess) return 0;
        return n;
    }
};

}  // namespace sensei
