// viscous.cu -- the viscous flux F_nu,n of Eq. governing on the device.
//
// tau_ij from Stokes's hypothesis, Theta_i = u_j tau_ij + k dT/dx_i with a
// constant mu and k dT = mu gamma / ((gamma - 1) Pr) d(p / rho) (the paper
// gives neither the viscosity law nor the face-gradient discretisation;
// these are the readings used).  The gradients of (u, v, w, p / rho) at a
// face between cells L and R (direction d, tangential directions e, f) are
//   d/dxi   = phi_R - phi_L,
//   d/deta  = [(phi_L + phi_R)(+e) - (phi_L + phi_R)(-e)] / 4, likewise zeta,
//   grad = sum_a d/dxi_a * (Sbar_a(L) + Sbar_a(R)) / (|Omega_L| + |Omega_R|),
// Sbar_a the mean of a cell's two a-face vectors (the metric identity
// grad xi_a = Sbar_a / |Omega|), a ghost cell carrying the geometry of the
// cell it copies.  The tangential differences read the block-edge ghosts.
//
// Per grid (and whenever the boundary rules change) the face gradient
// metrics grad xi_a of every face.  Per stage three kernels: the primitives
// (u, v, w, p / rho) of every ghosted cell; F_nu . S of every face, once;
// per interior cell the sum over its faces (R_nu), which the stencil kernel
// subtracts from the inviscid residual.  A face's one value enters both of
// its cells, so the pair cancels exactly in conservation sums.
#include <math.h>

#include <algorithm>

#include "blocks.cuh"

namespace sensei {
namespace {

__device__ __forceinline__ double rcp2(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    for (int n = 0; n < 2; ++n) r = fma(r, fma(-d, r, 1.0), r);
    return r;
}

// (u, v, w, p / rho) of every entry of each block's ghosted state array
__global__ void vis_prims_kernel(VisBatch p)
{
    const int b = blockIdx.y;
    const BlockDev &B = p.blocks[b];
    const double *U = slot64(B, p.user[b], p.slot);
    const long long n = B.L.sv;
    const double gm1 = p.gamma - 1.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double rho = U[e], mx = U[n + e], my = U[2 * n + e], mz = U[3 * n + e], E = U[4 * n + e];
        const double ir = rcp2(rho);
        const double u = mx * ir, v = my * ir, w = mz * ir;
        const double pr = gm1 * (E - 0.5 * (mx * u + my * v + mz * w));
        B.wv[e] = u;
        B.wv[n + e] = v;
        B.wv[2 * n + e] = w;
        B.wv[3 * n + e] = pr * ir;
    }
}

// The cell whose geometry cell c (of a face's two cells) carries: itself
// inside the block; behind a periodic face the opposite side's cell; behind
// an interface the neighbour block's cell; behind a physical boundary the
// boundary cell it mirrors.
__device__ __forceinline__ const BlockDev *metric_cell(const BlockDev *blocks, const BlockDev *B, int c[3])
{
    const int n[3] = {B->ni, B->nj, B->nk};
    for (int a = 0; a < 3; ++a) {
        if (c[a] >= 0 && c[a] < n[a]) continue;
        const int hi = c[a] >= n[a];
        const int f = 2 * a + hi;
        const int layer = hi ? c[a] - n[a] + 1 : -c[a];
        const int type = B->bc_type[f];
        if (type == SENSEI_BC_PERIODIC) {
            c[a] = hi ? c[a] - n[a] : c[a] + n[a];
        } else if (type == SENSEI_BC_INTERFACE) {
            const BlockDev *N = &blocks[B->nbr[f]];
            const int m[3] = {N->ni, N->nj, N->nk};
            c[a] = (B->nbr_face[f] & 1) ? m[a] - layer : layer - 1;
            return N;
        } else {
            c[a] = min(max(c[a], 0), n[a] - 1);
        }
    }
    return B;
}

__device__ __forceinline__ long long mindex(const BlockDev *B, int i, int j, int k)
{
    return (long long)k * B->ml.mplane + (long long)j * B->ml.mpitch + i;
}

// faces of family d of block B in node-grid order: m = k*mplane + j*mpitch + i
// with i <= ni (d = 0), j <= nj (d = 1), k <= nk (d = 2), the others inside
__device__ __forceinline__ bool face_of(const BlockDev &B, int d, long long m, int &i, int &j, int &k)
{
    k = (int)(m / B.ml.mplane);
    const long long r = m - (long long)k * B.ml.mplane;
    j = (int)(r / B.ml.mpitch);
    i = (int)(r - (long long)j * B.ml.mpitch);
    return i < B.ni + (d == 0) && j < B.nj + (d == 1) && k < B.nk + (d == 2);
}

// The face-gradient metrics of every d-face, into gvis[(d * GVIS + n) *
// mvolume + m]: n = 3 a + c, grad xi_a (component c) for a = d, e, f (the
// face's normal, then its two tangential index directions), (Sbar_a(L) +
// Sbar_a(R)) / (|Omega_L| + |Omega_R|), the tangential two already times the
// 1/4 of their central differences (exact); n = 9 + c, the face's area
// vector S; n = 12 + a, grad xi_a . S.  Depends on the boundary rules (the
// geometry a ghost cell carries): rerun when they change.
__global__ void vis_metrics_kernel(const BlockDev *blocks)
{
    const int b = blockIdx.y, d = blockIdx.z;
    const BlockDev &B = blocks[b];
    const int ndir = B.nk == 1 ? 2 : 3;
    if (d >= ndir) return;
    const long long mv = B.ml.mvolume;
    const int dirs[3] = {d, d == 0 ? 1 : 0, d == 2 ? 1 : 2};
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < mv; m += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        if (!face_of(B, d, m, i, j, k)) continue;
        int Lc[3] = {i - (d == 0), j - (d == 1), k - (d == 2)}, Rc[3] = {i, j, k};
        const BlockDev *bL = metric_cell(blocks, &B, Lc);
        const BlockDev *bR = metric_cell(blocks, &B, Rc);
        const long long mL = mindex(bL, Lc[0], Lc[1], Lc[2]), mR = mindex(bR, Rc[0], Rc[1], Rc[2]);
        const double ivs = 1.0 / (bL->vol[mL] + bR->vol[mR]);
        double *g = B.gvis + (long long)(d * GVIS) * mv + m;
        const double *fn = B.fn + (long long)(d * 4) * mv + m;
        const double A = fn[3 * mv];
        const double S[3] = {fn[0] * A, fn[mv] * A, fn[2 * mv] * A};
        for (int c = 0; c < 3; ++c) g[(9 + c) * mv] = S[c];
        for (int a = 0; a < 3; ++a) {
            const bool on = dirs[a] < ndir;
            const double *sa = bL->sbar + (long long)(dirs[a] * 4) * bL->ml.mvolume + mL;
            const double *sb = bR->sbar + (long long)(dirs[a] * 4) * bR->ml.mvolume + mR;
            const double w = a == 0 ? ivs : 0.25 * ivs;
            double gs = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double x = on ? (sa[c * bL->ml.mvolume] + sb[c * bR->ml.mvolume]) * w : 0.0;
                g[(a * 3 + c) * mv] = x;
                gs = fma(x, S[c], gs);
            }
            g[(12 + a) * mv] = gs;
        }
    }
}

// F_nu . S of every d-face into fvis[(d * NV + q) * mvolume + m], each face once
__global__ void __launch_bounds__(256, 2) vis_face_kernel(VisBatch p)
{
    const int b = blockIdx.y, d = blockIdx.z;
    const BlockDev &B = p.blocks[b];
    const int ndir = B.nk == 1 ? 2 : 3;
    if (d >= ndir) return;
    const long long mv = B.ml.mvolume;
    const long long sv = B.L.sv;
    const double *wv = B.wv;
    const int e = d == 0 ? 1 : 0;
    const int f = d == 2 ? 1 : 2;
    const long long offd = d == 0 ? 1 : (d == 1 ? B.L.sj : B.L.sk);
    const long long offe = e == 0 ? 1 : B.L.sj;
    const long long offf = f == 1 ? B.L.sj : B.L.sk;
    const bool has_f = f < ndir;
    const double mu = p.mu, kcond = p.kcond, mu2 = 2.0 * p.mu, mu23 = 2.0 / 3.0 * p.mu;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < mv; m += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        if (!face_of(B, d, m, i, j, k)) continue;
        const long long cR = cell_index(B.L, i, j, k), cL = cR - offd;
        double pL[4], pR[4], dxi[4], deta[4], dzeta[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            pL[q] = wv[q * sv + cL];
            pR[q] = wv[q * sv + cR];
            dxi[q] = pR[q] - pL[q];
            // tangential central differences, (+1) minus (-1) (their 1/4 is
            // in the metrics)
            deta[q] = (wv[q * sv + cL + offe] + wv[q * sv + cR + offe]) - (wv[q * sv + cL - offe] + wv[q * sv + cR - offe]);
            dzeta[q] = has_f ? (wv[q * sv + cL + offf] + wv[q * sv + cR + offf]) -
                                   (wv[q * sv + cL - offf] + wv[q * sv + cR - offf])
                             : 0.0;
        }
        const double *g = B.gvis + (long long)(d * GVIS) * mv + m;
        double gx[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) gx[a][c] = g[(a * 3 + c) * mv];
        // the velocity gradient (the temperature's enters only as grad T . S)
        double grad[3][3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) grad[q][c] = fma(dzeta[q], gx[2][c], fma(deta[q], gx[1][c], dxi[q] * gx[0][c]));
        // tau (symmetric: six entries) = mu (grad u + grad u^T) - 2/3 mu div u I
        const double d23 = mu23 * (grad[0][0] + grad[1][1] + grad[2][2]);
        const double t00 = fma(mu2, grad[0][0], -d23), t11 = fma(mu2, grad[1][1], -d23),
                     t22 = fma(mu2, grad[2][2], -d23);
        const double t01 = mu * (grad[0][1] + grad[1][0]), t02 = mu * (grad[0][2] + grad[2][0]),
                     t12 = mu * (grad[1][2] + grad[2][1]);
        // the face's area vector
        const double S0 = g[9 * mv], S1 = g[10 * mv], S2 = g[11 * mv];
        double *out = B.fvis + (long long)(d * NV) * mv + m;
        const double r1 = fma(t02, S2, fma(t01, S1, t00 * S0));
        const double r2 = fma(t12, S2, fma(t11, S1, t01 * S0));
        const double r3 = fma(t22, S2, fma(t12, S1, t02 * S0));
        out[0] = 0.0;
        out[mv] = r1;
        out[2 * mv] = r2;
        out[3 * mv] = r3;
        // Theta . S = (u tau + k grad T) . S = u . (tau S) + k grad T . S
        // (tau symmetric), u the face mean (uL + uR)/2
        const double uts = fma(pL[2] + pR[2], r3, fma(pL[1] + pR[1], r2, (pL[0] + pR[0]) * r1));
        const double gts = fma(dzeta[3], g[14 * mv], fma(deta[3], g[13 * mv], dxi[3] * g[12 * mv]));
        out[4 * mv] = fma(0.5, uts, kcond * gts);
    }
}

// R_nu = sum over a cell's faces of F_nu . S_out (dense interior layout)
__global__ void __launch_bounds__(256) vis_sum_kernel(VisBatch p)
{
    const int b = blockIdx.y;
    const BlockDev &B = p.blocks[b];
    const long long nint = (long long)B.ni * B.nj * B.nk;
    const long long mv = B.ml.mvolume;
    const int ndir = B.nk == 1 ? 2 : 3;
    for (long long rc = blockIdx.x * (long long)blockDim.x + threadIdx.x; rc < nint;
         rc += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(rc % B.ni);
        const int j = (int)((rc / B.ni) % B.nj);
        const int k = (int)(rc / ((long long)B.ni * B.nj));
        const long long m = mindex(&B, i, j, k);
        double acc[NV] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int d = 0; d < ndir; ++d) {
            const long long step = d == 0 ? 1 : (d == 1 ? B.ml.mpitch : B.ml.mplane);
            const double *F = B.fvis + (long long)(d * NV) * mv + m;
#pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] += F[q * mv + step] - F[q * mv];
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) B.rvis[q * nint + rc] = acc[q];
    }
}

}  // namespace

cudaError_t launch_vis_metrics(const BlockDev *blocks, int nblocks, long long max_faces, cudaStream_t s)
{
    const unsigned gx = (unsigned)std::max<long long>(1, std::min<long long>((max_faces + 255) / 256, 1024));
    vis_metrics_kernel<<<dim3(gx, (unsigned)nblocks, 3), 256, 0, s>>>(blocks);
    return cudaGetLastError();
}

cudaError_t launch_viscous(const VisBatch &p, long long max_state, long long max_faces, long long max_cells,
                           cudaStream_t s)
{
    const unsigned g1 = (unsigned)std::max<long long>(1, std::min<long long>((max_state + 255) / 256, 1024));
    vis_prims_kernel<<<dim3(g1, (unsigned)p.nblocks), 256, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned g2 = (unsigned)std::max<long long>(1, std::min<long long>((max_faces + 255) / 256, 1024));
    vis_face_kernel<<<dim3(g2, (unsigned)p.nblocks, 3), 256, 0, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned g3 = (unsigned)std::max<long long>(1, std::min<long long>((max_cells + 255) / 256, 1024));
    vis_sum_kernel<<<dim3(g3, (unsigned)p.nblocks), 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace sensei
