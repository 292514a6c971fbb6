// geometry.cu -- grid metrics and ghost-cell (boundary) kernels.
//
// Metrics: the face area vectors Delta s * n and cell volumes |Omega| of
// Eq. residual / Eq. spatial_residual (Sec. 3.1), computed once per grid.
// Ghost cells: boundary enforcement kept on the device (Sec. 5, "Ghost cell
// extrapolation on the GPU"), two layers per boundary face.
#include <math.h>

#include <algorithm>

#include "blocks.cuh"

namespace sensei {
namespace {

struct P3 {
    double x, y, z;
};

__device__ __forceinline__ P3 load_node(const double *X, long long nn, int ni, int nj, int i, int j, int k)
{
    long long q = ((long long)k * (nj + 1) + j) * (ni + 1) + i;
    return P3{X[q], X[nn + q], X[2 * nn + q]};
}

// Area vector of a quadrilateral from its corners in cyclic order: half the
// cross product of the two diagonals (exact for the bilinear face).
__device__ __forceinline__ P3 quad_area(P3 a, P3 b, P3 c, P3 d)
{
    P3 e{c.x - a.x, c.y - a.y, c.z - a.z};
    P3 f{d.x - b.x, d.y - b.y, d.z - b.z};
    return P3{0.5 * (e.y * f.z - e.z * f.y), 0.5 * (e.z * f.x - e.x * f.z), 0.5 * (e.x * f.y - e.y * f.x)};
}

// (centroid - o) . s with the corners' offsets from o formed first (exact
// for nearby points)
__device__ __forceinline__ double centroid_dot(P3 a, P3 b, P3 c, P3 d, P3 o, P3 s)
{
    const double cx = (a.x - o.x) + (b.x - o.x) + (c.x - o.x) + (d.x - o.x);
    const double cy = (a.y - o.y) + (b.y - o.y) + (c.y - o.y) + (d.y - o.y);
    const double cz = (a.z - o.z) + (b.z - o.z) + (c.z - o.z) + (d.z - o.z);
    return 0.25 * (cx * s.x + cy * s.y + cz * s.z);
}

// Corners of the three face families at lowest node (i, j, k), ordered so
// that the area vector points toward increasing i, j or k.
struct FaceCorners {
    P3 p[4];
};

__device__ __forceinline__ FaceCorners corners(const double *X, long long nn, int ni, int nj, int fam, int i, int j,
                                               int k)
{
    FaceCorners c;
    if (fam == 0) {
        c.p[0] = load_node(X, nn, ni, nj, i, j, k);
        c.p[1] = load_node(X, nn, ni, nj, i, j + 1, k);
        c.p[2] = load_node(X, nn, ni, nj, i, j + 1, k + 1);
        c.p[3] = load_node(X, nn, ni, nj, i, j, k + 1);
    } else if (fam == 1) {
        c.p[0] = load_node(X, nn, ni, nj, i, j, k);
        c.p[1] = load_node(X, nn, ni, nj, i, j, k + 1);
        c.p[2] = load_node(X, nn, ni, nj, i + 1, j, k + 1);
        c.p[3] = load_node(X, nn, ni, nj, i + 1, j, k);
    } else {
        c.p[0] = load_node(X, nn, ni, nj, i, j, k);
        c.p[1] = load_node(X, nn, ni, nj, i + 1, j, k);
        c.p[2] = load_node(X, nn, ni, nj, i + 1, j + 1, k);
        c.p[3] = load_node(X, nn, ni, nj, i, j + 1, k);
    }
    return c;
}

__global__ void metrics_kernel(int ni, int nj, int nk, const double *__restrict__ X, MetricsOut mo, MetricLayout ml)
{
    long long total = (long long)(ni + 1) * (nj + 1) * (nk + 1);
    long long nn = total;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % (ni + 1));
        int j = (int)((t / (ni + 1)) % (nj + 1));
        int k = (int)(t / ((long long)(ni + 1) * (nj + 1)));
        long long m = k * ml.mplane + j * ml.mpitch + i;
        bool in_j = j < nj, in_k = k < nk, in_i = i < ni;
        bool has[3] = {in_j && in_k, in_i && in_k, in_i && in_j};
        for (int fam = 0; fam < 3; ++fam) {
            if (!has[fam]) continue;
            FaceCorners c = corners(X, nn, ni, nj, fam, i, j, k);
            P3 s = quad_area(c.p[0], c.p[1], c.p[2], c.p[3]);
            double a = sqrt(s.x * s.x + s.y * s.y + s.z * s.z);
            double inv = a > 0.0 ? 1.0 / a : 0.0;
            double v[4] = {s.x * inv, s.y * inv, s.z * inv, a};
            for (int q = 0; q < 4; ++q) mo.n[fam][q][m] = v[q];
        }
        if (in_i && in_j && in_k) {
            // |Omega| = (1/3) sum over the six faces of centroid . outward area
            // vector, the centroids measured from the cell's corner node (the
            // area vectors of the closed cell sum to zero, so the origin does
            // not change the volume, and a corner of the cell keeps every term
            // of the cell's size instead of |x| h^2 terms cancelling to h^3);
            // the mean area vector of the two d-faces gives the spectral
            // radius of the time-step bound.
            const P3 o = load_node(X, nn, ni, nj, i, j, k);
            double vol = 0.0;
            for (int fam = 0; fam < 3; ++fam) {
                int di = fam == 0, dj = fam == 1, dk = fam == 2;
                FaceCorners lo = corners(X, nn, ni, nj, fam, i, j, k);
                FaceCorners hi = corners(X, nn, ni, nj, fam, i + di, j + dj, k + dk);
                P3 slo = quad_area(lo.p[0], lo.p[1], lo.p[2], lo.p[3]);
                P3 shi = quad_area(hi.p[0], hi.p[1], hi.p[2], hi.p[3]);
                vol += centroid_dot(hi.p[0], hi.p[1], hi.p[2], hi.p[3], o, shi) -
                       centroid_dot(lo.p[0], lo.p[1], lo.p[2], lo.p[3], o, slo);
                P3 sb{0.5 * (slo.x + shi.x), 0.5 * (slo.y + shi.y), 0.5 * (slo.z + shi.z)};
                mo.sbar[fam][0][m] = sb.x;
                mo.sbar[fam][1][m] = sb.y;
                mo.sbar[fam][2][m] = sb.z;
                mo.sbar[fam][3][m] = sqrt(sb.x * sb.x + sb.y * sb.y + sb.z * sb.z);
                if (mo.vol32)
                    for (int q = 0; q < 4; ++q) mo.sbar32[fam][q][m] = (float)mo.sbar[fam][q][m];
            }
            vol = vol / 3.0;
            mo.vol[m] = vol;
            mo.ivol[m] = 1.0 / vol;
            if (mo.vol32) mo.vol32[m] = (float)vol;
        }
    }
}

// The FP32 records of the FP32 stencil: record (tile_i, tile_j, k) holds
// the tile's i-faces, j-faces and upper k-faces (unit normal, area) and
// 1/|Omega| of its cells, rounded to FP32; entries outside the block are 0.
__global__ void pack_records_kernel(BlockDev B)
{
    const long long nrec = (long long)B.tiles_i * B.tiles_j * B.nk;
    const long long mv = B.ml.mvolume;
    float *rec = const_cast<float *>(B.rec32);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrec * REC;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / REC;
        int e = (int)(t - r * REC);
        const int tile_i = (int)(r % B.tiles_i);
        const int tile_j = (int)((r / B.tiles_i) % B.tiles_j);
        const int k = (int)(r / ((long long)B.tiles_i * B.tiles_j));
        const int i0 = tile_i * TI, j0 = tile_j * TJ;
        double v = 0.0;
        if (e < REC_I) {
            const int q = e / (TJ * (TI + 1)), rem = e % (TJ * (TI + 1));
            const int i = i0 + rem % (TI + 1), j = j0 + rem / (TI + 1);
            if (i <= B.ni && j < B.nj) v = B.fn[q * mv + k * B.ml.mplane + j * B.ml.mpitch + i];
        } else if ((e -= REC_I) < REC_J) {
            const int q = e / ((TJ + 1) * TI), rem = e % ((TJ + 1) * TI);
            const int i = i0 + rem % TI, j = j0 + rem / TI;
            if (i < B.ni && j <= B.nj) v = B.fn[(4 + q) * mv + k * B.ml.mplane + j * B.ml.mpitch + i];
        } else if ((e -= REC_J) < REC_K) {
            const int q = e / (TJ * TI), rem = e % (TJ * TI);
            const int i = i0 + rem % TI, j = j0 + rem / TI;
            if (i < B.ni && j < B.nj && B.nk > 1)
                v = B.fn[(8 + q) * mv + (k + 1) * B.ml.mplane + j * B.ml.mpitch + i];
        } else {
            e -= REC_K;
            const int i = i0 + e % TI, j = j0 + e / TI;
            if (i < B.ni && j < B.nj) v = B.ivol[k * B.ml.mplane + j * B.ml.mpitch + i];
        }
        rec[t] = (float)v;
    }
}

// ------------------------------------------------------------------------
// ghost cells: every boundary face of every block of one buffer slot
// ------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T *slot_buffer(const BlockDev &B, double *user, int slot);
template <>
__device__ __forceinline__ double *slot_buffer<double>(const BlockDev &B, double *user, int slot)
{
    return slot64(B, user, slot);
}
template <>
__device__ __forceinline__ float *slot_buffer<float>(const BlockDev &B, double *, int slot)
{
    return slot32(B, slot);
}

// One ghost cell: layer `layer` of face f at tangential position (t1, t2).
// (t1, t2) may lie one family's ghost layers outside the face (the
// block-edge ghosts of the viscous face gradients); the rule then reads that
// family's ghosts, which the face pass has filled, and a wall takes the
// normal of the nearest boundary face.
template <typename T>
__device__ __forceinline__ void fill_one(const BCBatch &p, const BlockDev &B, int b, int f, int layer, int t1, int t2)
{
    T *U = slot_buffer<T>(B, p.user[b], p.slot);
    const int type = B.bc_type[f];
    if (type == SENSEI_BC_EXTERNAL) return;   // written by the caller
    int gi, gj, gk, mi, mj, mk, a, bb, c;
    face_cells(f, B.ni, B.nj, B.nk, t1, t2, layer, 0, gi, gj, gk, a, bb, c);
    T q[NV];
    if (type == SENSEI_BC_PERIODIC || type == SENSEI_BC_SLIP_WALL) {
        // periodic: the opposite face's cell layer-1 inside; wall: the
        // mirror image of the cell layer-1 inside this face
        const int src_face = type == SENSEI_BC_PERIODIC ? (f ^ 1) : f;
        face_cells(src_face, B.ni, B.nj, B.nk, t1, t2, 1, layer - 1, a, bb, c, mi, mj, mk);
        const long long sc = cell_index(B.L, mi, mj, mk);
        for (int v = 0; v < NV; ++v) q[v] = U[sc + v * B.L.sv];
        if (type == SENSEI_BC_SLIP_WALL) {
            const int n1 = f < 2 ? B.nj : B.ni, n2 = f < 4 ? B.nk : B.nj;
            double nx, ny, nz;
            boundary_normal(B, f, min(max(t1, 0), n1 - 1), min(max(t2, 0), n2 - 1), nx, ny, nz);
            const T tx = (T)nx, ty = (T)ny, tz = (T)nz;
            const T mn = q[1] * tx + q[2] * ty + q[3] * tz;
            q[1] -= T(2) * mn * tx;
            q[2] -= T(2) * mn * ty;
            q[3] -= T(2) * mn * tz;
        }
    } else if (type == SENSEI_BC_EXTRAPOLATE) {
        const long long sc = cell_index(B.L, a, bb, c);
        for (int v = 0; v < NV; ++v) q[v] = U[sc + v * B.L.sv];
    } else if (type == SENSEI_BC_INFLOW) {
        const double *w = B.bc_prim[f];
        const double rho = w[0], u = w[1], v = w[2], ww = w[3], pr = w[4];
        q[0] = (T)rho;
        q[1] = (T)(rho * u);
        q[2] = (T)(rho * v);
        q[3] = (T)(rho * ww);
        q[4] = (T)(pr / (p.gamma - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww));
    } else {   // SENSEI_BC_INTERFACE: the neighbour's cell layer-1 inside its face
        const int nb = B.nbr[f];
        const BlockDev &N = p.blocks[nb];
        face_cells(B.nbr_face[f], N.ni, N.nj, N.nk, t1, t2, 1, layer - 1, a, bb, c, mi, mj, mk);
        const T *NU = slot_buffer<T>(N, p.user[nb], p.slot);
        const long long sc = cell_index(N.L, mi, mj, mk);
        for (int v = 0; v < NV; ++v) q[v] = NU[sc + v * N.L.sv];
    }
    const long long gc = cell_index(B.L, gi, gj, gk);
    for (int v = 0; v < NV; ++v) U[gc + v * B.L.sv] = q[v];
}

// The two cell layers next to face f of one state array (heterogeneous
// co-execution): pack copies the interior layers l = 0, 1 inside the face
// into buf[v][l][t2][t1]; unpack writes buf into the ghost layers l + 1
// outside it (a neighbour's interior layer l is this block's ghost layer
// l + 1).
__global__ void face_exchange_kernel(BlockDev B, double *u, int f, double *buf, int unpack)
{
    const int n1 = f < 2 ? B.nj : B.ni, n2 = f < 4 ? B.nk : B.nj;
    const long long face = (long long)n1 * n2, per = NG * face, total = NV * per;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(t / per);
        const long long r = t - v * per;
        const int l = (int)(r / face);
        const long long q = r - l * face;
        const int t2 = (int)(q / n1), t1 = (int)(q - (long long)t2 * n1);
        int gi, gj, gk, mi, mj, mk;
        face_cells(f, B.ni, B.nj, B.nk, t1, t2, l + 1, l, gi, gj, gk, mi, mj, mk);
        if (unpack)
            u[cell_index(B.L, gi, gj, gk) + v * B.L.sv] = buf[t];
        else
            buf[t] = u[cell_index(B.L, mi, mj, mk) + v * B.L.sv];
    }
}

template <typename T>
__global__ void bc_kernel(BCBatch p)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < p.total;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = find_block_bc(p.blocks, p.nblocks, t);
        const BlockDev &B = p.blocks[b];
        long long r = t - B.bc0;
        const int nfaces = B.nk == 1 ? 4 : 6;
        int f = 0;
        while (f < nfaces - 1 && r >= face_units(B, f)) {
            r -= face_units(B, f);
            ++f;
        }
        const int n1 = f < 2 ? B.nj : B.ni;
        const int layer = 1 + (int)(r % 2);
        const long long pos = r / 2;
        fill_one<T>(p, B, b, f, layer, (int)(pos % n1), (int)(pos / n1));
    }
}

// q = 0..3 -> -2, -1, n, n + 1: the ghost positions of one index
__device__ __forceinline__ int ghost_pos(int q, int n) { return q < 2 ? q - 2 : n + q - 2; }

// The block-edge ghosts (two indices outside the block) read by the viscous
// face gradients, after every face's own ghosts: i-faces fill those at j- or
// k-ghost positions, j-faces those at k-ghost positions (the rule of the
// lower face family).  One grid row (blockIdx.y) per block.
template <typename T>
__global__ void edge_kernel(BCBatch p)
{
    const int b = blockIdx.y;
    const BlockDev &B = p.blocks[b];
    const bool two_d = B.nk == 1;
    const long long pi = two_d ? 4 : 4LL * B.nk + 4LL * B.nj;   // positions per i-face
    const long long pj = two_d ? 0 : 4LL * B.ni;                // positions per j-face
    const long long total = 2 * 2 * (pi + pj);                   // two faces per family, two layers
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const int layer = 1 + (int)(u & 1);
        long long r = u >> 1;
        int f, t1, t2;
        if (r < 2 * pi) {
            f = (int)(r / pi);
            long long q = r - f * pi;
            if (two_d) {
                t1 = ghost_pos((int)q, B.nj);
                t2 = 0;
            } else if (q < 4LL * B.nk) {
                t1 = ghost_pos((int)(q % 4), B.nj);
                t2 = (int)(q / 4);
            } else {
                q -= 4LL * B.nk;
                t1 = (int)(q / 4);
                t2 = ghost_pos((int)(q % 4), B.nk);
            }
        } else {
            r -= 2 * pi;
            f = 2 + (int)(r / pj);
            const long long q = r - (f - 2) * pj;
            t1 = (int)(q / 4);
            t2 = ghost_pos((int)(q % 4), B.nk);
        }
        fill_one<T>(p, B, b, f, layer, t1, t2);
    }
}

}  // namespace

cudaError_t launch_metrics(int ni, int nj, int nk, const double *X, const MetricsOut &mo, const MetricLayout &ml,
                           cudaStream_t s)
{
    long long total = (long long)(ni + 1) * (nj + 1) * (nk + 1);
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    metrics_kernel<<<(unsigned)blocks, 256, 0, s>>>(ni, nj, nk, X, mo, ml);
    return cudaGetLastError();
}

cudaError_t launch_pack_records(const BlockDev &B, cudaStream_t s)
{
    if (!B.rec32) return cudaSuccess;
    const long long total = (long long)B.tiles_i * B.tiles_j * B.nk * REC;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    pack_records_kernel<<<(unsigned)blocks, 256, 0, s>>>(B);
    return cudaGetLastError();
}

// x = hi + lo with hi the float nearest to x and lo the float nearest to the
// remainder (exact in double): the double-float form of the face metrics
__global__ void split_df64_kernel(const double *__restrict__ x, float2 *__restrict__ out, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double v = x[e];
        const float hi = __double2float_rn(v);
        out[e] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

cudaError_t launch_split_df64(const BlockDev &B, cudaStream_t s)
{
    if (!B.fdf) return cudaSuccess;
    const long long n = 12LL * B.ml.mvolume;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    split_df64_kernel<<<(unsigned)blocks, 256, 0, s>>>(B.fn, const_cast<float2 *>(B.fdf), n);
    return cudaGetLastError();
}

cudaError_t launch_edges(const BCBatch &p, int max_units, cudaStream_t s)
{
    const dim3 grid((unsigned)std::max(1, std::min((max_units + 255) / 256, 64)), (unsigned)p.nblocks);
    if (p.slot >= SLOT_X0)
        edge_kernel<float><<<grid, 256, 0, s>>>(p);
    else
        edge_kernel<double><<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_face_exchange(const BlockDev &B, double *u, int f, double *buf, int unpack, cudaStream_t s)
{
    const long long n1 = f < 2 ? B.nj : B.ni, n2 = f < 4 ? B.nk : B.nj;
    const long long total = NV * NG * n1 * n2;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    face_exchange_kernel<<<blocks, 256, 0, s>>>(B, u, f, buf, unpack);
    return cudaGetLastError();
}

cudaError_t launch_bc(const BCBatch &p, cudaStream_t s)
{
    if (p.total == 0) return cudaSuccess;
    long long blocks = (p.total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (p.slot == SLOT_X0 || p.slot == SLOT_X1)
        bc_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(p);
    else
        bc_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace sensei
