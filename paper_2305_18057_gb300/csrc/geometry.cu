// geometry.cu -- grid metrics and ghost-cell (boundary) kernels.
//
// Metrics: the face area vectors Delta s * n and cell volumes |Omega| of
// Eq. residual / Eq. spatial_residual (Sec. 3.1), computed once per grid.
// Ghost cells: boundary enforcement kept on the device (Sec. 5, "Ghost cell
// extrapolation on the GPU"), two layers per boundary face.
#include <math.h>

#include "sensei_internal.cuh"

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

__device__ __forceinline__ double centroid_dot(P3 a, P3 b, P3 c, P3 d, P3 s)
{
    return 0.25 * ((a.x + b.x + c.x + d.x) * s.x + (a.y + b.y + c.y + d.y) * s.y + (a.z + b.z + c.z + d.z) * s.z);
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
            for (int q = 0; q < 4; ++q) {
                mo.n[fam][q][m] = v[q];
                if (mo.n32[fam][q]) mo.n32[fam][q][m] = (float)v[q];
            }
        }
        if (in_i && in_j && in_k) {
            // |Omega| = (1/3) sum over the six faces of centroid . outward area
            // vector; the mean area vector of the two d-faces gives the
            // spectral radius of the time-step bound.
            double vol = 0.0;
            for (int fam = 0; fam < 3; ++fam) {
                int di = fam == 0, dj = fam == 1, dk = fam == 2;
                FaceCorners lo = corners(X, nn, ni, nj, fam, i, j, k);
                FaceCorners hi = corners(X, nn, ni, nj, fam, i + di, j + dj, k + dk);
                P3 slo = quad_area(lo.p[0], lo.p[1], lo.p[2], lo.p[3]);
                P3 shi = quad_area(hi.p[0], hi.p[1], hi.p[2], hi.p[3]);
                vol += centroid_dot(hi.p[0], hi.p[1], hi.p[2], hi.p[3], shi) -
                       centroid_dot(lo.p[0], lo.p[1], lo.p[2], lo.p[3], slo);
                P3 sb{0.5 * (slo.x + shi.x), 0.5 * (slo.y + shi.y), 0.5 * (slo.z + shi.z)};
                mo.sbar[fam][0][m] = sb.x;
                mo.sbar[fam][1][m] = sb.y;
                mo.sbar[fam][2][m] = sb.z;
                mo.sbar[fam][3][m] = sqrt(sb.x * sb.x + sb.y * sb.y + sb.z * sb.z);
            }
            vol = vol / 3.0;
            mo.vol[m] = vol;
            mo.ivol[m] = 1.0 / vol;
            if (mo.ivol32) mo.ivol32[m] = (float)(1.0 / vol);
        }
    }
}

// ------------------------------------------------------------------------
// ghost cells
// ------------------------------------------------------------------------

__device__ __forceinline__ long long cell_at(const StateLayout &L, int i, int j, int k)
{
    return L.off + (long long)k * L.sk + (long long)j * L.sj + i;
}

// ghost cell of face f, layer g (1 next to the boundary, 2 outer), and the
// interior cell m cells inside the boundary (m = 0: the boundary cell)
__device__ __forceinline__ void face_cells(int f, int ni, int nj, int nk, int t1, int t2, int g, int m, int &gi,
                                           int &gj, int &gk_, int &mi, int &mj, int &mk)
{
    switch (f) {
    case 0: gi = -g; gj = t1; gk_ = t2; mi = m; mj = t1; mk = t2; break;
    case 1: gi = ni - 1 + g; gj = t1; gk_ = t2; mi = ni - 1 - m; mj = t1; mk = t2; break;
    case 2: gi = t1; gj = -g; gk_ = t2; mi = t1; mj = m; mk = t2; break;
    case 3: gi = t1; gj = nj - 1 + g; gk_ = t2; mi = t1; mj = nj - 1 - m; mk = t2; break;
    case 4: gi = t1; gj = t2; gk_ = -g; mi = t1; mj = t2; mk = m; break;
    default: gi = t1; gj = t2; gk_ = nk - 1 + g; mi = t1; mj = t2; mk = nk - 1 - m; break;
    }
}

template <typename T>
__global__ void bc_kernel(BCParamsT<T> p)
{
    long long total = 0;
    for (int f = 0; f < p.nfaces; ++f) total += p.count[f];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int f = 0;
        long long r = t;
        while (r >= p.count[f]) {
            r -= p.count[f];
            ++f;
        }
        int n1 = f < 2 ? p.nj : p.ni;
        int layer = 1 + (int)(r % 2);
        long long pos = r / 2;
        int t1 = (int)(pos % n1);
        int t2 = (int)(pos / n1);
        const FaceBC<T> &bc = p.f[f];
        int gi, gj, gk, mi, mj, mk;
        T q[NV];
        if (bc.type == SENSEI_BC_PERIODIC || bc.type == SENSEI_BC_SLIP_WALL) {
            // periodic: the opposite face's layer-1 cell inside; wall: mirror
            int src_face = bc.type == SENSEI_BC_PERIODIC ? (f ^ 1) : f;
            int a, b, c;
            face_cells(f, p.ni, p.nj, p.nk, t1, t2, layer, 0, gi, gj, gk, a, b, c);
            face_cells(src_face, p.ni, p.nj, p.nk, t1, t2, 1, layer - 1, a, b, c, mi, mj, mk);
            long long sc = cell_at(p.L, mi, mj, mk);
            for (int v = 0; v < NV; ++v) q[v] = p.U[sc + v * p.L.sv];
            if (bc.type == SENSEI_BC_SLIP_WALL) {
                int fam = f >> 1;
                int bi = mi, bj = mj, bk = mk;   // boundary face index: the cell's own minus face,
                if (f == 1) bi = p.ni;           // or the block's plus face
                if (f == 3) bj = p.nj;
                if (f == 5) bk = p.nk;
                if (f == 0) bi = 0;
                if (f == 2) bj = 0;
                if (f == 4) bk = 0;
                long long fm = bk * p.ml.mplane + bj * p.ml.mpitch + bi;
                const T nx = (T)p.fm.n[fam][0][fm], ny = (T)p.fm.n[fam][1][fm], nz = (T)p.fm.n[fam][2][fm];
                const T mn = q[1] * nx + q[2] * ny + q[3] * nz;
                q[1] -= T(2) * mn * nx;
                q[2] -= T(2) * mn * ny;
                q[3] -= T(2) * mn * nz;
            }
        } else if (bc.type == SENSEI_BC_EXTRAPOLATE) {
            face_cells(f, p.ni, p.nj, p.nk, t1, t2, layer, 0, gi, gj, gk, mi, mj, mk);
            long long sc = cell_at(p.L, mi, mj, mk);
            for (int v = 0; v < NV; ++v) q[v] = p.U[sc + v * p.L.sv];
        } else if (bc.type == SENSEI_BC_INFLOW) {
            face_cells(f, p.ni, p.nj, p.nk, t1, t2, layer, 0, gi, gj, gk, mi, mj, mk);
            double rho = bc.prim[0], u = bc.prim[1], v = bc.prim[2], w = bc.prim[3], pr = bc.prim[4];
            q[0] = (T)rho;
            q[1] = (T)(rho * u);
            q[2] = (T)(rho * v);
            q[3] = (T)(rho * w);
            q[4] = (T)(pr / (p.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w));
        } else {   // SENSEI_BC_INTERFACE: neighbour's layer-1 cell inside its face
            int a, b, c;
            face_cells(f, p.ni, p.nj, p.nk, t1, t2, layer, 0, gi, gj, gk, a, b, c);
            face_cells(bc.nbr_face, bc.nni, bc.nnj, bc.nnk, t1, t2, 1, layer - 1, a, b, c, mi, mj, mk);
            long long sc = cell_at(bc.nL, mi, mj, mk);
            for (int v = 0; v < NV; ++v) q[v] = bc.nbr[sc + v * bc.nL.sv];
        }
        long long gc = cell_at(p.L, gi, gj, gk);
        for (int v = 0; v < NV; ++v) p.U[gc + v * p.L.sv] = q[v];
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

template <typename T>
static cudaError_t launch_bc_t(const BCParamsT<T> &p, cudaStream_t s)
{
    long long total = 0;
    for (int f = 0; f < p.nfaces; ++f) total += p.count[f];
    if (total == 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    bc_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_bc(const BCParamsT<double> &p, cudaStream_t s) { return launch_bc_t(p, s); }
cudaError_t launch_bc(const BCParamsT<float> &p, cudaStream_t s) { return launch_bc_t(p, s); }

}  // namespace sensei
