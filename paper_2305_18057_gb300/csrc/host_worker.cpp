// host_worker.cpp -- the host-thread worker of heterogeneous CPU + GPU
// co-execution (Sec. 4: the workload of one time step split between the
// host cores and the GPU, the interface ghost layers exchanged every
// Runge-Kutta stage; Sec. 6, Eq. hete: the ideal split by the two speeds).
//
// One 3D block on the host, FP64, the same method as the library's FP64
// kernels: face area vectors and volumes from the nodes (Sec. 3.1), MUSCL
// reconstruction of the primitive (or conserved) variables with the minmod /
// van Leer slope or the unlimited kappa form (Eq. flux), the Roe flux with
// Harten's entropy fix on the acoustic waves (three-wave form) of F_{i,n}
// (Eq. governing), the flux-difference residual R = sum F.S_out (Eq.
// residual), the Shu-Osher stages of SSPRK(2,2), (3,3), (4,2) (Eq.
// runge_kutta with the 1/|Omega| of Eq. spatial_residual), the CFL time
// step min |Omega| / sum_d (|u.Sbar_d| + c |Sbar_d|).  Host threads (OpenMP)
// take (k, j) rows of cells.  Ghost rules as on the GPU; a face of type
// SENSEI_BC_EXTERNAL keeps the ghost layers the caller writes
// (sensei_host_face_exchange).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "sensei.h"

namespace {

constexpr int NV = 5;
constexpr int NG = 2;

struct V3 {
    double x, y, z;
};

inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
// area vector of a quadrilateral (corners in cyclic order): half the cross
// product of its diagonals
inline V3 quad_area(V3 a, V3 b, V3 c, V3 d)
{
    const V3 e = sub(c, a), f = sub(d, b);
    return {0.5 * (e.y * f.z - e.z * f.y), 0.5 * (e.z * f.x - e.x * f.z), 0.5 * (e.x * f.y - e.y * f.x)};
}
// (centroid - o) . s, the corners' offsets from o formed first
inline double centroid_dot(V3 a, V3 b, V3 c, V3 d, V3 o, V3 s)
{
    const double cx = (a.x - o.x) + (b.x - o.x) + (c.x - o.x) + (d.x - o.x);
    const double cy = (a.y - o.y) + (b.y - o.y) + (c.y - o.y) + (d.y - o.y);
    const double cz = (a.z - o.z) + (b.z - o.z) + (c.z - o.z) + (d.z - o.z);
    return 0.25 * (cx * s.x + cy * s.y + cz * s.z);
}

// Shu-Osher coefficients (alpha, beta, gdt) of U^(s) = alpha U^n + beta
// U^(s-1) - gdt dt R / |Omega| for SSPRK(2,2), (3,3), (4,2)
const double RK[3][4][3] = {
    {{0.0, 1.0, 1.0}, {0.5, 0.5, 0.5}},
    {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}},
    {{0.0, 1.0, 1.0 / 3.0}, {0.0, 1.0, 1.0 / 3.0}, {0.0, 1.0, 1.0 / 3.0}, {0.25, 0.75, 0.25}},
};
const int RK_STAGES[3] = {2, 3, 4};

}  // namespace

struct sensei_host_block {
    int ni, nj, nk;
    long sj, sk, sv;   // state layout: element v*sv + (k+2)*sk + (j+2)*sj + (i+2)
    double gamma, kappa, eps, fix;
    int limiter, cons, threads;
    int bc[6];
    double prim[6][NV];
    // face metrics, node-grid layout (ni+1)(nj+1)(nk+1): unit normal and
    // area of the face of family d with lowest corner node (i, j, k)
    std::vector<double> fn[3][4];
    std::vector<double> vol, sbar[3][4];   // cell arrays [k][j][i]
    std::vector<double> U, st[2], W, R, Fk, Fj;

    long cell(int i, int j, int k) const { return (long)(k + NG) * sk + (long)(j + NG) * sj + (i + NG); }
    long node(int i, int j, int k) const { return ((long)k * (nj + 1) + j) * (ni + 1) + i; }
    long icell(int i, int j, int k) const { return ((long)k * nj + j) * ni + i; }
    double *slot(int s) { return s == 0 ? U.data() : st[s - 1].data(); }
};

namespace {

void set_threads(const sensei_host_block *h)
{
#ifdef _OPENMP
    omp_set_num_threads(h->threads);
#else
    (void)h;
#endif
}

void metrics(sensei_host_block *h, const double *X)
{
    const int ni = h->ni, nj = h->nj, nk = h->nk;
    const long nn = (long)(ni + 1) * (nj + 1) * (nk + 1);
    auto node = [&](int i, int j, int k) {
        const long q = h->node(i, j, k);
        return V3{X[q], X[nn + q], X[2 * nn + q]};
    };
    // corners of the face of family d at lowest node (i, j, k), the area
    // vector toward increasing index
    auto corners = [&](int d, int i, int j, int k, V3 p[4]) {
        p[0] = node(i, j, k);
        if (d == 0) {
            p[1] = node(i, j + 1, k);
            p[2] = node(i, j + 1, k + 1);
            p[3] = node(i, j, k + 1);
        } else if (d == 1) {
            p[1] = node(i, j, k + 1);
            p[2] = node(i + 1, j, k + 1);
            p[3] = node(i + 1, j, k);
        } else {
            p[1] = node(i + 1, j, k);
            p[2] = node(i + 1, j + 1, k);
            p[3] = node(i, j + 1, k);
        }
    };
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 4; ++q) h->fn[d][q].assign(nn, 0.0);
    const long nc = (long)ni * nj * nk;
    h->vol.assign(nc, 0.0);
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 4; ++q) h->sbar[d][q].assign(nc, 0.0);
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nk; ++k)
        for (int j = 0; j <= nj; ++j)
            for (int i = 0; i <= ni; ++i) {
                const bool has[3] = {j < nj && k < nk, i < ni && k < nk, i < ni && j < nj};
                const long m = h->node(i, j, k);
                for (int d = 0; d < 3; ++d) {
                    if (!has[d]) continue;
                    V3 p[4];
                    corners(d, i, j, k, p);
                    const V3 s = quad_area(p[0], p[1], p[2], p[3]);
                    const double a = sqrt(s.x * s.x + s.y * s.y + s.z * s.z);
                    const double inv = a > 0.0 ? 1.0 / a : 0.0;
                    h->fn[d][0][m] = s.x * inv;
                    h->fn[d][1][m] = s.y * inv;
                    h->fn[d][2][m] = s.z * inv;
                    h->fn[d][3][m] = a;
                }
                if (i < ni && j < nj && k < nk) {
                    const V3 o = node(i, j, k);
                    double v = 0.0;
                    const long c = h->icell(i, j, k);
                    for (int d = 0; d < 3; ++d) {
                        V3 lo[4], hi[4];
                        corners(d, i, j, k, lo);
                        corners(d, i + (d == 0), j + (d == 1), k + (d == 2), hi);
                        const V3 slo = quad_area(lo[0], lo[1], lo[2], lo[3]);
                        const V3 shi = quad_area(hi[0], hi[1], hi[2], hi[3]);
                        v += centroid_dot(hi[0], hi[1], hi[2], hi[3], o, shi) -
                             centroid_dot(lo[0], lo[1], lo[2], lo[3], o, slo);
                        const V3 sb{0.5 * (slo.x + shi.x), 0.5 * (slo.y + shi.y), 0.5 * (slo.z + shi.z)};
                        h->sbar[d][0][c] = sb.x;
                        h->sbar[d][1][c] = sb.y;
                        h->sbar[d][2][c] = sb.z;
                        h->sbar[d][3][c] = sqrt(sb.x * sb.x + sb.y * sb.y + sb.z * sb.z);
                    }
                    h->vol[c] = v / 3.0;
                }
            }
}

// ghost cell of layer g (1 next to the face) and interior cell m inside
// (0 = the boundary cell) of face f at tangential (t1, t2)
void face_cells(const sensei_host_block *h, int f, int t1, int t2, int g, int m, int &gi, int &gj, int &gk, int &mi,
                int &mj, int &mk)
{
    const int ni = h->ni, nj = h->nj, nk = h->nk;
    switch (f) {
    case 0: gi = -g; gj = t1; gk = t2; mi = m; mj = t1; mk = t2; break;
    case 1: gi = ni - 1 + g; gj = t1; gk = t2; mi = ni - 1 - m; mj = t1; mk = t2; break;
    case 2: gi = t1; gj = -g; gk = t2; mi = t1; mj = m; mk = t2; break;
    case 3: gi = t1; gj = nj - 1 + g; gk = t2; mi = t1; mj = nj - 1 - m; mk = t2; break;
    case 4: gi = t1; gj = t2; gk = -g; mi = t1; mj = t2; mk = m; break;
    default: gi = t1; gj = t2; gk = nk - 1 + g; mi = t1; mj = t2; mk = nk - 1 - m; break;
    }
}

void face_extent(const sensei_host_block *h, int f, int &n1, int &n2)
{
    n1 = f < 2 ? h->nj : h->ni;
    n2 = f < 4 ? h->nk : h->nj;
}

// unit normal of boundary face f at tangential (t1, t2)
void boundary_normal(const sensei_host_block *h, int f, int t1, int t2, double n[3])
{
    int i, j, k;
    if (f < 2) {
        i = f == 0 ? 0 : h->ni;
        j = t1;
        k = t2;
    } else if (f < 4) {
        i = t1;
        j = f == 2 ? 0 : h->nj;
        k = t2;
    } else {
        i = t1;
        j = t2;
        k = f == 4 ? 0 : h->nk;
    }
    const long m = h->node(i, j, k);
    for (int q = 0; q < 3; ++q) n[q] = h->fn[f >> 1][q][m];
}

void fill_ghosts(sensei_host_block *h, double *u)
{
    for (int f = 0; f < 6; ++f) {
        const int type = h->bc[f];
        if (type == SENSEI_BC_EXTERNAL) continue;
        int n1, n2;
        face_extent(h, f, n1, n2);
#pragma omp parallel for schedule(static)
        for (int t2 = 0; t2 < n2; ++t2)
            for (int t1 = 0; t1 < n1; ++t1)
                for (int g = 1; g <= NG; ++g) {
                    int gi, gj, gk, mi, mj, mk, a, b, c;
                    face_cells(h, f, t1, t2, g, 0, gi, gj, gk, a, b, c);
                    double q[NV];
                    if (type == SENSEI_BC_PERIODIC || type == SENSEI_BC_SLIP_WALL) {
                        const int src = type == SENSEI_BC_PERIODIC ? (f ^ 1) : f;
                        face_cells(h, src, t1, t2, 1, g - 1, a, b, c, mi, mj, mk);
                        const long sc = h->cell(mi, mj, mk);
                        for (int v = 0; v < NV; ++v) q[v] = u[v * h->sv + sc];
                        if (type == SENSEI_BC_SLIP_WALL) {
                            double n[3];
                            boundary_normal(h, f, t1, t2, n);
                            const double mn = q[1] * n[0] + q[2] * n[1] + q[3] * n[2];
                            q[1] -= 2.0 * mn * n[0];
                            q[2] -= 2.0 * mn * n[1];
                            q[3] -= 2.0 * mn * n[2];
                        }
                    } else if (type == SENSEI_BC_EXTRAPOLATE) {
                        const long sc = h->cell(a, b, c);
                        for (int v = 0; v < NV; ++v) q[v] = u[v * h->sv + sc];
                    } else {   // inflow: the fixed freestream
                        const double *w = h->prim[f];
                        q[0] = w[0];
                        q[1] = w[0] * w[1];
                        q[2] = w[0] * w[2];
                        q[3] = w[0] * w[3];
                        q[4] = w[4] / (h->gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
                    }
                    const long gc = h->cell(gi, gj, gk);
                    for (int v = 0; v < NV; ++v) u[v * h->sv + gc] = q[v];
                }
    }
}

// reconstruction variables of every cell with its ghost layers in i, j, k
// (primitive W = (rho, u, v, w, p), or the conserved Q)
void recon_vars(sensei_host_block *h, const double *u)
{
    const long sv = h->sv;
    const double gm1 = h->gamma - 1.0;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = -NG; k < h->nk + NG; ++k)
        for (int j = -NG; j < h->nj + NG; ++j) {
            const long c0 = h->cell(-NG, j, k);
            for (int i = 0; i < h->ni + 2 * NG; ++i) {
                const long c = c0 + i;
                const double r = u[c], mx = u[sv + c], my = u[2 * sv + c], mz = u[3 * sv + c], e = u[4 * sv + c];
                if (h->cons) {
                    h->W[c] = r;
                    h->W[sv + c] = mx;
                    h->W[2 * sv + c] = my;
                    h->W[3 * sv + c] = mz;
                    h->W[4 * sv + c] = e;
                } else {
                    const double ir = 1.0 / r;
                    const double vx = mx * ir, vy = my * ir, vz = mz * ir;
                    h->W[c] = r;
                    h->W[sv + c] = vx;
                    h->W[2 * sv + c] = vy;
                    h->W[3 * sv + c] = vz;
                    h->W[4 * sv + c] = gm1 * (e - 0.5 * (mx * vx + my * vy + mz * vz));
                }
            }
        }
}

// MUSCL: plus state of cell 1 and minus state of cell 2 of a line w0..w3
inline void line_states(const sensei_host_block *h, double w0, double w1, double w2, double w3, double &L, double &R)
{
    const double dm = w1 - w0, d0 = w2 - w1, dp = w3 - w2;
    if (h->limiter == SENSEI_LIM_NONE) {
        const double c1 = h->eps * (1.0 - h->kappa) * 0.25, c2 = h->eps * (1.0 + h->kappa) * 0.25;
        L = w1 + (c1 * dm + c2 * d0);
        R = w2 - (c2 * d0 + c1 * dp);
        return;
    }
    double s1, s2;
    if (h->limiter == SENSEI_LIM_MINMOD) {
        auto mm = [](double a, double b) { return a * b > 0.0 ? (fabs(a) <= fabs(b) ? a : b) : 0.0; };
        s1 = mm(dm, d0);
        s2 = mm(d0, dp);
    } else {
        auto vl = [](double a, double b) { return a * b > 0.0 ? 2.0 * a * b / (a + b) : 0.0; };
        s1 = vl(dm, d0);
        s2 = vl(d0, dp);
    }
    L = w1 + 0.5 * h->eps * s1;
    R = w2 - 0.5 * h->eps * s2;
}

inline void to_prim(double gm1, const double q[NV], double w[NV])
{
    const double ir = 1.0 / q[0];
    w[0] = q[0];
    w[1] = q[1] * ir;
    w[2] = q[2] * ir;
    w[3] = q[3] * ir;
    w[4] = gm1 * (q[4] - 0.5 * (q[1] * w[1] + q[2] * w[2] + q[3] * w[3]));
}

// Roe flux A [ (F(W_L) + F(W_R)) / 2 - sum_k |lam_k| alpha_k r_k / 2 ] through
// a face of unit normal n and area A, Harten's fix |lam| < delta = fix a =>
// (lam^2 / delta + delta) / 2 on the acoustic waves
inline void roe_flux(const sensei_host_block *h, const double wl[NV], const double wr[NV], const double n[3], double A,
                     double F[NV])
{
    const double g = h->gamma, gm1 = g - 1.0;
    const double rl = wl[0], ul = wl[1], vl = wl[2], zl = wl[3], pl = wl[4];
    const double rr = wr[0], ur = wr[1], vr = wr[2], zr = wr[3], pr = wr[4];
    const double vnl = n[0] * ul + n[1] * vl + n[2] * zl, vnr = n[0] * ur + n[1] * vr + n[2] * zr;
    const double hl = g / gm1 * pl / rl + 0.5 * (ul * ul + vl * vl + zl * zl);
    const double hr = g / gm1 * pr / rr + 0.5 * (ur * ur + vr * vr + zr * zr);
    const double s = sqrt(rr / rl), wgt = 1.0 / (1.0 + s);
    const double rho = sqrt(rl * rr);
    const double u = (ul + s * ur) * wgt, v = (vl + s * vr) * wgt, w = (zl + s * zr) * wgt;
    const double H = (hl + s * hr) * wgt;
    const double q2 = u * u + v * v + w * w;
    const double a = sqrt(gm1 * (H - 0.5 * q2));
    const double vn = n[0] * u + n[1] * v + n[2] * w;
    const double dr = rr - rl, dp = pr - pl, dvn = vnr - vnl;
    double l1 = fabs(vn - a), l2 = fabs(vn), l3 = fabs(vn + a);
    const double delta = h->fix * a;
    if (l1 < delta) l1 = 0.5 * (l1 * l1 / delta + delta);
    if (l3 < delta) l3 = 0.5 * (l3 * l3 / delta + delta);
    const double a2 = a * a;
    const double c1 = l1 * (dp - rho * a * dvn) / (2.0 * a2);
    const double c3 = l3 * (dp + rho * a * dvn) / (2.0 * a2);
    const double c2 = l2 * (dr - dp / a2);
    const double du[3] = {ur - ul - dvn * n[0], vr - vl - dvn * n[1], zr - zl - dvn * n[2]};
    const double vel[3] = {u, v, w};
    double D[NV];
    D[0] = c1 + c2 + c3;
    for (int q = 0; q < 3; ++q)
        D[1 + q] = c1 * (vel[q] - a * n[q]) + c2 * vel[q] + c3 * (vel[q] + a * n[q]) + l2 * rho * du[q];
    D[4] = c1 * (H - a * vn) + c2 * 0.5 * q2 + c3 * (H + a * vn) +
           l2 * rho * (u * du[0] + v * du[1] + w * du[2]);
    const double ml = rl * vnl, mr = rr * vnr;
    const double fl[NV] = {ml, ml * ul + pl * n[0], ml * vl + pl * n[1], ml * zl + pl * n[2], rl * hl * vnl};
    const double fr[NV] = {mr, mr * ur + pr * n[0], mr * vr + pr * n[1], mr * zr + pr * n[2], rr * hr * vnr};
    for (int q = 0; q < NV; ++q) F[q] = 0.5 * A * ((fl[q] + fr[q]) - D[q]);
}

// the face flux between cells c and c + st of the reconstruction-variable
// array (line c - st .. c + 2 st), metrics at node index m of family d
inline void face_flux(const sensei_host_block *h, long c, long st, int d, long m, double F[NV])
{
    const long sv = h->sv;
    double L[NV], R[NV];
    for (int v = 0; v < NV; ++v) {
        const double *w = h->W.data() + v * sv + c;
        line_states(h, w[-st], w[0], w[st], w[2 * st], L[v], R[v]);
    }
    const double n[3] = {h->fn[d][0][m], h->fn[d][1][m], h->fn[d][2][m]};
    if (h->cons) {
        double wl[NV], wr[NV];
        to_prim(h->gamma - 1.0, L, wl);
        to_prim(h->gamma - 1.0, R, wr);
        roe_flux(h, wl, wr, n, h->fn[d][3][m], F);
    } else {
        roe_flux(h, L, R, n, h->fn[d][3][m], F);
    }
}

// R = sum over the six faces of F.S_out (Eq. residual) of the slot's state
// (ghosts in place) into h->R [v][k][j][i]: the k- and j-face fluxes of
// every face first, then per row the i-face fluxes and the sums; every pass
// shares its (k, j) rows out among the host threads
void residual(sensei_host_block *h, const double *u)
{
    const int ni = h->ni, nj = h->nj, nk = h->nk;
    const long nc = (long)ni * nj * nk, plane = (long)ni * nj;
    const long fkv = (long)(nk + 1) * plane;           // variable stride of Fk
    const long fjv = (long)nk * (nj + 1) * ni;          // variable stride of Fj
    recon_vars(h, u);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k <= nk; ++k)
        for (int j = 0; j < nj; ++j)
            for (int i = 0; i < ni; ++i) {
                double F[NV];
                face_flux(h, h->cell(i, j, k - 1), h->sk, 2, h->node(i, j, k), F);
                for (int v = 0; v < NV; ++v) h->Fk[v * fkv + (long)k * plane + (long)j * ni + i] = F[v];
            }
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j <= nj; ++j)
            for (int i = 0; i < ni; ++i) {
                double F[NV];
                face_flux(h, h->cell(i, j - 1, k), h->sj, 1, h->node(i, j, k), F);
                for (int v = 0; v < NV; ++v) h->Fj[v * fjv + ((long)k * (nj + 1) + j) * ni + i] = F[v];
            }
#pragma omp parallel
    {
        std::vector<double> fi((size_t)NV * (ni + 1));
#pragma omp for collapse(2) schedule(static)
        for (int k = 0; k < nk; ++k)
            for (int j = 0; j < nj; ++j) {
                for (int i = 0; i <= ni; ++i) {
                    double F[NV];
                    face_flux(h, h->cell(i - 1, j, k), 1, 0, h->node(i, j, k), F);
                    for (int v = 0; v < NV; ++v) fi[(size_t)v * (ni + 1) + i] = F[v];
                }
                for (int i = 0; i < ni; ++i) {
                    const long c = h->icell(i, j, k);
                    for (int v = 0; v < NV; ++v) {
                        const double *fk = h->Fk.data() + v * fkv;
                        const double *fj = h->Fj.data() + v * fjv + (long)k * (nj + 1) * ni;
                        double r = fi[(size_t)v * (ni + 1) + i + 1] - fi[(size_t)v * (ni + 1) + i];
                        r += fj[(long)(j + 1) * ni + i] - fj[(long)j * ni + i];
                        r += fk[(long)(k + 1) * plane + (long)j * ni + i] - fk[(long)k * plane + (long)j * ni + i];
                        h->R[(long)v * nc + c] = r;
                    }
                }
            }
    }
}

}  // namespace

extern "C" {

sensei_status sensei_host_create(int ni, int nj, int nk, const double *nodes, const sensei_scheme *scheme, int threads,
                                 sensei_host_block **out)
{
    if (!out) return SENSEI_ERR_INVALID_ARG;
    *out = nullptr;
    if (ni < NG || nj < NG || nk < NG || !nodes || !scheme || threads < 1) return SENSEI_ERR_INVALID_ARG;
    if (scheme->precision != SENSEI_FP64 || scheme->mu != 0.0) return SENSEI_ERR_UNSUPPORTED;
    if (!(scheme->gamma > 1.0) || scheme->limiter < SENSEI_LIM_NONE || scheme->limiter > SENSEI_LIM_VANLEER)
        return SENSEI_ERR_INVALID_ARG;
    sensei_host_block *h = new (std::nothrow) sensei_host_block();
    if (!h) return SENSEI_ERR_INVALID_ARG;
    h->ni = ni;
    h->nj = nj;
    h->nk = nk;
    h->sj = ni + 2 * NG;
    h->sk = h->sj * (nj + 2 * NG);
    h->sv = h->sk * (nk + 2 * NG);
    h->gamma = scheme->gamma;
    h->kappa = scheme->kappa;
    h->eps = scheme->eps;
    h->fix = scheme->entropy_fix;
    h->limiter = scheme->limiter;
    h->cons = scheme->reconstruct_conserved ? 1 : 0;
    h->threads = threads;
    for (int f = 0; f < 6; ++f) h->bc[f] = -1;
    set_threads(h);
    metrics(h, nodes);
    const size_t n = (size_t)NV * h->sv;
    h->U.assign(n, 0.0);
    h->st[0].assign(n, 0.0);
    h->st[1].assign(n, 0.0);
    h->W.assign(n, 0.0);
    h->R.assign((size_t)NV * ni * nj * nk, 0.0);
    h->Fk.assign((size_t)NV * (nk + 1) * ni * nj, 0.0);
    h->Fj.assign((size_t)NV * nk * (nj + 1) * ni, 0.0);
    *out = h;
    return SENSEI_OK;
}

sensei_status sensei_host_destroy(sensei_host_block *h)
{
    delete h;
    return SENSEI_OK;
}

sensei_status sensei_host_set_bc(sensei_host_block *h, int face, int type, const double *prim)
{
    if (!h || face < 0 || face > 5) return SENSEI_ERR_INVALID_ARG;
    if (type != SENSEI_BC_PERIODIC && type != SENSEI_BC_INFLOW && type != SENSEI_BC_EXTRAPOLATE &&
        type != SENSEI_BC_SLIP_WALL && type != SENSEI_BC_EXTERNAL)
        return SENSEI_ERR_INVALID_ARG;
    if (type == SENSEI_BC_INFLOW) {
        if (!prim) return SENSEI_ERR_INVALID_ARG;
        for (int v = 0; v < NV; ++v) h->prim[face][v] = prim[v];
    }
    h->bc[face] = type;
    return SENSEI_OK;
}

sensei_status sensei_host_layout(const sensei_host_block *h, sensei_layout *out)
{
    if (!h || !out) return SENSEI_ERR_INVALID_ARG;
    out->stride_j = h->sj;
    out->stride_k = h->sk;
    out->stride_var = h->sv;
    out->offset = (long long)NG * h->sk + NG * h->sj + NG;
    out->elems = (long long)NV * h->sv;
    out->ghost_i = NG;
    out->ghost_j = NG;
    out->ghost_k = NG;
    out->elem_bytes = (int)sizeof(double);
    return SENSEI_OK;
}

double *sensei_host_state(sensei_host_block *h) { return h ? h->U.data() : nullptr; }

sensei_status sensei_host_fill_ghosts(sensei_host_block *h)
{
    if (!h) return SENSEI_ERR_INVALID_ARG;
    for (int f = 0; f < 6; ++f)
        if (h->bc[f] < 0) return SENSEI_ERR_STATE;
    set_threads(h);
    fill_ghosts(h, h->U.data());
    return SENSEI_OK;
}

sensei_status sensei_host_residual(sensei_host_block *h, double *R)
{
    if (!h || !R) return SENSEI_ERR_INVALID_ARG;
    sensei_status st = sensei_host_fill_ghosts(h);
    if (st != SENSEI_OK) return st;
    residual(h, h->U.data());
    memcpy(R, h->R.data(), sizeof(double) * h->R.size());
    return SENSEI_OK;
}

sensei_status sensei_host_dt_min(sensei_host_block *h, double cfl, double *out)
{
    if (!h || !out || !(cfl > 0.0)) return SENSEI_ERR_INVALID_ARG;
    set_threads(h);
    const int ni = h->ni, nj = h->nj, nk = h->nk;
    const double *u = h->U.data();
    const long sv = h->sv;
    double best = INFINITY;
#pragma omp parallel for collapse(2) schedule(static) reduction(min : best)
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j)
            for (int i = 0; i < ni; ++i) {
                const long c = h->cell(i, j, k), ic = h->icell(i, j, k);
                double q[NV], w[NV];
                for (int v = 0; v < NV; ++v) q[v] = u[v * sv + c];
                to_prim(h->gamma - 1.0, q, w);
                const double a = sqrt(h->gamma * w[4] / w[0]);
                double sum = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double un = w[1] * h->sbar[d][0][ic] + w[2] * h->sbar[d][1][ic] + w[3] * h->sbar[d][2][ic];
                    sum += fabs(un) + a * h->sbar[d][3][ic];
                }
                best = std::min(best, h->vol[ic] / sum);
            }
    *out = cfl * best;
    return SENSEI_OK;
}

sensei_status sensei_host_stage(sensei_host_block *h, int rk, int stage, double dt)
{
    if (!h || rk < SENSEI_RK2_SSP || rk > SENSEI_RK4_SSP2 || !(dt > 0.0)) return SENSEI_ERR_INVALID_ARG;
    const int S = RK_STAGES[rk];
    if (stage < 0 || stage >= S) return SENSEI_ERR_INVALID_ARG;
    for (int f = 0; f < 6; ++f)
        if (h->bc[f] < 0) return SENSEI_ERR_STATE;
    set_threads(h);
    // stage inputs U -> ST0 -> ST1 -> ST0 ..., the last stage writes U
    double *in = stage == 0 ? h->U.data() : h->st[(stage - 1) % 2].data();
    double *out = stage == S - 1 ? h->U.data() : h->st[stage % 2].data();
    const double *co = RK[rk][stage];
    fill_ghosts(h, in);
    residual(h, in);
    // U^n lives in U until the last stage overwrites it (every other stage
    // writes a stage buffer)
    const double *un = h->U.data();
    const int ni = h->ni, nj = h->nj, nk = h->nk;
    const long nc = (long)ni * nj * nk, sv = h->sv;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j)
            for (int i = 0; i < ni; ++i) {
                const long c = h->cell(i, j, k), ic = h->icell(i, j, k);
                const double f = -co[2] * dt / h->vol[ic];
                for (int v = 0; v < NV; ++v) {
                    double x = co[1] * in[v * sv + c] + f * h->R[(long)v * nc + ic];
                    if (co[0] != 0.0) x += co[0] * un[v * sv + c];
                    out[v * sv + c] = x;
                }
            }
    return SENSEI_OK;
}

sensei_status sensei_host_face_exchange(sensei_host_block *h, int stage, int face, double *buf, int unpack)
{
    if (!h || !buf || face < 0 || face > 5 || stage < 0 || stage > 3) return SENSEI_ERR_INVALID_ARG;
    set_threads(h);
    // the state a stage reads: U for stage 0, else the previous stage's buffer
    double *u = stage == 0 ? h->U.data() : h->st[(stage - 1) % 2].data();
    int n1, n2;
    face_extent(h, face, n1, n2);
    const long per = (long)NG * n1 * n2;
    // one (variable, layer, t2) row of n1 cells per iteration: along i
    // (j- and k-faces) a contiguous row, along j (i-faces) stride sj
#pragma omp parallel for collapse(3) schedule(static)
    for (int v = 0; v < NV; ++v)
        for (int l = 0; l < NG; ++l)
            for (int t2 = 0; t2 < n2; ++t2) {
                int gi, gj, gk, mi, mj, mk;
                face_cells(h, face, 0, t2, l + 1, l, gi, gj, gk, mi, mj, mk);
                const long st = face < 2 ? h->sj : 1;
                double *row = u + v * h->sv + (unpack ? h->cell(gi, gj, gk) : h->cell(mi, mj, mk));
                double *b = buf + (long)v * per + ((long)l * n2 + t2) * n1;
                if (unpack)
                    for (int t1 = 0; t1 < n1; ++t1) row[t1 * st] = b[t1];
                else
                    for (int t1 = 0; t1 < n1; ++t1) b[t1] = row[t1 * st];
            }
    return SENSEI_OK;
}

}  // extern "C"
