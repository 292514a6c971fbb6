/*
 * sensei_oracle.c -- plain FP64 CPU oracle for the explicit finite-volume
 * Euler residual and Runge-Kutta stage update of the SENSEI solver
 * (arXiv 2305.18057, Sec. 2 "Finite Volume CFD Solver", Sec. 3
 * "Discretization", and the MUSCL paragraph of Sec. 5).
 *
 * TEST INFRASTRUCTURE.  This is the reference the CUDA library is checked
 * against.  Only the tests, __graft_entry__.smoke() and the CPU-baseline leg
 * of bench.py load it.  It shares no source, header, table or helper with the
 * CUDA path, and the CUDA path never calls it.
 *
 * Style: IEEE double everywhere, scalar loops in the order the paper states
 * the method, compiled with -O2 -ffp-contract=off (no fused multiply-add, so
 * every product and sum rounds exactly as written).  Nothing here is blocked,
 * fused or reordered for speed.
 *
 * Layout conventions (all arrays C-ordered, variable index slowest):
 *   nodes   X[3][nk+1][nj+1][ni+1]            (x, y, z of the grid nodes)
 *   state   U[5][nk+2gk][nj+4][ni+4]          (conserved Q of Eq. governing,
 *                                              2 ghost layers per side; gk=2 in
 *                                              3D, gk=0 in 2D where nk==1)
 *   interior R[5][nk][nj][ni]
 *   i-faces Si[3][nk][nj][ni+1], j-faces Sj[3][nk][nj+1][ni],
 *   k-faces Sk[3][nk+1][nj][ni], volumes vol[nk][nj][ni].
 * A 2D block is a one-cell-deep slab (nk == 1); it has f = 4 faces per cell
 * (Eq. residual), so its k-faces are never used.
 *
 * Threads: built with OpenMP, the loops over k-planes whose iterations are
 * independent (every face flux, the per-cell sums of Eq. residual, the
 * Runge-Kutta stage and final updates, the local time steps) may run on
 * several host threads (ora_set_threads; 1 by default).  Each iteration
 * computes the same values in the same order whatever the thread count;
 * the reductions (norms, the global time-step minimum) stay serial, so the
 * results are bitwise independent of the thread count.
 *
 * Parity status: every routine here is pinned by a CPU test (closed forms,
 * invariants, exact Riemann and oblique-shock solutions, brute force); see
 * tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 5   /* rho, rho*u, rho*v, rho*w, rho*e_t  (Eq. governing, vector Q) */
#define NG 2   /* ghost layers: the MUSCL stencil of Eq. flux reaches i-1..i+2 */

enum { ORA_BC_PERIODIC = 0, ORA_BC_INFLOW = 1, ORA_BC_EXTRAPOLATE = 2,
       ORA_BC_SLIP_WALL = 3, ORA_BC_INTERFACE = 4, ORA_BC_UNSET = -1 };
enum { ORA_LIM_NONE = 0, ORA_LIM_MINMOD = 1, ORA_LIM_VANLEER = 2 };
enum { ORA_RK2_SSP = 0, ORA_RK3_SSP = 1, ORA_RK4_SSP2 = 2 };

typedef struct {
    int ni, nj, nk, gk;
    long sj, sk, sv;                 /* strides of the ghosted cell arrays */
    double *Si, *Sj, *Sk, *vol;      /* metrics, owned */
    int bc_type[6];
    double bc_prim[6][NV];
    int bc_nbr[6], bc_nbr_face[6];
} ora_block;

typedef struct {
    int nb;
    ora_block *b;
    double gamma;
    int limiter;
    double kappa, eps;
    int recon_conserved;
    double fix_delta;                /* Harten entropy-fix width, times the Roe sound speed */
    double mu, prandtl;              /* viscous flux F_nu (mu = 0: Euler) */
} ora_grid;

/* ------------------------------------------------------------------------ */
/* indexing                                                                  */
/* ------------------------------------------------------------------------ */

static long cell(const ora_block *b, int i, int j, int k)
{
    return (long)(k + b->gk) * b->sk + (long)(j + NG) * b->sj + (long)(i + NG);
}

static long node_index(const ora_block *b, int i, int j, int k)
{
    return ((long)k * (b->nj + 1) + j) * (b->ni + 1) + i;
}

static long interior(const ora_block *b, int i, int j, int k)
{
    return ((long)k * b->nj + j) * b->ni + i;
}

static long n_interior(const ora_block *b)
{
    return (long)b->ni * b->nj * b->nk;
}

static int is2d(const ora_block *b) { return b->nk == 1; }

/* i-faces: index i in 0..ni, cell i-1 on the minus side, cell i on the plus side */
static long fi_index(const ora_block *b, int i, int j, int k)
{
    return ((long)k * b->nj + j) * (b->ni + 1) + i;
}
static long fj_index(const ora_block *b, int i, int j, int k)
{
    return ((long)k * (b->nj + 1) + j) * b->ni + i;
}
static long fk_index(const ora_block *b, int i, int j, int k)
{
    return ((long)k * b->nj + j) * b->ni + i;
}
static long n_fi(const ora_block *b) { return (long)b->nk * b->nj * (b->ni + 1); }
static long n_fj(const ora_block *b) { return (long)b->nk * (b->nj + 1) * b->ni; }
static long n_fk(const ora_block *b) { return (long)(b->nk + 1) * b->nj * b->ni; }

/* ------------------------------------------------------------------------ */
/* geometry: face area vectors and cell volumes (Delta s, n, |Omega| of      */
/* Eq. residual and Eq. spatial_residual)                                    */
/* ------------------------------------------------------------------------ */

static void get_node(const double *X, const ora_block *b, int i, int j, int k, double p[3])
{
    long n = (long)(b->ni + 1) * (b->nj + 1) * (b->nk + 1);
    long q = node_index(b, i, j, k);
    p[0] = X[q];
    p[1] = X[n + q];
    p[2] = X[2 * n + q];
}

static void sub3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[0] - b[0];
    r[1] = a[1] - b[1];
    r[2] = a[2] - b[2];
}

static void cross3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* Area vector of the quadrilateral with corners p0,p1,p2,p3 in cyclic order:
 * half the cross product of its diagonals, (p2-p0) x (p3-p1) / 2.  It is the
 * exact area vector of the bilinear face through the four nodes. */
static void quad_area(const double p0[3], const double p1[3], const double p2[3],
                      const double p3[3], double S[3])
{
    double d1[3], d2[3], c[3];
    sub3(p2, p0, d1);
    sub3(p3, p1, d2);
    cross3(d1, d2, c);
    S[0] = 0.5 * c[0];
    S[1] = 0.5 * c[1];
    S[2] = 0.5 * c[2];
}

/* Centroid of the four corners measured from the point o: the corners'
 * offsets from o are formed first (exact for nearby points), then averaged. */
static void quad_centroid_from(const double p0[3], const double p1[3], const double p2[3],
                               const double p3[3], const double o[3], double c[3])
{
    for (int a = 0; a < 3; ++a)
        c[a] = 0.25 * ((p0[a] - o[a]) + (p1[a] - o[a]) + (p2[a] - o[a]) + (p3[a] - o[a]));
}

/* The corner nodes of the three face families, ordered so that the area
 * vector points toward increasing i, j or k on a right-handed grid. */
static void iface_nodes(const double *X, const ora_block *b, int i, int j, int k, double p[4][3])
{
    get_node(X, b, i, j, k, p[0]);
    get_node(X, b, i, j + 1, k, p[1]);
    get_node(X, b, i, j + 1, k + 1, p[2]);
    get_node(X, b, i, j, k + 1, p[3]);
}
static void jface_nodes(const double *X, const ora_block *b, int i, int j, int k, double p[4][3])
{
    get_node(X, b, i, j, k, p[0]);
    get_node(X, b, i, j, k + 1, p[1]);
    get_node(X, b, i + 1, j, k + 1, p[2]);
    get_node(X, b, i + 1, j, k, p[3]);
}
static void kface_nodes(const double *X, const ora_block *b, int i, int j, int k, double p[4][3])
{
    get_node(X, b, i, j, k, p[0]);
    get_node(X, b, i + 1, j, k, p[1]);
    get_node(X, b, i + 1, j + 1, k, p[2]);
    get_node(X, b, i, j + 1, k, p[3]);
}

static void compute_metrics(ora_block *b, const double *X)
{
    double p[4][3], S[3], c[3];
    long nfi = n_fi(b), nfj = n_fj(b), nfk = n_fk(b);
    for (int k = 0; k < b->nk; ++k)
        for (int j = 0; j < b->nj; ++j)
            for (int i = 0; i <= b->ni; ++i) {
                iface_nodes(X, b, i, j, k, p);
                quad_area(p[0], p[1], p[2], p[3], S);
                for (int a = 0; a < 3; ++a) b->Si[a * nfi + fi_index(b, i, j, k)] = S[a];
            }
    for (int k = 0; k < b->nk; ++k)
        for (int j = 0; j <= b->nj; ++j)
            for (int i = 0; i < b->ni; ++i) {
                jface_nodes(X, b, i, j, k, p);
                quad_area(p[0], p[1], p[2], p[3], S);
                for (int a = 0; a < 3; ++a) b->Sj[a * nfj + fj_index(b, i, j, k)] = S[a];
            }
    for (int k = 0; k <= b->nk; ++k)
        for (int j = 0; j < b->nj; ++j)
            for (int i = 0; i < b->ni; ++i) {
                kface_nodes(X, b, i, j, k, p);
                quad_area(p[0], p[1], p[2], p[3], S);
                for (int a = 0; a < 3; ++a) b->Sk[a * nfk + fk_index(b, i, j, k)] = S[a];
            }
    /* |Omega| = (1/3) * sum over the six faces of  centroid . outward area
     * vector (divergence theorem applied to the position vector).  The
     * position is measured from the cell's corner node (i, j, k): the closed
     * surface's area vectors sum to zero, so any origin gives the same
     * volume, and a corner of the cell keeps every term of the cell's own
     * size (measured from the coordinate origin, terms of size |x| h^2 would
     * cancel to a volume h^3, losing a factor |x|/h of accuracy). */
    for (int k = 0; k < b->nk; ++k)
        for (int j = 0; j < b->nj; ++j)
            for (int i = 0; i < b->ni; ++i) {
                double o[3];
                get_node(X, b, i, j, k, o);
                double v = 0.0;
                for (int side = 0; side < 2; ++side) {
                    double sgn = side ? 1.0 : -1.0;
                    iface_nodes(X, b, i + side, j, k, p);
                    quad_area(p[0], p[1], p[2], p[3], S);
                    quad_centroid_from(p[0], p[1], p[2], p[3], o, c);
                    v += sgn * (c[0] * S[0] + c[1] * S[1] + c[2] * S[2]);
                    jface_nodes(X, b, i, j + side, k, p);
                    quad_area(p[0], p[1], p[2], p[3], S);
                    quad_centroid_from(p[0], p[1], p[2], p[3], o, c);
                    v += sgn * (c[0] * S[0] + c[1] * S[1] + c[2] * S[2]);
                    kface_nodes(X, b, i, j, k + side, p);
                    quad_area(p[0], p[1], p[2], p[3], S);
                    quad_centroid_from(p[0], p[1], p[2], p[3], o, c);
                    v += sgn * (c[0] * S[0] + c[1] * S[1] + c[2] * S[2]);
                }
                b->vol[interior(b, i, j, k)] = v / 3.0;
            }
}

/* ------------------------------------------------------------------------ */
/* thermodynamics: Q <-> primitive W = (rho, u, v, w, p), calorically perfect */
/* gas, e_t = p/((gamma-1) rho) + |u|^2/2,  h_t = e_t + p/rho  (Sec. 2)      */
/* ------------------------------------------------------------------------ */

static void cons_to_prim(double gamma, const double Q[NV], double W[NV])
{
    double rho = Q[0];
    double u = Q[1] / rho, v = Q[2] / rho, w = Q[3] / rho;
    W[0] = rho;
    W[1] = u;
    W[2] = v;
    W[3] = w;
    W[4] = (gamma - 1.0) * (Q[4] - 0.5 * rho * (u * u + v * v + w * w));
}

static void prim_to_cons(double gamma, const double W[NV], double Q[NV])
{
    double rho = W[0];
    Q[0] = rho;
    Q[1] = rho * W[1];
    Q[2] = rho * W[2];
    Q[3] = rho * W[3];
    Q[4] = W[4] / (gamma - 1.0) + 0.5 * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

/* ------------------------------------------------------------------------ */
/* MUSCL extrapolation, Eq. flux (Sec. 5), written as printed: kappa-scheme  */
/* with limiter values Psi of consecutive-difference ratios.                 */
/*                                                                          */
/* Reading (the paper does not define r or Psi): Psi^+_{f} limits the       */
/* difference across face f by the ratio (next difference)/(difference at f) */
/* and Psi^-_{f} by (previous difference)/(difference at f).  The product   */
/* Psi(num/den)*den is taken as 0 when den == 0 (the limited slope of a flat */
/* difference is zero).                                                     */
/* ------------------------------------------------------------------------ */

static double psi(int limiter, double r)
{
    switch (limiter) {
    case ORA_LIM_MINMOD: return fmax(0.0, fmin(1.0, r));
    case ORA_LIM_VANLEER: return (r + fabs(r)) / (1.0 + fabs(r));
    default: return 1.0;
    }
}

static double psi_times(int limiter, double num, double den)
{
    if (limiter == ORA_LIM_NONE) return den;
    if (den == 0.0) return 0.0;
    return psi(limiter, num / den) * den;
}

/* Left and right states at face i+1/2 from q[0..3] = Q_{i-1}, Q_i, Q_{i+1}, Q_{i+2}. */
static void muscl_face(int limiter, double kappa, double eps, const double q[4],
                       double *qL, double *qR)
{
    double dm = q[1] - q[0];   /* Q_i     - Q_{i-1}  (difference at face i-1/2) */
    double d0 = q[2] - q[1];   /* Q_{i+1} - Q_i      (difference at face i+1/2) */
    double dp = q[3] - q[2];   /* Q_{i+2} - Q_{i+1}  (difference at face i+3/2) */
    double plus_im = psi_times(limiter, d0, dm);   /* Psi^+_{i-1/2} (Q_i - Q_{i-1})     */
    double minus_ip = psi_times(limiter, dm, d0);  /* Psi^-_{i+1/2} (Q_{i+1} - Q_i)     */
    double plus_ip = psi_times(limiter, dp, d0);   /* Psi^+_{i+1/2} (Q_{i+1} - Q_i)     */
    double minus_ipp = psi_times(limiter, d0, dp); /* Psi^-_{i+3/2} (Q_{i+2} - Q_{i+1}) */
    *qL = q[1] + eps / 4.0 * ((1.0 - kappa) * plus_im + (1.0 + kappa) * minus_ip);
    *qR = q[2] - eps / 4.0 * ((1.0 + kappa) * plus_ip + (1.0 - kappa) * minus_ipp);
}

/* ------------------------------------------------------------------------ */
/* inviscid normal flux F_{i,n} of Eq. governing and the Roe flux            */
/* ------------------------------------------------------------------------ */

/* F_{i,n}(W) for the unit normal n (Eq. governing, second vector). */
static void euler_flux(double gamma, const double W[NV], const double n[3], double F[NV])
{
    double rho = W[0], u = W[1], v = W[2], w = W[3], p = W[4];
    double Vn = n[0] * u + n[1] * v + n[2] * w;
    double rho_et = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
    double rho_ht = rho_et + p;
    F[0] = rho * Vn;
    F[1] = rho * u * Vn + n[0] * p;
    F[2] = rho * v * Vn + n[1] * p;
    F[3] = rho * w * Vn + n[2] * p;
    F[4] = rho_ht * Vn;
}

typedef struct {
    double lam[3];          /* V_n - a, V_n, V_n + a at the Roe average */
    double a, rho, u, v, w, H, Vn, q2;
    double dp, dVn, drho, du, dv, dw;
} roe_state;

/* Roe-averaged state and jumps between W_L and W_R across the unit normal n
 * (the paper names no flux function; the Roe approximate Riemann solver in
 * its three-wave form is the reading used here). */
static void roe_average(double gamma, const double WL[NV], const double WR[NV],
                        const double n[3], roe_state *s)
{
    double HL = (WL[4] / (gamma - 1.0) + 0.5 * WL[0] * (WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3]) + WL[4]) / WL[0];
    double HR = (WR[4] / (gamma - 1.0) + 0.5 * WR[0] * (WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3]) + WR[4]) / WR[0];
    double R = sqrt(WR[0] / WL[0]);
    s->rho = R * WL[0];
    s->u = (WL[1] + R * WR[1]) / (1.0 + R);
    s->v = (WL[2] + R * WR[2]) / (1.0 + R);
    s->w = (WL[3] + R * WR[3]) / (1.0 + R);
    s->H = (HL + R * HR) / (1.0 + R);
    s->q2 = s->u * s->u + s->v * s->v + s->w * s->w;
    s->a = sqrt((gamma - 1.0) * (s->H - 0.5 * s->q2));
    s->Vn = n[0] * s->u + n[1] * s->v + n[2] * s->w;
    s->lam[0] = s->Vn - s->a;
    s->lam[1] = s->Vn;
    s->lam[2] = s->Vn + s->a;
    s->drho = WR[0] - WL[0];
    s->du = WR[1] - WL[1];
    s->dv = WR[2] - WL[2];
    s->dw = WR[3] - WL[3];
    s->dp = WR[4] - WL[4];
    s->dVn = n[0] * s->du + n[1] * s->dv + n[2] * s->dw;
}

/* Sum over the three waves of  lam_k * alpha_k * r_k, with the wave speeds
 * given by the caller (|lam| with the entropy fix for the flux; lam itself
 * for the Roe-property check).  alpha_k r_k: acoustic waves
 * (dp -/+ rho a dVn)/(2 a^2) (1, u -/+ a n, H -/+ a Vn); entropy and shear
 * waves (drho - dp/a^2)(1, u, q^2/2) + rho (0, du - dVn n, u.du - Vn dVn). */
static void roe_wave_sum(const roe_state *s, const double n[3], const double lam[3], double D[NV])
{
    double a2 = s->a * s->a;
    double al1 = (s->dp - s->rho * s->a * s->dVn) / (2.0 * a2);
    double al3 = (s->dp + s->rho * s->a * s->dVn) / (2.0 * a2);
    double al2 = s->drho - s->dp / a2;
    double r1[NV] = {1.0, s->u - s->a * n[0], s->v - s->a * n[1], s->w - s->a * n[2], s->H - s->a * s->Vn};
    double r3[NV] = {1.0, s->u + s->a * n[0], s->v + s->a * n[1], s->w + s->a * n[2], s->H + s->a * s->Vn};
    double r2[NV] = {1.0, s->u, s->v, s->w, 0.5 * s->q2};
    double sh[NV] = {0.0, s->du - s->dVn * n[0], s->dv - s->dVn * n[1], s->dw - s->dVn * n[2],
                     s->u * s->du + s->v * s->dv + s->w * s->dw - s->Vn * s->dVn};
    for (int q = 0; q < NV; ++q)
        D[q] = lam[0] * al1 * r1[q] + lam[1] * (al2 * r2[q] + s->rho * sh[q]) + lam[2] * al3 * r3[q];
}

/* Harten's entropy fix on the acoustic waves: |lam| below delta = fix * a is
 * replaced by (lam^2 + delta^2)/(2 delta).  fix == 0 switches it off. */
static double fixed_abs(double lam, double delta)
{
    if (fabs(lam) < delta) return (lam * lam + delta * delta) / (2.0 * delta);
    return fabs(lam);
}

/* Roe flux through a face with area vector S = n |S|:
 * |S| * [ (F(W_L) + F(W_R))/2 - (1/2) sum_k |lam_k| alpha_k r_k ]. */
static void roe_flux(double gamma, double fix, const double WL[NV], const double WR[NV],
                     const double S[3], double Fh[NV])
{
    double area = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    double n[3] = {S[0] / area, S[1] / area, S[2] / area};
    double FL[NV], FR[NV], D[NV], lam[3];
    roe_state s;
    euler_flux(gamma, WL, n, FL);
    euler_flux(gamma, WR, n, FR);
    roe_average(gamma, WL, WR, n, &s);
    double delta = fix * s.a;
    lam[0] = fixed_abs(s.lam[0], delta);
    lam[1] = fabs(s.lam[1]);
    lam[2] = fixed_abs(s.lam[2], delta);
    roe_wave_sum(&s, n, lam, D);
    for (int q = 0; q < NV; ++q)
        Fh[q] = area * (0.5 * (FL[q] + FR[q]) - 0.5 * D[q]);
}

/* ------------------------------------------------------------------------ */
/* boundary conditions / ghost cells (Sec. 5 "Ghost cell extrapolation")     */
/* face numbering: 0 imin, 1 imax, 2 jmin, 3 jmax, 4 kmin, 5 kmax            */
/* ------------------------------------------------------------------------ */

/* For face f of block b, ghost layer g (1 = next to the boundary, 2 = outer)
 * at tangential position (t1, t2), return the ghost cell and the interior
 * cell that lies m cells inside the boundary (m = 0 is the boundary cell). */
static long ghost_cell(const ora_block *b, int f, int g, int t1, int t2)
{
    switch (f) {
    case 0: return cell(b, -g, t1, t2);
    case 1: return cell(b, b->ni - 1 + g, t1, t2);
    case 2: return cell(b, t1, -g, t2);
    case 3: return cell(b, t1, b->nj - 1 + g, t2);
    case 4: return cell(b, t1, t2, -g);
    default: return cell(b, t1, t2, b->nk - 1 + g);
    }
}

static long inner_cell(const ora_block *b, int f, int m, int t1, int t2)
{
    switch (f) {
    case 0: return cell(b, m, t1, t2);
    case 1: return cell(b, b->ni - 1 - m, t1, t2);
    case 2: return cell(b, t1, m, t2);
    case 3: return cell(b, t1, b->nj - 1 - m, t2);
    case 4: return cell(b, t1, t2, m);
    default: return cell(b, t1, t2, b->nk - 1 - m);
    }
}

static void face_extent(const ora_block *b, int f, int *n1, int *n2)
{
    if (f < 2) { *n1 = b->nj; *n2 = b->nk; }
    else if (f < 4) { *n1 = b->ni; *n2 = b->nk; }
    else { *n1 = b->ni; *n2 = b->nj; }
}

/* unit normal of the boundary face of face family f at tangential (t1, t2) */
static void boundary_normal(const ora_block *b, int f, int t1, int t2, double n[3])
{
    double S[3];
    for (int a = 0; a < 3; ++a) {
        switch (f) {
        case 0: S[a] = b->Si[a * n_fi(b) + fi_index(b, 0, t1, t2)]; break;
        case 1: S[a] = b->Si[a * n_fi(b) + fi_index(b, b->ni, t1, t2)]; break;
        case 2: S[a] = b->Sj[a * n_fj(b) + fj_index(b, t1, 0, t2)]; break;
        case 3: S[a] = b->Sj[a * n_fj(b) + fj_index(b, t1, b->nj, t2)]; break;
        case 4: S[a] = b->Sk[a * n_fk(b) + fk_index(b, t1, t2, 0)]; break;
        default: S[a] = b->Sk[a * n_fk(b) + fk_index(b, t1, t2, b->nk)]; break;
        }
    }
    double area = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    n[0] = S[0] / area;
    n[1] = S[1] / area;
    n[2] = S[2] / area;
}

/* Ghost cells of face f.  edges = 0: the face's own ghosts (tangential
 * positions inside the face).  edges = 1: the block-edge ghosts the viscous
 * face gradients read (two indices outside the block), filled after every
 * face's own ghosts by the rule of the lower face family: an i-face fills
 * its ghosts at j- or k-ghost positions, a j-face those at k-ghost
 * positions; the rule then reads ghosts of the other family (its own
 * block's, or for an interface the neighbour's), already in place. */
static void fill_face_range(const ora_grid *g, int bi, int f, double *const *U, int edges)
{
    const ora_block *b = &g->b[bi];
    double *u = U[bi];
    int n1, n2;
    face_extent(b, f, &n1, &n2);
    int type = b->bc_type[f];
    double Qinf[NV];
    if (type == ORA_BC_INFLOW) prim_to_cons(g->gamma, b->bc_prim[f], Qinf);
    /* the tangential ranges: the second tangential index has no ghosts in 2D */
    int fam = f >> 1;
    int g1 = edges && fam == 0 ? NG : 0;                       /* t1 = j for i-faces, i otherwise */
    int g2 = edges && fam < 2 && !is2d(b) ? NG : 0;           /* t2 = k for i- and j-faces */
    for (int t2 = -g2; t2 < n2 + g2; ++t2)
        for (int t1 = -g1; t1 < n1 + g1; ++t1) {
            int out1 = t1 < 0 || t1 >= n1, out2 = t2 < 0 || t2 >= n2;
            if (edges ? (out1 + out2 != 1) : (out1 || out2)) continue;
            for (int layer = 1; layer <= NG; ++layer) {
                long gc = ghost_cell(b, f, layer, t1, t2);
                if (type == ORA_BC_PERIODIC) {
                    /* the opposite face's interior: ghost layer g of face f is
                     * the cell g-1 cells inside the opposite boundary */
                    long src = inner_cell(b, f ^ 1, layer - 1, t1, t2);
                    for (int q = 0; q < NV; ++q) u[q * b->sv + gc] = u[q * b->sv + src];
                } else if (type == ORA_BC_INFLOW) {
                    for (int q = 0; q < NV; ++q) u[q * b->sv + gc] = Qinf[q];
                } else if (type == ORA_BC_EXTRAPOLATE) {
                    long src = inner_cell(b, f, 0, t1, t2);
                    for (int q = 0; q < NV; ++q) u[q * b->sv + gc] = u[q * b->sv + src];
                } else if (type == ORA_BC_SLIP_WALL) {
                    /* mirror image of the interior cell layer-1 cells inside:
                     * density and total energy copied, momentum reflected,
                     * m_g = m - 2 (m . n) n (at an edge, n of the nearest
                     * boundary face) */
                    long src = inner_cell(b, f, layer - 1, t1, t2);
                    double n[3];
                    boundary_normal(b, f, t1 < 0 ? 0 : (t1 >= n1 ? n1 - 1 : t1), t2 < 0 ? 0 : (t2 >= n2 ? n2 - 1 : t2),
                                    n);
                    double m[3] = {u[1 * b->sv + src], u[2 * b->sv + src], u[3 * b->sv + src]};
                    double mn = m[0] * n[0] + m[1] * n[1] + m[2] * n[2];
                    u[0 * b->sv + gc] = u[0 * b->sv + src];
                    u[1 * b->sv + gc] = m[0] - 2.0 * mn * n[0];
                    u[2 * b->sv + gc] = m[1] - 2.0 * mn * n[1];
                    u[3 * b->sv + gc] = m[2] - 2.0 * mn * n[2];
                    u[4 * b->sv + gc] = u[4 * b->sv + src];
                } else if (type == ORA_BC_INTERFACE) {
                    /* point-matched neighbour face with aligned tangential
                     * indices: ghost layer g is the neighbour's cell g-1
                     * inside its face */
                    const ora_block *nb = &g->b[b->bc_nbr[f]];
                    long src = inner_cell(nb, b->bc_nbr_face[f], layer - 1, t1, t2);
                    const double *un = U[b->bc_nbr[f]];
                    for (int q = 0; q < NV; ++q) u[q * b->sv + gc] = un[q * nb->sv + src];
                }
            }
        }
}

static void fill_face(const ora_grid *g, int bi, int f, double *const *U) { fill_face_range(g, bi, f, U, 0); }

/* ------------------------------------------------------------------------ */
/* residual, Eq. residual: R_h = sum over the f faces of                     */
/*                               (F_{i,n} - F_{nu,n}) Delta s - |Omega| S_h  */
/* with R taken on the outward area vector of each face, so that            */
/* |Omega| dU/dt = -R (Eq. spatial_residual).                                */
/* ------------------------------------------------------------------------ */

/* Face flux between the 4-cell stencil c[0..3] (cells i-1, i, i+1, i+2 along
 * one index direction; the face lies between c[1] and c[2]). */
static void stencil_flux(const ora_grid *g, const ora_block *b, const double *u,
                         const long c[4], const double S[3], double F[NV])
{
    double V[4][NV];        /* the reconstructed variables of the four cells */
    double L[NV], Rr[NV], WL[NV], WR[NV];
    for (int m = 0; m < 4; ++m) {
        double Q[NV];
        for (int q = 0; q < NV; ++q) Q[q] = u[q * b->sv + c[m]];
        if (g->recon_conserved)
            for (int q = 0; q < NV; ++q) V[m][q] = Q[q];
        else
            cons_to_prim(g->gamma, Q, V[m]);
    }
    for (int q = 0; q < NV; ++q) {
        double s[4] = {V[0][q], V[1][q], V[2][q], V[3][q]};
        muscl_face(g->limiter, g->kappa, g->eps, s, &L[q], &Rr[q]);
    }
    if (g->recon_conserved) {
        cons_to_prim(g->gamma, L, WL);
        cons_to_prim(g->gamma, Rr, WR);
    } else {
        memcpy(WL, L, sizeof L);
        memcpy(WR, Rr, sizeof Rr);
    }
    roe_flux(g->gamma, g->fix_delta, WL, WR, S, F);
}

/* ------------------------------------------------------------------------ */
/* viscous flux F_nu,n of Eq. governing (Stokes's hypothesis; Theta = work  */
/* of the viscous stresses + heat conduction).  The paper gives neither the */
/* viscosity law nor the face-gradient discretisation; the readings used:   */
/* constant mu, heat conductivity mu c_p / Pr (so that k grad T =            */
/* mu gamma / ((gamma - 1) Pr) grad(p / rho)), and face gradients from      */
/* computational-space central differences and the metric identity         */
/* grad xi_a = Sbar_a / |Omega|, both averaged over the face's two cells.   */
/* ------------------------------------------------------------------------ */

/* the viscous variables (u, v, w, p / rho) of a ghosted cell */
static void vis_vars(const ora_grid *g, const ora_block *b, const double *u, int i, int j, int k, double phi[4])
{
    double Q[NV], W[NV];
    long c0 = cell(b, i, j, k);
    for (int q = 0; q < NV; ++q) Q[q] = u[q * b->sv + c0];
    cons_to_prim(g->gamma, Q, W);
    phi[0] = W[1];
    phi[1] = W[2];
    phi[2] = W[3];
    phi[3] = W[4] / W[0];
}

/* area vector of face family a at face index (i, j, k) (lowest-corner) */
static void face_vector(const ora_block *b, int a, int i, int j, int k, double S[3])
{
    for (int c = 0; c < 3; ++c) {
        if (a == 0) S[c] = b->Si[c * n_fi(b) + fi_index(b, i, j, k)];
        else if (a == 1) S[c] = b->Sj[c * n_fj(b) + fj_index(b, i, j, k)];
        else S[c] = b->Sk[c * n_fk(b) + fk_index(b, i, j, k)];
    }
}

/* Sbar_a of interior cell (i, j, k): the mean of its two a-face vectors */
static void cell_sbar(const ora_block *b, int a, int i, int j, int k, double S[3])
{
    double s0[3], s1[3];
    face_vector(b, a, i, j, k, s0);
    face_vector(b, a, i + (a == 0), j + (a == 1), k + (a == 2), s1);
    for (int c = 0; c < 3; ++c) S[c] = 0.5 * (s0[c] + s1[c]);
}

static int clampi(int x, int n) { return x < 0 ? 0 : (x >= n ? n - 1 : x); }

/* The cell whose geometry a cell of a face stencil carries: an interior
 * cell its own; a ghost cell (outside in one direction) that of the cell it
 * copies -- the opposite side's cell for a periodic face, the neighbour
 * block's cell for an interface -- or, behind a physical boundary, the
 * boundary cell it mirrors. */
static const ora_block *metric_cell(const ora_grid *g, const ora_block *b, int c[3])
{
    int n[3] = {b->ni, b->nj, b->nk};
    for (int a = 0; a < 3; ++a) {
        if (c[a] >= 0 && c[a] < n[a]) continue;
        int hi = c[a] >= n[a];
        int f = 2 * a + hi;
        int layer = hi ? c[a] - n[a] + 1 : -c[a];     /* 1 next to the boundary */
        int type = b->bc_type[f];
        if (type == ORA_BC_PERIODIC) {
            c[a] = hi ? c[a] - n[a] : c[a] + n[a];
        } else if (type == ORA_BC_INTERFACE) {
            const ora_block *nb = &g->b[b->bc_nbr[f]];
            int nf = b->bc_nbr_face[f];
            int m[3] = {nb->ni, nb->nj, nb->nk};
            c[a] = (nf & 1) ? m[a] - layer : layer - 1;
            return nb;
        } else {
            c[a] = clampi(c[a], n[a]);
        }
    }
    return b;
}

/* F_nu . S through the d-face between cells L = (i, j, k) - e_d and
 * R = (i, j, k) (face index (i, j, k), area vector S toward +d). */
static void viscous_flux(const ora_grid *g, const ora_block *b, const double *u, int d, int i, int j, int k,
                         const double S[3], double F[NV])
{
    int ndir = is2d(b) ? 2 : 3;
    int L[3] = {i - (d == 0), j - (d == 1), k - (d == 2)};
    int R[3] = {i, j, k};
    /* the tangential families e, f of direction d */
    int e = d == 0 ? 1 : 0;
    int f = d == 2 ? 1 : 2;
    double pL[4], pR[4], dxi[4], deta[4], dzeta[4];
    vis_vars(g, b, u, L[0], L[1], L[2], pL);
    vis_vars(g, b, u, R[0], R[1], R[2], pR);
    for (int q = 0; q < 4; ++q) {
        dxi[q] = pR[q] - pL[q];
        deta[q] = 0.0;
        dzeta[q] = 0.0;
    }
    for (int t = 0; t < 2; ++t) {
        int a = t == 0 ? e : f;
        if (a >= ndir) continue;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int Lp[3] = {L[0], L[1], L[2]}, Rp[3] = {R[0], R[1], R[2]};
            Lp[a] += sgn;
            Rp[a] += sgn;
            double qa[4], qb[4];
            vis_vars(g, b, u, Lp[0], Lp[1], Lp[2], qa);
            vis_vars(g, b, u, Rp[0], Rp[1], Rp[2], qb);
            for (int q = 0; q < 4; ++q) acc[q] += sgn * (qa[q] + qb[q]);
        }
        for (int q = 0; q < 4; ++q) {
            if (t == 0) deta[q] = 0.25 * acc[q];
            else dzeta[q] = 0.25 * acc[q];
        }
    }
    /* grad xi_a at the face: (Sbar_a(L) + Sbar_a(R)) / (|Omega_L| + |Omega_R|),
     * a ghost cell carrying the geometry of the cell it copies */
    int Lc[3] = {L[0], L[1], L[2]}, Rc[3] = {R[0], R[1], R[2]};
    const ora_block *bL = metric_cell(g, b, Lc), *bR = metric_cell(g, b, Rc);
    double vsum = bL->vol[interior(bL, Lc[0], Lc[1], Lc[2])] + bR->vol[interior(bR, Rc[0], Rc[1], Rc[2])];
    double gx[3][3];   /* gx[m] = grad of the m-th computational coordinate (d, e, f) */
    int dirs[3] = {d, e, f};
    for (int m = 0; m < 3; ++m) {
        if (dirs[m] >= ndir) {
            gx[m][0] = gx[m][1] = gx[m][2] = 0.0;
            continue;
        }
        double sa[3], sb[3];
        cell_sbar(bL, dirs[m], Lc[0], Lc[1], Lc[2], sa);
        cell_sbar(bR, dirs[m], Rc[0], Rc[1], Rc[2], sb);
        for (int c = 0; c < 3; ++c) gx[m][c] = (sa[c] + sb[c]) / vsum;
    }
    double grad[4][3];
    for (int q = 0; q < 4; ++q)
        for (int c = 0; c < 3; ++c) grad[q][c] = dxi[q] * gx[0][c] + deta[q] * gx[1][c] + dzeta[q] * gx[2][c];
    double mu = g->mu;
    double div = grad[0][0] + grad[1][1] + grad[2][2];
    double tau[3][3];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) tau[a][c] = mu * (grad[a][c] + grad[c][a]) - (a == c ? 2.0 / 3.0 * mu * div : 0.0);
    double ub[3] = {0.5 * (pL[0] + pR[0]), 0.5 * (pL[1] + pR[1]), 0.5 * (pL[2] + pR[2])};
    double kappa = mu * g->gamma / ((g->gamma - 1.0) * g->prandtl);
    double theta[3];
    for (int c = 0; c < 3; ++c) theta[c] = ub[0] * tau[0][c] + ub[1] * tau[1][c] + ub[2] * tau[2][c] + kappa * grad[3][c];
    F[0] = 0.0;
    for (int a = 0; a < 3; ++a) F[1 + a] = tau[a][0] * S[0] + tau[a][1] * S[1] + tau[a][2] * S[2];
    F[4] = theta[0] * S[0] + theta[1] * S[1] + theta[2] * S[2];
}

static void block_residual(const ora_grid *g, int bi, double *const *U, double *R, const double *src)
{
    const ora_block *b = &g->b[bi];
    const double *u = U[bi];
    long nfi = n_fi(b), nfj = n_fj(b), nfk = n_fk(b);
    double *Fi = calloc((size_t)NV * nfi, sizeof(double));
    double *Fj = calloc((size_t)NV * nfj, sizeof(double));
    double *Fk = is2d(b) ? NULL : calloc((size_t)NV * nfk, sizeof(double));

    /* every face flux once */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < b->nk; ++k)
        for (int j = 0; j < b->nj; ++j)
            for (int i = 0; i <= b->ni; ++i) {
                double S[3], F[NV];
                long c[4];
                for (int m = 0; m < 4; ++m) c[m] = cell(b, i - 2 + m, j, k);
                for (int a = 0; a < 3; ++a) S[a] = b->Si[a * nfi + fi_index(b, i, j, k)];
                stencil_flux(g, b, u, c, S, F);
                if (g->mu > 0.0) {
                    double Fv[NV];
                    viscous_flux(g, b, u, 0, i, j, k, S, Fv);
                    for (int q = 0; q < NV; ++q) F[q] -= Fv[q];
                }
                for (int q = 0; q < NV; ++q) Fi[q * nfi + fi_index(b, i, j, k)] = F[q];
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < b->nk; ++k)
        for (int j = 0; j <= b->nj; ++j)
            for (int i = 0; i < b->ni; ++i) {
                double S[3], F[NV];
                long c[4];
                for (int m = 0; m < 4; ++m) c[m] = cell(b, i, j - 2 + m, k);
                for (int a = 0; a < 3; ++a) S[a] = b->Sj[a * nfj + fj_index(b, i, j, k)];
                stencil_flux(g, b, u, c, S, F);
                if (g->mu > 0.0) {
                    double Fv[NV];
                    viscous_flux(g, b, u, 1, i, j, k, S, Fv);
                    for (int q = 0; q < NV; ++q) F[q] -= Fv[q];
                }
                for (int q = 0; q < NV; ++q) Fj[q * nfj + fj_index(b, i, j, k)] = F[q];
            }
    if (!is2d(b)) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k <= b->nk; ++k)
            for (int j = 0; j < b->nj; ++j)
                for (int i = 0; i < b->ni; ++i) {
                    double S[3], F[NV];
                    long c[4];
                    for (int m = 0; m < 4; ++m) c[m] = cell(b, i, j, k - 2 + m);
                    for (int a = 0; a < 3; ++a) S[a] = b->Sk[a * nfk + fk_index(b, i, j, k)];
                    stencil_flux(g, b, u, c, S, F);
                    if (g->mu > 0.0) {
                        double Fv[NV];
                        viscous_flux(g, b, u, 2, i, j, k, S, Fv);
                        for (int q = 0; q < NV; ++q) F[q] -= Fv[q];
                    }
                    for (int q = 0; q < NV; ++q) Fk[q * nfk + fk_index(b, i, j, k)] = F[q];
                }
    }

    /* sum over the faces of each cell with the outward sign:
     * (F_{i+1/2} - F_{i-1/2}) + (F_{j+1/2} - F_{j-1/2}) + (F_{k+1/2} - F_{k-1/2}) - |Omega| S */
    long nint = n_interior(b);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < b->nk; ++k)
        for (int j = 0; j < b->nj; ++j)
            for (int i = 0; i < b->ni; ++i) {
                long c0 = interior(b, i, j, k);
                for (int q = 0; q < NV; ++q) {
                    double r = Fi[q * nfi + fi_index(b, i + 1, j, k)] - Fi[q * nfi + fi_index(b, i, j, k)];
                    r += Fj[q * nfj + fj_index(b, i, j + 1, k)] - Fj[q * nfj + fj_index(b, i, j, k)];
                    if (!is2d(b))
                        r += Fk[q * nfk + fk_index(b, i, j, k + 1)] - Fk[q * nfk + fk_index(b, i, j, k)];
                    if (src) r -= src[q * nint + c0];
                    R[q * nint + c0] = r;
                }
            }
    free(Fi);
    free(Fj);
    free(Fk);
}

/* ------------------------------------------------------------------------ */
/* time step: dt = CFL * min over cells of |Omega| / sum_d (|u . Sbar_d| +   */
/* c |Sbar_d|), Sbar_d the mean of the cell's two d-face area vectors.  The  */
/* paper states no time-step rule; this spectral-radius bound is the reading */
/* used.                                                                     */
/* ------------------------------------------------------------------------ */

/* the viscous part of the spectral radius of direction d (zero for mu = 0):
 * 4 max(4/3, gamma) mu / (Pr rho) |Sbar_d|^2 / |Omega| (the paper gives no
 * time-step rule; the factor 4 and the max form are the reading used) */
static double viscous_radius(const ora_grid *g, double rho, double vol, const double Sb[3])
{
    if (!(g->mu > 0.0)) return 0.0;
    double f = g->gamma > 4.0 / 3.0 ? g->gamma : 4.0 / 3.0;
    return 4.0 * f * g->mu / (g->prandtl * rho) * (Sb[0] * Sb[0] + Sb[1] * Sb[1] + Sb[2] * Sb[2]) / vol;
}

static double block_dt_min(const ora_grid *g, int bi, const double *u)
{
    const ora_block *b = &g->b[bi];
    long nfi = n_fi(b), nfj = n_fj(b), nfk = n_fk(b);
    double best = INFINITY;
    for (int k = 0; k < b->nk; ++k)
        for (int j = 0; j < b->nj; ++j)
            for (int i = 0; i < b->ni; ++i) {
                double Q[NV], W[NV];
                long c0 = cell(b, i, j, k);
                for (int q = 0; q < NV; ++q) Q[q] = u[q * b->sv + c0];
                cons_to_prim(g->gamma, Q, W);
                double c = sqrt(g->gamma * W[4] / W[0]);
                double sum = 0.0;
                for (int d = 0; d < (is2d(b) ? 2 : 3); ++d) {
                    double Sb[3];
                    for (int a = 0; a < 3; ++a) {
                        double s0, s1;
                        if (d == 0) {
                            s0 = b->Si[a * nfi + fi_index(b, i, j, k)];
                            s1 = b->Si[a * nfi + fi_index(b, i + 1, j, k)];
                        } else if (d == 1) {
                            s0 = b->Sj[a * nfj + fj_index(b, i, j, k)];
                            s1 = b->Sj[a * nfj + fj_index(b, i, j + 1, k)];
                        } else {
                            s0 = b->Sk[a * nfk + fk_index(b, i, j, k)];
                            s1 = b->Sk[a * nfk + fk_index(b, i, j, k + 1)];
                        }
                        Sb[a] = 0.5 * (s0 + s1);
                    }
                    double uS = W[1] * Sb[0] + W[2] * Sb[1] + W[3] * Sb[2];
                    double mag = sqrt(Sb[0] * Sb[0] + Sb[1] * Sb[1] + Sb[2] * Sb[2]);
                    sum += fabs(uS) + c * mag;
                    sum += viscous_radius(g, W[0], b->vol[interior(b, i, j, k)], Sb);
                }
                double t = b->vol[interior(b, i, j, k)] / sum;
                if (t < best) best = t;
            }
    return best;
}

/* ------------------------------------------------------------------------ */
/* explicit Runge-Kutta, Eq. runge_kutta in its Butcher form:               */
/*   U^i     = U^n - dt * sum_{j<i} a_ij R^j / |Omega|                       */
/*   U^{n+1} = U^n - dt * sum_i   b_i  R^i / |Omega|                         */
/* The 1/|Omega| comes from Eq. spatial_residual, which the printed          */
/* Eq. runge_kutta leaves implicit.  Coefficients (the paper defers them to  */
/* Ferracina & Spijker): the optimal strong-stability-preserving methods     */
/* SSPRK(2,2), SSPRK(3,3) and SSPRK(4,2).                                    */
/* ------------------------------------------------------------------------ */

static int rk_tableau(int rk, double a[4][4], double b[4])
{
    memset(a, 0, 16 * sizeof(double));
    memset(b, 0, 4 * sizeof(double));
    if (rk == ORA_RK2_SSP) {
        a[1][0] = 1.0;
        b[0] = 0.5;
        b[1] = 0.5;
        return 2;
    }
    if (rk == ORA_RK3_SSP) {
        a[1][0] = 1.0;
        a[2][0] = 0.25;
        a[2][1] = 0.25;
        b[0] = 1.0 / 6.0;
        b[1] = 1.0 / 6.0;
        b[2] = 2.0 / 3.0;
        return 3;
    }
    if (rk == ORA_RK4_SSP2) {
        for (int i = 1; i < 4; ++i)
            for (int j = 0; j < i; ++j) a[i][j] = 1.0 / 3.0;
        for (int i = 0; i < 4; ++i) b[i] = 0.25;
        return 4;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* exported API                                                              */
/* ------------------------------------------------------------------------ */

void ora_destroy(ora_grid *g)
{
    if (!g) return;
    for (int bi = 0; bi < g->nb; ++bi) {
        free(g->b[bi].Si);
        free(g->b[bi].Sj);
        free(g->b[bi].Sk);
        free(g->b[bi].vol);
    }
    free(g->b);
    free(g);
}

/* dims: 3 ints (ni, nj, nk) per block; nodes: one X[3][nk+1][nj+1][ni+1] per block */
ora_grid *ora_create(int nb, const int *dims, const double *const *nodes, double gamma,
                     int limiter, double kappa, double eps, int recon_conserved, double fix_delta)
{
    ora_grid *g = calloc(1, sizeof(ora_grid));
    g->nb = nb;
    g->b = calloc((size_t)nb, sizeof(ora_block));
    g->gamma = gamma;
    g->limiter = limiter;
    g->kappa = kappa;
    g->eps = eps;
    g->recon_conserved = recon_conserved;
    g->fix_delta = fix_delta;
    for (int bi = 0; bi < nb; ++bi) {
        ora_block *b = &g->b[bi];
        b->ni = dims[3 * bi];
        b->nj = dims[3 * bi + 1];
        b->nk = dims[3 * bi + 2];
        b->gk = (b->nk == 1) ? 0 : NG;
        b->sj = b->ni + 2 * NG;
        b->sk = b->sj * (b->nj + 2 * NG);
        b->sv = b->sk * (b->nk + 2 * b->gk);
        b->Si = calloc((size_t)3 * n_fi(b), sizeof(double));
        b->Sj = calloc((size_t)3 * n_fj(b), sizeof(double));
        b->Sk = calloc((size_t)3 * n_fk(b), sizeof(double));
        b->vol = calloc((size_t)n_interior(b), sizeof(double));
        for (int f = 0; f < 6; ++f) {
            b->bc_type[f] = ORA_BC_UNSET;
            b->bc_nbr[f] = -1;
            b->bc_nbr_face[f] = -1;
        }
        compute_metrics(b, nodes[bi]);
    }
    return g;
}

/* returns 0 on success, nonzero on an inconsistent description */
int ora_set_bc(ora_grid *g, int bi, int f, int type, const double *prim, int nbr, int nbr_face)
{
    if (bi < 0 || bi >= g->nb || f < 0 || f > 5) return 1;
    ora_block *b = &g->b[bi];
    b->bc_type[f] = type;
    if (type == ORA_BC_INFLOW) {
        if (!prim) return 2;
        for (int q = 0; q < NV; ++q) b->bc_prim[f][q] = prim[q];
    }
    if (type == ORA_BC_INTERFACE) {
        if (nbr < 0 || nbr >= g->nb || nbr_face < 0 || nbr_face > 5) return 3;
        if ((nbr_face >> 1) != (f >> 1) || nbr_face == f) return 4;   /* aligned: opposite side, same axis */
        int n1, n2, m1, m2;
        face_extent(b, f, &n1, &n2);
        face_extent(&g->b[nbr], nbr_face, &m1, &m2);
        if (n1 != m1 || n2 != m2) return 5;
        b->bc_nbr[f] = nbr;
        b->bc_nbr_face[f] = nbr_face;
    }
    return 0;
}

void ora_get_metrics(const ora_grid *g, int bi, double *Si, double *Sj, double *Sk, double *vol)
{
    const ora_block *b = &g->b[bi];
    memcpy(Si, b->Si, sizeof(double) * 3 * n_fi(b));
    memcpy(Sj, b->Sj, sizeof(double) * 3 * n_fj(b));
    memcpy(Sk, b->Sk, sizeof(double) * 3 * n_fk(b));
    memcpy(vol, b->vol, sizeof(double) * n_interior(b));
}

void ora_fill_ghosts(const ora_grid *g, double *const *U)
{
    for (int bi = 0; bi < g->nb; ++bi)
        for (int f = 0; f < (is2d(&g->b[bi]) ? 4 : 6); ++f) fill_face(g, bi, f, U);
    /* the block-edge ghosts of the viscous face gradients, from the face
     * ghosts of every block */
    if (g->mu > 0.0)
        for (int bi = 0; bi < g->nb; ++bi)
            for (int f = 0; f < (is2d(&g->b[bi]) ? 4 : 6); ++f) fill_face_range(g, bi, f, U, 1);
}

/* viscosity (constant mu >= 0; 0 = Euler) and Prandtl number of F_nu */
void ora_set_viscosity(ora_grid *g, double mu, double prandtl)
{
    g->mu = mu;
    g->prandtl = prandtl;
}

/* R_h of every block from states whose ghost layers are already filled;
 * src (may be NULL, or hold NULL entries) is |Omega| S_h per interior cell. */
void ora_residual(const ora_grid *g, double *const *U, double *const *R, const double *const *src)
{
    for (int bi = 0; bi < g->nb; ++bi) block_residual(g, bi, U, R[bi], src ? src[bi] : NULL);
}

/* min over all cells of |Omega| / sum_d (|u . Sbar_d| + c |Sbar_d|); dt = CFL times this */
double ora_dt_min(const ora_grid *g, double *const *U)
{
    double best = INFINITY;
    for (int bi = 0; bi < g->nb; ++bi) {
        double t = block_dt_min(g, bi, U[bi]);
        if (t < best) best = t;
    }
    return best;
}

/* out[0..4] L2 = sqrt(sum R^2 / N), out[5..9] max |R|, out[10..14] sum |Omega| U,
 * with sums in block, k, j, i order over all interior cells. */
void ora_norms(const ora_grid *g, double *const *R, double *const *U, double *out)
{
    double s2[NV] = {0}, mx[NV] = {0}, cons[NV] = {0};
    long N = 0;
    for (int bi = 0; bi < g->nb; ++bi) {
        const ora_block *b = &g->b[bi];
        long nint = n_interior(b);
        N += nint;
        for (int k = 0; k < b->nk; ++k)
            for (int j = 0; j < b->nj; ++j)
                for (int i = 0; i < b->ni; ++i) {
                    long c0 = interior(b, i, j, k);
                    for (int q = 0; q < NV; ++q) {
                        double r = R[bi][q * nint + c0];
                        s2[q] += r * r;
                        if (fabs(r) > mx[q]) mx[q] = fabs(r);
                        cons[q] += b->vol[c0] * U[bi][q * b->sv + cell(b, i, j, k)];
                    }
                }
    }
    for (int q = 0; q < NV; ++q) {
        out[q] = sqrt(s2[q] / (double)N);
        out[NV + q] = mx[q];
        out[2 * NV + q] = cons[q];
    }
}

/* local time step of one cell: cfl * |Omega| / sum_d (|u . Sbar_d| + c |Sbar_d|),
 * the same spectral-radius bound as block_dt_min, without the minimum */
static double cell_dt(const ora_grid *g, const ora_block *b, const double *u, int i, int j, int k, double cfl)
{
    long nfi = n_fi(b), nfj = n_fj(b), nfk = n_fk(b);
    double Q[NV], W[NV];
    long c0 = cell(b, i, j, k);
    for (int q = 0; q < NV; ++q) Q[q] = u[q * b->sv + c0];
    cons_to_prim(g->gamma, Q, W);
    double c = sqrt(g->gamma * W[4] / W[0]);
    double sum = 0.0;
    for (int d = 0; d < (is2d(b) ? 2 : 3); ++d) {
        double Sb[3];
        for (int a = 0; a < 3; ++a) {
            double s0, s1;
            if (d == 0) {
                s0 = b->Si[a * nfi + fi_index(b, i, j, k)];
                s1 = b->Si[a * nfi + fi_index(b, i + 1, j, k)];
            } else if (d == 1) {
                s0 = b->Sj[a * nfj + fj_index(b, i, j, k)];
                s1 = b->Sj[a * nfj + fj_index(b, i, j + 1, k)];
            } else {
                s0 = b->Sk[a * nfk + fk_index(b, i, j, k)];
                s1 = b->Sk[a * nfk + fk_index(b, i, j, k + 1)];
            }
            Sb[a] = 0.5 * (s0 + s1);
        }
        double uS = W[1] * Sb[0] + W[2] * Sb[1] + W[3] * Sb[2];
        double mag = sqrt(Sb[0] * Sb[0] + Sb[1] * Sb[1] + Sb[2] * Sb[2]);
        sum += fabs(uS) + c * mag;
        sum += viscous_radius(g, W[0], b->vol[interior(b, i, j, k)], Sb);
    }
    return cfl * b->vol[interior(b, i, j, k)] / sum;
}

static double rk_step_impl(const ora_grid *g, double *const *U, const double *const *src, int rk,
                           double cfl, double dt, double *norms, int local);

/* One explicit RK step (Eq. runge_kutta, Butcher form) of all blocks, in
 * place.  dt > 0 is used as given; dt <= 0 means dt = cfl * ora_dt_min(U^n).
 * norms (15 doubles, may be NULL) receives ora_norms of R(U^n) and U^n.
 * src (may be NULL) is |Omega| S_h per interior cell, constant over the step.
 * Returns the dt used. */
double ora_rk_step(const ora_grid *g, double *const *U, const double *const *src, int rk,
                   double cfl, double dt, double *norms)
{
    return rk_step_impl(g, U, src, rk, cfl, dt, norms, 0);
}

/* The same step with local time stepping (a convergence accelerator for
 * steady states, which the paper's inlet case is): every cell advances
 * with its own step dt_c = cfl |Omega_c| / sum_d (|u . Sbar_d| + c |Sbar_d|),
 * evaluated on U^n and frozen over the stages.  Returns the smallest dt_c. */
double ora_rk_step_local(const ora_grid *g, double *const *U, const double *const *src, int rk,
                         double cfl, double *norms)
{
    return rk_step_impl(g, U, src, rk, cfl, 0.0, norms, 1);
}

static double rk_step_impl(const ora_grid *g, double *const *U, const double *const *src, int rk,
                           double cfl, double dt, double *norms, int local)
{
    double a[4][4], bw[4];
    int s = rk_tableau(rk, a, bw);
    if (s == 0) return -1.0;
    int nb = g->nb;
    double **Un = calloc((size_t)nb, sizeof(double *));     /* U^n, ghosted */
    double **Ui = calloc((size_t)nb, sizeof(double *));     /* stage state */
    double ***Rs = calloc((size_t)s, sizeof(double **));    /* R^1..R^s */
    for (int i = 0; i < s; ++i) Rs[i] = calloc((size_t)nb, sizeof(double *));
    for (int bi = 0; bi < nb; ++bi) {
        const ora_block *b = &g->b[bi];
        size_t ncell = (size_t)NV * b->sv;
        Un[bi] = malloc(ncell * sizeof(double));
        Ui[bi] = malloc(ncell * sizeof(double));
        memcpy(Un[bi], U[bi], ncell * sizeof(double));
        for (int i = 0; i < s; ++i) Rs[i][bi] = calloc((size_t)NV * n_interior(b), sizeof(double));
    }
    ora_fill_ghosts(g, Un);
    double **dtc = calloc((size_t)nb, sizeof(double *));   /* per-cell steps */
    for (int bi = 0; bi < nb; ++bi) {
        const ora_block *b = &g->b[bi];
        dtc[bi] = malloc(sizeof(double) * n_interior(b));
        if (local) {
#pragma omp parallel for schedule(static)
            for (int k = 0; k < b->nk; ++k)
                for (int j = 0; j < b->nj; ++j)
                    for (int ii = 0; ii < b->ni; ++ii)
                        dtc[bi][interior(b, ii, j, k)] = cell_dt(g, b, Un[bi], ii, j, k, cfl);
        }
    }
    if (local) {
        dt = INFINITY;
        for (int bi = 0; bi < nb; ++bi)
            for (long c0 = 0; c0 < n_interior(&g->b[bi]); ++c0)
                if (dtc[bi][c0] < dt) dt = dtc[bi][c0];
    } else {
        if (!(dt > 0.0)) dt = cfl * ora_dt_min(g, Un);
        for (int bi = 0; bi < nb; ++bi)
            for (long c0 = 0; c0 < n_interior(&g->b[bi]); ++c0) dtc[bi][c0] = dt;
    }

    for (int i = 0; i < s; ++i) {
        for (int bi = 0; bi < nb; ++bi) {
            const ora_block *b = &g->b[bi];
            long nint = n_interior(b);
            memcpy(Ui[bi], Un[bi], sizeof(double) * NV * b->sv);
#pragma omp parallel for schedule(static)
            for (int k = 0; k < b->nk; ++k)
                for (int j = 0; j < b->nj; ++j)
                    for (int ii = 0; ii < b->ni; ++ii) {
                        long c0 = interior(b, ii, j, k), cg = cell(b, ii, j, k);
                        for (int q = 0; q < NV; ++q) {
                            double acc = 0.0;
                            for (int jj = 0; jj < i; ++jj) acc += a[i][jj] * Rs[jj][bi][q * nint + c0];
                            Ui[bi][q * b->sv + cg] = Un[bi][q * b->sv + cg] - dtc[bi][c0] * acc / b->vol[c0];
                        }
                    }
        }
        ora_fill_ghosts(g, Ui);
        ora_residual(g, Ui, Rs[i], src);
    }
    if (norms) ora_norms(g, Rs[0], Un, norms);

    for (int bi = 0; bi < nb; ++bi) {
        const ora_block *b = &g->b[bi];
        long nint = n_interior(b);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < b->nk; ++k)
            for (int j = 0; j < b->nj; ++j)
                for (int ii = 0; ii < b->ni; ++ii) {
                    long c0 = interior(b, ii, j, k), cg = cell(b, ii, j, k);
                    for (int q = 0; q < NV; ++q) {
                        double acc = 0.0;
                        for (int i = 0; i < s; ++i) acc += bw[i] * Rs[i][bi][q * nint + c0];
                        U[bi][q * b->sv + cg] = Un[bi][q * b->sv + cg] - dtc[bi][c0] * acc / b->vol[c0];
                    }
                }
    }
    for (int bi = 0; bi < nb; ++bi) {
        free(Un[bi]);
        free(Ui[bi]);
        free(dtc[bi]);
        for (int i = 0; i < s; ++i) free(Rs[i][bi]);
    }
    free(dtc);
    for (int i = 0; i < s; ++i) free(Rs[i]);
    free(Rs);
    free(Un);
    free(Ui);
    return dt;
}

/* ---- host threads --------------------------------------------------------- */

/* Host threads for the loops over k-planes (n >= 1); returns the count in
 * effect: 1 when built without OpenMP. */
int ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---- pointwise entry points for the pin tests ---------------------------- */

void ora_rk_tableau(int rk, double *a16, double *b4, int *stages)
{
    double a[4][4], b[4];
    *stages = rk_tableau(rk, a, b);
    memcpy(a16, a, sizeof a);
    memcpy(b4, b, sizeof b);
}

void ora_euler_flux(double gamma, const double *W, const double *S, double *F)
{
    double area = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    double n[3] = {S[0] / area, S[1] / area, S[2] / area};
    euler_flux(gamma, W, n, F);
    for (int q = 0; q < NV; ++q) F[q] *= area;
}

void ora_roe_flux(double gamma, double fix, const double *WL, const double *WR, const double *S, double *F)
{
    roe_flux(gamma, fix, WL, WR, S, F);
}

/* |S| sum_k lam_k alpha_k r_k with signed wave speeds: by Roe's property this
 * is F(W_R).S - F(W_L).S. */
void ora_roe_jump(double gamma, const double *WL, const double *WR, const double *S, double *J)
{
    double area = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    double n[3] = {S[0] / area, S[1] / area, S[2] / area};
    roe_state s;
    double D[NV];
    roe_average(gamma, WL, WR, n, &s);
    roe_wave_sum(&s, n, s.lam, D);
    for (int q = 0; q < NV; ++q) J[q] = area * D[q];
}

void ora_muscl(int limiter, double kappa, double eps, const double *q4, double *qL, double *qR)
{
    muscl_face(limiter, kappa, eps, q4, qL, qR);
}

double ora_psi(int limiter, double r) { return psi(limiter, r); }

void ora_cons_to_prim(double gamma, const double *Q, double *W) { cons_to_prim(gamma, Q, W); }
void ora_prim_to_cons(double gamma, const double *W, double *Q) { prim_to_cons(gamma, W, Q); }
