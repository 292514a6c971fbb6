// stencil.cuh -- the fused residual / Runge-Kutta stage kernel.
//
// One CTA owns a TI x TJ column of cells and marches up a chunk of k-planes
// (2.5-D blocking).  Per plane:
//   P0  primitives W = (rho, u, v, w, p) of the plane, with a 2-cell halo in
//       i and j, into shared memory (the interior from the per-thread
//       k-window registers, the halo ring from global memory);
//   P1  MUSCL face states of every cell for the i and j directions, each
//       limited slope computed once per cell and direction (Eq. flux; the
//       limiter-reuse idea of Sec. 5 kept on chip instead of in a global
//       array);
//   P2  the Roe flux of every face of the tile, once per face, through one
//       loop and one copy of the flux code: each column's k-face above the
//       plane (kept in registers), then the i- and j-faces (into shared
//       memory);
//   P3  R = sum over the faces of F.S_out - |Omega| S_h (Eq. residual), then
//       either R is written out (residual mode) or the Runge-Kutta stage
//       update out = alpha U^n + beta U^(s-1) - gdt dt R / |Omega| is applied
//       (Eq. runge_kutta, Shu-Osher form), with FP64 norm partials.
// The reconstruction/flux arithmetic type is R (double, float, or the
// double-float pair df64); the state, the update and every reduction are
// FP64.
#pragma once

#include <math.h>

#include "blocks.cuh"
#include "df64.cuh"

// CTAs per SM the register allocation must allow: 2 (FP64 and double-float
// arithmetic; shared memory, 107 KB per CTA, allows no more).
template <typename R>
struct MinCtas {
    static constexpr int value = 2;
};

namespace sensei {

template <typename R>
struct SmemLayout {
    // sW[NV][TJ+4][TI+4], sP_i[2][NV][TJ][TI+2], sP_j[2][NV][TJ+2][TI],
    // sF_i[NV][TJ][TI+1], sF_j[NV][TJ+1][TI], sK[2][NV][NTHREADS] (each
    // thread's own column at planes k+1 and k+2), reduction scratch
    static constexpr int W = NV * (TJ + 4) * (TI + 4);
    static constexpr int PI = 2 * NV * TJ * (TI + 2);
    static constexpr int PJ = 2 * NV * (TJ + 2) * TI;
    static constexpr int FI = NV * TJ * (TI + 1);
    static constexpr int FJ = NV * (TJ + 1) * TI;
    static constexpr int K = 2 * NV * NTHREADS;
    static constexpr int elems = W + PI + PJ + FI + FJ + K;
    static constexpr int red_doubles = 3 * NV * (NTHREADS / 32);
    static constexpr size_t bytes = sizeof(R) * (size_t)elems + sizeof(double) * red_doubles + 16;
};

// Reciprocal and reciprocal square root of positive normal numbers by
// Newton-Raphson refinement of the hardware approximations.  FP64: the PTX
// rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64 seeds carry 20 correct bits
// (measured on sm_103a); each Newton step doubles that: STEPS = 1 gives
// ~1e-12 relative error (used where the value only scales the Roe
// dissipation or a limited slope), STEPS = 2 reaches the correctly rounded
// value (used where it enters the state or the central flux).  The
// reciprocal step is r' = r + r (1 - d r); the rsqrt step
// y' = y + (y/2) (1 - x y^2).  FP32: the approximations alone (below).
template <int STEPS>
__device__ __forceinline__ double rcp_nr(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
#pragma unroll
    for (int n = 0; n < STEPS; ++n) {
        double e = fma(-d, r, 1.0);
        r = fma(r, e, r);
    }
    return r;
}

// x / 2 for a positive normal x (x >= 2^-1021): FP64 lowers the exponent
// by one on the integer pipe, off the narrow FP64 pipe (exact); FP32 and
// double-float multiply by 0.5 on the FP32 pipe (exact)
__device__ __forceinline__ double half_pos(double x)
{
    return __hiloint2double(__double2hiint(x) - 0x00100000, __double2loint(x));
}
__device__ __forceinline__ float half_pos(float x) { return 0.5f * x; }
__device__ __forceinline__ df64 half_pos(df64 x) { return df64(0.5f * x.hi, 0.5f * x.lo); }

// |x| with the sign bit cleared on the integer pipe (FP64); FP32 and
// double-float as usual
__device__ __forceinline__ double abs_bits(double x)
{
    return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x));
}
__device__ __forceinline__ float abs_bits(float x) { return fabsf(x); }
__device__ __forceinline__ df64 abs_bits(df64 x) { return fabs(x); }

template <int STEPS>
__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
#pragma unroll
    for (int n = 0; n < STEPS; ++n) {
        double e = fma(-(x * y), y, 1.0);
        y = fma(half_pos(y), e, y);
    }
    return y;
}

template <typename R, int STEPS>
__device__ __forceinline__ R rcp_t(R x);
template <>
__device__ __forceinline__ double rcp_t<double, 1>(double x) { return rcp_nr<1>(x); }
template <>
__device__ __forceinline__ double rcp_t<double, 2>(double x) { return rcp_nr<2>(x); }
// FP32: the single-precision approximations (about 1 ulp), flush-to-zero
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ float rcp_t<float, 1>(float x) { return rcp_approx(x); }
template <>
__device__ __forceinline__ float rcp_t<float, 2>(float x) { return rcp_approx(x); }

template <typename R>
__device__ __forceinline__ R rsqrt1_t(R x);
template <>
__device__ __forceinline__ double rsqrt1_t<double>(double x) { return rsqrt_nr<1>(x); }
template <>
__device__ __forceinline__ float rsqrt1_t<float>(float x) { return rsqrt_approx(x); }
// double-float: one Newton step from the single-precision approximation
// (23 -> about 46 bits) in both cases
template <>
__device__ __forceinline__ df64 rcp_t<df64, 1>(df64 x) { return rcp_df(x); }
template <>
__device__ __forceinline__ df64 rcp_t<df64, 2>(df64 x) { return rcp_df(x); }
template <>
__device__ __forceinline__ df64 rsqrt1_t<df64>(df64 x) { return rsqrt_df(x); }

// x > 0 (nonzero, not NaN) and the sign of x, from the bit pattern (integer
// pipe, keeps compares off the FP64 pipe)
__device__ __forceinline__ bool positive(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool positive(float x) { return __float_as_int(x) > 0; }
__device__ __forceinline__ bool same_sign(double a, double b) { return (__double2hiint(a) ^ __double2hiint(b)) >= 0; }
__device__ __forceinline__ bool same_sign(float a, float b) { return (__float_as_int(a) ^ __float_as_int(b)) >= 0; }
// 0 < x < infinity (finite, positive, not NaN) from the bit pattern
__device__ __forceinline__ bool positive_finite(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool positive_finite(float x)
{
    const int b = __float_as_int(x);
    return b > 0 && b < 0x7f800000;
}
// a < b for a, b >= 0 (or NaN, which compares false) by the bit patterns
__device__ __forceinline__ bool lt_nonneg(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
__device__ __forceinline__ bool lt_nonneg(float a, float b) { return __float_as_int(a) < __float_as_int(b); }
// the double-float forms: the sign is the high part's; magnitudes compare
// the high parts, then the (sign-adjusted) low parts
__device__ __forceinline__ bool positive(df64 x) { return positive(x.hi); }
__device__ __forceinline__ bool positive_finite(df64 x) { return positive_finite(x.hi); }
__device__ __forceinline__ bool same_sign(df64 a, df64 b) { return same_sign(a.hi, b.hi); }
__device__ __forceinline__ bool lt_nonneg(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
// |a| <= |b| by the bit patterns of the magnitudes
__device__ __forceinline__ bool abs_le(double a, double b)
{
    return (__double_as_longlong(a) & 0x7fffffffffffffffLL) <= (__double_as_longlong(b) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool abs_le(float a, float b)
{
    return (__float_as_int(a) & 0x7fffffff) <= (__float_as_int(b) & 0x7fffffff);
}
__device__ __forceinline__ bool abs_le(df64 a, df64 b)
{
    const float ah = fabsf(a.hi), bh = fabsf(b.hi);
    if (ah != bh) return ah < bh;
    const float al = a.hi < 0.0f ? -a.lo : a.lo, bl = b.hi < 0.0f ? -b.lo : b.lo;
    return al <= bl;
}

// FP64 <-> FP32 conversions on the integer pipe, from the IEEE-754 binary64
// and binary32 layouts: GB300 has 2 FP64 lanes per SM, so the conversion
// instructions of the FP64 pipe would bound the FP32-arithmetic kernels.
// double -> float: exponent rebiased by 1023 - 127, the top 23 fraction bits
// kept and rounded by the next bit (ties away from zero; a carry into the
// exponent is the correct result); values below the float normal range go
// to +-0, above it to +-inf, NaN stays NaN.
__device__ __forceinline__ float to_f32(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned frac = (unsigned)(b >> 29) & 0x7fffffu;
    const unsigned rnd = (unsigned)(b >> 28) & 1u;
    unsigned r = sign | ((unsigned)e << 23) | frac;
    r += rnd;
    const bool nan = ((hi >> 20) & 0x7ffu) == 0x7ffu && (b & 0xfffffffffffffULL) != 0;
    r = e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u | (nan ? 0x400000u : 0u)) : r);
    return __uint_as_float(r);
}

// float -> double, exact for normal floats (subnormals go to +-0)
__device__ __forceinline__ double to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    const unsigned hi = e == 0u ? sign : (sign | ((e == 255u ? 0x7ffu : e + 896u) << 20) | (m >> 3));
    const unsigned lo = e == 0u ? 0u : (m << 29);
    return __hiloint2double((int)hi, (int)lo);
}

template <typename To, typename From>
__device__ __forceinline__ To cvt(From x);
template <>
__device__ __forceinline__ double cvt<double, double>(double x) { return x; }
template <>
__device__ __forceinline__ float cvt<float, float>(float x) { return x; }
template <>
__device__ __forceinline__ float cvt<float, double>(double x) { return to_f32(x); }
template <>
__device__ __forceinline__ double cvt<double, float>(float x) { return to_f64(x); }
// double <-> double-float: the split rounds on the integer pipe; the
// remainder takes one FP64 subtraction
template <>
__device__ __forceinline__ df64 cvt<df64, double>(double x)
{
    const float h = to_f32(x);
    return df64(h, to_f32(x - to_f64(h)));
}
template <>
__device__ __forceinline__ double cvt<double, df64>(df64 x) { return to_f64(x.hi) + to_f64(x.lo); }
template <>
__device__ __forceinline__ df64 cvt<df64, df64>(df64 x) { return x; }

// conserved -> primitive; true if rho > 0, p > 0 and both finite
template <typename R>
__device__ __forceinline__ bool to_prim(const R q[NV], R gm1, R w[NV])
{
    R ir = rcp_t<R, 2>(q[0]);
    R u = q[1] * ir, v = q[2] * ir, ww = q[3] * ir;
    R p = gm1 * fma(R(-0.5), fma(q[3], ww, fma(q[2], v, q[1] * u)), q[4]);
    w[0] = q[0];
    w[1] = u;
    w[2] = v;
    w[3] = ww;
    w[4] = p;
    return positive_finite(q[0]) && positive_finite(p);
}

// MUSCL extrapolation to the two faces of one cell (Eq. flux), per variable:
//   plus-side state  W_c + d_plus   (left state of face c+1/2)
//   minus-side state W_c - d_minus  (right state of face c-1/2)
// Limited: d_plus = d_minus = (eps/2) sigma with sigma the minmod or van Leer
// slope of the two differences (the printed kappa form reduces to this for a
// symmetric limiter).  Unlimited: the kappa form,
//   d_plus  = eps/4 [(1-kappa) dm + (1+kappa) dp],
//   d_minus = eps/4 [(1+kappa) dm + (1-kappa) dp].
template <typename R, int LIM>
__device__ __forceinline__ void face_states(R wm, R w0, R wp, R c1, R c2, R half_eps, R &plus, R &minus)
{
    R dm = w0 - wm, dp = wp - w0;
    if (LIM == SENSEI_LIM_NONE) {
        plus = w0 + (c1 * dm + c2 * dp);
        minus = w0 - (c2 * dm + c1 * dp);
    } else {
        // the limited slope sigma, then W +- (eps / 2) sigma as one fused
        // multiply-add each
        R sig, scale;
        if (LIM == SENSEI_LIM_MINMOD) {
            // minmod: the smaller difference if both have the same sign (a
            // zero difference gives 0 either way); sign and magnitude tests
            // on the bit patterns
            R m = abs_le(dm, dp) ? dm : copysign(dp, dm);
            sig = same_sign(dm, dp) ? m : R(0);
            scale = half_eps;
        } else {
            // van Leer: 2 dm dp / (dm + dp) when dm dp > 0 (the factor 2
            // joins eps / 2); the reciprocal only scales a limited slope,
            // one Newton step suffices
            R pr = dm * dp;
            R r = rcp_t<R, 1>(dm + dp);
            sig = positive(pr) ? pr * r : R(0);
            scale = R(2) * half_eps;
        }
        plus = fma(sig, scale, w0);
        minus = fma(-sig, scale, w0);
    }
}

// a1 b1 + a2 b2 + a3 b3 (+ a4 b4 + a5 b5) as a chain of fused multiply-adds
// (FP64 and FP32), or in the double-float form as one accumulation with a
// single renormalisation
template <typename R>
__device__ __forceinline__ R dot3(R a1, R b1, R a2, R b2, R a3, R b3)
{
    return fma(a3, b3, fma(a2, b2, a1 * b1));
}
template <>
__device__ __forceinline__ df64 dot3<df64>(df64 a1, df64 b1, df64 a2, df64 b2, df64 a3, df64 b3)
{
    return acc_done(acc_fma(a3, b3, acc_fma(a2, b2, acc_mul(a1, b1))));
}
template <typename R>
__device__ __forceinline__ R dot5(R a1, R b1, R a2, R b2, R a3, R b3, R a4, R b4, R a5, R b5)
{
    return fma(a5, b5, fma(a4, b4, fma(a3, b3, fma(a2, b2, a1 * b1))));
}
template <>
__device__ __forceinline__ df64 dot5<df64>(df64 a1, df64 b1, df64 a2, df64 b2, df64 a3, df64 b3, df64 a4, df64 b4,
                                           df64 a5, df64 b5)
{
    return acc_done(acc_fma(a5, b5, acc_fma(a4, b4, acc_fma(a3, b3, acc_fma(a2, b2, acc_mul(a1, b1))))));
}

// Roe flux through a face of unit normal n and area A between primitive
// states wl, wr: A/2 [F(wl) + F(wr) - sum_k |lam_k| alpha_k r_k], three-wave
// form, Harten's entropy fix on the acoustic waves (delta = fix * a).
// Arranged for few operations: A/2 joins the wave speeds, so the flux is
// one fused multiply-add per component; the energy row of the dissipation
// uses D_4 = u . (D_1, D_2, D_3) + (H - q^2) s13 - q^2/2 c2 (exact algebra
// on the three-wave sum); halvings of positive values on the integer pipe.
template <typename R>
__device__ __forceinline__ void roe_flux(const R wl[NV], const R wr[NV], R nx, R ny, R nz, R A, R gm1, R kg,
                                         R fix, R ifix, R F[NV])
{
    const R rl = wl[0], ul = wl[1], vl = wl[2], zl = wl[3], pl = wl[4];
    const R rr = wr[0], ur = wr[1], vr = wr[2], zr = wr[3], pr = wr[4];
    // products and sums as explicit fused multiply-adds (FP64 contracts them
    // anyway; double-float forms each in one operation)
    const R vnl = dot3(nx, ul, ny, vl, nz, zl);
    const R vnr = dot3(nx, ur, ny, vr, nz, zr);
    const R rhl = fma(half_pos(rl), dot3(ul, ul, vl, vl, zl, zl), kg * pl);   // rho h_t
    const R rhr = fma(half_pos(rr), dot3(ur, ur, vr, vr, zr, zr), kg * pr);
    const R ml = rl * vnl, mr = rr * vnr;
    const R psum = pl + pr;
    R c[NV];
    c[0] = ml + mr;
    c[1] = dot3(ml, ul, mr, ur, nx, psum);
    c[2] = dot3(ml, vl, mr, vr, ny, psum);
    c[3] = dot3(ml, zl, mr, zr, nz, psum);
    c[4] = fma(rhr, vnr, rhl * vnl);
    // Roe average with weights sqrt(rho): with q = 1/sqrt(rl rr) and
    // t = sqrt(rr/rl) = rr q, phi = (phi_l + t phi_r)/(1+t), the averaged
    // density sqrt(rl rr) = rl rr q and the averaged enthalpy
    // (H_l + t H_r)/(1+t) with H_l + t H_r = (rhl rr + t rhr rl) q^2.
    // These only enter the dissipation term: one Newton step suffices.
    const R rlr = rl * rr;
    const R qq = rsqrt1_t(rlr);
    const R t = rr * qq;
    const R wL = rcp_t<R, 1>(R(1) + t);
    const R u = wL * fma(t, ur, ul), v = wL * fma(t, vr, vl), w = wL * fma(t, zr, zl);
    const R H = wL * (fma(t * rhr, rl, rhl * rr) * (qq * qq));
    const R rho = rlr * qq;
    const R q2 = dot3(u, u, v, v, w, w);
    const R hq2 = R(0.5) * q2;
    const R a2 = gm1 * (H - hq2);
    const R ia = rsqrt1_t(a2);
    const R a = a2 * ia;
    const R ia2 = ia * ia;
    const R vn = dot3(nx, u, ny, v, nz, w);
    const R dr = rr - rl, dp = pr - pl, du = ur - ul, dv = vr - vl, dw = zr - zl, dvn = vnr - vnl;
    R l1 = abs_bits(vn - a), l3 = abs_bits(vn + a);
    R l2 = abs_bits(vn);
    const R delta = fix * a;
    // |lambda| < delta on the integer pipe (both are >= 0)
    // (lambda^2 / delta + delta) / 2 with 1/delta = ia / fix
    if (lt_nonneg(l1, delta)) l1 = R(0.5) * fma(l1 * l1, ia * ifix, delta);
    if (lt_nonneg(l3, delta)) l3 = R(0.5) * fma(l3 * l3, ia * ifix, delta);
    // the wave speeds times A/2
    const R h = R(0.5) * A;
    l1 = h * l1;
    l2 = h * l2;
    l3 = h * l3;
    const R rad = rho * a * dvn;
    const R hia2 = half_pos(ia2);
    const R c1w = l1 * ((dp - rad) * hia2);
    const R c3w = l3 * ((dp + rad) * hia2);
    const R c2w = l2 * fma(-dp, ia2, dr);
    const R cs = l2 * rho;
    const R s13 = c1w + c3w, d13 = c3w - c1w;
    const R D0 = s13 + c2w;
    const R g = fma(a, d13, -(cs * dvn));
    const R D1 = dot3(u, D0, nx, g, cs, du);
    const R D2 = dot3(v, D0, ny, g, cs, dv);
    const R D3 = dot3(w, D0, nz, g, cs, dw);
    const R D4 = dot5(u, D1, v, D2, w, D3, H - q2, s13, -hq2, c2w);
    F[0] = fma(h, c[0], -D0);
    F[1] = fma(h, c[1], -D1);
    F[2] = fma(h, c[2], -D2);
    F[3] = fma(h, c[3], -D3);
    F[4] = fma(h, c[4], -D4);
}

// The face flux from the two reconstructed states (primitive, or conserved
// when p.cons is set).
// One inlined copy of the Roe flux per call site (the branch only converts
// the states).
template <typename R>
__device__ __forceinline__ void face_flux(R L[NV], R Rt[NV], R nx, R ny, R nz, R A, R gm1, R kg, R fix, R ifix, int cons,
                                          R F[NV])
{
    R wl[NV], wr[NV];
    if (cons) {
        to_prim(L, gm1, wl);
        to_prim(Rt, gm1, wr);
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            wl[v] = L[v];
            wr[v] = Rt[v];
        }
    }
    roe_flux(wl, wr, nx, ny, nz, A, gm1, kg, fix, ifix, F);
}

// Loads a cell of the stage input (storage type TS) as the arithmetic type R.
template <typename R, typename TS>
struct CellLoader {
    const TS *in;
    StateLayout L;
    int ni, nj, nk;
    __device__ __forceinline__ bool inside(int i, int j, int k) const
    {
        return i >= -NG && i < ni + NG && j >= -NG && j < nj + NG && k >= -L.gk && k < nk + L.gk;
    }
    __device__ __forceinline__ void raw(int i, int j, int k, R q[NV]) const
    {
        if (inside(i, j, k)) {
            const TS *c = in + L.off + (long long)k * L.sk + (long long)j * L.sj + i;
#pragma unroll
            for (int v = 0; v < NV; ++v) q[v] = cvt<R, TS>(__ldg(c + v * L.sv));
        } else {   // outside the ghosted box: a harmless state, never used by a valid face
            q[0] = R(1);
            q[1] = q[2] = q[3] = R(0);
            q[4] = R(2.5);
        }
    }
};

// One face-metric value (index into the 12 arrays of mvolume) in the
// arithmetic type: converted from FP64, or, for double-float, read from the
// copy split once at grid set-up.
template <typename R>
__device__ __forceinline__ R face_metric(const double *fm, const float2 *, long long idx)
{
    return cvt<R, double>(fm[idx]);
}
template <>
__device__ __forceinline__ df64 face_metric<df64>(const double *, const float2 *fdm, long long idx)
{
    const float2 v = __ldg(fdm + idx);
    return df64(v.x, v.y);
}

// Convert a loaded cell to the reconstructed variables; flag non-physical
// interior cells.
template <typename R>
__device__ __forceinline__ void to_recon(const R q[NV], R gm1, int cons, bool interior, unsigned *err, R out[NV])
{
    R w[NV];
    bool ok = to_prim(q, gm1, w);
    if (interior && !ok) atomicOr(err, ERR_NONPHYSICAL);
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = cons ? q[v] : w[v];
}

// Face metrics of one block in the arithmetic type R.


// The output buffer of a stage for block n: FP64 (the caller's U or an FP64
// stage state) or FP32 (an FP32 stage state).
template <typename T>
__device__ __forceinline__ T *out_buffer(const BlockDev &N, double *user, int slot);
template <>
__device__ __forceinline__ double *out_buffer<double>(const BlockDev &N, double *user, int slot)
{
    return slot64(N, user, slot);
}
template <>
__device__ __forceinline__ float *out_buffer<float>(const BlockDev &N, double *, int slot)
{
    return slot32(N, slot);
}

// The ghost push: the new value q of a boundary cell is written into every
// ghost cell it feeds (the ghost rules of the boundary fill, applied from
// the producing side): interface and periodic ghosts of layer m+1 for the
// cell m cells inside a face, the mirrored wall ghost of layer m+1, both
// extrapolation ghosts from the boundary cell; inflow ghosts are fixed and
// caller-written (external) ghosts are the caller's.
//
// It is held per work item in affine form: for each face f,
// the ghost cell that cell m of the face's line (t1, t2) feeds is element
// off + t1 a1 + t2 a2 + m a3 of the target array dst (the neighbour's for
// an interface, the block's own otherwise), variables sv apart.  kind:
// PUSH_NONE (inflow, caller-written), PUSH_COPY (interface, periodic: the
// ghost of layer m+1), PUSH_EXTRAP (from the boundary cell into both
// layers), PUSH_WALL (the mirrored ghost of layer m+1).  Set up once per
// item by one thread per face (push_face_setup), used by push_affine (NF:
// the block's faces, 4 in 2D), so that a boundary cell's push is inlined
// arithmetic with no per-cell walk through the block descriptors.
enum { PUSH_NONE = 0, PUSH_COPY = 1, PUSH_EXTRAP = 2, PUSH_WALL = 3 };
struct PushFace {
    void *dst;
    long long off, a1, a2, a3, sv;
    int kind;
};

template <typename R>
__device__ __forceinline__ void push_face_setup(const BatchParams<R> &p, const BlockDev &B, int b, int f,
                                                PushFace &pf)
{
    const int type = B.bc_type[f];
    const BlockDev *T = &B;
    double *user = p.user[b];
    int tf = f;
    pf.kind = PUSH_NONE;
    pf.dst = nullptr;
    pf.off = pf.a1 = pf.a2 = pf.a3 = pf.sv = 0;
    if (type == SENSEI_BC_INTERFACE) {
        T = &p.blocks[B.nbr[f]];
        user = p.user[B.nbr[f]];
        tf = B.nbr_face[f];
        pf.kind = PUSH_COPY;
    } else if (type == SENSEI_BC_PERIODIC) {
        tf = f ^ 1;
        pf.kind = PUSH_COPY;
    } else if (type == SENSEI_BC_EXTRAPOLATE) {
        pf.kind = PUSH_EXTRAP;
    } else if (type == SENSEI_BC_SLIP_WALL) {
        pf.kind = PUSH_WALL;
    }
    if (pf.kind == PUSH_NONE) return;
    pf.dst = p.out_slot >= SLOT_X0 ? (void *)slot32(*T, p.out_slot) : (void *)slot64(*T, user, p.out_slot);
    int gi, gj, gk, a, c, d;
    long long e[4];
    const int probe[4][3] = {{0, 0, 1}, {1, 0, 1}, {0, 1, 1}, {0, 0, 2}};   // (t1, t2, layer)
    for (int n = 0; n < 4; ++n) {
        face_cells(tf, T->ni, T->nj, T->nk, probe[n][0], probe[n][1], probe[n][2], 0, gi, gj, gk, a, c, d);
        e[n] = cell_index(T->L, gi, gj, gk);
    }
    pf.off = e[0];
    pf.a1 = e[1] - e[0];
    pf.a2 = e[2] - e[0];
    pf.a3 = e[3] - e[0];
    pf.sv = T->L.sv;
}

template <typename T, int NF>
__device__ __forceinline__ void push_affine(const PushFace *pf, const BlockDev &B, int i, int j, int k,
                                            const T q[NV])
{
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int m = f == 0 ? i : f == 1 ? B.ni - 1 - i : f == 2 ? j : f == 3 ? B.nj - 1 - j : f == 4 ? k
                                                                                                   : B.nk - 1 - k;
        const int kind = pf[f].kind;
        if (m > 1 || kind == PUSH_NONE || (kind == PUSH_EXTRAP && m != 0)) continue;
        int t1, t2;
        tangential(f, i, j, k, t1, t2);
        T *dst = reinterpret_cast<T *>(pf[f].dst);
        const long long g = pf[f].off + t1 * pf[f].a1 + t2 * pf[f].a2 + m * pf[f].a3, sv = pf[f].sv;
        if (kind == PUSH_WALL) {
            double nx, ny, nz;
            boundary_normal(B, f, t1, t2, nx, ny, nz);
            const T tx = (T)nx, ty = (T)ny, tz = (T)nz;
            const T mn = q[1] * tx + q[2] * ty + q[3] * tz;
            dst[g] = q[0];
            dst[g + sv] = q[1] - T(2) * mn * tx;
            dst[g + 2 * sv] = q[2] - T(2) * mn * ty;
            dst[g + 3 * sv] = q[3] - T(2) * mn * tz;
            dst[g + 4 * sv] = q[4];
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) dst[g + v * sv] = q[v];
            if (kind == PUSH_EXTRAP) {
#pragma unroll
                for (int v = 0; v < NV; ++v) dst[g + pf[f].a3 + v * sv] = q[v];
            }
        }
    }
}

// PLAIN: a Runge-Kutta stage of the Euler equations with one global step
// (the accumulating update, no local steps, no viscous residual), the
// stencil's common case, with those runtime choices fixed at compile time so
// that it carries none of the others' code (fewer registers and spills); the
// general instantiation serves residuals, local steps and viscous grids.
template <typename R, typename TS, int LIM, bool TWO_D, bool PART, bool PLAIN>
__global__ void __launch_bounds__(NTHREADS, MinCtas<R>::value) stencil_kernel(const __grid_constant__ BatchParams<R> p)
{
    const int mode = PLAIN ? MODE_ACCUM : p.mode;
    const bool local_dt = PLAIN ? false : p.local != 0;
    const bool vis = PLAIN ? false : p.vis != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SL = SmemLayout<R>;
    R *sW = reinterpret_cast<R *>(smem_raw);
    R *sPi = sW + SL::W;
    R *sPj = sPi + SL::PI;
    R *sFi = sPj + SL::PJ;
    R *sFj = sFi + SL::FI;
    R *sK = sFj + SL::FJ;
    double *sRed = reinterpret_cast<double *>(sK + SL::K + ((SL::elems * sizeof(R)) % 8 ? 1 : 0));
    __shared__ BlockDev sB;
    __shared__ PushFace sPush[6];   // the item's ghost push, face by face

    constexpr int WP = TI + 4;                 // sW row pitch
    constexpr int WPL = (TJ + 4) * WP;         // sW variable plane
    auto W_at = [&](int v, int r, int c) -> R & { return sW[v * WPL + (r + 2) * WP + (c + 2)]; };
    constexpr int PIP = TI + 2, PIV = TJ * PIP, PIS = NV * PIV;
    constexpr int PJP = TI, PJV = (TJ + 2) * PJP, PJS = NV * PJV;
    constexpr int FIP = TI + 1, FIV = TJ * FIP;
    constexpr int FJP = TI, FJV = (TJ + 1) * FJP;
    constexpr int NFACES = TWO_D ? 4 : 6;

    const int t = threadIdx.x;
    const int ti = t % TI, tj = t / TI;

    const R gm1 = p.gamma - R(1);
    const R kg = p.gamma / gm1;
    const R c1 = p.eps * (R(1) - p.kappa) / R(4);
    const R c2 = p.eps * (R(1) + p.kappa) / R(4);
    const R half_eps = p.eps / R(2);
    const int cons = p.cons;
    const bool update = mode != MODE_RESIDUAL;
    const double dt = update ? p.dt_scale * *p.dt_slot : 0.0;

    // persistent: CTA x takes items x, x + grid, x + 2 grid, ...
    for (long long pos = blockIdx.x; pos < p.nitems; pos += gridDim.x) {
        const long long item = p.order ? p.order[pos] : pos;
        const int b = find_block_item(p.blocks, p.nblocks, item);
        __syncthreads();   // the previous item is done with sB and the shared tiles
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
        const double *fm = B.fn;     // FP64 face metrics [family*4 + q][mvolume]
        const float2 *fdm = B.fdf;   // their double-float split (double-float grids)
        const TS *in = (p.in_slot == SLOT_X0 || p.in_slot == SLOT_X1)
                           ? reinterpret_cast<const TS *>(slot32(B, p.in_slot))
                           : reinterpret_cast<const TS *>(slot64(B, p.user[b], p.in_slot));
        const double *un = p.user[b];
        double *out64 = mode == MODE_ACCUM ? slot64(B, p.user[b], p.out_slot) : nullptr;
        CellLoader<R, TS> ld{in, L, B.ni, B.nj, B.nk};

        // per-thread FP64 norm accumulators (touched once per plane; under
        // the register budget the compiler may keep them in local memory)
        double nsq[NV], nmax[NV], ncons[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) nsq[v] = nmax[v] = ncons[v] = 0.0;

        // per-thread k-window of the own column: the centre plane (in
        // registers until the plane's P0 puts it in sW), planes k+1 and k+2
        // in sK[kb] and sK[kb ^ 1] (each thread its own entries), the
        // plus-side k-state of the centre plane and the flux of its lower
        // k-face in registers.  The window opens one plane early: the
        // iteration k = k0 - 1 only forms the flux of face k0 - 1/2, through
        // the same face loop as every other face.
        R Wc[NV], Pp[NV], Fkm[NV];
        int kb = 0;
        if (!TWO_D) {
            R q[NV];
            R Wm2[NV], W0[NV], W1[NV];
            ld.raw(ci, cj, k0 - 2, q);
            to_recon(q, gm1, cons, false, p.err, Wm2);
            ld.raw(ci, cj, k0 - 1, q);
            to_recon(q, gm1, cons, false, p.err, Wc);
            ld.raw(ci, cj, k0, q);
            to_recon(q, gm1, cons, col_valid, p.err, W0);
            ld.raw(ci, cj, k0 + 1, q);
            to_recon(q, gm1, cons, col_valid && k0 + 1 < B.nk, p.err, W1);
            // plus-side state of plane k0 - 1 (left state of face k0 - 1/2)
            R dummy;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                face_states<R, LIM>(Wm2[v], Wc[v], W0[v], c1, c2, half_eps, Pp[v], dummy);
                sK[v * NTHREADS + t] = W0[v];
                sK[(NV + v) * NTHREADS + t] = W1[v];
                Fkm[v] = R(0);
            }
        }

        for (int k = TWO_D ? k0 : k0 - 1; k < k1; ++k) {
            const bool warm = !TWO_D && k < k0;
            // ---- P0: the centre plane with its halo into shared memory
            R pre[NV];
            if (!TWO_D) {
                ld.raw(ci, cj, k + 3, pre);   // prefetch the plane entering the window
#pragma unroll
                for (int v = 0; v < NV; ++v) W_at(v, tj, ti) = Wc[v];
                // halo ring: 2 columns each side of the TJ rows, 2 rows each side of the TI columns
                for (int e = warm ? NTHREADS : t; e < 4 * TJ + 4 * TI; e += NTHREADS) {
                    int r, c;
                    if (e < 4 * TJ) {
                        r = e >> 2;
                        int sd = e & 3;
                        c = sd < 2 ? sd - 2 : TI + sd - 2;
                    } else {
                        int e2 = e - 4 * TJ;
                        int sd = e2 / TI;
                        c = e2 % TI;
                        r = sd < 2 ? sd - 2 : TJ + sd - 2;
                    }
                    R q[NV];
                    R w[NV];
                    ld.raw(i0 + c, j0 + r, k, q);
                    to_recon(q, gm1, cons, false, p.err, w);
#pragma unroll
                    for (int v = 0; v < NV; ++v) W_at(v, r, c) = w[v];
                }
            } else {
                for (int e = t; e < (TJ + 4) * (TI + 4); e += NTHREADS) {
                    int r = e / (TI + 4) - 2, c = e % (TI + 4) - 2;
                    bool corner = (r < 0 || r >= TJ) && (c < 0 || c >= TI);
                    if (corner) continue;
                    R q[NV];
                    R w[NV];
                    int gi = i0 + c, gj = j0 + r;
                    ld.raw(gi, gj, 0, q);
                    to_recon(q, gm1, cons,
                             gi >= 0 && gi < B.ni && gj >= 0 && gj < B.nj && r >= 0 && r < TJ && c >= 0 && c < TI,
                             p.err, w);
#pragma unroll
                    for (int v = 0; v < NV; ++v) W_at(v, r, c) = w[v];
                }
            }
            __syncthreads();

            // ---- P1: face states, i direction (cells -1..TI of every row)
            //      and j direction (rows -1..TJ of every column)
            for (int e = warm ? TJ * (TI + 2) + (TJ + 2) * TI : t; e < TJ * (TI + 2) + (TJ + 2) * TI; e += NTHREADS) {
                // the centre cell in sW, the stride to its neighbours along
                // the direction, and where its two face states go
                int wc, ws;
                R *dst;
                int dstride;
                if (e < TJ * (TI + 2)) {
                    int r = e / (TI + 2), c = e % (TI + 2) - 1;
                    wc = (r + 2) * WP + (c + 2);
                    ws = 1;
                    dst = sPi + r * PIP + (c + 1);
                    dstride = PIV;
                } else {
                    int e2 = e - TJ * (TI + 2);
                    int r = e2 / TI - 1, c = e2 % TI;
                    wc = (r + 2) * WP + (c + 2);
                    ws = WP;
                    dst = sPj + (r + 1) * PJP + c;
                    dstride = PJV;
                }
                const int side = dstride == PIV ? PIS : PJS;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const R *wv = sW + v * WPL + wc;
                    R pl, mn;
                    face_states<R, LIM>(wv[-ws], wv[0], wv[ws], c1, c2, half_eps, pl, mn);
                    dst[v * dstride] = pl;
                    dst[side + v * dstride] = mn;
                }
            }
            __syncthreads();

            // ---- P2: Roe flux of every face of the tile, once each, through
            //      one copy of the flux code: first each thread's own face
            //      k+1/2 (left = plus state of plane k, right = minus state
            //      of plane k+1), then the i-faces and j-faces from the
            //      shared face states
            const long long kpl = (long long)k * ml.mplane;
            constexpr int NKF = TWO_D ? 0 : NTHREADS;
            constexpr int NIJ = TJ * (TI + 1) + (TJ + 1) * TI;
            R Fkp[NV], Ppn[NV], Rk[NV];
            if (!TWO_D) {
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    face_states<R, LIM>(W_at(v, tj, ti), sK[(kb * NV + v) * NTHREADS + t],
                                        sK[((kb ^ 1) * NV + v) * NTHREADS + t], c1, c2, half_eps, Ppn[v], Rk[v]);
            }
#pragma unroll 1
            for (int e = t; e < (warm ? NKF : NKF + NIJ); e += NTHREADS) {
                R Lf[NV], Rf[NV], F[NV];
                int fam, fi, fj;
                long long fplane;
                R *dst = nullptr;
                int vstride = 0;
                bool valid;
                if (e < NKF) {   // e == t
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        Lf[v] = Pp[v];
                        Rf[v] = Rk[v];
                    }
                    fam = 2;
                    fi = min(ci, B.ni - 1);
                    fj = min(cj, B.nj - 1);
                    fplane = (long long)(k + 1) * ml.mplane;
                    valid = true;
                } else if (e < NKF + TJ * (TI + 1)) {
                    const int f = e - NKF;
                    const int r = f / (TI + 1), c = f % (TI + 1);   // face between cells c-1 and c of row r
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        Lf[v] = sPi[v * PIV + r * PIP + c];
                        Rf[v] = sPi[PIS + v * PIV + r * PIP + (c + 1)];
                    }
                    fam = 0;
                    fi = i0 + c;
                    fj = j0 + r;
                    fplane = kpl;
                    dst = sFi + r * FIP + c;
                    vstride = FIV;
                    valid = fi <= B.ni && fj < B.nj;
                } else {
                    const int f = e - NKF - TJ * (TI + 1);
                    const int r = f / TI, c = f % TI;              // face between rows r-1 and r of column c
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        Lf[v] = sPj[v * PJV + r * PJP + c];
                        Rf[v] = sPj[PJS + v * PJV + (r + 1) * PJP + c];
                    }
                    fam = 1;
                    fi = i0 + c;
                    fj = j0 + r;
                    fplane = kpl;
                    dst = sFj + r * FJP + c;
                    vstride = FJV;
                    valid = fi < B.ni && fj <= B.nj;
                }
                R nx = R(1), ny = R(0), nz = R(0), A = R(0);
                if (valid) {
                    const long long m = (long long)(fam * 4) * ml.mvolume + fplane + (long long)fj * ml.mpitch + fi;
                    nx = face_metric<R>(fm, fdm, m);
                    ny = face_metric<R>(fm, fdm, ml.mvolume + m);
                    nz = face_metric<R>(fm, fdm, 2 * ml.mvolume + m);
                    A = face_metric<R>(fm, fdm, 3 * ml.mvolume + m);
                }
                face_flux(Lf, Rf, nx, ny, nz, A, gm1, kg, p.fix, p.ifix, cons, F);
                if (e < NKF) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fkp[v] = F[v];
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) dst[v * vstride] = F[v];
                }
            }
            __syncthreads();

            // ---- P3: residual, update, ghost push, norms
            if (col_valid && !warm) {
                const long long cell = L.off + (long long)k * L.sk + (long long)cj * L.sj + ci;
                const long long mc = kpl + (long long)cj * ml.mpitch + ci;
                R rres[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    R rr = (sFi[v * FIV + tj * FIP + ti + 1] - sFi[v * FIV + tj * FIP + ti]) +
                           (sFj[v * FJV + (tj + 1) * FJP + ti] - sFj[v * FJV + tj * FJP + ti]);
                    if (!TWO_D) rr += Fkp[v] - Fkm[v];
                    rres[v] = rr;
                }
                const bool boundary = ci < 2 || ci >= B.ni - 2 || cj < 2 || cj >= B.nj - 2 ||
                                      (!TWO_D && (k < 2 || k >= B.nk - 2));
                {
                    const double ivol = B.ivol[mc];
                    const double vol = B.vol[mc];
                    const double coef = local_dt ? -p.gdt * B.dtv[mc] : -p.gdt * dt * ivol;
                    const long long rc = ((long long)k * B.nj + cj) * B.ni + ci;
                    const long long nint = (long long)B.ni * B.nj * B.nk;
                    double q64[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        double r = cvt<double, R>(rres[v]);
                        if (vis) r -= B.rvis[v * nint + rc];   // R = sum (F_i - F_nu) . S
                        if (mode == MODE_RESIDUAL && p.src[b]) r -= p.src[b][v * nint + rc];
                        const double uin = cvt<double, TS>(in[cell + v * L.sv]);
                        if (mode == MODE_ACCUM) {
                            double val = p.beta * uin + coef * r;
                            if (p.alpha != 0.0) val += p.alpha * un[cell + v * L.sv];
                            out64[cell + v * L.sv] = val;
                            q64[v] = val;
                        } else {
                            p.rout[b][v * nint + rc] = r;
                        }
                        if (PART && p.partials) {
                            nsq[v] = fma(r, r, nsq[v]);
                            nmax[v] = fmax(nmax[v], fabs(r));
                            ncons[v] = fma(vol, uin, ncons[v]);
                        }
                    }
                    if (p.push && boundary && mode == MODE_ACCUM) push_affine<double, NFACES>(sPush, B, ci, cj, k, q64);
                }
            }
            if (!TWO_D) {
                R q[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    Fkm[v] = Fkp[v];
                    Pp[v] = Ppn[v];
                    Wc[v] = sK[(kb * NV + v) * NTHREADS + t];
                    q[v] = pre[v];
                }
                R w3[NV];
                to_recon(q, gm1, cons, col_valid && k + 3 < B.nk, p.err, w3);
#pragma unroll
                for (int v = 0; v < NV; ++v) sK[(kb * NV + v) * NTHREADS + t] = w3[v];
                kb ^= 1;
            }
        }

        // ---- FP64 norm partials of this item, fixed-order reduction
        if (PART && p.partials) {
            const int lane = t & 31, warp = t >> 5;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double a = nsq[v], bm = nmax[v], c = ncons[v];
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
                    double x = sRed[t * (NTHREADS / 32) + w];
                    acc = kind == 1 ? fmax(acc, x) : acc + x;
                }
                p.partials[item * 3 * NV + t] = acc;
            }
        }
    }
}

// PART: the variant that accumulates the norm partials (the first stage of
// a step, residual evaluations); the other stages run without its registers
template <typename R, typename TS, bool PART>
struct StencilLauncher {
    using Fn = void (*)(const BatchParams<R>);
    template <bool PLAIN>
    static Fn pick_plain(int limiter, bool two_d)
    {
        switch (limiter) {
        case SENSEI_LIM_NONE: return two_d ? stencil_kernel<R, TS, SENSEI_LIM_NONE, true, PART, PLAIN>
                                           : stencil_kernel<R, TS, SENSEI_LIM_NONE, false, PART, PLAIN>;
        case SENSEI_LIM_MINMOD: return two_d ? stencil_kernel<R, TS, SENSEI_LIM_MINMOD, true, PART, PLAIN>
                                             : stencil_kernel<R, TS, SENSEI_LIM_MINMOD, false, PART, PLAIN>;
        default: return two_d ? stencil_kernel<R, TS, SENSEI_LIM_VANLEER, true, PART, PLAIN>
                              : stencil_kernel<R, TS, SENSEI_LIM_VANLEER, false, PART, PLAIN>;
        }
    }
    static Fn pick(int limiter, bool two_d, bool plain)
    {
        return plain ? pick_plain<true>(limiter, two_d) : pick_plain<false>(limiter, two_d);
    }
    // a Runge-Kutta stage of the Euler equations with one global step
    static bool plain(const BatchParams<R> &p) { return p.mode == MODE_ACCUM && !p.local && !p.vis; }
    static cudaError_t prepare(Fn fn)
    {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SmemLayout<R>::bytes);
        if (e != cudaSuccess) return e;
        // all of the unified L1/shared storage as shared memory, so that the
        // register-limited number of CTAs per SM is not cut by the carveout
        return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    static cudaError_t launch(const BatchParams<R> &p, int limiter, bool two_d, int grid, cudaStream_t s)
    {
        Fn fn = pick(limiter, two_d, plain(p));
        cudaError_t e = prepare(fn);
        if (e != cudaSuccess) return e;
        fn<<<grid, NTHREADS, SmemLayout<R>::bytes, s>>>(p);
        return cudaGetLastError();
    }
    // the smaller of the plain and the general instantiation's resident CTAs
    static int ctas_per_sm(int limiter, bool two_d)
    {
        int best = 1 << 30;
        for (int pl = 0; pl < 2; ++pl) {
            Fn fn = pick(limiter, two_d, pl != 0);
            if (prepare(fn) != cudaSuccess) return 0;
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NTHREADS, SmemLayout<R>::bytes) != cudaSuccess)
                return 0;
            best = n < best ? n : best;
        }
        return best;
    }
};

}  // namespace sensei
