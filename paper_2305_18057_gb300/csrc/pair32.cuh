// pair32.cuh -- paired FP32 arithmetic for the 3D FP32 stencil: two
// independent face computations carried in one register pair and advanced
// by one packed instruction (add / mul / fma on .f32x2, sm_100 and later),
// which halves the issue slots of the MUSCL reconstruction and the Roe flux.
// Reciprocals, square roots, compares and selects act on each half.
//
// Every packed operation rounds each half exactly as its scalar FP32
// counterpart would.  The formulas are those of the scalar FP32 code in
// stencil.cuh (face_states, roe_flux, to_prim); a few products that the
// scalar code fuses with a negated addend are rounded separately here, so
// that no sign-flip constant is needed (packed arithmetic has no negation
// modifier), which moves results by a rounding of FP32.
#pragma once

#include "stencil.cuh"

namespace sensei {

struct P2 {
    float2 v;
};

__device__ __forceinline__ P2 mk2(float a, float b)
{
    P2 r;
    r.v = make_float2(a, b);
    return r;
}
__device__ __forceinline__ P2 sp2(float a) { return mk2(a, a); }
__device__ __forceinline__ P2 operator+(P2 a, P2 b)
{
    P2 r;
    r.v = __fadd2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ P2 operator*(P2 a, P2 b)
{
    P2 r;
    r.v = __fmul2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ P2 pfma(P2 a, P2 b, P2 c)
{
    P2 r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
}
// a - b: the packed subtraction of PTX (sub.rn.f32x2), no constant operand
__device__ __forceinline__ P2 operator-(P2 a, P2 b)
{
    unsigned long long x, y, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.v.x), "f"(a.v.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.v.x), "f"(b.v.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    P2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.v.x), "=f"(o.v.y) : "l"(r));
    return o;
}
__device__ __forceinline__ P2 pabs(P2 a) { return mk2(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ P2 prcp(P2 a) { return mk2(rcp_approx(a.v.x), rcp_approx(a.v.y)); }
__device__ __forceinline__ P2 prsqrt(P2 a) { return mk2(rsqrt_approx(a.v.x), rsqrt_approx(a.v.y)); }
// per half: c > 0 (bit pattern: positive, nonzero, not NaN) ? a : 0
__device__ __forceinline__ P2 keep_if_pos(P2 c, P2 a)
{
    return mk2(positive(c.v.x) ? a.v.x : 0.0f, positive(c.v.y) ? a.v.y : 0.0f);
}
// per half: l < d (both >= 0, by the bit patterns) ? a : b
__device__ __forceinline__ P2 sel_lt(P2 l, P2 d, P2 a, P2 b)
{
    return mk2(lt_nonneg(l.v.x, d.v.x) ? a.v.x : b.v.x, lt_nonneg(l.v.y, d.v.y) ? a.v.y : b.v.y);
}

// The two MUSCL face states (Eq. flux) of the face between cells 1 and 2 of
// a line of four cells w0..w3 of one variable: the plus-side state of cell 1
// (left state) and the minus-side state of cell 2 (right state).  Limited:
// W -+ (eps/2) sigma with the minmod or van Leer slope of the cell's two
// differences; unlimited: the kappa form.  c1 = eps (1 - kappa) / 4,
// c2 = eps (1 + kappa) / 4, he = eps / 2.
template <int LIM>
__device__ __forceinline__ void line_states2(P2 w0, P2 w1, P2 w2, P2 w3, P2 c1, P2 c2, P2 he, P2 &L, P2 &R)
{
    // he: eps / 2 (minmod) or eps (van Leer, where the factor 2 of the
    // slope joins it); the minus-side state is w2 - sigma he
    const P2 dm = w1 - w0, d0 = w2 - w1, dp = w3 - w2;
    if (LIM == SENSEI_LIM_NONE) {
        L = w1 + pfma(c2, d0, c1 * dm);
        R = w2 - pfma(c1, dp, c2 * d0);
    } else if (LIM == SENSEI_LIM_MINMOD) {
        float s1[2], s2[2];
        const float a[2] = {dm.v.x, dm.v.y}, b[2] = {d0.v.x, d0.v.y}, c[2] = {dp.v.x, dp.v.y};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float m1 = abs_le(a[h], b[h]) ? a[h] : copysignf(b[h], a[h]);
            s1[h] = same_sign(a[h], b[h]) ? m1 : 0.0f;
            const float m2 = abs_le(b[h], c[h]) ? b[h] : copysignf(c[h], b[h]);
            s2[h] = same_sign(b[h], c[h]) ? m2 : 0.0f;
        }
        L = pfma(mk2(s1[0], s1[1]), he, w1);
        R = w2 - mk2(s2[0], s2[1]) * he;
    } else {
        // van Leer: 2 dm dp / (dm + dp) when dm dp > 0 (he carries the 2)
        const P2 pr1 = dm * d0, pr2 = d0 * dp;
        const P2 s1 = keep_if_pos(pr1, pr1 * prcp(dm + d0));
        const P2 s2 = keep_if_pos(pr2, pr2 * prcp(d0 + dp));
        L = pfma(s1, he, w1);
        R = w2 - s2 * he;
    }
}

// conserved -> primitive of a pair of cells; ok_x: the x half is physical
__device__ __forceinline__ void to_prim2(const P2 q[NV], P2 gm1, P2 w[NV], bool &ok_x)
{
    const P2 ir = prcp(q[0]);
    const P2 u = q[1] * ir, v = q[2] * ir, ww = q[3] * ir;
    const P2 p = gm1 * pfma(sp2(-0.5f), pfma(q[3], ww, pfma(q[2], v, q[1] * u)), q[4]);
    w[0] = q[0];
    w[1] = u;
    w[2] = v;
    w[3] = ww;
    w[4] = p;
    ok_x = positive_finite(q[0].v.x) && positive_finite(p.v.x);
}

// The Roe flux of two faces at once (three-wave form, Harten's entropy fix
// on the acoustic waves, delta = fix * a): the operations of roe_flux in
// stencil.cuh, each on a pair.  nx, ny, nz: unit normals; A: areas.
__device__ __forceinline__ void roe_flux2(const P2 wl[NV], const P2 wr[NV], P2 nx, P2 ny, P2 nz, P2 A, P2 gm1, P2 kg,
                                          P2 fix, P2 ifix, P2 F[NV])
{
    const P2 half = sp2(0.5f);
    const P2 rl = wl[0], ul = wl[1], vl = wl[2], zl = wl[3], pl = wl[4];
    const P2 rr = wr[0], ur = wr[1], vr = wr[2], zr = wr[3], pr = wr[4];
    const P2 vnl = pfma(nz, zl, pfma(ny, vl, nx * ul));
    const P2 vnr = pfma(nz, zr, pfma(ny, vr, nx * ur));
    const P2 rhl = pfma(half * rl, pfma(zl, zl, pfma(vl, vl, ul * ul)), kg * pl);
    const P2 rhr = pfma(half * rr, pfma(zr, zr, pfma(vr, vr, ur * ur)), kg * pr);
    const P2 ml = rl * vnl, mr = rr * vnr;
    const P2 psum = pl + pr;
    P2 c[NV];
    c[0] = ml + mr;
    c[1] = pfma(nx, psum, pfma(mr, ur, ml * ul));
    c[2] = pfma(ny, psum, pfma(mr, vr, ml * vl));
    c[3] = pfma(nz, psum, pfma(mr, zr, ml * zl));
    c[4] = pfma(rhr, vnr, rhl * vnl);
    const P2 rlr = rl * rr;
    const P2 qq = prsqrt(rlr);
    const P2 t = rr * qq;
    const P2 wL = prcp(sp2(1.0f) + t);
    const P2 u = wL * pfma(t, ur, ul), v = wL * pfma(t, vr, vl), w = wL * pfma(t, zr, zl);
    const P2 H = wL * (pfma(t * rhr, rl, rhl * rr) * (qq * qq));
    const P2 rho = rlr * qq;
    const P2 q2 = pfma(w, w, pfma(v, v, u * u));
    const P2 hq2 = half * q2;
    const P2 a2 = gm1 * (H - hq2);
    const P2 ia = prsqrt(a2);
    const P2 a = a2 * ia;
    const P2 ia2 = ia * ia;
    const P2 vn = pfma(nz, w, pfma(ny, v, nx * u));
    const P2 dr = rr - rl, dp = pr - pl, du = ur - ul, dv = vr - vl, dw = zr - zl, dvn = vnr - vnl;
    P2 l1 = pabs(vn - a), l3 = pabs(vn + a);
    P2 l2 = pabs(vn);
    const P2 delta = fix * a;
    const P2 iad = ia * ifix;
    l1 = sel_lt(l1, delta, half * pfma(l1 * l1, iad, delta), l1);
    l3 = sel_lt(l3, delta, half * pfma(l3 * l3, iad, delta), l3);
    const P2 h = half * A;
    l1 = h * l1;
    l2 = h * l2;
    l3 = h * l3;
    const P2 rad = rho * a * dvn;
    const P2 hia2 = half * ia2;
    const P2 c1w = l1 * ((dp - rad) * hia2);
    const P2 c3w = l3 * ((dp + rad) * hia2);
    const P2 c2w = l2 * (dr - dp * ia2);
    const P2 cs = l2 * rho;
    const P2 s13 = c1w + c3w, d13 = c3w - c1w;
    const P2 D0 = s13 + c2w;
    const P2 g = a * d13 - cs * dvn;
    const P2 D1 = pfma(cs, du, pfma(nx, g, u * D0));
    const P2 D2 = pfma(cs, dv, pfma(ny, g, v * D0));
    const P2 D3 = pfma(cs, dw, pfma(nz, g, w * D0));
    const P2 D4 = pfma(H - q2, s13, pfma(w, D3, pfma(v, D2, u * D1))) - hq2 * c2w;
    F[0] = h * c[0] - D0;
    F[1] = h * c[1] - D1;
    F[2] = h * c[2] - D2;
    F[3] = h * c[3] - D3;
    F[4] = h * c[4] - D4;
}

// Flux of a pair of faces from the two reconstructed states (primitive, or
// conserved when cons is set).
__device__ __forceinline__ void face_flux2(P2 L[NV], P2 Rt[NV], P2 nx, P2 ny, P2 nz, P2 A, P2 gm1, P2 kg, P2 fix,
                                           P2 ifix, int cons, P2 F[NV])
{
    if (cons) {
        P2 wl[NV], wr[NV];
        bool ok;
        to_prim2(L, gm1, wl, ok);
        to_prim2(Rt, gm1, wr, ok);
        roe_flux2(wl, wr, nx, ny, nz, A, gm1, kg, fix, ifix, F);
    } else {
        roe_flux2(L, Rt, nx, ny, nz, A, gm1, kg, fix, ifix, F);
    }
}

// double -> float for the FP32 stencil's tiles (integer pipe): round to
// nearest, ties away from zero, as to_f32; magnitudes below the float normal
// range give +-0; magnitudes of 2^128 and above, infinities and NaNs give a
// NaN (a state that large is non-physical either way).  The exponent is
// rebiased by adding 2^30 to the word formed from the top exponent bits and
// mantissa (the low 8 exponent bits of a double in the float range are the
// float exponent minus 128, modulo 256).
__device__ __forceinline__ float to_f32_tile(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d) + 0x10000000ULL;   // rounding bit
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned m = __funnelshift_l(lo, hi, 3) + 0x40000000u;
    const unsigned sign = (unsigned)(__double_as_longlong(d) >> 32) & 0x80000000u;
    const unsigned ax = (unsigned)(__double_as_longlong(d) >> 32) & 0x7fffffffu;
    unsigned r = (m & 0x7fffffffu) | sign;
    r = ax < 0x38100000u ? sign : r;
    r = ax >= 0x47f00000u ? 0x7fffffffu : r;
    return __uint_as_float(r);
}

template <typename TS>
__device__ __forceinline__ float tile_f32(TS x);
template <>
__device__ __forceinline__ float tile_f32<double>(double x) { return to_f32_tile(x); }
template <>
__device__ __forceinline__ float tile_f32<float>(float x) { return x; }

}  // namespace sensei
