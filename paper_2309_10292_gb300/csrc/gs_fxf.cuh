// Fixed point with a float remainder for FP64 fields (GS_ARITH_FXF).
//
// GB300's FP64 pipe issues about two FMAs per clock per SM; its FP32 and
// integer pipes are 64 times wider.  A value x is held as a pair (X, l) with
//     x = (X + l) 2^-22,   X a 32-bit integer, |X| < 2^24,  l a float, |l| < 1,
// so that float(X) is exact and (X 2^-22, l 2^-22) is a double-single pair
// whose high part lies on a fixed grid.  That grid makes the six-neighbour
// sums and sum - 6u of the high parts exact integer additions (the low parts
// are summed in FP32 at 2^-22 of the magnitude); the products are float-pair
// products (an FMA recovers each high product's rounding error) with the
// coefficients stored as float pairs, pre-multiplied by dt and by 16 so that
// every product comes out in sixteenths of a unit.  Each product's high part
// is split at that grid into an integer count (exact, summed in 32 bits) and
// a float rest below 1/32 of a unit, and one rounding at the end puts the
// whole-unit part into X and the rest into l.  The storage grid is 2^-47
// absolute for |l| <= 1/2, and the float-pair products carry about 47
// significant bits, as double-single does: a step rounds at a few 1e-15,
// far inside the 1e-10 tolerance of the FP64 workload after 100 steps.
// Supported range: |u|, |v| < 4 (reported as GS_DERR_RANGE otherwise), and
// |du|, |dv| < 32 per step.  The operation structure
// follows gs_update term by term: u + dt (Du lap u - u v^2 + F (1 - u) +
// n r), v + dt (Dv lap v + u v^2 - (F + k) v), with lap x = (sum - 6x) / 6
// folded into Du / 6, Dv / 6.
#pragma once

#include <cmath>

#include "gs_common.cuh"
#include "gs_ds.cuh"

constexpr float kFxfUnit = 4194304.0f;             // 2^22: units per 1
constexpr float kFxfInvUnit = 1.0f / 4194304.0f;   // 2^-22

struct GsFxf {
    int32_t X;  // whole units
    float l;    // the rest, in units
};

// x -> (X, l).  hi + lo is x as double-single (gs_ds.cuh: hi the top 24
// bits, truncated); hi 2^22 has at most 24 bits, so its nearest integer X,
// the fraction hi 2^22 - X and float(X) are exact, and lo 2^22 joins the
// fraction with one rounding.  |x| >= 4, inf or NaN sets ovf.
GS_D GsFxf fxf_from_double(double x, bool& ovf)
{
    const GsDS d = ds_from_double(x);
    const float hs = __fmul_rn(d.hi, kFxfUnit);
    GsFxf r;
    r.X = __float2int_rn(hs);
    r.l = __fmaf_rn(d.lo, kFxfUnit, __fsub_rn(hs, __int2float_rn(r.X)));
    ovf = ((uint32_t)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu) >= 1025u;
    return r;
}

// (X + l) 2^-22 as the nearest double: X 2^-22 exactly by bit operations,
// l 2^-22 widened exactly (ds_widen), one FP64 add
GS_D double fxf_to_double(GsFxf a)
{
    const uint32_t s = a.X < 0 ? 0x80000000u : 0u;
    const uint32_t m = a.X < 0 ? 0u - (uint32_t)a.X : (uint32_t)a.X;
    const int lz = __clz(m);  // leading one at bit 31 - lz: X 2^-22 has biased exponent 1032 - lz
    const unsigned long long bits = ((unsigned long long)s << 32) | ((unsigned long long)(1032 - lz) << 52) |
                                    (((unsigned long long)m << (21 + lz)) & 0xFFFFFFFFFFFFFull);
    const double hx = m ? __longlong_as_double((long long)bits) : 0.0;
    return __dadd_rn(hx, ds_widen(__fmul_rn(a.l, kFxfInvUnit)));
}

// A pair kept in the 8 bytes of a double (X in the low word): the z-marching
// kernel converts each staged plane in place once, and the steps inside one
// gs_step call keep the fields in this form between steps.
GS_D double fxf_pack(GsFxf a)
{
    return __longlong_as_double(
        (long long)(((unsigned long long)__float_as_uint(a.l) << 32) | (unsigned long long)(uint32_t)a.X));
}

GS_D GsFxf fxf_unpack(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return GsFxf{(int32_t)(uint32_t)b, __uint_as_float((uint32_t)(b >> 32))};
}

// Coefficients as float pairs (c1 + c2 ~ the double value), all multiplied
// by dt and by 16 (products in sixteenths of a unit).
struct GsCoefFXF {
    float a1, a2;  // Du / 6 dt 16
    float b1, b2;  // Dv / 6 dt 16
    float f1, f2;  // (Du + F) dt 16
    float k1, k2;  // (Dv + F + k) dt 16
    float n1, n2;  // noise dt 4: the noise term per numerator (r = num 2^-24, 2^22 units, 16)
    float t1, t2;  // dt (u v^2 is formed in real units)
    int32_t KF;    // F dt in sixteenths of a unit, rounded ...
    float rF;      // ... and the rest
    int dt_one;    // dt == 1: the product (v^2) dt is skipped
};

inline void fxf_split_host(double d, float& hi, float& lo)
{
    hi = (float)d;
    lo = (float)(d - (double)hi);
}

inline GsCoefFXF gs_make_coef_fxf(double Du, double Dv, double F, double k, double dt, double noise)
{
    GsCoefFXF c;
    fxf_split_host(Du / 6.0 * dt * 16.0, c.a1, c.a2);
    fxf_split_host(Dv / 6.0 * dt * 16.0, c.b1, c.b2);
    fxf_split_host((Du + F) * dt * 16.0, c.f1, c.f2);
    fxf_split_host((Dv + F + k) * dt * 16.0, c.k1, c.k2);
    fxf_split_host(noise * dt * 4.0, c.n1, c.n2);
    fxf_split_host(dt, c.t1, c.t2);
    const double fs = F * dt * 67108864.0;  // 2^26 sixteenths of a unit per 1
    const double kf = std::nearbyint(fs);
    c.KF = (int32_t)kf;
    c.rF = (float)(fs - kf);
    c.dt_one = dt == 1.0;
    return c;
}

// (c1 + c2)(xh + xl) as p + e: p the rounded high product, e its rounding
// error (exact by FMA) plus the cross terms; c2 xl is below the result's
// rounding when c2 is 2^-24 of c1 (a coefficient split in two floats)
GS_D void fxf_mul(float c1, float c2, float xh, float xl, float& p, float& e)
{
    p = __fmul_rn(c1, xh);
    e = __fmaf_rn(c1, xh, -p);
    e = __fmaf_rn(c1, xl, e);
    e = __fmaf_rn(c2, xh, e);
}

// p + e in sixteenths of a unit -> the integer K nearest p and the float
// rest (p - K is exact: K and p are floats within 1/2 of each other, or p is
// already an integer)
GS_D void fxf_grid(float p, float e, int32_t& K, float& r)
{
    K = __float2int_rn(p);
    r = __fadd_rn(__fsub_rn(p, __int2float_rn(K)), e);
}

// The range check of the results: each new X, biased by 2^24, is OR-ed into
// one word (per thread, over as many cells as the caller likes); the word
// reaches 2^25 exactly when some result has |x'| >= 4.
GS_D bool fxf_range_bad(uint32_t rng) { return rng >= (1u << 25); }

// x + (T + t) / 16 units, T an integer count and t a float rest (both in
// sixteenths), renormalised to |l| <= 1/2; the new X joins the range word
GS_D GsFxf fxf_finish(GsFxf x, int32_t T, float t, uint32_t& rng)
{
    const int32_t Th = (T + 8) >> 4;  // whole units, rounded
    const float low = __int2float_rn(T - (Th << 4));
    const float l = __fmaf_rn(__fadd_rn(low, t), 0.0625f, x.l);
    const int32_t K = __float2int_rn(l);
    GsFxf r;
    r.X = x.X + Th + K;
    r.l = __fsub_rn(l, __int2float_rn(K));
    rng |= (uint32_t)(r.X + (1 << 24));
    return r;
}

// The six neighbours' sum: integer parts exactly, rests in FP32, in the
// neighbour order of gs_nsum (x-, x+, y-, y+, z-, z+)
GS_D void fxf_nsum(GsFxf xm, GsFxf xp, GsFxf ym, GsFxf yp, GsFxf zm, GsFxf zp, int32_t& S, float& SL)
{
    S = xm.X + xp.X + ym.X + yp.X + zm.X + zp.X;
    SL = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(xm.l, xp.l), ym.l), yp.l), zm.l), zp.l);
}

// gs_update in this arithmetic.  S*, SL*: the neighbour sums (fxf_nsum);
// rnum: the noise numerator (r = rnum / 2^24); rng: the range word
// (fxf_range_bad).  DT: 0 reads c.dt_one at run time, 1 knows dt == 1, 2
// knows dt != 1.
template <bool NOISE, int DT = 0>
GS_D void gs_update_fxf(const GsCoefFXF& c, GsFxf u, GsFxf v, int32_t SU, float SLU, int32_t SV, float SLV,
                        int32_t rnum, GsFxf& un, GsFxf& vn, uint32_t& rng)
{
    // the neighbour sums in units as float pairs (the integer sum rounded to
    // a float, and what that lost plus the rests' sum); Du lap u dt =
    // Du / 6 S dt - Du u dt, the second part joining F u dt in one product
    const float suh = __int2float_rn(SU), svh = __int2float_rn(SV);
    const float sul = __fadd_rn(SLU, __int2float_rn(SU - __float2int_rn(suh)));
    const float svl = __fadd_rn(SLV, __int2float_rn(SV - __float2int_rn(svh)));
    const float uh = __int2float_rn(u.X), vhu = __int2float_rn(v.X);
    // v in real units times 4, so that u (units) v^2 comes out in sixteenths
    const float vh = __fmul_rn(vhu, 4.0f * kFxfInvUnit), vl = __fmul_rn(v.l, 4.0f * kFxfInvUnit);
    // v^2 = w1 + w2 with every term: vl is an absolute rest (up to 1/2 unit),
    // not 2^-24 of vh, so vl^2 is not negligible (and always positive:
    // dropping it would bias u v^2)
    float w1 = __fmul_rn(vh, vh);
    float w2 = __fmaf_rn(vh, vh, -w1);
    w2 = __fmaf_rn(__fadd_rn(vh, vh), vl, w2);
    w2 = __fmaf_rn(vl, vl, w2);
    if (DT == 2 || (DT == 0 && !c.dt_one)) {
        float p, e;
        fxf_mul(c.t1, c.t2, w1, w2, p, e);
        w1 = p;
        w2 = e;
    }
    float q1, q2;  // u v^2 dt, with the rest-times-rest term w2 u.l for the same reason
    fxf_mul(w1, w2, uh, u.l, q1, q2);
    q2 = __fmaf_rn(w2, u.l, q2);
    float pa, ea, pb, eb, pf, ef, pk, ek;
    fxf_mul(c.a1, c.a2, suh, sul, pa, ea);   // Du / 6 S_u dt
    fxf_mul(c.b1, c.b2, svh, svl, pb, eb);   // Dv / 6 S_v dt
    fxf_mul(c.f1, c.f2, uh, u.l, pf, ef);    // (Du + F) u dt
    fxf_mul(c.k1, c.k2, vhu, v.l, pk, ek);   // (Dv + F + k) v dt
    int32_t Ka, Kb, Kq, Kf, Kk;
    float ra, rb, rq, rf, rk;
    fxf_grid(pa, ea, Ka, ra);
    fxf_grid(pb, eb, Kb, rb);
    fxf_grid(q1, q2, Kq, rq);
    fxf_grid(pf, ef, Kf, rf);
    fxf_grid(pk, ek, Kk, rk);
    // du dt = Du / 6 S_u - (Du + F) u - u v^2 + F + n r   (= Du lap u - u v^2 + F (1 - u) + n r)
    // dv dt = Dv / 6 S_v - (Dv + F + k) v + u v^2         (= Dv lap v + u v^2 - (F + k) v)
    int32_t Tu = Ka - Kq + c.KF - Kf;
    float tu = __fsub_rn(__fadd_rn(__fsub_rn(ra, rq), c.rF), rf);
    if (NOISE) {
        const float rn = __int2float_rn(rnum);
        float pn = __fmul_rn(c.n1, rn);
        float en = __fmaf_rn(c.n1, rn, -pn);
        en = __fmaf_rn(c.n2, rn, en);
        int32_t Kn;
        float rr;
        fxf_grid(pn, en, Kn, rr);
        Tu += Kn;
        tu = __fadd_rn(tu, rr);
    }
    const int32_t Tv = Kb + Kq - Kk;
    const float tv = __fsub_rn(__fadd_rn(rb, rq), rk);
    un = fxf_finish(u, Tu, tu, rng);
    vn = fxf_finish(v, Tv, tv, rng);
}

// A 2-cell group of cells whose inputs are packed pairs (fxf_pack); writes
// packed pairs (PACK) or FP64 values.
template <bool NOISE, bool PACK, int DT>
GS_D void gs_update_group_fxf(const GsCoefFXF& c, uint32_t pre, uint32_t kk2, const double* cu, const double* cv,
                              const double* pu, const double* pv, const double* nu, const double* nv,
                              const double* ymu, const double* ypu, const double* ymv, const double* ypv,
                              double xlu, double xru, double xlv, double xrv, double* ou, double* ov, uint32_t& rng)
{
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const GsFxf u = fxf_unpack(cu[e]), v = fxf_unpack(cv[e]);
        int32_t SU, SV;
        float SLU, SLV;
        fxf_nsum(fxf_unpack(e > 0 ? cu[0] : xlu), fxf_unpack(e < 1 ? cu[1] : xru), fxf_unpack(ymu[e]),
                 fxf_unpack(ypu[e]), fxf_unpack(pu[e]), fxf_unpack(nu[e]), SU, SLU);
        fxf_nsum(fxf_unpack(e > 0 ? cv[0] : xlv), fxf_unpack(e < 1 ? cv[1] : xrv), fxf_unpack(ymv[e]),
                 fxf_unpack(ypv[e]), fxf_unpack(pv[e]), fxf_unpack(nv[e]), SV, SLV);
        const int32_t rn = NOISE ? gs_group_num(pre, (uint32_t)e, kk2) : 0;
        GsFxf a, b;
        gs_update_fxf<NOISE, DT>(c, u, v, SU, SLU, SV, SLV, rn, a, b, rng);
        ou[e] = PACK ? fxf_pack(a) : fxf_to_double(a);
        ov[e] = PACK ? fxf_pack(b) : fxf_to_double(b);
    }
}
