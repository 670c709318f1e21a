// Double-single arithmetic for FP64 fields on a GPU whose FP64 pipe is
// narrow (about 2 FP64 FMAs per clock per SM on GB300, against 128 FP32
// lanes).  A value is a pair of floats (hi, lo) with x ~ hi + lo, about 48
// significant bits; the operations are the classical error-free
// transformations (Knuth's two-sum, Dekker's fast two-sum, the product error
// by a fused multiply-add), each written with explicit round-to-nearest
// intrinsics so that the compiler neither contracts nor reassociates them.
//
// Storage stays FP64.  The conversions use integer bit operations, not the
// FP64 pipe: hi takes the top 24 significant bits of the double (truncated),
// lo the remaining 29 bits rounded to 24; values below 2^-126 become 0 (the
// fields are O(1), so this is far below any tolerance).  Back to FP64 the
// two floats are widened exactly by bit operations and added with one FP64
// add.  The update follows gs_update's operation order term by term.
#pragma once

#include "gs_common.cuh"

struct GsDS {
    float hi, lo;
};

GS_D GsDS ds_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return GsDS{s, e};
}

// requires |a| >= |b| (or a == 0)
GS_D GsDS ds_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return GsDS{s, __fsub_rn(b, __fsub_rn(s, a))};
}

GS_D GsDS ds_add(GsDS x, GsDS y)
{
    GsDS s = ds_two_sum(x.hi, y.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return ds_fast_two_sum(s.hi, e);
}

GS_D GsDS ds_mul(GsDS x, GsDS y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return ds_fast_two_sum(p, e);
}

// product with a float that is exact (a small integer, -6, a noise numerator)
GS_D GsDS ds_mul_f(GsDS x, float c)
{
    const float p = __fmul_rn(x.hi, c);
    float e = __fmaf_rn(x.hi, c, -p);
    e = __fmaf_rn(x.lo, c, e);
    return ds_fast_two_sum(p, e);
}

GS_D GsDS ds_neg(GsDS x) { return GsDS{-x.hi, -x.lo}; }

GS_D GsDS ds_fma(GsDS a, GsDS b, GsDS c) { return ds_add(ds_mul(a, b), c); }

GS_D GsDS ds_from_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t h = (uint32_t)(b >> 32), l = (uint32_t)b;
    const uint32_t sign = h & 0x80000000u;
    const uint32_t ah = h & 0x7FFFFFFFu;  // |x|: biased exponent e at bits 20-30
    // hi: (h:l) << 3 puts e's low 8 bits at 23-30 and the top 23 stored bits
    // at 0-22; the float exponent e - 896 is e's low 8 bits with bit 7
    // flipped (896 = 3 * 256 + 128), exact for 897 <= e <= 1150
    const uint32_t hb = ((__funnelshift_l(l, h, 3) & 0x7FFFFFFFu) ^ 0x40000000u) | sign;
    const float hi = __uint_as_float(ah >= (897u << 20) ? hb : sign);
    // lo: the remaining 29 bits, weight 2^(e - 1075) = the float exponent
    // field of hi minus 52
    const float r = __uint2float_rn(l & 0x1FFFFFFFu);
    const float scale = __uint_as_float((hb & 0x7F800000u) - (52u << 23));
    const float lo = ah >= (949u << 20) ? __uint_as_float(sign | __float_as_uint(__fmul_rn(r, scale))) : 0.0f;
    return GsDS{hi, lo};
}

// exact float -> double by bits (float subnormals, never produced here, read as 0)
GS_D double ds_widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e8 = (u >> 23) & 0xFFu;
    if (e8 == 0) return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e8 + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}

GS_D double ds_to_double(GsDS a) { return __dadd_rn(ds_widen(a.hi), ds_widen(a.lo)); }

// Coefficients as double-single pairs (host): hi = nearest float, lo = the
// nearest float to the rest.
struct GsCoefDS {
    GsDS Du6, Dv6, F, Fk, dt, noise24, one;
    int dt_one;  // dt == 1 exactly: the products du * dt are skipped (same bits)
};

inline GsDS gs_ds_host(double d)
{
    const float hi = (float)d;
    return GsDS{hi, (float)(d - (double)hi)};
}

inline GsCoefDS gs_make_coef_ds(double Du, double Dv, double F, double k, double dt, double noise)
{
    GsCoefDS c;
    c.Du6 = gs_ds_host(Du / 6.0);
    c.Dv6 = gs_ds_host(Dv / 6.0);
    c.F = gs_ds_host(F);
    c.Fk = gs_ds_host(F + k);
    c.dt = gs_ds_host(dt);
    c.noise24 = gs_ds_host(noise / 16777216.0);
    c.one = GsDS{1.0f, 0.0f};
    c.dt_one = dt == 1.0;
    return c;
}

// sum of the six neighbours: the hi parts through error-free two-sums, their
// errors and the lo parts accumulated in one float, one renormalisation
GS_D GsDS ds_nsum(GsDS xm, GsDS xp, GsDS ym, GsDS yp, GsDS zm, GsDS zp)
{
    GsDS s = ds_two_sum(xm.hi, xp.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(xm.lo, xp.lo));
    s = ds_two_sum(s.hi, ym.hi);
    e = __fadd_rn(e, __fadd_rn(s.lo, ym.lo));
    s = ds_two_sum(s.hi, yp.hi);
    e = __fadd_rn(e, __fadd_rn(s.lo, yp.lo));
    s = ds_two_sum(s.hi, zm.hi);
    e = __fadd_rn(e, __fadd_rn(s.lo, zm.lo));
    s = ds_two_sum(s.hi, zp.hi);
    e = __fadd_rn(e, __fadd_rn(s.lo, zp.lo));
    return ds_fast_two_sum(s.hi, e);
}

// gs_update's steps in double-single (same order; rnum is the exact noise numerator)
template <bool NOISE>
GS_D void gs_update_ds(const GsCoefDS& c, GsDS u, GsDS v, GsDS su, GsDS sv, float rnum, GsDS& un, GsDS& vn)
{
    const GsDS lu = ds_add(ds_mul_f(u, -6.0f), su);            // sum - 6u
    const GsDS lv = ds_add(ds_mul_f(v, -6.0f), sv);
    const GsDS uvv = ds_mul(u, ds_mul(v, v));                   // u v^2
    GsDS du = ds_add(ds_mul(c.Du6, lu), ds_neg(uvv));           // Du lap u - u v^2
    du = ds_add(ds_mul(c.F, ds_add(c.one, ds_neg(u))), du);     // + F (1 - u)
    if (NOISE) du = ds_add(ds_mul_f(c.noise24, rnum), du);      // + n r
    GsDS dv = ds_add(ds_mul(c.Dv6, lv), uvv);                   // Dv lap v + u v^2
    dv = ds_add(ds_mul(ds_neg(c.Fk), v), dv);                   // - (F + k) v
    // u + dt du.  With dt = 1 the product is skipped: du leaves ds_add
    // through a fast two-sum, whose output it reproduces bit for bit, so the
    // result is identical either way.
    un = ds_add(c.dt_one ? du : ds_mul(du, c.dt), u);
    vn = ds_add(c.dt_one ? dv : ds_mul(dv, c.dt), v);
}

// A double-single pair kept in the 8 bytes of a double (hi in the low word):
// the z-marching kernel converts each staged plane in place once, so its
// neighbours are read already converted, and the steps inside one gs_step
// call keep the fields in this form between steps.
GS_D double ds_pack(GsDS a)
{
    return __longlong_as_double(
        (long long)(((unsigned long long)__float_as_uint(a.lo) << 32) | (unsigned long long)__float_as_uint(a.hi)));
}

GS_D GsDS ds_unpack(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return GsDS{__uint_as_float((uint32_t)b), __uint_as_float((uint32_t)(b >> 32))};
}

struct GsFromDouble {
    GS_D GsDS operator()(double x) const { return ds_from_double(x); }
};
struct GsFromPacked {
    GS_D GsDS operator()(double x) const { return ds_unpack(x); }
};

// A 2-cell group of FP64 cells (the z-marching kernels' double2 groups);
// `get` turns an input into a pair (conversion of an FP64 value, or a pair
// packed by ds_pack): the arithmetic is the same either way.  PACK: write
// the results as packed pairs (ds_pack) instead of FP64 values.
template <bool NOISE, typename Get = GsFromDouble, bool PACK = false>
GS_D void gs_update_group_ds(const GsCoefDS& c, uint32_t pre, uint32_t kk2, const double* cu, const double* cv,
                             const double* pu, const double* pv, const double* nu, const double* nv,
                             const double* ymu, const double* ypu, const double* ymv, const double* ypv,
                             double xlu, double xru, double xlv, double xrv, double* ou, double* ov, Get get = Get())
{
    GsDS u[2], v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        u[e] = get(cu[e]);
        v[e] = get(cv[e]);
    }
    const GsDS xlU = get(xlu), xrU = get(xru);
    const GsDS xlV = get(xlv), xrV = get(xrv);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const GsDS su = ds_nsum(e > 0 ? u[0] : xlU, e < 1 ? u[1] : xrU, get(ymu[e]), get(ypu[e]), get(pu[e]),
                                get(nu[e]));
        const GsDS sv = ds_nsum(e > 0 ? v[0] : xlV, e < 1 ? v[1] : xrV, get(ymv[e]), get(ypv[e]), get(pv[e]),
                                get(nv[e]));
        const float rn = NOISE ? (float)gs_group_num(pre, (uint32_t)e, kk2) : 0.0f;
        GsDS un, vn;
        gs_update_ds<NOISE>(c, u[e], v[e], su, sv, rn, un, vn);
        ou[e] = PACK ? ds_pack(un) : ds_to_double(un);
        ov[e] = PACK ? ds_pack(vn) : ds_to_double(vn);
    }
}
