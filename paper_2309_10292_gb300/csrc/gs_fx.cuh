// Fixed-point arithmetic for FP64 fields (GS_ARITH_FX).  GB300's FP64 pipe
// issues about two FMAs per clock per SM, so the FP64 stencil step is bound
// by it; its integer pipes are wide.  A value x is held as the 64-bit
// integer X = round(x * 2^52): the resolution 2^-52 equals the FP64 spacing
// at 1, and |x| < 2^11 fits.  The six-neighbour sums and the Laplacian's
// sum - 6 u are then exact integer additions, and only the products round
// (to the nearest multiple of 2^-52, ties upward), which keeps every step
// within a few 2^-52 of exact arithmetic: closer to the exact update than
// IEEE FP64 itself.  The operation structure follows gs_update term by term.
//
// Supported range: |u|, |v| < 2^10 (the Gray-Scott fields stay within about
// [-1, 2]).  A value outside it is reported (GS_DERR_RANGE) and clamped.
// Conversions use integer bit operations only, not the FP64 pipe.
#pragma once

#include <cmath>

#include "gs_common.cuh"

constexpr int kFxFrac = 52;                        // fractional bits
constexpr long long kFxOne = 1LL << kFxFrac;

// x -> round(x * 2^52); |x| >= 2^10 sets ovf and clamps the exponent
GS_D long long fx_from_double(double x, bool& ovf)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FFu);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int sh = e - 1023;  // x = m * 2^(sh - 52), X = m * 2^sh
    unsigned long long a;
    if (sh >= 0) {
        ovf = sh > 9;
        a = m << (sh > 9 ? 9 : sh);
    } else {
        ovf = false;
        const int r = -sh;  // round(m / 2^r), half up
        a = r > 54 ? 0ull : ((m >> (r - 1)) + 1ull) >> 1;
    }
    if (e == 0) a = 0;  // zero (and subnormals, far below the resolution)
    return (b >> 63) ? -(long long)a : (long long)a;
}

// X * 2^-52 as the nearest double (ties to even), by integer bit operations
GS_D double fx_to_double(long long X)
{
    if (X == 0) return 0.0;
    const unsigned long long sgn = X < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long a = X < 0 ? (unsigned long long)(-X) : (unsigned long long)X;
    const int lz = __clzll((long long)a);
    const unsigned long long n = a << lz;        // leading one at bit 63
    const unsigned long long q = n >> 11;        // 53 bits, leading one at bit 52
    const unsigned long long rem = n & 0x7FFull; // the 11 bits rounded off
    const unsigned long long up = (rem > 0x400ull || (rem == 0x400ull && (q & 1ull))) ? 1ull : 0ull;
    // value = n * 2^(-52 - lz): leading weight 2^(11 - lz), biased exponent
    // 1034 - lz; the leading one of q adds 1 to the exponent field, and a
    // rounding carry out of the mantissa moves into it as well
    const unsigned long long bits = ((unsigned long long)(1034 - lz - 1) << 52) + q + up;
    return __longlong_as_double((long long)(bits | sgn));
}

// round(a * b / 2^52) for the exact 128-bit product (rounded half up)
GS_D long long fx_mul(long long a, long long b)
{
    const long long hi = __mul64hi(a, b);
    const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
    const unsigned long long r = (lo >> kFxFrac) | ((unsigned long long)hi << (64 - kFxFrac));
    return (long long)(r + ((lo >> (kFxFrac - 1)) & 1ull));
}

struct GsCoefFX {
    long long Du6, Dv6, F, Fk, dt, noise;  // Du / 6, Dv / 6, F, F + k, dt, n in fixed point
    int dt_one;                            // dt == 1 exactly: the products du * dt are skipped
};

inline long long fx_host(double d) { return (long long)llround(ldexp(d, kFxFrac)); }

inline GsCoefFX gs_make_coef_fx(double Du, double Dv, double F, double k, double dt, double noise)
{
    GsCoefFX c;
    c.Du6 = fx_host(Du / 6.0);
    c.Dv6 = fx_host(Dv / 6.0);
    c.F = fx_host(F);
    c.Fk = fx_host(F + k);
    c.dt = fx_host(dt);
    c.noise = fx_host(noise);
    c.dt_one = dt == 1.0;
    return c;
}

// gs_update in fixed point.  su, sv: exact neighbour sums; rnum: the noise
// numerator (r = rnum / 2^24 is rnum << 28 in fixed point, exactly).
template <bool NOISE>
GS_D void gs_update_fx(const GsCoefFX& c, long long u, long long v, long long su, long long sv, int32_t rnum,
                       long long& un, long long& vn)
{
    const long long lu = su - ((u << 2) + (u << 1));         // sum - 6u (exact)
    const long long lv = sv - ((v << 2) + (v << 1));
    const long long uvv = fx_mul(u, fx_mul(v, v));           // u v^2
    long long du = fx_mul(c.Du6, lu) - uvv;                  // Du lap u - u v^2
    du += fx_mul(c.F, kFxOne - u);                           // + F (1 - u)
    if (NOISE) du += fx_mul(c.noise, (long long)rnum << 28); // + n r
    long long dv = fx_mul(c.Dv6, lv) + uvv;                  // Dv lap v + u v^2
    dv -= fx_mul(c.Fk, v);                                   // - (F + k) v
    un = u + (c.dt_one ? du : fx_mul(du, c.dt));             // u + dt du
    vn = v + (c.dt_one ? dv : fx_mul(dv, c.dt));
}

// A fixed-point value kept in the 8 bytes of a double (the z-marching
// kernel converts each staged plane in place once, and the steps inside one
// gs_step call keep the fields in this form between steps).
GS_D double fx_pack(long long X) { return __longlong_as_double(X); }
GS_D long long fx_unpack(double d) { return (long long)__double_as_longlong(d); }

// A 2-cell group of FP64 cells whose inputs are packed fixed-point values;
// writes packed values (PACK) or FP64 outputs.
template <bool NOISE, bool PACK = false>
GS_D void gs_update_group_fx(const GsCoefFX& c, uint32_t pre, uint32_t kk2, const double* cu, const double* cv,
                             const double* pu, const double* pv, const double* nu, const double* nv,
                             const double* ymu, const double* ypu, const double* ymv, const double* ypv,
                             double xlu, double xru, double xlv, double xrv, double* ou, double* ov)
{
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const long long u = fx_unpack(cu[e]), v = fx_unpack(cv[e]);
        const long long su = fx_unpack(e > 0 ? cu[0] : xlu) + fx_unpack(e < 1 ? cu[1] : xru) + fx_unpack(ymu[e]) +
                             fx_unpack(ypu[e]) + fx_unpack(pu[e]) + fx_unpack(nu[e]);
        const long long sv = fx_unpack(e > 0 ? cv[0] : xlv) + fx_unpack(e < 1 ? cv[1] : xrv) + fx_unpack(ymv[e]) +
                             fx_unpack(ypv[e]) + fx_unpack(pv[e]) + fx_unpack(nv[e]);
        const int32_t rn = NOISE ? gs_group_num(pre, (uint32_t)e, kk2) : 0;
        long long un, vn;
        gs_update_fx<NOISE>(c, u, v, su, sv, rn, un, vn);
        ou[e] = PACK ? fx_pack(un) : fx_to_double(un);
        ov[e] = PACK ? fx_pack(vn) : fx_to_double(vn);
    }
}
