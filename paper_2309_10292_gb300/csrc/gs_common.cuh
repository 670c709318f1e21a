// Device-side building blocks shared by every libgs stencil kernel.
//
//  * gs_fmix32 / gs_step_keys / gs_noise: the counter-based draw of the
//    noise term r of Eq. 1a (MurmurHash3 finaliser, two keyed rounds).
//  * GsCoef / gs_update: the per-cell forward-Euler update of Eq. 2a, 2b
//    with the Laplacian of Eq. 3.  Every kernel calls this one function with
//    the neighbour sum formed in the same order, and every operation is an
//    explicit round-to-nearest intrinsic, so all kernels (plain, z-marching,
//    temporally blocked, batched) produce bitwise-identical fields.
//  * mbarrier / TMA (cp.async.bulk.tensor) wrappers with bounded waits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define GS_HD __host__ __device__ __forceinline__
#define GS_D __device__ __forceinline__

// device error codes written to the object's error word
enum : int { GS_DERR_NONE = 0, GS_DERR_TIMEOUT = 1, GS_DERR_BADARG = 2, GS_DERR_RANGE = 3 };

// ---------------------------------------------------------------------------
// Noise: r(seed, t, c) in (-1, 1), exact in float and double.
// ---------------------------------------------------------------------------
GS_HD uint32_t gs_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

struct GsKeys {
    uint32_t k1, k2;
};

GS_HD GsKeys gs_step_keys(uint64_t seed, int64_t t)
{
    GsKeys k;
    k.k1 = gs_fmix32((uint32_t)seed ^ gs_fmix32((uint32_t)t ^ 0x9E3779B9u));
    k.k2 = gs_fmix32((uint32_t)(seed >> 32) ^ gs_fmix32(k.k1 ^ 0x7F4A7C15u));
    return k;
}

// signed odd numerator 2m + 1 - 2^24 of r = num / 2^24
GS_HD int32_t gs_noise_num(uint32_t c, GsKeys k)
{
    uint32_t h = gs_fmix32(gs_fmix32(c ^ k.k1) ^ k.k2);
    return 2 * (int32_t)(h >> 8) + 1 - (1 << 24);
}

template <typename T>
GS_D T gs_noise(uint32_t c, GsKeys k)
{
    // |num| < 2^24: the conversion and the power-of-two scale are exact
    return (T)gs_noise_num(c, k) * (T)(1.0 / 16777216.0);
}

// The same numerators for the V consecutive cells g + e (e < V) of one
// 16-byte group, g a multiple of V (V <= 4).  Because g + e = g ^ e and e
// only touches the two low bits, the first xor-shift of fmix32(c ^ k1) is
// pre ^ e with pre = x ^ (x >> 16), x = g ^ k1, computed once per group.
// The xor-shift by 16 is its own inverse (y ^ (y >> 16) ^ ((y ^ (y >> 16))
// >> 16) = y for 32-bit y), so the last xor-shift of the first round and the
// first xor-shift of the second, with k2 xored in between, reduce to one xor
// with kk2 = k2 ^ (k2 >> 16).  Bit for bit equal to gs_noise_num(g + e, k).
GS_HD uint32_t gs_group_pre(uint32_t g, GsKeys k)
{
    const uint32_t x = g ^ k.k1;
    return x ^ (x >> 16);
}

GS_HD uint32_t gs_kk2(GsKeys k) { return k.k2 ^ (k.k2 >> 16); }

GS_HD int32_t gs_group_num(uint32_t pre, uint32_t e, uint32_t kk2)
{
    uint32_t h = pre ^ e;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= kk2;  // = (y ^ (y >> 16) ^ k2) xor-shifted by 16, y = h before it
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return 2 * (int32_t)(h >> 8) + 1 - (1 << 24);
}

// ---------------------------------------------------------------------------
// Per-cell update.
// ---------------------------------------------------------------------------
template <typename T>
struct GsCoef {
    T Du6, Dv6;  // Du / 6, Dv / 6   (Eq. 3's 1/6 folded into the diffusion rate)
    T F, Fk;     // F, F + k
    T dt;
    T noise24;   // n / 2^24: the noise term n r = noise24 * num with r = num / 2^24 (exact scaling)
};

// Kernel-side coefficients from the model parameters (host).
template <typename T>
inline GsCoef<T> gs_make_coef(double Du, double Dv, double F, double k, double dt, double noise)
{
    GsCoef<T> c;
    c.Du6 = (T)(Du / 6.0);
    c.Dv6 = (T)(Dv / 6.0);
    c.F = (T)F;
    c.Fk = (T)(F + k);
    c.dt = (T)dt;
    c.noise24 = (T)noise * (T)(1.0 / 16777216.0);
    return c;
}

GS_D float gs_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
GS_D double gs_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
GS_D float gs_mul(float a, float b) { return __fmul_rn(a, b); }
GS_D double gs_mul(double a, double b) { return __dmul_rn(a, b); }
GS_D float gs_add(float a, float b) { return __fadd_rn(a, b); }
GS_D double gs_add(double a, double b) { return __dadd_rn(a, b); }
GS_D float gs_sub(float a, float b) { return __fsub_rn(a, b); }
GS_D double gs_sub(double a, double b) { return __dsub_rn(a, b); }

// Neighbour sum in the fixed order x-, x+, y-, y+, z-, z+ (Eq. 3).
template <typename T>
GS_D T gs_nsum(T xm, T xp, T ym, T yp, T zm, T zp)
{
    T s = gs_add(xm, xp);
    s = gs_add(s, ym);
    s = gs_add(s, yp);
    s = gs_add(s, zm);
    return gs_add(s, zp);
}

// One forward-Euler step of one cell (Eq. 1a, 1b, 2a, 2b).
//   su, sv: neighbour sums of u and v (gs_nsum order); rnum: the noise
//   numerator as T (r = rnum / 2^24; ignored when with_noise is false, which
//   equals adding n r = 0).  n r = noise24 * rnum exactly, so the fused
//   multiply-add rounds the same value as fma(n, r, du).
template <typename T, bool with_noise>
GS_D void gs_update(const GsCoef<T>& c, T u, T v, T su, T sv, T rnum, T& un, T& vn)
{
    T lu = gs_fma((T)-6, u, su);            // sum - 6u
    T lv = gs_fma((T)-6, v, sv);
    T uvv = gs_mul(u, gs_mul(v, v));        // u v^2
    T du = gs_fma(c.Du6, lu, -uvv);         // Du lap u - u v^2
    du = gs_fma(c.F, gs_sub((T)1, u), du);  // + F (1 - u)
    if (with_noise) du = gs_fma(c.noise24, rnum, du);  // + n r
    T dv = gs_fma(c.Dv6, lv, uvv);          // Dv lap v + u v^2
    dv = gs_fma(-c.Fk, v, dv);              // - (F + k) v
    un = gs_fma(du, c.dt, u);               // u + dt du
    vn = gs_fma(dv, c.dt, v);
}

// ---------------------------------------------------------------------------
// Timers and error reporting.
// ---------------------------------------------------------------------------
GS_D uint64_t gs_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

GS_D void gs_report(int* err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------
// mbarrier (shared memory, CTA scope) and TMA.
// ---------------------------------------------------------------------------
GS_D uint32_t gs_smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

GS_D void gs_mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gs_smem_addr(bar)), "r"(count)
                 : "memory");
}

GS_D void gs_fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

GS_D void gs_fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

GS_D void gs_mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gs_smem_addr(bar)) : "memory");
}

GS_D void gs_mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gs_smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

GS_D bool gs_mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(gs_smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` to complete, giving up after timeout_ns
// of global time.  Returns false on timeout.
GS_D bool gs_mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns)
{
    if (gs_mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gs_globaltimer();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (gs_mbar_try_wait(bar, parity)) return true;
        if (gs_globaltimer() - t0 > timeout_ns) return false;
    }
}

// 3D tiled TMA load global -> shared, completion signalled on `bar`.
// x must be a multiple of 16 bytes / element size (checked by the callers'
// plan validation: x is always a multiple of the vector width).
GS_D void gs_tma_load_3d(void* smem_dst, const void* tmap, uint64_t* bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(gs_smem_addr(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(gs_smem_addr(bar))
        : "memory");
}

GS_D void gs_prefetch_tmap(const void* tmap)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// vector types: 16 bytes of T
template <typename T>
struct GsVec;
template <>
struct GsVec<float> {
    using type = float4;
    static constexpr int N = 4;
};
template <>
struct GsVec<double> {
    using type = double2;
    static constexpr int N = 2;
};

template <typename T>
GS_D void gs_unpack(const typename GsVec<T>::type& p, T* a);
template <>
GS_D void gs_unpack<float>(const float4& p, float* a)
{
    a[0] = p.x; a[1] = p.y; a[2] = p.z; a[3] = p.w;
}
template <>
GS_D void gs_unpack<double>(const double2& p, double* a)
{
    a[0] = p.x; a[1] = p.y;
}
template <typename T>
GS_D typename GsVec<T>::type gs_pack(const T* a);
template <>
GS_D float4 gs_pack<float>(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
template <>
GS_D double2 gs_pack<double>(const double* a) { return make_double2(a[0], a[1]); }

// ---------------------------------------------------------------------------
// Grid-scope ordering for persistent kernels.
// ---------------------------------------------------------------------------
GS_D void gs_fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

GS_D unsigned gs_atom_add_release_gpu(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

GS_D unsigned gs_ld_acquire_gpu(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

GS_D int gs_ld_relaxed_gpu(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------------------
// Packed FP32 (two lanes per instruction, sm_100 family).  Each lane is an
// ordinary round-to-nearest single operation, so results equal the scalar
// intrinsics above bit for bit.  Off by default: on GB300 the z-march kernel
// measured 10-15 % slower with it (fewer instructions, longer schedule).
// ---------------------------------------------------------------------------
typedef unsigned long long gs_f2;

GS_D gs_f2 gs_pk(float a, float b)
{
    gs_f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
GS_D void gs_upk(gs_f2 r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
GS_D gs_f2 gs_add2(gs_f2 a, gs_f2 b)
{
    gs_f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
GS_D gs_f2 gs_mul2(gs_f2 a, gs_f2 b)
{
    gs_f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
GS_D gs_f2 gs_fma2(gs_f2 a, gs_f2 b, gs_f2 c)
{
    gs_f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Update of the 4 cells of one float4 group with packed arithmetic; the same
// operations in the same order as gs_update.  The u equation is carried with
// its sign flipped (w = -du) so every step is one fused multiply-add; since
// round-to-nearest is symmetric, w is exactly -du at every step and
// u + dt du = fma(w, -dt, u).
//   c*: centre, pm/pp: z-1 / z+1, ym/yp: y-1 / y+1, xl/xr: x neighbours of
//   the group's first / last cell, rn: noise numerators as float.
template <bool NOISE>
GS_D void gs_update4(const GsCoef<float>& c, const float (&cu)[4], const float (&cv)[4], const float (&pu)[4],
                     const float (&pv)[4], const float (&nu)[4], const float (&nv)[4], const float (&ymu)[4],
                     const float (&ypu)[4], const float (&ymv)[4], const float (&ypv)[4], float xlu, float xru,
                     float xlv, float xrv, const float (&rn)[4], float (&ou)[4], float (&ov)[4])
{
    const gs_f2 m6 = gs_pk(-6.f, -6.f), one = gs_pk(1.f, 1.f), m1 = gs_pk(-1.f, -1.f);
    const gs_f2 mDu6 = gs_pk(-c.Du6, -c.Du6), Dv6 = gs_pk(c.Dv6, c.Dv6);
    const gs_f2 mF = gs_pk(-c.F, -c.F), mFk = gs_pk(-c.Fk, -c.Fk);
    const gs_f2 dt = gs_pk(c.dt, c.dt), mdt = gs_pk(-c.dt, -c.dt), mn24 = gs_pk(-c.noise24, -c.noise24);
    // u and v, pairs (0,1) and (2,3)
    const gs_f2 xu[3] = {gs_pk(xlu, cu[0]), gs_pk(cu[1], cu[2]), gs_pk(cu[3], xru)};
    const gs_f2 xv[3] = {gs_pk(xlv, cv[0]), gs_pk(cv[1], cv[2]), gs_pk(cv[3], xrv)};
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int e = 2 * p;
        const gs_f2 u = gs_pk(cu[e], cu[e + 1]), v = gs_pk(cv[e], cv[e + 1]);
        gs_f2 su = gs_add2(xu[p], xu[p + 1]);
        su = gs_add2(su, gs_pk(ymu[e], ymu[e + 1]));
        su = gs_add2(su, gs_pk(ypu[e], ypu[e + 1]));
        su = gs_add2(su, gs_pk(pu[e], pu[e + 1]));
        su = gs_add2(su, gs_pk(nu[e], nu[e + 1]));
        gs_f2 sv = gs_add2(xv[p], xv[p + 1]);
        sv = gs_add2(sv, gs_pk(ymv[e], ymv[e + 1]));
        sv = gs_add2(sv, gs_pk(ypv[e], ypv[e + 1]));
        sv = gs_add2(sv, gs_pk(pv[e], pv[e + 1]));
        sv = gs_add2(sv, gs_pk(nv[e], nv[e + 1]));
        const gs_f2 lu = gs_fma2(m6, u, su);
        const gs_f2 lv = gs_fma2(m6, v, sv);
        const gs_f2 uvv = gs_mul2(u, gs_mul2(v, v));
        gs_f2 w = gs_fma2(mDu6, lu, uvv);         // -(Du lap u - u v^2)
        w = gs_fma2(mF, gs_fma2(u, m1, one), w);  // -(... + F (1 - u))
        if (NOISE) w = gs_fma2(mn24, gs_pk(rn[e], rn[e + 1]), w);  // -(... + n r)
        const gs_f2 un = gs_fma2(w, mdt, u);     // u + dt du
        gs_f2 dv = gs_fma2(Dv6, lv, uvv);
        dv = gs_fma2(mFk, v, dv);
        const gs_f2 vn = gs_fma2(dv, dt, v);
        gs_upk(un, ou[e], ou[e + 1]);
        gs_upk(vn, ov[e], ov[e + 1]);
    }
}

// One 16-byte group of V cells (FP32: 4, packed; FP64: 2, scalar).
template <typename T, bool NOISE>
GS_D void gs_update_group(const GsCoef<T>& c, uint32_t pre, uint32_t kk2, const T* cu, const T* cv, const T* pu,
                          const T* pv, const T* nu, const T* nv, const T* ymu, const T* ypu, const T* ymv,
                          const T* ypv, T xlu, T xru, T xlv, T xrv, T* ou, T* ov);

template <>
GS_D void gs_update_group<float, true>(const GsCoef<float>& c, uint32_t pre, uint32_t kk2, const float* cu,
                                       const float* cv, const float* pu, const float* pv, const float* nu,
                                       const float* nv, const float* ymu, const float* ypu, const float* ymv,
                                       const float* ypv, float xlu, float xru, float xlv, float xrv, float* ou,
                                       float* ov)
{
    float rn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) rn[e] = (float)gs_group_num(pre, (uint32_t)e, kk2);
#ifndef GS_PACKED_FP32
    // default: scalar instructions (measured faster on GB300 than the packed
    // form below, which stays available with -DGS_PACKED_FP32)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float su = gs_nsum(e > 0 ? cu[e - 1] : xlu, e < 3 ? cu[e + 1] : xru, ymu[e], ypu[e], pu[e], nu[e]);
        const float sv = gs_nsum(e > 0 ? cv[e - 1] : xlv, e < 3 ? cv[e + 1] : xrv, ymv[e], ypv[e], pv[e], nv[e]);
        gs_update<float, true>(c, cu[e], cv[e], su, sv, rn[e], ou[e], ov[e]);
    }
    return;
#endif
    gs_update4<true>(c, *(const float(*)[4])cu, *(const float(*)[4])cv, *(const float(*)[4])pu,
                     *(const float(*)[4])pv, *(const float(*)[4])nu, *(const float(*)[4])nv,
                     *(const float(*)[4])ymu, *(const float(*)[4])ypu, *(const float(*)[4])ymv,
                     *(const float(*)[4])ypv, xlu, xru, xlv, xrv, rn, *(float(*)[4])ou, *(float(*)[4])ov);
}

template <>
GS_D void gs_update_group<float, false>(const GsCoef<float>& c, uint32_t pre, uint32_t kk2, const float* cu,
                                        const float* cv, const float* pu, const float* pv, const float* nu,
                                        const float* nv, const float* ymu, const float* ypu, const float* ymv,
                                        const float* ypv, float xlu, float xru, float xlv, float xrv, float* ou,
                                        float* ov)
{
    const float rn[4] = {0.f, 0.f, 0.f, 0.f};
    (void)pre;
    (void)kk2;
#ifndef GS_PACKED_FP32
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float su = gs_nsum(e > 0 ? cu[e - 1] : xlu, e < 3 ? cu[e + 1] : xru, ymu[e], ypu[e], pu[e], nu[e]);
        const float sv = gs_nsum(e > 0 ? cv[e - 1] : xlv, e < 3 ? cv[e + 1] : xrv, ymv[e], ypv[e], pv[e], nv[e]);
        gs_update<float, false>(c, cu[e], cv[e], su, sv, 0.f, ou[e], ov[e]);
    }
    return;
#endif
    gs_update4<false>(c, *(const float(*)[4])cu, *(const float(*)[4])cv, *(const float(*)[4])pu,
                      *(const float(*)[4])pv, *(const float(*)[4])nu, *(const float(*)[4])nv,
                      *(const float(*)[4])ymu, *(const float(*)[4])ypu, *(const float(*)[4])ymv,
                      *(const float(*)[4])ypv, xlu, xru, xlv, xrv, rn, *(float(*)[4])ou, *(float(*)[4])ov);
}

template <bool NOISE>
GS_D void gs_update_group_d(const GsCoef<double>& c, uint32_t pre, uint32_t kk2, const double* cu,
                            const double* cv, const double* pu, const double* pv, const double* nu,
                            const double* nv, const double* ymu, const double* ypu, const double* ymv,
                            const double* ypv, double xlu, double xru, double xlv, double xrv, double* ou,
                            double* ov)
{
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const double su = gs_nsum(e > 0 ? cu[e - 1] : xlu, e < 1 ? cu[e + 1] : xru, ymu[e], ypu[e], pu[e], nu[e]);
        const double sv = gs_nsum(e > 0 ? cv[e - 1] : xlv, e < 1 ? cv[e + 1] : xrv, ymv[e], ypv[e], pv[e], nv[e]);
        const double rn = NOISE ? (double)gs_group_num(pre, (uint32_t)e, kk2) : 0.0;
        gs_update<double, NOISE>(c, cu[e], cv[e], su, sv, rn, ou[e], ov[e]);
    }
}

template <>
GS_D void gs_update_group<double, true>(const GsCoef<double>& c, uint32_t pre, uint32_t kk2, const double* cu,
                                        const double* cv, const double* pu, const double* pv, const double* nu,
                                        const double* nv, const double* ymu, const double* ypu,
                                        const double* ymv, const double* ypv, double xlu, double xru, double xlv,
                                        double xrv, double* ou, double* ov)
{
    gs_update_group_d<true>(c, pre, kk2, cu, cv, pu, pv, nu, nv, ymu, ypu, ymv, ypv, xlu, xru, xlv, xrv, ou, ov);
}

template <>
GS_D void gs_update_group<double, false>(const GsCoef<double>& c, uint32_t pre, uint32_t kk2, const double* cu,
                                         const double* cv, const double* pu, const double* pv, const double* nu,
                                         const double* nv, const double* ymu, const double* ypu,
                                         const double* ymv, const double* ypv, double xlu, double xru,
                                         double xlv, double xrv, double* ou, double* ov)
{
    gs_update_group_d<false>(c, pre, kk2, cu, cv, pu, pv, nu, nv, ymu, ypu, ymv, ypv, xlu, xru, xlv, xrv, ou, ov);
}
