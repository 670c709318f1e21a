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
enum : int { GS_DERR_NONE = 0, GS_DERR_TIMEOUT = 1, GS_DERR_BADARG = 2 };

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

// ---------------------------------------------------------------------------
// Per-cell update.
// ---------------------------------------------------------------------------
template <typename T>
struct GsCoef {
    T Du6, Dv6;  // Du / 6, Dv / 6   (Eq. 3's 1/6 folded into the diffusion rate)
    T F, Fk;     // F, F + k
    T dt, noise;
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
    c.noise = (T)noise;
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
//   su, sv: neighbour sums of u and v (gs_nsum order); r: the noise draw
//   (ignored when with_noise is false, which equals adding noise*0).
template <typename T, bool with_noise>
GS_D void gs_update(const GsCoef<T>& c, T u, T v, T su, T sv, T r, T& un, T& vn)
{
    T lu = gs_fma((T)-6, u, su);            // sum - 6u
    T lv = gs_fma((T)-6, v, sv);
    T uvv = gs_mul(u, gs_mul(v, v));        // u v^2
    T du = gs_fma(c.Du6, lu, -uvv);         // Du lap u - u v^2
    du = gs_fma(c.F, gs_sub((T)1, u), du);  // + F (1 - u)
    if (with_noise) du = gs_fma(c.noise, r, du);  // + n r
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
