// Gray-Scott stencil kernels for sm_103a.
//
//   gs_init_kernel       centred-cube initial state
//   gs_noise_kernel      r(seed, t, c) for a range of cells (Eq. 1a's r)
//   gs_naive_kernel      one thread per cell, periodic neighbours by index
//                        arithmetic; any L >= 1 (also the parity baseline)
//   gs_zmarch_kernel     persistent CTAs marching along z over x-y tiles.
//                        One producer warp streams each z-plane of the tile
//                        (plus its one-cell halo ring, wrapped periodically)
//                        into a shared-memory ring with TMA; consumer warps
//                        keep the z-1 / z / z+1 centre values in registers,
//                        read x/y neighbours from shared memory and write the
//                        new u, v with 16-byte stores.  Each cell's u and v
//                        are read from HBM once and written once per step:
//                        16 B/cell (FP32), 32 B/cell (FP64).
//
// All kernels apply gs_update (gs_common.cuh) with the same neighbour order,
// so they agree bit for bit.
#include <algorithm>
#include <cstdio>

#include <type_traits>

#include "gs_common.cuh"
#include "gs_ds.cuh"
#include "gs_fx.cuh"
#include "gs_fxf.cuh"
#include "gs_internal.h"

namespace gs {

// ---------------------------------------------------------------------------
// Initial state
// ---------------------------------------------------------------------------
template <typename T>
__global__ void gs_init_kernel(T* __restrict__ u, T* __restrict__ v, int L)
{
    const int64_t n = (int64_t)L * L * L;
    const int lo = L / 2 - 3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(i % L);
        int64_t r = i / L;
        int y = (int)(r % L);
        int z = (int)(r / L);
        bool in = x >= lo && x < lo + 6 && y >= lo && y < lo + 6 && z >= lo && z < lo + 6;
        u[i] = in ? (T)0.25 : (T)1.0;
        v[i] = in ? (T)0.33 : (T)0.0;
    }
}

template <typename T>
__global__ void gs_noise_kernel(T* __restrict__ out, int64_t n, GsKeys k)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = gs_noise<T>((uint32_t)i, k);
}

// ---------------------------------------------------------------------------
// Plain kernel: one thread per cell
// ---------------------------------------------------------------------------
template <typename T>
static GsCoef<T> make_coef(const Params& p)
{
    return gs_make_coef<T>(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
}

// AR: the arithmetic of FP64 fields (0: IEEE, 1: double-single, 2: fixed
// point, 3: fixed point with a float remainder).  IO (AR > 0): bit 0 = the
// inputs hold that arithmetic's packed values (else FP64 values, converted
// at use), bit 1 = write packed values (else FP64).
template <typename T, bool NOISE, int AR, int IO = 0>
__global__ void __launch_bounds__(256) gs_naive_kernel(const T* __restrict__ u, const T* __restrict__ v,
                                                       T* __restrict__ un, T* __restrict__ vn, int L,
                                                       GsCoef<T> c, GsCoefDS cds, GsCoefFX cfx, GsCoefFXF cfxf,
                                                       GsKeys k, int* err)
{
    constexpr bool IN_PACKED = (IO & 1) != 0, OUT_PACKED = (IO & 2) != 0;
    const int64_t n = (int64_t)L * L * L;
    const int64_t LL = (int64_t)L * L;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L);
        const int64_t r = i / L;
        const int y = (int)(r % L);
        const int z = (int)(r / L);
        const int64_t row = i - x;
        const int64_t pl = i - (int64_t)y * L;  // x + L*L*z
        const int64_t ixm = row + (x == 0 ? L - 1 : x - 1);
        const int64_t ixp = row + (x == L - 1 ? 0 : x + 1);
        const int64_t iym = pl + (int64_t)(y == 0 ? L - 1 : y - 1) * L;
        const int64_t iyp = pl + (int64_t)(y == L - 1 ? 0 : y + 1) * L;
        const int64_t base = i - (int64_t)z * LL;
        const int64_t izm = base + (int64_t)(z == 0 ? L - 1 : z - 1) * LL;
        const int64_t izp = base + (int64_t)(z == L - 1 ? 0 : z + 1) * LL;
        if constexpr (AR == 1) {
            // FP64 fields in double-single arithmetic (gs_ds.cuh)
            auto get = [&](double x) -> GsDS {
                if constexpr (IN_PACKED) return ds_unpack(x);
                else return ds_from_double(x);
            };
            const GsDS uc = get(u[i]), vc = get(v[i]);
            const GsDS su = ds_nsum(get(u[ixm]), get(u[ixp]), get(u[iym]), get(u[iyp]), get(u[izm]), get(u[izp]));
            const GsDS sv = ds_nsum(get(v[ixm]), get(v[ixp]), get(v[iym]), get(v[iyp]), get(v[izm]), get(v[izp]));
            const float rn = NOISE ? (float)gs_noise_num((uint32_t)i, k) : 0.0f;
            GsDS a, b;
            gs_update_ds<NOISE>(cds, uc, vc, su, sv, rn, a, b);
            un[i] = OUT_PACKED ? ds_pack(a) : ds_to_double(a);
            vn[i] = OUT_PACKED ? ds_pack(b) : ds_to_double(b);
        } else if constexpr (AR == 2) {
            // FP64 fields in fixed point (gs_fx.cuh)
            bool any = false;
            auto get = [&](double x) -> long long {
                if constexpr (IN_PACKED) {
                    return fx_unpack(x);
                } else {
                    bool o;
                    const long long r = fx_from_double(x, o);
                    any |= o;
                    return r;
                }
            };
            const long long uc = get(u[i]), vc = get(v[i]);
            const long long su = get(u[ixm]) + get(u[ixp]) + get(u[iym]) + get(u[iyp]) + get(u[izm]) + get(u[izp]);
            const long long sv = get(v[ixm]) + get(v[ixp]) + get(v[iym]) + get(v[iyp]) + get(v[izm]) + get(v[izp]);
            if (any) gs_report(err, GS_DERR_RANGE);
            const int32_t rn = NOISE ? gs_noise_num((uint32_t)i, k) : 0;
            long long a, b;
            gs_update_fx<NOISE>(cfx, uc, vc, su, sv, rn, a, b);
            un[i] = OUT_PACKED ? fx_pack(a) : fx_to_double(a);
            vn[i] = OUT_PACKED ? fx_pack(b) : fx_to_double(b);
        } else if constexpr (AR == 3) {
            // FP64 fields in fixed point with a float remainder (gs_fxf.cuh)
            bool any = false;
            auto get = [&](double x) -> GsFxf {
                if constexpr (IN_PACKED) {
                    return fxf_unpack(x);
                } else {
                    bool o;
                    const GsFxf r = fxf_from_double(x, o);
                    any |= o;
                    return r;
                }
            };
            const GsFxf uc = get(u[i]), vc = get(v[i]);
            int32_t SU, SV;
            float SLU, SLV;
            fxf_nsum(get(u[ixm]), get(u[ixp]), get(u[iym]), get(u[iyp]), get(u[izm]), get(u[izp]), SU, SLU);
            fxf_nsum(get(v[ixm]), get(v[ixp]), get(v[iym]), get(v[iyp]), get(v[izm]), get(v[izp]), SV, SLV);
            const int32_t rn = NOISE ? gs_noise_num((uint32_t)i, k) : 0;
            GsFxf a, b;
            uint32_t rng = 0;
            gs_update_fxf<NOISE>(cfxf, uc, vc, SU, SLU, SV, SLV, rn, a, b, rng);
            if (any || fxf_range_bad(rng)) gs_report(err, GS_DERR_RANGE);
            un[i] = OUT_PACKED ? fxf_pack(a) : fxf_to_double(a);
            vn[i] = OUT_PACKED ? fxf_pack(b) : fxf_to_double(b);
        } else {
            const T uc = u[i], vc = v[i];
            const T su = gs_nsum(u[ixm], u[ixp], u[iym], u[iyp], u[izm], u[izp]);
            const T sv = gs_nsum(v[ixm], v[ixp], v[iym], v[iyp], v[izm], v[izp]);
            T rn = (T)0;
            if (NOISE) rn = (T)gs_noise_num((uint32_t)i, k);
            T a, b;
            gs_update<T, NOISE>(c, uc, vc, su, sv, rn, a, b);
            un[i] = a;
            vn[i] = b;
        }
    }
}

static int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)num_sms() * 32;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

int launch_init(int dtype, int L, void* u, void* v, cudaStream_t s)
{
    const int64_t n = (int64_t)L * L * L;
    const int g = grid_for(n, 256);
    if (dtype == GS_F32)
        gs_init_kernel<float><<<g, 256, 0, s>>>((float*)u, (float*)v, L);
    else
        gs_init_kernel<double><<<g, 256, 0, s>>>((double*)u, (double*)v, L);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int launch_noise_field(int dtype, uint64_t seed, int64_t t, int64_t n, void* out, cudaStream_t s)
{
    if (n <= 0) return GS_OK;
    const int g = grid_for(n, 256);
    GsKeys k = gs_step_keys(seed, t);
    if (dtype == GS_F32)
        gs_noise_kernel<float><<<g, 256, 0, s>>>((float*)out, n, k);
    else
        gs_noise_kernel<double><<<g, 256, 0, s>>>((double*)out, n, k);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

template <typename T>
static int naive_t(int L, const void* u, const void* v, void* un, void* vn, const Params& p,
                   int64_t t, int* err, cudaStream_t s)
{
    const int64_t n = (int64_t)L * L * L;
    const int g = grid_for(n, 256);
    GsCoef<T> c = make_coef<T>(p);
    const GsCoefDS cds = gs_make_coef_ds(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
    const GsCoefFX cfx = gs_make_coef_fx(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
    const GsCoefFXF cfxf = gs_make_coef_fxf(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
    GsKeys k = gs_step_keys(p.seed, t);
    const bool nz = p.noise != 0.0;
    const T* cu = (const T*)u;
    const T* cv = (const T*)v;
    bool launched = false;
    if constexpr (std::is_same<T, double>::value) {
        if (p.arith == GS_ARITH_DS || p.arith == GS_ARITH_FX || p.arith == GS_ARITH_FXF) {
#define GS_NAIVE_AR(AR, IO)                                                                                       \
    (nz ? gs_naive_kernel<T, true, AR, IO><<<g, 256, 0, s>>>(cu, cv, (T*)un, (T*)vn, L, c, cds, cfx, cfxf, k, err) \
        : gs_naive_kernel<T, false, AR, IO><<<g, 256, 0, s>>>(cu, cv, (T*)un, (T*)vn, L, c, cds, cfx, cfxf, k, err))
#define GS_NAIVE_IO(AR)                      \
    switch (p.io & 3) {                      \
    case 0: GS_NAIVE_AR(AR, 0); break;       \
    case 1: GS_NAIVE_AR(AR, 1); break;       \
    case 2: GS_NAIVE_AR(AR, 2); break;       \
    default: GS_NAIVE_AR(AR, 3); break;      \
    }
            if (p.arith == GS_ARITH_DS) {
                GS_NAIVE_IO(1)
            } else if (p.arith == GS_ARITH_FX) {
                GS_NAIVE_IO(2)
            } else {
                GS_NAIVE_IO(3)
            }
#undef GS_NAIVE_IO
#undef GS_NAIVE_AR
            launched = true;
        }
    }
    if (!launched) {
        if (nz) gs_naive_kernel<T, true, 0><<<g, 256, 0, s>>>(cu, cv, (T*)un, (T*)vn, L, c, cds, cfx, cfxf, k, err);
        else gs_naive_kernel<T, false, 0><<<g, 256, 0, s>>>(cu, cv, (T*)un, (T*)vn, L, c, cds, cfx, cfxf, k, err);
    }
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int launch_naive(int dtype, int L, const void* u, const void* v, void* un, void* vn,
                 const Params& p, int64_t t, int* err, cudaStream_t s)
{
    return dtype == GS_F32 ? naive_t<float>(L, u, v, un, vn, p, t, err, s)
                           : naive_t<double>(L, u, v, un, vn, p, t, err, s);
}

// ---------------------------------------------------------------------------
// TMA-staged z-marching kernel
// ---------------------------------------------------------------------------
// Shared-memory stage layout, per field (u then v), each block 128-B aligned:
//   main  [ty][tx]   cells x0..x0+tx-1, y0..y0+ty-1 of plane z
//   top   [tx]       row (y0 - 1) mod L
//   bot   [tx]       row (y0 + nvy) mod L   (nvy = valid rows of the tile)
//   left  [ty][V]    columns (x0 - V .. x0 - 1) mod L
//   right [ty][V]    columns (x0 + nvx .. x0 + nvx + V - 1) mod L
struct ZLayout {
    int main_off, top_off, bot_off, left_off, right_off;  // elements
    int field_elems;   // elements per field per stage (padded)
    int stage_bytes;   // both fields
    int tx_bytes;      // bytes TMA writes per stage (what the barrier expects)
};

static inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

static ZLayout make_layout(int esz, int V, int tx, int ty)
{
    const int a = 128 / esz;  // elements per 128 B
    ZLayout l;
    l.main_off = 0;
    l.top_off = round_up(tx * ty, a);
    l.bot_off = l.top_off + round_up(tx, a);
    l.left_off = l.bot_off + round_up(tx, a);
    l.right_off = l.left_off + round_up(V * ty, a);
    l.field_elems = l.right_off + round_up(V * ty, a);
    l.stage_bytes = 2 * l.field_elems * esz;
    l.tx_bytes = 2 * (tx * ty + 2 * tx + 2 * V * ty) * esz;
    return l;
}

template <typename T>
struct ZArgs {
    T* un;
    T* vn;
    int L;
    int tx, ty, tz;          // tile
    int ntx, nty, ntiles;    // tiles along x, y and total (x fastest, then y, then z)
    int stages;
    ZLayout lay;
    GsCoef<T> c;
    GsCoefDS cds;            // the same coefficients as double-single pairs (DS kernels)
    GsCoefFX cfx;            // and in fixed point (FX kernels)
    GsCoefFXF cfxf;          // and as float pairs for the fixed point with a remainder (FXF kernels)
    GsKeys keys;
    int* err;
    uint64_t timeout_ns;
    int stall;               // failure injection: the producer issues nothing
    unsigned* tickets;       // [next ticket, CTAs done] (zeroed between launches), or null: round robin
    int alternate;           // odd z-chunks march down
};

// Work of the persistent CTAs: tiles in the order x fastest, then y, then
// z-chunk (the CTAs work on neighbouring tiles of the same z-chunk at a time,
// so the tiles' halo rows are L2 hits).  In the memory-bound IEEE kernels
// (ZArgs::alternate) odd z-chunks march down (nz < 0: planes z0 + nz - 1
// down to z0), so two neighbouring chunks read the halo planes they share at
// about the same time, the second read from L2.  The FP64 arithmetics on the
// FP32 and integer pipes are bound by instruction issue: they march up only,
// and keep one copy of their long per-plane code (both directions at once
// measured 1 % slower), and take tiles round robin (the counter measured
// 0.5 % slower there).
//
// With a ticket counter (ZArgs::tickets) the CTAs take work units in that
// order as they become free: units are the tiles, the last G / 2 of them
// (G = CTAs) cut along z into four pieces (alternating direction), so every
// CTA ends the launch within a fraction of a tile of the others.  Without
// one (the batch's per-instance baseline) CTA c takes tiles c, c + G, ...,
// and the partial last round is cut along z so that every CTA gets a share:
// each of its `rem` tiles becomes s = G / rem pieces of about nz / s planes.
struct ZSeg {
    int x0, y0, z0, nz;  // nz < 0: march down |nz| planes
};

// the segment `part` of `parts` of tile `tile` (false when it is empty)
template <typename T>
GS_D bool zmarch_piece(int tile, int part, int parts, const ZArgs<T>& a, ZSeg& g)
{
    const int txi = tile % a.ntx;
    const int tyi = (tile / a.ntx) % a.nty;
    const int tzi = tile / (a.ntx * a.nty);
    const int z0 = tzi * a.tz;
    const int nz = min(a.tz, a.L - z0);
    const int lo = nz * part / parts, hi = nz * (part + 1) / parts;
    if (hi <= lo) return false;  // more pieces than planes: this one is empty
    g.x0 = txi * a.tx;
    g.y0 = tyi * a.ty;
    g.z0 = z0 + lo;
    g.nz = a.alternate && ((tzi + part) & 1) ? lo - hi : hi - lo;
    return true;
}

// round robin: the next segment of CTA blockIdx.x (k counts its draws)
template <typename T>
GS_D bool zmarch_next_seg(int& k, const ZArgs<T>& a, ZSeg& g)
{
    const int G = gridDim.x, c = blockIdx.x;
    const int R = a.ntiles / G, rem = a.ntiles - R * G;
    for (;;) {
        int tile, part = 0, parts = 1;
        if (k < R) {
            tile = c + k * G;
        } else if (k == R && rem) {
            parts = G / rem;
            if (c >= rem * parts) return false;
            tile = R * G + c / parts;
            part = c % parts;
        } else {
            return false;
        }
        ++k;
        if (zmarch_piece(tile, part, parts, a, g)) return true;
    }
}

// ticket counter: the segment of the next free work unit (false: none left)
template <typename T>
GS_D bool zmarch_unit_seg(unsigned* tickets, const ZArgs<T>& a, ZSeg& g)
{
    const int m = min(a.ntiles, (int)gridDim.x / 2);
    const int whole = a.ntiles - m;
    for (;;) {
        const int u = (int)atomicAdd(&tickets[0], 1u);
        if (u < whole) {
            if (zmarch_piece(u, 0, 1, a, g)) return true;
        } else if (u < whole + 4 * m) {
            const int v = u - whole;
            if (zmarch_piece(whole + v / 4, v % 4, 4, a, g)) return true;
        } else {
            return false;
        }
    }
}

// AR: the arithmetic of FP64 fields (0: IEEE, 1: double-single, 2: fixed
// point, 3: fixed point with a float remainder).  IO (AR > 0): bit 0 = the
// input fields hold that arithmetic's packed values, bit 1 = write packed
// values; AR = 3: bit 2 = dt is 1 (its (v^2) dt product is skipped at
// compile time).  The other arithmetics reading FP64 values convert every
// staged plane in place once (CONV).
template <typename T, bool NOISE, int AR, int IO = 0>
GS_D void zmarch_body(const ZMaps& maps, const ZArgs<T>& a)
{
    constexpr bool DS = AR == 1;
    constexpr bool FXF = AR == 3;
    constexpr bool CONV = AR != 0 && (IO & 1) == 0;
    constexpr bool PACK = (IO & 2) != 0;
    constexpr int FXF_DT = (IO & 4) != 0 ? 1 : 2;
    constexpr int V = GsVec<T>::N;
    using VT = typename GsVec<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    // full / empty per stage; with CONV also `conv`: one arrival per consumer
    // warp once its part of the stage has been converted in place
    __shared__ __align__(8) uint64_t bars[(CONV ? 3 : 2) * 8];
    __shared__ volatile int abort_flag;
    // the segments the producer hands to the consumers, in order, through
    // four slots: (x0, y0, z0, +-nz), nz == 0 after the last.  The producer
    // writes a slot before it releases the segment's first plane (that
    // mbarrier arrival orders it) and reuses it four segments later, at
    // least 12 planes on, when the consumers have read it long before (the
    // ring holds at most 8 stages)
    __shared__ int4 s_seg[4];

    const int S = a.stages;
    uint64_t* full = bars;
    uint64_t* empty = bars + S;
    uint64_t* conv = bars + 2 * S;  // CONV only
    const int nxv = a.tx / V;
    const int ncons = nxv * a.ty;
    const int cons_threads = (ncons + 31) & ~31;
    const int cons_warps = cons_threads >> 5;
    const int tid = threadIdx.x;
    const int L = a.L;
    T* ring = reinterpret_cast<T*>(smem);

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            gs_mbar_init(&full[s], 1);
            gs_mbar_init(&empty[s], cons_warps);
            if constexpr (CONV) gs_mbar_init(&conv[s], cons_warps);
        }
        abort_flag = 0;
        gs_fence_mbar_init();
    }
    __syncthreads();

    if (tid >= cons_threads) {
        // ------------------------------ producer warp ------------------------------
        if (tid != cons_threads) return;
        uint32_t seq = 0;           // planes issued (for the drain)
        int ps = 0;                 // stage of the next plane
        uint32_t pph = 0;           // its round's parity
        bool wrapped = false;       // every stage used once: wait for the consumers' release
        // with a ticket counter: the last CTA to finish (after every CTA drew
        // its last ticket; the fence orders this CTA's draws before its count)
        // zeroes the counter for the next launch
        auto finish = [&]() {
            if (!a.tickets) return;
            __threadfence();
            if (atomicAdd(&a.tickets[1], 1u) == gridDim.x - 1) {
                a.tickets[0] = 0;
                a.tickets[1] = 0;
            }
        };
        if (!a.stall) {
            for (int f = 0; f < 2; ++f)
                for (int m = 0; m < 3; ++m) gs_prefetch_tmap(&maps.m[f][m]);
            int wk = 0, kd = 0;
            ZSeg sg;
            for (;;) {
                const bool more = a.tickets ? zmarch_unit_seg(a.tickets, a, sg) : zmarch_next_seg(wk, a, sg);
                // the stage of the segment's first plane (or of the end marker)
                if (wrapped && !gs_mbar_wait(&empty[ps], pph ^ 1u, a.timeout_ns)) {
                    gs_report(a.err, GS_DERR_TIMEOUT);
                    abort_flag = 1;
                    goto drain;
                }
                if (abort_flag) goto drain;
                if (!more) {
                    s_seg[kd & 3] = make_int4(0, 0, 0, 0);
                    gs_mbar_arrive(&full[ps]);  // no copy: the phase completes here
                    ++seq;
                    if (++ps == S) { ps = 0; pph ^= 1u; wrapped = true; }
                    break;
                }
                s_seg[kd & 3] = make_int4(sg.x0, sg.y0, sg.z0, sg.nz);
                ++kd;
                const bool down = sg.nz < 0;
                const int x0 = sg.x0, y0 = sg.y0, z0 = sg.z0, nz = down ? -sg.nz : sg.nz;
                const int nvx = min(a.tx, L - x0), nvy = min(a.ty, L - y0);
                const int ytop = (y0 - 1 + L) % L, ybot = (y0 + nvy) % L;
                const int xl = (x0 - V + L) % L, xr = (x0 + nvx) % L;
                int zp = down ? (z0 + nz) % L : (z0 - 1 + L) % L;
                for (int j = 0; j < nz + 2; ++j) {
                    if (j > 0 && wrapped) {
                        if (!gs_mbar_wait(&empty[ps], pph ^ 1u, a.timeout_ns)) {
                            gs_report(a.err, GS_DERR_TIMEOUT);
                            abort_flag = 1;
                            goto drain;
                        }
                    }
                    if (abort_flag) goto drain;
                    gs_mbar_arrive_expect_tx(&full[ps], a.lay.tx_bytes);
                    for (int f = 0; f < 2; ++f) {
                        T* b = ring + (size_t)ps * (a.lay.stage_bytes / sizeof(T)) + f * a.lay.field_elems;
                        gs_tma_load_3d(b + a.lay.main_off, &maps.m[f][0], &full[ps], x0, y0, zp);
                        gs_tma_load_3d(b + a.lay.top_off, &maps.m[f][1], &full[ps], x0, ytop, zp);
                        gs_tma_load_3d(b + a.lay.bot_off, &maps.m[f][1], &full[ps], x0, ybot, zp);
                        gs_tma_load_3d(b + a.lay.left_off, &maps.m[f][2], &full[ps], xl, y0, zp);
                        gs_tma_load_3d(b + a.lay.right_off, &maps.m[f][2], &full[ps], xr, y0, zp);
                    }
                    ++seq;
                    if (++ps == S) { ps = 0; pph ^= 1u; wrapped = true; }
                    if (down)
                        zp = zp == 0 ? L - 1 : zp - 1;
                    else
                        zp = zp + 1 == L ? 0 : zp + 1;
                }
            }
        }
        finish();
        return;
    drain:
        // let every copy this thread issued land before the CTA can exit
        // (fixed 2 s budget: copies in flight always complete within it)
        for (uint32_t q = (seq > (uint32_t)S ? seq - S : 0); q < seq; ++q)
            gs_mbar_wait(&full[q % S], (q / S) & 1, 2000000000ull);
        finish();
        return;
    }

    // ------------------------------- consumer warps --------------------------------
    const int xv = tid % nxv;
    const int row = tid / nxv;  // >= ty for the padding threads of the last warp
    const int lane = tid & 31;
    const size_t stage_elems = a.lay.stage_bytes / sizeof(T);
    const int64_t LL = (int64_t)L * L;
    const uint32_t kk2 = gs_kk2(a.keys);
    int cs = 0;        // stage of the next plane to consume
    uint32_t cph = 0;  // its round's parity

    auto advance = [&]() {
        if (++cs == S) { cs = 0; cph ^= 1u; }
    };
    auto release = [&](int s) {
        // CONV: the in-place conversion wrote the stage; order those writes
        // before the copy engine's next fill of it
        if constexpr (CONV) gs_fence_proxy_async();
        __syncwarp();
        if (lane == 0) gs_mbar_arrive(&empty[s]);
    };
    auto wait_full = [&]() -> bool {
        if (gs_mbar_wait(&full[cs], cph, a.timeout_ns)) return true;
        gs_report(a.err, GS_DERR_TIMEOUT);
        abort_flag = 1;
        return false;
    };

    // planes z-1, z, z+1 of this thread's group in three register sets that
    // rotate by renaming (the loop below is unrolled by 3)
    T qu[3][V], qv[3][V];
    bool range_bad = false;  // FXF: some result out of range (reported once, at the end)
    int kd = 0;
    for (;;) {
        // the next segment's first plane, and with it its descriptor
        if (!wait_full()) return;
        const int4 dsc = s_seg[kd & 3];
        ++kd;
        if (dsc.w == 0) break;  // no segment left (nothing follows the marker's stage)
        // one segment, marching up (planes z0, z0 + 1, ...) or down (DESC:
        // z0 + nz - 1, z0 + nz - 2, ...); either way each cell takes z-1 as
        // its lower and z+1 as its upper neighbour, so the update is the
        // same to the bit
        auto run = [&](auto desc_tag) -> bool {
            constexpr bool DESC = decltype(desc_tag)::value;
            const int x0 = dsc.x, y0 = dsc.y, z0 = dsc.z, nz = DESC ? -dsc.w : dsc.w;
            const int nvx = min(a.tx, L - x0), nvy = min(a.ty, L - y0);
            const bool active = row < nvy && xv * V < nvx;
            const int rr = row < a.ty ? row : 0;  // padding threads read a valid address
            const int moff = a.lay.main_off + rr * a.tx + xv * V;
            // y neighbours (top / bottom halo rows at the tile's edges)
            const int om = row > 0 ? a.lay.main_off + (row - 1) * a.tx + xv * V : a.lay.top_off + xv * V;
            const int op = row + 1 < nvy ? a.lay.main_off + (row + 1) * a.tx + xv * V : a.lay.bot_off + xv * V;
            // x neighbours of the group's end cells: from the adjacent lanes when
            // they hold the same row's neighbouring groups (conflict-free), else
            // from shared memory (halo columns, or a group in another warp)
            const bool has_r = xv * V + V < nvx;
            const bool l_smem = xv == 0 || lane == 0;
            const bool r_smem = !has_r || lane == 31;
            const int oxl = xv > 0 ? moff - 1 : a.lay.left_off + rr * V + (V - 1);
            const int oxr = has_r ? moff + V : a.lay.right_off + rr * V;
            int64_t gidx = (int64_t)(DESC ? z0 + nz - 1 : z0) * LL + (int64_t)(y0 + row) * L + x0 + xv * V;

            // CONV: convert this thread's cells of stage s, and the halo entries
            // only it reads, to packed double-single pairs (DS), fixed-point
            // values (FX) or fixed-point pairs (FXF) in place, then announce it;
            // every FP64 value is converted once per pass instead of at each use
            auto convert_stage = [&](int s) {
                if constexpr (CONV) {
                    bool ovf = false;
                    if (active) {
#pragma unroll
                        for (int f = 0; f < 2; ++f) {
                            T* bf = ring + s * stage_elems + f * a.lay.field_elems;
                            auto cvt = [&](int off) {
                                if constexpr (DS) {
                                    bf[off] = ds_pack(ds_from_double(bf[off]));
                                } else if constexpr (AR == 2) {
                                    bool o;
                                    bf[off] = fx_pack(fx_from_double(bf[off], o));
                                    ovf |= o;
                                } else {
                                    bool o;
                                    bf[off] = fxf_pack(fxf_from_double(bf[off], o));
                                    ovf |= o;
                                }
                            };
#pragma unroll
                            for (int e = 0; e < V; ++e) {
                                cvt(moff + e);
                                if (row == 0) cvt(a.lay.top_off + xv * V + e);
                                if (row + 1 == nvy) cvt(a.lay.bot_off + xv * V + e);
                            }
                            if (xv == 0) cvt(oxl);
                            if (!has_r) cvt(oxr);
                        }
                    }
                    if constexpr (AR >= 2) {
                        if (__any_sync(0xffffffffu, ovf) && lane == 0) gs_report(a.err, GS_DERR_RANGE);
                    }
                    (void)ovf;
                    __syncwarp();
                    if (lane == 0) gs_mbar_arrive(&conv[s]);
                }
            };
            auto load_centre = [&](T (&u)[V], T (&v)[V]) {
                const T* b = ring + cs * stage_elems;
                gs_unpack<T>(*reinterpret_cast<const VT*>(b + moff), u);
                gs_unpack<T>(*reinterpret_cast<const VT*>(b + a.lay.field_elems + moff), v);
            };
            // one plane: P, C, N are planes z-1, z, z+1 (N is loaded here); the
            // centre plane's stage is released afterwards
            int sc = 0;
            uint32_t scp = 0;  // the centre stage's round parity
            auto plane = [&](T (&pu)[V], T (&pv)[V], T (&cu)[V], T (&cv)[V], T (&nu)[V], T (&nv)[V]) -> bool {
                // z-1 and z+1 of the centre plane: P and N marching up, N and P down
                auto pick = [&](T (&up)[V], T (&dn)[V]) -> T (&)[V] {
                    if constexpr (DESC) return dn; else return up;
                };
                T (&zmu)[V] = pick(pu, nu);
                T (&zmv)[V] = pick(pv, nv);
                T (&zpu)[V] = pick(nu, pu);
                T (&zpv)[V] = pick(nv, pv);
                const int sn = cs;
                const uint32_t snp = cph;
                if (!wait_full()) return false;
                convert_stage(cs);
                load_centre(nu, nv);
                // x neighbours of the group's end cells from the adjacent lanes;
                // the FP64 arithmetics on the FP32 and integer pipes read them all
                // from shared memory instead (four loads issue fewer instructions
                // than eight 32-bit shuffles and the edge lanes' loads)
                T shlu{}, shlv{}, shru{}, shrv{};
                if constexpr (AR == 0) {
                    shlu = __shfl_up_sync(0xffffffffu, cu[V - 1], 1);
                    shlv = __shfl_up_sync(0xffffffffu, cv[V - 1], 1);
                    shru = __shfl_down_sync(0xffffffffu, cu[0], 1);
                    shrv = __shfl_down_sync(0xffffffffu, cv[0], 1);
                }
                if constexpr (CONV) {
                    // every warp's part of the centre stage is converted
                    if (!gs_mbar_wait(&conv[sc], scp, a.timeout_ns)) {
                        gs_report(a.err, GS_DERR_TIMEOUT);
                        abort_flag = 1;
                        return false;
                    }
                }
                if (active) {
                    T outu[V], outv[V];
                    const T* bu = ring + sc * stage_elems;
                    const T* bv = bu + a.lay.field_elems;
                    T ymu[V], ypu[V], ymv[V], ypv[V];
                    gs_unpack<T>(*reinterpret_cast<const VT*>(bu + om), ymu);
                    gs_unpack<T>(*reinterpret_cast<const VT*>(bu + op), ypu);
                    gs_unpack<T>(*reinterpret_cast<const VT*>(bv + om), ymv);
                    gs_unpack<T>(*reinterpret_cast<const VT*>(bv + op), ypv);
                    T xlu = shlu, xlv = shlv, xru = shru, xrv = shrv;
                    if (AR != 0 || l_smem) { xlu = bu[oxl]; xlv = bv[oxl]; }
                    if (AR != 0 || r_smem) { xru = bu[oxr]; xrv = bv[oxr]; }
                    const uint32_t pre = NOISE ? gs_group_pre((uint32_t)gidx, a.keys) : 0u;
                    if constexpr (DS)
                        gs_update_group_ds<NOISE, GsFromPacked, PACK>(a.cds, pre, kk2, cu, cv, zmu, zmv, zpu, zpv, ymu,
                                                                      ypu, ymv, ypv, xlu, xru, xlv, xrv, outu, outv);
                    else if constexpr (AR == 2)
                        gs_update_group_fx<NOISE, PACK>(a.cfx, pre, kk2, cu, cv, zmu, zmv, zpu, zpv, ymu, ypu, ymv, ypv,
                                                        xlu, xru, xlv, xrv, outu, outv);
                    else if constexpr (FXF) {
                        uint32_t rng = 0;
                        gs_update_group_fxf<NOISE, PACK, FXF_DT>(a.cfxf, pre, kk2, cu, cv, zmu, zmv, zpu, zpv, ymu, ypu,
                                                                 ymv, ypv, xlu, xru, xlv, xrv, outu, outv, rng);
                        range_bad |= fxf_range_bad(rng);
                    }
                    else
                        gs_update_group<T, NOISE>(a.c, pre, kk2, cu, cv, zmu, zmv, zpu, zpv, ymu, ypu, ymv, ypv, xlu,
                                                  xru, xlv, xrv, outu, outv);
                    *reinterpret_cast<VT*>(a.un + gidx) = gs_pack<T>(outu);
                    *reinterpret_cast<VT*>(a.vn + gidx) = gs_pack<T>(outv);
                }
                release(sc);
                sc = sn;
                scp = snp;
                advance();
                gidx += DESC ? -LL : LL;
                return true;
            };

            // the plane before the first: centre values only (waited for above)
            if (!wait_full()) return false;
            convert_stage(cs);
            load_centre(qu[0], qv[0]);
            release(cs);
            advance();
            // the first plane
            sc = cs;
            scp = cph;
            if (!wait_full()) return false;
            convert_stage(cs);
            load_centre(qu[1], qv[1]);
            advance();

            int zi = 0;
            for (; zi + 3 <= nz; zi += 3) {
                if (!plane(qu[0], qv[0], qu[1], qv[1], qu[2], qv[2])) return false;
                if (!plane(qu[1], qv[1], qu[2], qv[2], qu[0], qv[0])) return false;
                if (!plane(qu[2], qv[2], qu[0], qv[0], qu[1], qv[1])) return false;
            }
            // remainder (each tile reloads planes z0 - 1 and z0 into q0, q1)
            if (zi < nz && !plane(qu[0], qv[0], qu[1], qv[1], qu[2], qv[2])) return false;
            if (zi + 1 < nz && !plane(qu[1], qv[1], qu[2], qv[2], qu[0], qv[0])) return false;
            release(sc);  // the plane after the last (only its centre was used)
            return !abort_flag;
        };
        bool ok;
        if constexpr (AR == 0)
            ok = dsc.w < 0 ? run(std::true_type{}) : run(std::false_type{});
        else
            ok = run(std::false_type{});  // these march up only
        if (!ok) return;
    }
    if (range_bad) gs_report(a.err, GS_DERR_RANGE);
}

template <typename T, bool NOISE, int AR, int IO>
__global__ void gs_zmarch_kernel(const __grid_constant__ ZMaps maps, const ZArgs<T> a)
{
    zmarch_body<T, NOISE, AR, IO>(maps, a);
}

// The fixed point with a remainder, capped at 72 registers (which its
// packed-step form needs anyway): 7 warps of 72 fit one SM sub-partition's
// 16K registers, so tiles of up to 25 warps (128 x 12 cells) fit an SM.
template <bool NOISE, int IO>
__global__ void __maxnreg__(72) gs_zmarch_fxf_kernel(const __grid_constant__ ZMaps maps, const ZArgs<double> a)
{
    zmarch_body<double, NOISE, 3, IO>(maps, a);
}

// The 64-bit fixed point, capped at 72 registers as well: its long 64-bit
// multiply chains leave it latency-bound, and the cap lets 25-warp tiles fit.
template <bool NOISE, int IO>
__global__ void __maxnreg__(72) gs_zmarch_fx_kernel(const __grid_constant__ ZMaps maps, const ZArgs<double> a)
{
    zmarch_body<double, NOISE, 2, IO>(maps, a);
}

bool zmarch_supported(int dtype, int L)
{
    const int V = dtype == GS_F32 ? 4 : 2;
    return L >= V && L % V == 0;
}

int zmarch_validate(int dtype, int L, const ZPlan& pl)
{
    const int V = dtype == GS_F32 ? 4 : 2;
    const int esz = elem_size(dtype);
    if (!zmarch_supported(dtype, L))
        return fail(GS_EINVAL, "z-march kernel needs L %% %d == 0 (L=%d)", V, L);
    if (pl.tx < V || pl.tx % V || pl.tx > 256 || pl.tx > L)
        return fail(GS_EINVAL, "tile_x=%d must be a multiple of %d in [%d, min(256, L)]", pl.tx, V, V);
    if (pl.ty < 1 || pl.ty > 256 || pl.ty > L)
        return fail(GS_EINVAL, "tile_y=%d must be in [1, min(256, L)]", pl.ty);
    if (pl.tz < 1) return fail(GS_EINVAL, "tile_z=%d must be >= 1", pl.tz);
    if (pl.stages < 3 || pl.stages > 8) return fail(GS_EINVAL, "stages=%d must be in [3, 8]", pl.stages);
    const int ncons = (pl.tx / V) * pl.ty;
    if (((ncons + 31) & ~31) + 32 > 1024)
        return fail(GS_EINVAL, "tile %dx%d needs more than 1024 threads", pl.tx, pl.ty);
    ZLayout lay = make_layout(esz, V, pl.tx, pl.ty);
    if ((size_t)lay.stage_bytes * pl.stages > 200 * 1024)
        return fail(GS_EINVAL, "tile %dx%d with %d stages needs %d B of shared memory", pl.tx, pl.ty,
                    pl.stages, lay.stage_bytes * pl.stages);
    return GS_OK;
}

int zmarch_encode(int dtype, int L, const ZPlan& pl, void* u, void* v, ZMaps* maps)
{
    const int V = dtype == GS_F32 ? 4 : 2;
    void* f[2] = {u, v};
    for (int i = 0; i < 2; ++i) {
        CUresult r0 = encode_tiled_3d(&maps->m[i][0], dtype, f[i], L, pl.tx, pl.ty);
        CUresult r1 = encode_tiled_3d(&maps->m[i][1], dtype, f[i], L, pl.tx, 1);
        CUresult r2 = encode_tiled_3d(&maps->m[i][2], dtype, f[i], L, V, pl.ty);
        if (r0 != CUDA_SUCCESS || r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
            return fail(GS_ECUDA, "cuTensorMapEncodeTiled failed (%d, %d, %d) for L=%d tile %dx%d",
                        (int)r0, (int)r1, (int)r2, L, pl.tx, pl.ty);
    }
    return GS_OK;
}

template <typename T, bool NOISE, int AR, int IO = 0>
static int zmarch_launch_t(int L, const ZPlan& pl, const ZMaps& maps, void* un, void* vn,
                           const Params& p, int64_t t, int* d_err, uint64_t timeout_ns,
                           int stall, unsigned* tickets, cudaStream_t s)
{
    constexpr int V = GsVec<T>::N;
    ZArgs<T> a;
    a.un = (T*)un;
    a.vn = (T*)vn;
    a.L = L;
    a.tx = pl.tx;
    a.ty = pl.ty;
    a.tz = pl.tz;
    a.ntx = (L + pl.tx - 1) / pl.tx;
    a.nty = (L + pl.ty - 1) / pl.ty;
    const int ntz = (L + pl.tz - 1) / pl.tz;
    a.ntiles = a.ntx * a.nty * ntz;
    a.stages = pl.stages;
    a.lay = make_layout(sizeof(T), V, pl.tx, pl.ty);
    a.c = make_coef<T>(p);
    a.cds = gs_make_coef_ds(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
    a.cfx = gs_make_coef_fx(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
    a.cfxf = gs_make_coef_fxf(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
    a.keys = gs_step_keys(p.seed, t);
    a.err = d_err;
    a.timeout_ns = timeout_ns;
    a.stall = stall;
    a.tickets = AR == 0 ? tickets : nullptr;
    a.alternate = AR == 0;
    const int ncons = (pl.tx / V) * pl.ty;
    const int threads = ((ncons + 31) & ~31) + 32;
    const size_t smem = (size_t)a.lay.stage_bytes * pl.stages;
    void (*kern)(const ZMaps, const ZArgs<T>) = nullptr;
    if constexpr (AR == 3)
        kern = gs_zmarch_fxf_kernel<NOISE, IO>;
    else if constexpr (AR == 2)
        kern = gs_zmarch_fx_kernel<NOISE, IO>;
    else
        kern = gs_zmarch_kernel<T, NOISE, AR, IO>;
    GS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return fail(GS_EINVAL, "z-march tile %dx%d does not fit on an SM", pl.tx, pl.ty);
    const int grid = std::min(a.ntiles, per_sm * num_sms());
    kern<<<grid, threads, smem, s>>>(maps, a);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int launch_zmarch(int dtype, int L, const ZPlan& pl, const ZMaps& maps, void* un, void* vn,
                  const Params& p, int64_t t, int* d_err, uint64_t timeout_ns, int stall,
                  unsigned* tickets, cudaStream_t s)
{
    const bool noise = p.noise != 0.0;
    if (dtype == GS_F32)
        return noise ? zmarch_launch_t<float, true, 0>(L, pl, maps, un, vn, p, t, d_err, timeout_ns, stall, tickets, s)
                     : zmarch_launch_t<float, false, 0>(L, pl, maps, un, vn, p, t, d_err, timeout_ns, stall, tickets, s);
    if (p.arith == GS_ARITH_DS || p.arith == GS_ARITH_FX || p.arith == GS_ARITH_FXF) {
#define GS_ZM(AR, IO)                                                                                            \
    return noise ? zmarch_launch_t<double, true, AR, IO>(L, pl, maps, un, vn, p, t, d_err, timeout_ns, stall, tickets, s) \
                 : zmarch_launch_t<double, false, AR, IO>(L, pl, maps, un, vn, p, t, d_err, timeout_ns, stall, tickets, s)
#define GS_ZM_IO(AR)          \
    switch (p.io & 3) {       \
    case 0: GS_ZM(AR, 0);     \
    case 1: GS_ZM(AR, 1);     \
    case 2: GS_ZM(AR, 2);     \
    default: GS_ZM(AR, 3);    \
    }
        if (p.arith == GS_ARITH_DS) GS_ZM_IO(1)
        if (p.arith == GS_ARITH_FX) GS_ZM_IO(2)
        switch ((p.io & 3) | (p.dt == 1.0 ? 4 : 0)) {
        case 0: GS_ZM(3, 0);
        case 1: GS_ZM(3, 1);
        case 2: GS_ZM(3, 2);
        case 3: GS_ZM(3, 3);
        case 4: GS_ZM(3, 4);
        case 5: GS_ZM(3, 5);
        case 6: GS_ZM(3, 6);
        default: GS_ZM(3, 7);
        }
#undef GS_ZM_IO
#undef GS_ZM
    }
    return noise ? zmarch_launch_t<double, true, 0>(L, pl, maps, un, vn, p, t, d_err, timeout_ns, stall, tickets, s)
                 : zmarch_launch_t<double, false, 0>(L, pl, maps, un, vn, p, t, d_err, timeout_ns, stall, tickets, s);
}

}  // namespace gs
