// Temporally blocked Gray-Scott stencil: D time steps per pass over HBM
// (FP32).
//
// Each CTA owns an x-y tile of TX x TY cells and a z-chunk of TZ planes.  Its
// region is the tile plus a halo of HX = 4 cells in x and D rows in y
// (periodic wrap by modular addressing), one group of 4 cells per thread, and
// tb_item (gs_tblock.cuh) stages, steps and stores it: level s applies step
// t + s - 1 where level s-1 is valid, the region shrinking by one cell per
// level in x and y.  HBM traffic per cell and pass: one read and one write of
// u and v (16 B) plus halo re-reads of neighbouring tiles (mostly L2 hits),
// for D steps.
//
// Requirements (checked by tblock_validate): L % TX == 0, L % TY == 0,
// TX % 4 == 0, 2 <= D <= 8, at most 512 threads.  Depths 5-8 use the deep
// variant further down (all levels in shared memory).
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "gs_common.cuh"
#include "gs_internal.h"
#include "gs_tblock.cuh"

namespace gs {

struct TbArgs {
    const float* u;
    const float* v;
    float* un;
    float* vn;
    int L;
    int tx, ty, tz;
    int ntx, nty, ntiles;
    int W, H, G;          // region width (cells), height (rows), groups per row
    int plane_elems;      // H * W (one field of one plane)
    GsCoef<float> c;
    GsKeys keys[8];       // step t + s - 1 for level s
    unsigned* tickets;    // [next ticket, CTAs done] (zeroed between launches), or null: round robin
};

// The tiles of a launch, in x, y, z order.  With a ticket counter each CTA
// takes the next free tile when it finishes one: thread 0 draws one tile
// ahead into a two-slot shared buffer (the barrier that ends every tile
// orders the hand-off), and the last CTA to finish zeroes the counter for
// the next launch.  Without one, CTA c takes tiles c, c + G, ...
struct TbTiles {
    const TbArgs& a;
    int* slot;  // two shared-memory slots
    int k = 0;
    GS_D int draw() { return a.tickets ? (int)atomicAdd(&a.tickets[0], 1u) : (int)blockIdx.x + (k++) * (int)gridDim.x; }
    GS_D void start()
    {
        if (threadIdx.x == 0) slot[0] = draw();
        __syncthreads();
    }
    // tile n of this CTA (>= ntiles: none left); thread 0 draws tile n + 1
    GS_D int get(int n)
    {
        const int tile = slot[n & 1];
        if (threadIdx.x == 0 && tile < a.ntiles) slot[(n + 1) & 1] = draw();
        return tile;
    }
    GS_D void finish()
    {
        if (threadIdx.x != 0 || !a.tickets) return;
        __threadfence();
        if (atomicAdd(&a.tickets[1], 1u) == gridDim.x - 1) {
            a.tickets[0] = 0;
            a.tickets[1] = 0;
        }
    }
};

// Shared memory: level-0 ring of kTbStages planes, then for each level
// 1..D-1 a ring of 3 planes; each plane holds u then v, H rows x W cells.
template <bool NOISE, int D>
__global__ void __launch_bounds__(512, 1) gs_tblock_kernel(const TbArgs a)
{
    constexpr int V = 4;
    constexpr int HX = 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    float* lev = ring + (size_t)kTbStages * 2 * a.plane_elems;
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = a.G, W = a.W, H = a.H, L = a.L;

    // this thread's place in the region (the same for every tile)
    TbThread<D> th;
    th.real = tid < G * H;
    const int gx = th.real ? tid % G : 0;
    const int row = th.real ? tid / G : 0;
    th.o = row * W + gx * V;
    th.oym = (row > 0 ? row - 1 : row) * W + gx * V;
    th.oyp = (row < H - 1 ? row + 1 : row) * W + gx * V;
    // x neighbours from the adjacent lanes when they hold this row's
    // neighbouring groups, else from shared memory (clamped inside the region)
    th.lsh = gx > 0 && lane > 0;
    th.rsh = gx < G - 1 && lane < 31;
    th.oxl = gx > 0 ? th.o - 1 : th.o;
    th.oxr = gx < G - 1 ? th.o + V : th.o + V - 1;
#pragma unroll
    for (int s = 1; s <= D; ++s) {
        th.act[s] = th.real && row >= s && row < H - s && gx * V + V > s && gx * V < W - s;
        th.wact[s] = true;  // not used (rows of 10-18 groups rarely leave a whole warp idle)
    }
    th.store = th.real && row >= D && row < D + a.ty && gx * V >= HX && gx * V < HX + a.tx;
    uint32_t kk2[D];
#pragma unroll
    for (int s = 0; s < D; ++s) kk2[s] = gs_kk2(a.keys[s]);

    __shared__ int s_tile[2];
    TbTiles tiles{a, s_tile};
    tiles.start();
    for (int n = 0;; ++n) {
        const int tile = tiles.get(n);
        if (tile >= a.ntiles) break;
        const int txi = tile % a.ntx;
        const int tyi = (tile / a.ntx) % a.nty;
        const int tzi = tile / (a.ntx * a.nty);
        const int x0 = txi * a.tx, y0 = tyi * a.ty, z0 = tzi * a.tz;
        const int xg = (x0 - HX + gx * V + L) % L;
        const int yg = (y0 - D + row + L) % L;
        tb_item<NOISE, D, false>(a.u, a.v, a.un, a.vn, L, (uint32_t)yg * (uint32_t)L + (uint32_t)xg, z0, min(a.tz, L - z0),
                          a.c, a.keys, kk2, th, ring, lev, a.plane_elems);
    }
    tiles.finish();
}

// ---------------------------------------------------------------------------
// Deep temporal blocking (D = 5..8).  Same schedule (level s computes plane
// j = p + 1 - 2(s-1) at iteration p, so one barrier per iteration orders
// everything), but no register FIFOs: every level keeps its planes in a
// 4-plane shared ring (level s reads planes j-1, j, j+1 of level s-1 while
// level s-1 writes plane j+2 into the fourth slot), and all neighbours come
// from shared memory.  The x halo is 8 cells (two groups).  Shared memory
// limits the tiles to about 16 x 8 at D = 8, so the halo recomputation is
// large; the autotuner includes these depths but they do not beat depth 1.
// ---------------------------------------------------------------------------
constexpr int kTbDeepHX = 8;
constexpr int kTbDeepRing = 4;

template <bool NOISE, int D>
__global__ void __launch_bounds__(512, 1) gs_tblock_deep_kernel(const TbArgs a)
{
    constexpr int V = 4;
    constexpr int HX = kTbDeepHX;
    constexpr int S = kTbStages;
    constexpr int R = kTbDeepRing;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    float* lev = ring + (size_t)S * 2 * a.plane_elems;
    const int tid = threadIdx.x;
    const int G = a.G, W = a.W, H = a.H, L = a.L;
    const int PE = a.plane_elems;
    const bool real = tid < G * H;
    const int gx = real ? tid % G : 0;
    const int row = real ? tid / G : 0;
    const uint32_t LL = (uint32_t)L * (uint32_t)L;
    // offsets of this thread's group and its neighbours (clamped inside the region)
    const int o = row * W + gx * V;
    const int oym = (row > 0 ? row - 1 : row) * W + gx * V;
    const int oyp = (row < H - 1 ? row + 1 : row) * W + gx * V;
    const int oxl = gx > 0 ? o - 1 : o;
    const int oxr = gx < G - 1 ? o + V : o + V - 1;
    bool act[D + 1];
#pragma unroll
    for (int s = 1; s <= D; ++s)
        act[s] = real && row >= s && row < H - s && gx * V + V > s && gx * V < W - s;
    const bool store = real && row >= D && row < D + a.ty && gx * V >= HX && gx * V < HX + a.tx;
    uint32_t kk2[D];
#pragma unroll
    for (int s = 0; s < D; ++s) kk2[s] = gs_kk2(a.keys[s]);

    __shared__ int s_tile[2];
    TbTiles tiles{a, s_tile};
    tiles.start();
    for (int n = 0;; ++n) {
        const int tile = tiles.get(n);
        if (tile >= a.ntiles) break;
        const int txi = tile % a.ntx;
        const int tyi = (tile / a.ntx) % a.nty;
        const int tzi = tile / (a.ntx * a.nty);
        const int x0 = txi * a.tx, y0 = tyi * a.ty, z0 = tzi * a.tz;
        const int nz = min(a.tz, L - z0);
        const int xg = (x0 - HX + gx * V + L) % L;
        const int yg = (y0 - D + row + L) % L;
        const uint32_t rowoff = (uint32_t)yg * (uint32_t)L + (uint32_t)xg;
        const int zlo = z0 - D;                 // global z of local level-0 plane 0
        const int nplanes = nz + 2 * D;         // level-0 planes z0-D .. z0+nz+D-1
        const int niter = nz + 3 * D - 3;       // level D finishes local plane nz+D-1 at it = nz+3D-4

        auto issue = [&](int jl) {
            if (real && jl < nplanes) {
                int zq = zlo + jl;
                zq += zq < 0 ? L : 0;
                zq -= zq >= L ? L : 0;
                const size_t gidx = (size_t)zq * LL + rowoff;
                float* st = ring + (size_t)(jl % S) * 2 * PE;
                tb_cp16(st + o, a.u + gidx);
                tb_cp16(st + PE + o, a.v + gidx);
            }
            tb_commit();
        };
#pragma unroll
        for (int jl = 0; jl < S - 1; ++jl) issue(jl);
        tb_wait<S - 4>();  // planes 0, 1, 2 complete
        __syncthreads();

        for (int it = 0; it < niter; ++it) {
            issue(it + S - 1);
#pragma unroll
            for (int s = 1; s <= D; ++s) {
                const int j = it + 1 - 2 * (s - 1);
                if (j < s || j > nz + 2 * D - 1 - s || !act[s]) continue;
                // level s-1 planes j-1, j, j+1
                const float* pm;
                const float* pc;
                const float* pp;
                if (s == 1) {
                    pm = ring + (size_t)((j - 1) % S) * 2 * PE;
                    pc = ring + (size_t)(j % S) * 2 * PE;
                    pp = ring + (size_t)((j + 1) % S) * 2 * PE;
                } else {
                    const float* lb = lev + (size_t)(s - 2) * R * 2 * PE;
                    pm = lb + (size_t)((j - 1) % R) * 2 * PE;
                    pc = lb + (size_t)(j % R) * 2 * PE;
                    pp = lb + (size_t)((j + 1) % R) * 2 * PE;
                }
                float cu[4], cv[4], zmu[4], zmv[4], zpu[4], zpv[4], ymu[4], ypu[4], ymv[4], ypv[4];
                gs_unpack<float>(*reinterpret_cast<const float4*>(pc + o), cu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pc + PE + o), cv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pm + o), zmu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pm + PE + o), zmv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pp + o), zpu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pp + PE + o), zpv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pc + oym), ymu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pc + oyp), ypu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pc + PE + oym), ymv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pc + PE + oyp), ypv);
                const float xlu = pc[oxl], xlv = pc[PE + oxl], xru = pc[oxr], xrv = pc[PE + oxr];
                int zq = zlo + j;
                zq += zq < 0 ? L : 0;
                zq -= zq >= L ? L : 0;
                const uint32_t g = (uint32_t)zq * LL + rowoff;
                const uint32_t pre = NOISE ? gs_group_pre(g, a.keys[s - 1]) : 0u;
                float ou[4], ov[4];
                gs_update_group<float, NOISE>(a.c, pre, kk2[s - 1], cu, cv, zmu, zmv, zpu, zpv, ymu, ypu, ymv, ypv,
                                              xlu, xru, xlv, xrv, ou, ov);
                if (s < D) {
                    float* wb = lev + ((size_t)(s - 1) * R + (size_t)(j % R)) * 2 * PE;
                    *reinterpret_cast<float4*>(wb + o) = gs_pack<float>(ou);
                    *reinterpret_cast<float4*>(wb + PE + o) = gs_pack<float>(ov);
                } else if (store) {
                    *reinterpret_cast<float4*>(a.un + (size_t)zq * LL + rowoff) = gs_pack<float>(ou);
                    *reinterpret_cast<float4*>(a.vn + (size_t)zq * LL + rowoff) = gs_pack<float>(ov);
                }
            }
            tb_wait<S - 4>();  // planes up to it + 3 complete
            __syncthreads();
        }
        tb_wait<0>();
        __syncthreads();
    }
    tiles.finish();
}

static int tblock_halo_x(int depth) { return depth <= 4 ? 4 : kTbDeepHX; }

static size_t tblock_smem(int depth, int W, int H)
{
    const int planes = depth <= 4 ? kTbStages + 3 * (depth - 1) : kTbStages + kTbDeepRing * (depth - 1);
    return (size_t)planes * 2 * W * H * sizeof(float);
}

int tblock_validate(int dtype, int L, const ZPlan& pl)
{
    if (dtype != GS_F32) return fail(GS_EINVAL, "temporal blocking is built for FP32 only");
    if (pl.depth < 2 || pl.depth > 8) return fail(GS_EINVAL, "depth=%d must be in [2, 8]", pl.depth);
    if (pl.tx < 4 || pl.tx % 4 || L % pl.tx) return fail(GS_EINVAL, "tile_x=%d must be a multiple of 4 dividing L=%d", pl.tx, L);
    if (pl.ty < 1 || L % pl.ty) return fail(GS_EINVAL, "tile_y=%d must divide L=%d", pl.ty, L);
    if (pl.tz < 1) return fail(GS_EINVAL, "tile_z=%d must be >= 1", pl.tz);
    const int HX = tblock_halo_x(pl.depth);
    if (L < 2 * HX || L < 2 * pl.depth + 4) return fail(GS_EINVAL, "L=%d too small for depth %d", L, pl.depth);
    const int W = pl.tx + 2 * HX, H = pl.ty + 2 * pl.depth, G = W / 4;
    if (G * H > 512) return fail(GS_EINVAL, "tile %dx%d at depth %d needs %d threads (> 512)", pl.tx, pl.ty, pl.depth, G * H);
    const size_t smem = tblock_smem(pl.depth, W, H);
    if (smem > 227 * 1024)
        return fail(GS_EINVAL, "tile %dx%d at depth %d needs %zu B of shared memory", pl.tx, pl.ty, pl.depth, smem);
    return GS_OK;
}

template <bool NOISE, int D>
static int tblock_launch_t(int L, const ZPlan& pl, const void* u, const void* v, void* un, void* vn,
                           const Params& p, int64_t t, unsigned* tickets, cudaStream_t s)
{
    TbArgs a;
    a.u = (const float*)u;
    a.v = (const float*)v;
    a.un = (float*)un;
    a.vn = (float*)vn;
    a.L = L;
    a.tx = pl.tx;
    a.ty = pl.ty;
    a.tz = pl.tz;
    a.ntx = L / pl.tx;
    a.nty = L / pl.ty;
    a.ntiles = a.ntx * a.nty * ((L + pl.tz - 1) / pl.tz);
    a.W = pl.tx + 2 * tblock_halo_x(D);
    a.H = pl.ty + 2 * D;
    a.G = a.W / 4;
    a.plane_elems = a.W * a.H;
    a.c = gs_make_coef<float>(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
    for (int i = 0; i < 8; ++i) a.keys[i] = gs_step_keys(p.seed, t + (i < D ? i : 0));
    a.tickets = tickets;
    const int threads = (a.G * a.H + 31) & ~31;
    const size_t smem = tblock_smem(D, a.W, a.H);
    void (*kern)(const TbArgs) = nullptr;
    if constexpr (D <= 4)
        kern = gs_tblock_kernel<NOISE, D>;
    else
        kern = gs_tblock_deep_kernel<NOISE, D>;
    GS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return fail(GS_EINVAL, "temporal-blocking tile %dx%d depth %d does not fit on an SM", pl.tx, pl.ty, D);
    const int grid = std::min(a.ntiles, per_sm * num_sms());
    kern<<<grid, threads, smem, s>>>(a);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int launch_tblock(int L, const ZPlan& pl, const void* u, const void* v, void* un, void* vn, const Params& p,
                  int64_t t, unsigned* tickets, cudaStream_t s)
{
    const bool nz = p.noise != 0.0;
#define GS_TB_CASE(DD) \
    case DD: return nz ? tblock_launch_t<true, DD>(L, pl, u, v, un, vn, p, t, tickets, s) : tblock_launch_t<false, DD>(L, pl, u, v, un, vn, p, t, tickets, s);
    switch (pl.depth) {
        GS_TB_CASE(2)
        GS_TB_CASE(3)
        GS_TB_CASE(4)
        GS_TB_CASE(5)
        GS_TB_CASE(6)
        GS_TB_CASE(7)
        GS_TB_CASE(8)
    default: return fail(GS_EINVAL, "depth=%d must be in [2, 8]", pl.depth);
    }
#undef GS_TB_CASE
}

}  // namespace gs
