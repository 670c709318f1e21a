// Temporally blocked Gray-Scott stencil: D time steps per pass over HBM
// (FP32).
//
// Each CTA owns an x-y tile of TX x TY cells and a z-chunk of TZ planes.  It
// stages the tile plus a halo of HX = 4 cells in x and D rows in y (periodic
// wrap by modular addressing) plane by plane into a shared-memory ring with
// 16-byte cp.async copies, one group of 4 cells per thread.  Level s = 1..D
// applies step t+s-1 (gs_update, same arithmetic as every other kernel) to the
// region where level s-1 is valid, which shrinks by one cell per level; level
// s keeps its planes in a 4-plane shared ring.  Level s computes plane
// q = p - 2(s - 1) at iteration p, i.e. it lags level s-1 by two planes, so
// every plane it reads was written in an earlier iteration and one
// __syncthreads per iteration orders everything.  Level D writes the tile's
// interior to HBM.  HBM traffic per cell and pass: one read and one write of
// u and v (16 B) plus the halo re-reads of neighbouring tiles (mostly L2
// hits), for D steps.
//
// Requirements (checked by tblock_validate): L % TX == 0, L % TY == 0,
// TX % 4 == 0, 2 <= D <= 4.
#include <algorithm>
#include <cstdio>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {

constexpr int kTbStages = 5;  // level-0 ring depth (planes)
constexpr int kTbLevelRing = 4;

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
    GsKeys keys[4];       // step t + s - 1 for level s
};

GS_D void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(gs_smem_addr(smem)), "l"(gmem) : "memory");
}
GS_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
GS_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <bool NOISE, int D>
__global__ void __launch_bounds__(1024) gs_tblock_kernel(const TbArgs a)
{
    constexpr int V = 4;
    constexpr int HX = 4;
    constexpr int S = kTbStages;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);          // S planes x 2 fields
    float* lev = ring + (size_t)S * 2 * a.plane_elems;         // (D-1) levels x 4 planes x 2 fields
    const int tid = threadIdx.x;
    const int G = a.G, W = a.W, H = a.H, L = a.L;
    const int PE = a.plane_elems;
    const bool real = tid < G * H;
    const int gx = real ? tid % G : 0;
    const int row = real ? tid / G : 0;
    const long long LL = (long long)L * L;

    // shared-memory offsets of this thread's group and its neighbours (clamped
    // inside the region; clamped values only feed cells that are never used)
    const int o = row * W + gx * V;
    const int oym = (row > 0 ? row - 1 : row) * W + gx * V;
    const int oyp = (row < H - 1 ? row + 1 : row) * W + gx * V;
    const int oxl = gx > 0 ? o - 1 : o;
    const int oxr = gx < G - 1 ? o + V : o + V - 1;
    // level s is valid on rows [s, H - s) and cells [s, W - s) of the region
    bool act[D + 1];
#pragma unroll
    for (int s = 1; s <= D; ++s)
        act[s] = real && row >= s && row < H - s && gx * V + V > s && gx * V < W - s;
    const bool store = real && row >= D && row < D + a.ty && gx * V >= HX && gx * V < HX + a.tx;
    uint32_t kk2[D];
#pragma unroll
    for (int s = 0; s < D; ++s) kk2[s] = gs_kk2(a.keys[s]);

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int txi = tile % a.ntx;
        const int tyi = (tile / a.ntx) % a.nty;
        const int tzi = tile / (a.ntx * a.nty);
        const int x0 = txi * a.tx, y0 = tyi * a.ty, z0 = tzi * a.tz;
        const int nz = min(a.tz, L - z0);
        const int xg = (x0 - HX + gx * V + L) % L;    // global x of the group's first cell
        const int yg = (y0 - D + row + L) % L;        // global y of the row
        const long long rowoff = (long long)yg * L + xg;
        const int zlo = z0 - D;                       // global z of local level-0 plane 0
        const int nplanes = nz + 2 * D;               // level-0 planes z0-D .. z0+nz+D-1
        const int niter = nz + 3 * D - 3;             // level 1 runs planes j = 1 .. nz+2D-2

        auto issue = [&](int j) {
            if (real && j < nplanes) {
                const int zq = ((zlo + j) % L + L) % L;
                const long long g = (long long)zq * LL + rowoff;
                float* st = ring + (size_t)(j % S) * 2 * PE;
                cp_async16(st + o, a.u + g);
                cp_async16(st + PE + o, a.v + g);
            }
            cp_async_commit();
        };
        // prologue: planes 0 .. S-2 in flight; planes 0, 1, 2 complete
#pragma unroll
        for (int j = 0; j < S - 1; ++j) issue(j);
        cp_async_wait<S - 4>();
        __syncthreads();

        for (int it = 0; it < niter; ++it) {
            issue(it + S - 1);
#pragma unroll
            for (int s = 1; s <= D; ++s) {
                // level s computes local plane j = it + 1 - 2 (s - 1) (level-0 numbering)
                const int j = it + 1 - 2 * (s - 1);
                // needed range of level s: local planes s .. nz + 2D - 1 - s
                if (j < s || j > nz + 2 * D - 1 - s || !act[s]) continue;
                const float *pb, *cb, *nb;  // level s-1 planes j-1, j, j+1 (u; v at +PE)
                if (s == 1) {
                    pb = ring + (size_t)((j - 1) % S) * 2 * PE;
                    cb = ring + (size_t)(j % S) * 2 * PE;
                    nb = ring + (size_t)((j + 1) % S) * 2 * PE;
                } else {
                    const float* lb = lev + (size_t)(s - 2) * kTbLevelRing * 2 * PE;
                    pb = lb + (size_t)((j - 1) % kTbLevelRing) * 2 * PE;
                    cb = lb + (size_t)(j % kTbLevelRing) * 2 * PE;
                    nb = lb + (size_t)((j + 1) % kTbLevelRing) * 2 * PE;
                }
                float cu[4], cv[4], pu[4], pv[4], nu[4], nv[4], ymu[4], ypu[4], ymv[4], ypv[4], ou[4], ov[4];
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + o), cu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + PE + o), cv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pb + o), pu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(pb + PE + o), pv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(nb + o), nu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(nb + PE + o), nv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + oym), ymu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + oyp), ypu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + PE + oym), ymv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + PE + oyp), ypv);
                const float xlu = cb[oxl], xru = cb[oxr], xlv = cb[PE + oxl], xrv = cb[PE + oxr];
                const int zq = ((zlo + j) % L + L) % L;
                const long long g = (long long)zq * LL + rowoff;
                const uint32_t pre = NOISE ? gs_group_pre((uint32_t)g, a.keys[s - 1]) : 0u;
                gs_update_group<float, NOISE>(a.c, pre, kk2[s - 1], cu, cv, pu, pv, nu, nv, ymu, ypu, ymv, ypv,
                                              xlu, xru, xlv, xrv, ou, ov);
                if (s < D) {
                    float* wb = lev + (size_t)(s - 1) * kTbLevelRing * 2 * PE + (size_t)(j % kTbLevelRing) * 2 * PE;
                    *reinterpret_cast<float4*>(wb + o) = gs_pack<float>(ou);
                    *reinterpret_cast<float4*>(wb + PE + o) = gs_pack<float>(ov);
                } else if (store) {
                    *reinterpret_cast<float4*>(a.un + g) = gs_pack<float>(ou);
                    *reinterpret_cast<float4*>(a.vn + g) = gs_pack<float>(ov);
                }
            }
            cp_async_wait<S - 4>();
            __syncthreads();
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

int tblock_validate(int dtype, int L, const ZPlan& pl)
{
    if (dtype != GS_F32) return fail(GS_EINVAL, "temporal blocking is built for FP32 only");
    if (pl.depth < 2 || pl.depth > 4) return fail(GS_EINVAL, "depth=%d must be in [2, 4]", pl.depth);
    if (pl.tx < 4 || pl.tx % 4 || L % pl.tx) return fail(GS_EINVAL, "tile_x=%d must be a multiple of 4 dividing L=%d", pl.tx, L);
    if (pl.ty < 1 || L % pl.ty) return fail(GS_EINVAL, "tile_y=%d must divide L=%d", pl.ty, L);
    if (pl.tz < 1) return fail(GS_EINVAL, "tile_z=%d must be >= 1", pl.tz);
    if (L < 4 + 2 * pl.depth) return fail(GS_EINVAL, "L=%d too small for depth %d", L, pl.depth);
    const int W = pl.tx + 8, H = pl.ty + 2 * pl.depth, G = W / 4;
    if (G * H > 1024) return fail(GS_EINVAL, "tile %dx%d at depth %d needs %d threads (> 1024)", pl.tx, pl.ty, pl.depth, G * H);
    const size_t smem = (size_t)(kTbStages + kTbLevelRing * (pl.depth - 1)) * 2 * W * H * sizeof(float);
    if (smem > 227 * 1024)
        return fail(GS_EINVAL, "tile %dx%d at depth %d needs %zu B of shared memory", pl.tx, pl.ty, pl.depth, smem);
    return GS_OK;
}

template <bool NOISE, int D>
static int tblock_launch_t(int L, const ZPlan& pl, const void* u, const void* v, void* un, void* vn,
                           const Params& p, int64_t t, cudaStream_t s)
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
    a.W = pl.tx + 8;
    a.H = pl.ty + 2 * D;
    a.G = a.W / 4;
    a.plane_elems = a.W * a.H;
    a.c = gs_make_coef<float>(p.Du, p.Dv, p.F, p.k, p.dt, p.noise);
    for (int i = 0; i < 4; ++i) a.keys[i] = gs_step_keys(p.seed, t + (i < D ? i : 0));
    const int threads = (a.G * a.H + 31) & ~31;
    const size_t smem = (size_t)(kTbStages + kTbLevelRing * (D - 1)) * 2 * a.plane_elems * sizeof(float);
    auto kern = gs_tblock_kernel<NOISE, D>;
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
                  int64_t t, cudaStream_t s)
{
    const bool nz = p.noise != 0.0;
    switch (pl.depth) {
    case 2: return nz ? tblock_launch_t<true, 2>(L, pl, u, v, un, vn, p, t, s) : tblock_launch_t<false, 2>(L, pl, u, v, un, vn, p, t, s);
    case 3: return nz ? tblock_launch_t<true, 3>(L, pl, u, v, un, vn, p, t, s) : tblock_launch_t<false, 3>(L, pl, u, v, un, vn, p, t, s);
    case 4: return nz ? tblock_launch_t<true, 4>(L, pl, u, v, un, vn, p, t, s) : tblock_launch_t<false, 4>(L, pl, u, v, un, vn, p, t, s);
    default: return fail(GS_EINVAL, "depth=%d must be in [2, 4]", pl.depth);
    }
}

}  // namespace gs
