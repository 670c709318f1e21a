// One temporally blocked work item (FP32, D = 2..4 steps per pass over HBM):
// the schedule shared by the single-grid kernel (gs_tblock_kernel, x-y tiles
// with an x halo) and the batched one (gs_batch_tb_kernel, full-row tiles
// with the x wrap inside the row).
//
// The item's region is W x H cells per plane (the tile plus its halo), one
// group of 4 cells per thread.  Level s = 1..D applies step t + s - 1
// (gs_update_group, the arithmetic of every other kernel) to the region where
// level s-1 is valid, which shrinks by one cell (row) per level.  Level s
// computes plane j = p + 1 - 2 (s - 1) at iteration p (two planes behind
// level s-1), so every input of every level was produced in an earlier
// iteration: the levels of one iteration are independent (the instruction-
// level parallelism that hides latency), levels run from the top down and
// each reads its input FIFO before the level below pushes.  The z-1 / z / z+1
// values of a thread's own group come from per-level register FIFOs, x
// neighbours from the adjacent lanes (or shared memory at a warp or row edge),
// and only the y neighbours from shared memory (a 3-plane ring per level), so
// one __syncthreads per iteration orders everything.  Each thread stages its
// own group of the level-0 planes with 16-byte cp.async copies into a 5-plane
// ring; level D writes the tile's interior to HBM.
#pragma once

#include <type_traits>

#include "gs_common.cuh"

namespace gs {

constexpr int kTbStages = 5;  // level-0 ring depth (planes)

GS_D void tb_cp16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(gs_smem_addr(smem)), "l"(gmem) : "memory");
}
GS_D void tb_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
GS_D void tb_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// A thread's place in the item's region: shared-memory offsets of its group
// (o) and of its neighbours (y clamped inside the region: clamped values only
// feed cells no level keeps; x from the caller's rule), whether its left /
// right neighbour group sits in the adjacent lane of the same row, which
// levels it computes (act) and whether some lane of its warp does (wact:
// with WSKIP a warp with no lane at a level skips it), and whether it stores
// level D.
template <int D>
struct TbThread {
    int o, oym, oyp, oxl, oxr;
    bool real, lsh, rsh, store;
    bool act[D + 1], wact[D + 1];
};

// Stage, step and store one item: planes z0 - D .. z0 + nz + D - 1 of the
// fields u, v (L^3, x fastest), written back for planes z0 .. z0 + nz - 1 of
// un, vn.  rowoff: global offset (y L + x) of this thread's group within a
// plane.  keys / kk2: the noise keys of steps t .. t + D - 1.  ring: 2 S PE
// floats, lev: 6 (D - 1) PE floats (PE >= W H, a multiple of 4).  WSKIP:
// whole warps skip the levels none of their lanes computes (worth it when
// rows fill whole warps, as in the batch's full-row tiles; elsewhere it only
// costs registers).
template <bool NOISE, int D, bool WSKIP>
GS_D void tb_item(const float* __restrict__ u, const float* __restrict__ v, float* __restrict__ un,
                  float* __restrict__ vn, int L, uint32_t rowoff, int z0, int nz, const GsCoef<float>& c,
                  const GsKeys* keys, const uint32_t* kk2, const TbThread<D>& th, float* ring, float* lev, int PE)
{
    constexpr int S = kTbStages;
    const uint32_t LL = (uint32_t)L * (uint32_t)L;
    const int o = th.o;
    const int zlo = z0 - D;            // global z of local level-0 plane 0
    const int nplanes = nz + 2 * D;    // level-0 planes z0-D .. z0+nz+D-1
    const int niter = nz + 3 * D - 3;  // level D finishes local plane nz+D-1 at it = nz+3D-4

    auto issue = [&](int jl) {
        if (th.real && jl < nplanes) {
            int zq = zlo + jl;
            zq += zq < 0 ? L : 0;
            zq -= zq >= L ? L : 0;
            const size_t gidx = (size_t)zq * LL + rowoff;
            float* st = ring + (size_t)(jl % S) * 2 * PE;
            tb_cp16(st + o, u + gidx);
            tb_cp16(st + PE + o, v + gidx);
        }
        tb_commit();
    };
#pragma unroll
    for (int jl = 0; jl < S - 1; ++jl) issue(jl);
    tb_wait<S - 4>();  // planes 0, 1, 2 complete
    __syncthreads();

    // register FIFOs of this thread's group: level s planes (oldest, middle, newest)
    float fu[D][3][4], fv[D][3][4];
    gs_unpack<float>(*reinterpret_cast<const float4*>(ring + o), fu[0][1]);
    gs_unpack<float>(*reinterpret_cast<const float4*>(ring + PE + o), fv[0][1]);
    gs_unpack<float>(*reinterpret_cast<const float4*>(ring + 2 * PE + o), fu[0][2]);
    gs_unpack<float>(*reinterpret_cast<const float4*>(ring + 3 * PE + o), fv[0][2]);

    // One iteration: levels from the top down.  FULL (the steady state,
    // every level in range) drops the range and activity tests, so the
    // iteration is one straight-line block the compiler can interleave
    // across levels: inactive lanes of an active warp compute values nobody
    // reads and only `store` guards the write to HBM.
    auto iteration = [&](const int it, auto full_tag) {
        constexpr bool FULL = decltype(full_tag)::value;
        issue(it + S - 1);
        const int zb = zlo + it + 1;  // global z of level 1's plane, unwrapped
#pragma unroll
        for (int s = D; s >= 1; --s) {
            // level s computes local plane j = it + 1 - 2 (s - 1) from level
            // s-1 planes j-1, j, j+1: all produced in earlier iterations
            const int j = it + 1 - 2 * (s - 1);
            // a warp with no lane at level s leaves it (and its FIFO and
            // level plane, which no active lane reads) alone
            if constexpr (WSKIP) {
                if (!th.wact[s]) continue;
            }
            if (s == 1) {
                // level 0 "computes" by loading: push local plane it + 2 (complete)
                const float* nb = ring + (size_t)((it + 2) % S) * 2 * PE;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    fu[0][0][e] = fu[0][1][e]; fu[0][1][e] = fu[0][2][e];
                    fv[0][0][e] = fv[0][1][e]; fv[0][1][e] = fv[0][2][e];
                }
                gs_unpack<float>(*reinterpret_cast<const float4*>(nb + o), fu[0][2]);
                gs_unpack<float>(*reinterpret_cast<const float4*>(nb + PE + o), fv[0][2]);
            }
            // centre plane of level s-1 (for y and x neighbours)
            const float* cb = s == 1 ? ring + (size_t)(j % S) * 2 * PE
                                     : lev + ((size_t)(s - 2) * 3 + (size_t)(j % 3)) * 2 * PE;
            const float(&cu)[4] = fu[s - 1][1];
            const float(&cv)[4] = fv[s - 1][1];
            // x neighbours by shuffle (all lanes of the warp take part)
            float xlu = __shfl_up_sync(0xffffffffu, cu[3], 1);
            float xlv = __shfl_up_sync(0xffffffffu, cv[3], 1);
            float xru = __shfl_down_sync(0xffffffffu, cu[0], 1);
            float xrv = __shfl_down_sync(0xffffffffu, cv[0], 1);
            if (!FULL && !(j >= s && j <= nz + 2 * D - 1 - s)) continue;
            float ou[4] = {0.f, 0.f, 0.f, 0.f}, ov[4] = {0.f, 0.f, 0.f, 0.f};
            int zq = zb - 2 * (s - 1);
            zq += zq < 0 ? L : 0;
            zq -= zq >= L ? L : 0;
            if (FULL || th.act[s]) {
                if (!th.lsh) { xlu = cb[th.oxl]; xlv = cb[PE + th.oxl]; }
                if (!th.rsh) { xru = cb[th.oxr]; xrv = cb[PE + th.oxr]; }
                float ymu[4], ypu[4], ymv[4], ypv[4];
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + th.oym), ymu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + th.oyp), ypu);
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + PE + th.oym), ymv);
                gs_unpack<float>(*reinterpret_cast<const float4*>(cb + PE + th.oyp), ypv);
                const uint32_t g = (uint32_t)zq * LL + rowoff;
                const uint32_t pre = NOISE ? gs_group_pre(g, keys[s - 1]) : 0u;
                gs_update_group<float, NOISE>(c, pre, kk2[s - 1], cu, cv, fu[s - 1][0], fv[s - 1][0], fu[s - 1][2],
                                              fv[s - 1][2], ymu, ypu, ymv, ypv, xlu, xru, xlv, xrv, ou, ov);
                if (s < D) {
                    float* wb = lev + ((size_t)(s - 1) * 3 + (size_t)(j % 3)) * 2 * PE;
                    *reinterpret_cast<float4*>(wb + o) = gs_pack<float>(ou);
                    *reinterpret_cast<float4*>(wb + PE + o) = gs_pack<float>(ov);
                } else if (th.store) {
                    *reinterpret_cast<float4*>(un + (size_t)zq * LL + rowoff) = gs_pack<float>(ou);
                    *reinterpret_cast<float4*>(vn + (size_t)zq * LL + rowoff) = gs_pack<float>(ov);
                }
            }
            if (s < D) {
                // push level s plane j (values of inactive lanes are never used)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    fu[s][0][e] = fu[s][1][e]; fu[s][1][e] = fu[s][2][e]; fu[s][2][e] = ou[e];
                    fv[s][0][e] = fv[s][1][e]; fv[s][1][e] = fv[s][2][e]; fv[s][2][e] = ov[e];
                }
            }
        }
        tb_wait<S - 4>();  // planes up to it + 3 complete
        __syncthreads();
    };
    // every level is in range for it in [3D-3, nz+2D-3]
    const int steady_end = nz + 2 * D - 2;
    int it = 0;
    for (; it < 3 * D - 3; ++it) iteration(it, std::false_type{});
    // unrolled by 3: the FIFO rotation becomes register renaming
#pragma unroll 3
    for (; it < steady_end; ++it) iteration(it, std::true_type{});
    for (; it < niter; ++it) iteration(it, std::false_type{});
    tb_wait<0>();
    __syncthreads();
}

}  // namespace gs
