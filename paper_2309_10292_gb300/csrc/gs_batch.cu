// Batched Gray-Scott: many independent periodic grids of different sizes
// and (F, k) advanced together by one persistent kernel.
//
// Work decomposition.  Each plane of instance i (edge L_i, 4 <= L_i <= 256)
// is cut into runs of 256 V consecutive cells in row-major order (one group
// of V cells per consumer thread), times a z-chunk of tz planes.  Every tile
// but the last of a plane is therefore full whatever L_i is (row-shaped
// tiles leave threads idle when L_i does not divide 256 V: 10 rows of 96 use
// 960 of 1024 cells, and the tenth tile of a 96^2 plane only 6 rows).  A tile
// is staged as the whole rows it touches, so the x wrap is an index wrap
// inside shared memory (no x-halo copies).  Work items are numbered instance
// by instance, and the CTAs take them in that order from a ticket counter
// (each CTA's next item is the next free one, so a step ends within a
// fraction of an item on every CTA; the last grid / 2 items are cut along z
// into four pieces for the same reason).  Neighbouring z-chunks march in
// opposite directions, so the halo planes two chunks share are read by both
// at about the same time (once from HBM, once from L2).  The allocation-free
// step keeps the static order instead: CTA b takes items b, b + grid, ...
//
// Per item a producer warp streams the planes z0-1 .. z0+nz with TMA (a box
// of the tile's rows + two wrapped halo rows per field, per-instance tensor
// maps in global memory) into a shared-memory ring; 256 consumer threads
// hold z-1/z/z+1 in registers and store u', v' with 16-byte writes, exactly
// like the single grid z-march kernel and with the same per-cell update, so
// results are bitwise equal to running each instance alone.
//
// Between steps all CTAs meet at a grid barrier in global memory (an
// arrival counter, reset before every launch).  Every wait is bounded: on
// expiry the kernel records GS_ETIMEOUT in the control block and all CTAs
// leave after letting their own copies land.  The n-step run (counter reset +
// kernel) is captured once per n as a CUDA graph and replayed with one
// cudaGraphLaunch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <map>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "gs_common.cuh"
#include "gs_internal.h"
#include "gs_tblock.cuh"

namespace gs {

constexpr int kBatchConsumers = 256;
constexpr int kBatchThreads = kBatchConsumers + 32;

struct BInst {
    int L;
    int ty;         // rows of a tile's TMA box (the most rows a 256 V-cell run touches)
    int nty, ntz;   // tiles per plane, z-chunks
    int item0, nitems;
    uint32_t seed_lo, seed_hi;
    double F, Fk;
    long long off[2][2];  // element offsets of buffer [set][field] in the arena
};

struct BCtrl {
    long long t;    // step counter of the current state
    int cur;        // buffer set holding the current state
    unsigned bar;   // grid barrier arrivals (reset before every launch) ...
    unsigned next;  // ... and the work-item tickets of a dynamic launch (with it)
    int err;        // device error word
    int pad[2];
};
static_assert(offsetof(BCtrl, next) == offsetof(BCtrl, bar) + sizeof(unsigned), "bar and next reset together");

template <typename T>
struct BArgs {
    T* arena;
    const BInst* inst;
    const int4* items;        // work item -> (instance, y0, z0, nz); nz < 0: march down |nz| planes
    const CUtensorMap* maps;  // [inst][set][field][kind]: kind 0 tile box, 1 halo row
    BCtrl* ctrl;
    int nitems, tz, stages;
    int main_elems, row_elems, field_elems;  // shared-memory stage layout (elements)
    long long nsteps;
    T Du6, Dv6, dt, noise24;
    uint64_t timeout_ns;
    int fault;    // 1: the producer issues no copies; 2: CTA 0 never arrives at the grid barrier
    int dynamic;  // 1: CTAs take items in table order from a ticket counter; 0: CTA b takes b, b + grid, ...
};

// What the consumers need of one work item, written to shared memory by the
// producer thread before it releases the item's first plane (the release of
// that mbarrier arrival orders it), so the consumers start an item without
// waiting on the item and instance tables in global memory.  kBatchDescs
// slots are reused round robin: the producer fills slot k + kBatchDescs only
// after the consumers freed a stage issued kBatchDescs items later than item
// k's first plane (an item has at least 3 planes, the end-of-step marker one,
// and the ring at most 8 stages, so they read slot k long before).  A
// descriptor with nz == 0 marks the end of the CTA's items for the step; it
// travels through one ring stage (a plain arrival, no copy).
constexpr int kBatchDescs = 4;
template <typename T>
struct BDesc {
    T* un;
    T* vn;             // output fields of this step
    T F, Fk;
    GsKeys keys;       // noise keys of the instance and step
    uint32_t kk2;
    int L, c0, z0, nz;  // nz < 0: march down |nz| planes
};

GS_D bool wait_or_abort(uint64_t* bar, uint32_t parity, uint64_t timeout_ns, volatile int* abort_flag)
{
    if (gs_mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gs_globaltimer();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (gs_mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gs_globaltimer() - t0 > timeout_ns) return false;
    }
}

// All threads of the CTA call this.  Returns false once any CTA failed.
GS_D bool batch_grid_sync(BCtrl* ctrl, unsigned target, uint64_t timeout_ns, bool skip_arrive,
                          volatile int* s_abort)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = *s_abort == 0;
        if (ok && !skip_arrive) {
            __threadfence();
            gs_atom_add_release_gpu(&ctrl->bar, 1u);
        }
        if (ok) {
            uint64_t t0 = 0;
            bool timing = false;
            // the arrival counter and the target both wrap modulo 2^32 on long
            // runs (steps x CTAs); their signed difference stays exact because
            // the counter is never more than one step's arrivals away from it
            while ((int)(gs_ld_acquire_gpu(&ctrl->bar) - target) < 0) {
                if (gs_ld_relaxed_gpu(&ctrl->err)) {
                    ok = false;
                    break;
                }
                if (!timing) {
                    t0 = gs_globaltimer();
                    timing = true;
                } else if (gs_globaltimer() - t0 > timeout_ns) {
                    gs_report(&ctrl->err, GS_DERR_TIMEOUT);
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!ok) *s_abort = 1;
        __threadfence();
    }
    __syncthreads();
    return *s_abort == 0;
}

// Register cap (measured on GB300, FP32, noise on, 256 mixed grids): 76
// registers runs 1.3 % faster than 80, 6 % faster than the 88-94 the
// compiler takes under __launch_bounds__(288, 2), and without any bound it
// settles on 72 with spills (10 % slower).  FP64 spills below about 90.
template <typename T, bool NOISE>
__global__ void __maxnreg__(sizeof(T) == 4 ? 76 : 96) gs_batch_kernel(const __grid_constant__ BArgs<T> a)
{
    constexpr int V = GsVec<T>::N;
    using VT = typename GsVec<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[16];
    __shared__ volatile int s_abort;
    __shared__ BDesc<T> s_desc[kBatchDescs];

    const int S = a.stages;
    uint64_t* full = bars;
    uint64_t* empty = bars + S;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    T* ring = reinterpret_cast<T*>(smem);
    const int stage_elems = 2 * a.field_elems;
    const int top_off = a.main_elems, bot_off = a.main_elems + a.row_elems;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            gs_mbar_init(&full[s], 1);
            gs_mbar_init(&empty[s], kBatchConsumers / 32);
        }
        s_abort = 0;
        gs_fence_mbar_init();
    }
    __syncthreads();

    const long long t0 = a.ctrl->t;
    const int cur0 = a.ctrl->cur;
    // ring position, advanced identically by producer and consumers: stage
    // index and the parity of its current round (no runtime division)
    int cs = 0;
    uint32_t cph = 0;
    uint32_t seq = 0;      // planes issued by the producer (for its drain)
    uint32_t kl = 0;       // items taken by this CTA (descriptor slot kl % kBatchDescs)
    bool wrapped = false;  // producer: every stage used once
    auto advance = [&]() {
        if (++cs == S) { cs = 0; cph ^= 1u; wrapped = true; }
    };
    long long s = 0;
    for (; s < a.nsteps; ++s) {
        const int in = (cur0 + (int)(s & 1)) & 1, out = in ^ 1;
        const long long t = t0 + s;
        if (tid < kBatchConsumers) {
            // ------------------------------ consumers ------------------------------
            // planes z-1, z, z+1 in three register sets rotated by renaming
            T qu[3][V], qv[3][V];
            for (;;) {
                // the next item's first plane, and with it its descriptor
                if (!wait_or_abort(&full[cs], cph, a.timeout_ns, &s_abort)) {
                    gs_report(&a.ctrl->err, GS_DERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                const BDesc<T> d = s_desc[kl % kBatchDescs];
                ++kl;
                if (d.nz == 0) {
                    // no more items for this CTA in this step
                    __syncwarp();
                    if (lane == 0) gs_mbar_arrive(&empty[cs]);
                    advance();
                    break;
                }
                // One item, marching up (DESC false: planes z0, z0+1, ...) or
                // down (DESC true, d.nz < 0: planes z0+nz-1, z0+nz-2, ...).
                // Either way each cell sees z-1 as its lower and z+1 as its
                // upper neighbour, so the update is the same to the bit.
                // Returns false when a wait for a stage ran out.
                auto run = [&](auto desc_tag) -> bool {
                    constexpr bool DESC = decltype(desc_tag)::value;
                    const int L = d.L;
                    const int c0 = d.c0, z0 = d.z0, nz = DESC ? -d.nz : d.nz;
                    // the tile: cells c0 .. c0 + C - 1 of each plane (row
                    // major), staged as the whole rows ya .. yb (box rows from
                    // ya; rows past yb are not used) plus halo rows ya - 1,
                    // yb + 1.  This thread's group: cell c0 + V tid.
                    const int C = min(kBatchConsumers * V, L * L - c0);
                    const int ya = c0 / L, nrows = (c0 + C - 1) / L - ya + 1;
                    const bool active = V * tid < C;
                    const int q = (active ? V * tid : 0) + c0 - ya * L;  // offset from the box's first row
                    const int row = q / L, x = q - row * L;
                    const int moff = q;
                    const int rowbase = row * L;
                    GsCoef<T> c;
                    c.Du6 = a.Du6; c.Dv6 = a.Dv6; c.dt = a.dt; c.noise24 = a.noise24;
                    c.F = d.F; c.Fk = d.Fk;
                    const GsKeys keys = d.keys;
                    const uint32_t kk2 = d.kk2;
                    T* un = d.un;
                    T* vn = d.vn;
                    const long long LL = (long long)L * L;
                    const int om = row > 0 ? moff - L : top_off + x;
                    const int op = row + 1 < nrows ? moff + L : bot_off + x;
                    // x neighbours from the adjacent lanes within a row: the
                    // tile's last active group always ends a row (a partial
                    // tile is the last of its plane), so no active lane
                    // reads an inactive one
                    const bool l_smem = x == 0 || lane == 0;
                    const bool r_smem = x + V == L || lane == 31;
                    const int oxl = x > 0 ? moff - 1 : rowbase + L - 1;  // periodic in x
                    const int oxr = x + V < L ? moff + V : rowbase;
                    long long g = (long long)(DESC ? z0 + nz - 1 : z0) * LL + (long long)(ya * L + q);

                    auto load = [&](T (&u)[V], T (&v)[V]) {
                        gs_unpack<T>(*reinterpret_cast<const VT*>(ring + cs * stage_elems + moff), u);
                        gs_unpack<T>(*reinterpret_cast<const VT*>(ring + cs * stage_elems + a.field_elems + moff), v);
                    };
                    int sc = 0;
                    // one plane: P, C, N are the previous, current and next
                    // planes of the march (N loaded here)
                    auto plane = [&](T (&pu)[V], T (&pv)[V], T (&cu)[V], T (&cv)[V], T (&nu)[V],
                                     T (&nv)[V]) -> bool {
                        const int sn = cs;
                        if (!wait_or_abort(&full[sn], cph, a.timeout_ns, &s_abort)) return false;
                        load(nu, nv);
                        const T shlu = __shfl_up_sync(0xffffffffu, cu[V - 1], 1);
                        const T shlv = __shfl_up_sync(0xffffffffu, cv[V - 1], 1);
                        const T shru = __shfl_down_sync(0xffffffffu, cu[0], 1);
                        const T shrv = __shfl_down_sync(0xffffffffu, cv[0], 1);
                        if (active) {
                            const T* bu = ring + sc * stage_elems;
                            const T* bv = bu + a.field_elems;
                            T ymu[V], ypu[V], ymv[V], ypv[V], ou[V], ov[V];
                            gs_unpack<T>(*reinterpret_cast<const VT*>(bu + om), ymu);
                            gs_unpack<T>(*reinterpret_cast<const VT*>(bu + op), ypu);
                            gs_unpack<T>(*reinterpret_cast<const VT*>(bv + om), ymv);
                            gs_unpack<T>(*reinterpret_cast<const VT*>(bv + op), ypv);
                            T xlu = shlu, xlv = shlv, xru = shru, xrv = shrv;
                            if (l_smem) { xlu = bu[oxl]; xlv = bv[oxl]; }
                            if (r_smem) { xru = bu[oxr]; xrv = bv[oxr]; }
                            const uint32_t pre = NOISE ? gs_group_pre((uint32_t)g, keys) : 0u;
                            if constexpr (DESC)
                                gs_update_group<T, NOISE>(c, pre, kk2, cu, cv, nu, nv, pu, pv, ymu, ypu, ymv, ypv,
                                                          xlu, xru, xlv, xrv, ou, ov);
                            else
                                gs_update_group<T, NOISE>(c, pre, kk2, cu, cv, pu, pv, nu, nv, ymu, ypu, ymv, ypv,
                                                          xlu, xru, xlv, xrv, ou, ov);
                            *reinterpret_cast<VT*>(un + g) = gs_pack<T>(ou);
                            *reinterpret_cast<VT*>(vn + g) = gs_pack<T>(ov);
                        }
                        __syncwarp();
                        if (lane == 0) gs_mbar_arrive(&empty[sc]);
                        sc = sn;
                        advance();
                        g += DESC ? -LL : LL;
                        return true;
                    };

                    load(qu[0], qv[0]);  // the first plane (waited for above)
                    __syncwarp();
                    if (lane == 0) gs_mbar_arrive(&empty[cs]);
                    advance();
                    sc = cs;
                    if (!wait_or_abort(&full[cs], cph, a.timeout_ns, &s_abort)) return false;
                    load(qu[1], qv[1]);
                    advance();
                    bool ok = true;
                    int zi = 0;
                    for (; ok && zi + 3 <= nz; zi += 3) {
                        ok = plane(qu[0], qv[0], qu[1], qv[1], qu[2], qv[2]) &&
                             plane(qu[1], qv[1], qu[2], qv[2], qu[0], qv[0]) &&
                             plane(qu[2], qv[2], qu[0], qv[0], qu[1], qv[1]);
                    }
                    // remainder (each item reloads its first two planes into q0, q1)
                    if (ok && zi < nz) ok = plane(qu[0], qv[0], qu[1], qv[1], qu[2], qv[2]);
                    if (ok && zi + 1 < nz) ok = plane(qu[1], qv[1], qu[2], qv[2], qu[0], qv[0]);
                    if (!ok) return false;
                    __syncwarp();
                    if (lane == 0) gs_mbar_arrive(&empty[sc]);
                    return true;
                };
                if (!(d.nz < 0 ? run(std::true_type{}) : run(std::false_type{}))) {
                    gs_report(&a.ctrl->err, GS_DERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
            }
            gs_fence_proxy_async_global();  // this step's stores before the next step's TMA reads
        } else if (tid == kBatchConsumers && a.fault != 1) {
            // ------------------------------ producer -------------------------------
            gs_fence_proxy_async_global();  // the previous step's stores (acquired at the barrier)
            // the step's tickets: nitems items and one failed draw per CTA, so
            // step s of the launch draws base .. base + nitems + grid - 1
            const unsigned base = (unsigned)((unsigned long long)s * (unsigned)(a.nitems + gridDim.x));
            int k = 0;
            auto draw = [&]() -> int {
                return a.dynamic ? (int)(atomicAdd(&a.ctrl->next, 1u) - base) : blockIdx.x + (k++) * gridDim.x;
            };
            int item = draw();  // the next ticket is drawn one item ahead (its latency hides behind the copies)
            for (;;) {
                if (item >= a.nitems || s_abort) {
                    // end of this CTA's items: the marker through one stage
                    const int sl = cs;
                    if (s_abort || (wrapped && !wait_or_abort(&empty[sl], cph ^ 1u, a.timeout_ns, &s_abort))) {
                        if (!s_abort) {
                            gs_report(&a.ctrl->err, GS_DERR_TIMEOUT);
                            s_abort = 1;
                        }
                        break;
                    }
                    s_desc[kl % kBatchDescs].nz = 0;
                    gs_mbar_arrive(&full[sl]);
                    ++kl;
                    ++seq;
                    advance();
                    break;
                }
                const int4 it = a.items[item];
                item = draw();
                const int ii = it.x;
                const BInst& I = a.inst[ii];
                const GsKeys keys = gs_step_keys(((uint64_t)I.seed_hi << 32) | I.seed_lo, t);
                const int L = I.L, ty = I.ty;
                const bool desc = it.w < 0;  // march down from the top plane
                const int c0 = it.y, z0 = it.z, nz = desc ? -it.w : it.w;
                const int C = min(kBatchConsumers * V, L * L - c0);
                const int y0 = c0 / L, y1 = (c0 + C - 1) / L;  // rows of the tile
                const int ytop = (y0 - 1 + L) % L, ybot = (y1 + 1) % L;
                const uint32_t bytes = 2u * (uint32_t)(L * ty + 2 * L) * (uint32_t)sizeof(T);
                const CUtensorMap* mu = a.maps + (((size_t)ii * 2 + in) * 2 + 0) * 2;
                const CUtensorMap* mv = a.maps + (((size_t)ii * 2 + in) * 2 + 1) * 2;
                bool failed = false;
                int zp = desc ? (z0 + nz) % L : (z0 - 1 + L) % L;
                for (int j = 0; j < nz + 2; ++j) {
                    const int sl = cs;
                    if (wrapped && !wait_or_abort(&empty[sl], cph ^ 1u, a.timeout_ns, &s_abort)) {
                        failed = true;
                        break;
                    }
                    if (j == 0) {
                        BDesc<T>& d = s_desc[kl % kBatchDescs];
                        d.un = a.arena + I.off[out][0];
                        d.vn = a.arena + I.off[out][1];
                        d.F = (T)I.F;
                        d.Fk = (T)I.Fk;
                        d.keys = keys;
                        d.kk2 = gs_kk2(keys);
                        d.L = L;
                        d.c0 = c0;
                        d.z0 = z0;
                        d.nz = it.w;
                    }
                    gs_mbar_arrive_expect_tx(&full[sl], bytes);
                    T* b = ring + sl * stage_elems;
                    gs_tma_load_3d(b, &mu[0], &full[sl], 0, y0, zp);
                    gs_tma_load_3d(b + top_off, &mu[1], &full[sl], 0, ytop, zp);
                    gs_tma_load_3d(b + bot_off, &mu[1], &full[sl], 0, ybot, zp);
                    b += a.field_elems;
                    gs_tma_load_3d(b, &mv[0], &full[sl], 0, y0, zp);
                    gs_tma_load_3d(b + top_off, &mv[1], &full[sl], 0, ytop, zp);
                    gs_tma_load_3d(b + bot_off, &mv[1], &full[sl], 0, ybot, zp);
                    ++seq;
                    advance();
                    if (desc)
                        zp = zp == 0 ? L - 1 : zp - 1;
                    else
                        zp = zp + 1 == L ? 0 : zp + 1;
                }
                ++kl;
                if (failed) {
                    gs_report(&a.ctrl->err, GS_DERR_TIMEOUT);
                    s_abort = 1;
                }
            }
        }
        const bool skip = a.fault == 2 && blockIdx.x == 0;
        if (!batch_grid_sync(a.ctrl, (unsigned)((unsigned long long)(s + 1) * gridDim.x), a.timeout_ns, skip,
                             &s_abort))
            break;
    }
    if (tid == kBatchConsumers && s_abort) {
        // a failure stopped the consumers: let every copy this thread issued
        // land before the CTA can leave (fixed budget; copies always complete)
        for (uint32_t q = (seq > (uint32_t)S ? seq - S : 0); q < seq; ++q)
            gs_mbar_wait(&full[q % S], (q / S) & 1, 2000000000ull);
    }
    if (blockIdx.x == 0 && tid == 0 && s == a.nsteps) {
        a.ctrl->t = t0 + a.nsteps;
        a.ctrl->cur = (cur0 + (int)(a.nsteps & 1)) & 1;
    }
}

// ---------------------------------------------------------------------------
// Temporally blocked batch (FP32, D = 2..4 steps per pass over HBM).
//
// The single-grid kernel's schedule (tb_item, gs_tblock.cuh) on the batch's
// full-row tiles: a work item is ty_i rows of instance i by a z-chunk, and
// its region is the whole row (the x wrap is an index wrap in shared memory,
// so no cell is recomputed in x) by ty_i + 2D rows (the y halo shrinks by
// one row per level).  ty_i is the largest divisor of L_i with
// (L_i / 4) (ty_i + 2D) groups fitting the 512 threads, one group of 4 cells
// per thread.  The CTAs take items from the ticket counter in table order
// (the last grid / 2 cut in four along z), and all meet at the grid barrier
// after each pass (D steps).
// ---------------------------------------------------------------------------
constexpr int kBtbThreads = 512;
constexpr int kBtbStages = kTbStages;  // level-0 ring (7 planes measured no faster)
constexpr int kBtbMaxDepth = 4;

// rows per tile of the blocked form for edge L and depth D (0: no tile fits)
static int btb_rows(int L, int D)
{
    const int G = L / 4;
    for (int ty = L; ty >= 1; --ty)
        if (L % ty == 0 && G * (ty + 2 * D) <= kBtbThreads) return ty;
    return 0;
}

// floats per field and plane of the blocked form's shared-memory planes
static int btb_plane_elems(const std::vector<int>& L, int D)
{
    int pe = 0;
    for (int l : L) pe = std::max(pe, (btb_rows(l, D) + 2 * D) * l);
    return (pe + 31) / 32 * 32;
}

static size_t btb_smem_bytes(int pe, int D) { return (size_t)(2 * kBtbStages + 6 * (D - 1)) * pe * sizeof(float); }

struct BtbArgs {
    float* arena;
    const BInst* inst;
    const int* rows;    // ty_i of the blocked form, per instance
    const int4* items;  // (instance, y0, z0, nz)
    BCtrl* ctrl;
    int nitems;
    int pe;             // floats per field and plane of the shared-memory planes
    long long npasses;
    float Du6, Dv6, dt, noise24;
    uint64_t timeout_ns;
    int fault;          // 2: CTA 0 never arrives at the grid barrier
};

template <bool NOISE, int D>
__global__ void __launch_bounds__(kBtbThreads, 1) gs_batch_tb_kernel(const __grid_constant__ BtbArgs a)
{
    constexpr int V = 4;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ volatile int s_abort;
    __shared__ int s_item[2];  // this CTA's current and next item (thread 0 draws one ahead)
    float* ring = reinterpret_cast<float*>(smem);
    const int PE = a.pe;
    float* lev = ring + (size_t)kBtbStages * 2 * PE;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) s_abort = 0;
    __syncthreads();
    const long long t0 = a.ctrl->t;
    const int cur0 = a.ctrl->cur;
    long long pass = 0;
    for (; pass < a.npasses; ++pass) {
        const int in = (cur0 + (int)(pass & 1)) & 1, out = in ^ 1;
        const long long tp = t0 + pass * D;
        // items from the ticket counter in table order, as in the single-step
        // kernel: every CTA draws one ticket past the pass's items, so pass p
        // draws p (nitems + grid) .. p (nitems + grid) + nitems + grid - 1; the
        // barrier that ends each item orders the hand-off of the next
        const unsigned base = (unsigned)((unsigned long long)pass * (unsigned)(a.nitems + gridDim.x));
        auto draw = [&]() -> int { return (int)(atomicAdd(&a.ctrl->next, 1u) - base); };
        if (tid == 0) s_item[0] = draw();
        __syncthreads();
        for (int n = 0;; ++n) {
            const int item = s_item[n & 1];
            if (item >= a.nitems) break;
            if (tid == 0) s_item[(n + 1) & 1] = draw();
            const int4 itm = a.items[item];
            const BInst& I = a.inst[itm.x];
            const int L = I.L, G = L / V, W = L;
            const int ty = a.rows[itm.x];
            const int H = ty + 2 * D;
            // this thread's place in the item's region: x periodic within the
            // row, y clamped inside the region
            TbThread<D> th;
            th.real = tid < G * H;
            const int gx = th.real ? tid % G : 0;
            const int row = th.real ? tid / G : 0;
            th.o = row * W + gx * V;
            th.oym = (row > 0 ? row - 1 : row) * W + gx * V;
            th.oyp = (row < H - 1 ? row + 1 : row) * W + gx * V;
            th.lsh = gx > 0 && lane > 0;
            th.rsh = gx < G - 1 && lane < 31;
            th.oxl = gx > 0 ? th.o - 1 : row * W + W - 1;
            th.oxr = gx < G - 1 ? th.o + V : row * W;
#pragma unroll
            for (int s = 1; s <= D; ++s) {
                th.act[s] = th.real && row >= s && row < H - s;
                th.wact[s] = __any_sync(0xffffffffu, th.act[s]);
            }
            th.store = th.real && row >= D && row < D + ty;
            GsCoef<float> c;
            c.Du6 = a.Du6; c.Dv6 = a.Dv6; c.dt = a.dt; c.noise24 = a.noise24;
            c.F = (float)I.F; c.Fk = (float)I.Fk;
            const uint64_t seed = ((uint64_t)I.seed_hi << 32) | I.seed_lo;
            GsKeys keys[D];
            uint32_t kk2[D];
#pragma unroll
            for (int s = 0; s < D; ++s) {
                keys[s] = gs_step_keys(seed, tp + s);
                kk2[s] = gs_kk2(keys[s]);
            }
            const int yg = (itm.y - D + row + L) % L;
            tb_item<NOISE, D, true>(a.arena + I.off[in][0], a.arena + I.off[in][1], a.arena + I.off[out][0],
                              a.arena + I.off[out][1], L, (uint32_t)yg * (uint32_t)L + (uint32_t)(gx * V), itm.z,
                              itm.w, c, keys, kk2, th, ring, lev, PE);
        }
        const bool skip = a.fault == 2 && blockIdx.x == 0;
        if (!batch_grid_sync(a.ctrl, (unsigned)((unsigned long long)(pass + 1) * gridDim.x), a.timeout_ns, skip,
                             &s_abort))
            break;
    }
    if (blockIdx.x == 0 && tid == 0 && pass == a.npasses) {
        a.ctrl->t = t0 + a.npasses * D;
        a.ctrl->cur = (cur0 + (int)(a.npasses & 1)) & 1;
    }
}

}  // namespace gs

using namespace gs;

struct gs_batch {
    int n = 0, dtype = GS_F32;
    double Du = 0, Dv = 0, dt = 0, noise = 0;
    uint64_t seed = 0;
    std::vector<int> L;
    std::vector<double> F, k;
    std::vector<BInst> h_inst;
    void* arena = nullptr;
    BInst* d_inst = nullptr;
    std::vector<int4> base_items;           // (instance, y0, z0, +-nz) before the tail split
    int4* d_items = nullptr;                // the table the kernel walks
    int items_cap = 0;                      // capacity of d_items
    int items_grid = -1;                    // grid the device table was cut for (-1: none yet)
    CUtensorMap* d_maps = nullptr;
    BCtrl* d_ctrl = nullptr;
    std::vector<ZPlan> zplan;               // per-instance plan of the sequential path
    std::vector<ZMaps> zmaps[2];            // per-instance tensor maps of the sequential path
    int nitems = 0, tz = 32, stages = 8, main_elems = 0, row_elems = 0, field_elems = 0;
    size_t arena_bytes = 0;
    int grid = 0;
    int64_t t = 0;
    int cur = 0;
    bool ctrl_dirty = true;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    std::map<int64_t, cudaGraphExec_t> graphs;
    int64_t launches = 0;
    uint64_t timeout_ns = 2000000000ull;
    int fault = 0;
    bool cooperative = true;
    // temporally blocked form (depth > 1, FP32): rows per tile per instance,
    // its own work-item table (cut for its own grid) and plane stride
    int depth = 1;
    int* d_tb_rows = nullptr;
    std::vector<int4> tb_base_items;
    int4* d_tb_items = nullptr;
    int tb_items_cap = 0, tb_nitems = 0, tb_items_grid = -1, tb_pe = 0, tb_grid = 0;
};

// The work item of z-chunk zc of a single-step table: (instance, c0, z0,
// +-nz), marching up the chunk for even zc and down it (nz stored negated)
// for odd zc.  Adjacent chunks then meet at their shared halo planes at the
// same time (both ends, or both starts, of items that run side by side), so
// the second read of those planes finds them in L2 instead of HBM.
static int4 march_item(int i, int y0, int z0, int nz, int zc)
{
    return make_int4(i, y0, z0, (zc & 1) ? -nz : nz);
}

// Tiles of the single-step kernel: runs of tile_cells = 256 V consecutive
// cells of a plane in row-major order (one group of V cells per consumer
// thread), so every tile but the last of a plane is full whatever L is.
// A tile is staged as the whole rows it touches; run_box_rows is the most
// rows any tile of an L^2 plane touches (the height of its TMA box).
static int run_tiles(int L, int tile_cells) { return (L * L + tile_cells - 1) / tile_cells; }
static int run_box_rows(int L, int tile_cells)
{
    int rows = 0;
    for (int c0 = 0; c0 < L * L; c0 += tile_cells) {
        const int C = std::min(tile_cells, L * L - c0);
        rows = std::max(rows, (c0 + C - 1) / L - c0 / L + 1);
    }
    return rows;
}

// the work items of instances [0, n) for the single-step kernel, instance by
// instance, tiles of a plane fastest: (instance, first cell, z0, +-nz)
static void plain_items(const BInst* inst, int n, int tz, int tile_cells, std::vector<int4>& out)
{
    out.clear();
    for (int i = 0; i < n; ++i) {
        const BInst& I = inst[i];
        for (int j = 0; j < I.nty * I.ntz; ++j) {
            const int c0 = (j % I.nty) * tile_cells, zc = j / I.nty, z0 = zc * tz;
            out.push_back(march_item(i, c0, z0, std::min(tz, I.L - z0), zc));
        }
    }
}

// For a launch whose CTAs take items from a ticket counter in table order:
// cut the last m items along z into up to f pieces each (with `alternate`,
// alternating their direction), so the last items taken are short and the
// CTAs finish a step within a fraction of an item of one another.  Every
// cell is still updated once.
static void split_last(const std::vector<int4>& base, int m, int f, bool alternate, std::vector<int4>& out)
{
    const int n = (int)base.size();
    m = std::min(std::max(m, 0), n);
    out.assign(base.begin(), base.end() - m);
    for (int q = n - m; q < n; ++q) {
        const int4 it = base[q];
        const bool desc = it.w < 0;
        const int nz = desc ? -it.w : it.w;
        const int parts = std::min(f, nz);
        for (int p = 0; p < parts; ++p) {
            const int za = nz * p / parts, zb = nz * (p + 1) / parts;
            const bool d = alternate ? desc != ((p & 1) != 0) : desc;
            out.push_back(make_int4(it.x, it.y, it.z + za, d ? za - zb : zb - za));
        }
    }
}

// upload `items` as the kernel's table (growing the device buffer if needed)
static int upload_items(gs_batch* b, const std::vector<int4>& items)
{
    if ((int)items.size() > b->items_cap) {
        int4* d = nullptr;
        GS_CUDA_TRY(guarded_malloc((void**)&d, sizeof(int4) * items.size()));
        guarded_free(b->d_items);
        b->d_items = d;
        b->items_cap = (int)items.size();
    }
    GS_CUDA_TRY(cudaMemcpy(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    b->nitems = (int)items.size();
    return GS_OK;
}

// upload the blocked form's work-item table (growing its device buffer if needed)
static int upload_tb_items(gs_batch* b, const std::vector<int4>& items)
{
    if ((int)items.size() > b->tb_items_cap) {
        int4* d = nullptr;
        GS_CUDA_TRY(guarded_malloc((void**)&d, sizeof(int4) * items.size()));
        guarded_free(b->d_tb_items);
        b->d_tb_items = d;
        b->tb_items_cap = (int)items.size();
    }
    GS_CUDA_TRY(cudaMemcpy(b->d_tb_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    b->tb_nitems = (int)items.size();
    return GS_OK;
}

// (Re)build the blocked form's tables for depth D and the current z-chunk:
// rows per tile per instance, base work items (instance by instance, y tiles
// fastest), plane stride.  GS_EINVAL when some instance has no tile that fits.
static int build_tb_tables(gs_batch* b, int D)
{
    std::vector<int> rows(b->n);
    for (int i = 0; i < b->n; ++i) {
        rows[i] = btb_rows(b->L[i], D);
        if (rows[i] < 1)
            return fail(GS_EINVAL, "depth %d: instance %d (L=%d) has no blocked tile within %d threads", D, i,
                        b->L[i], kBtbThreads);
    }
    b->tb_base_items.clear();
    for (int i = 0; i < b->n; ++i) {
        const int L = b->L[i], nty = L / rows[i], ntz = (L + b->tz - 1) / b->tz;
        for (int j = 0; j < nty * ntz; ++j) {
            const int y0 = (j % nty) * rows[i], z0 = (j / nty) * b->tz;
            b->tb_base_items.push_back(make_int4(i, y0, z0, std::min(b->tz, L - z0)));
        }
    }
    GS_CUDA_TRY(cudaStreamSynchronize(b->stream));  // no launch still reads the old tables
    if (!b->d_tb_rows) GS_CUDA_TRY(guarded_malloc((void**)&b->d_tb_rows, sizeof(int) * b->n));
    GS_CUDA_TRY(cudaMemcpy(b->d_tb_rows, rows.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice));
    const int rc = upload_tb_items(b, b->tb_base_items);
    if (rc) return rc;
    b->tb_pe = btb_plane_elems(b->L, D);
    b->tb_items_grid = -1;
    return GS_OK;
}

static int batch_upload_ctrl(gs_batch* b)
{
    BCtrl h{};
    h.t = b->t;
    h.cur = b->cur;
    h.bar = 0;
    h.err = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&b->d_ctrl->t, &h.t, sizeof(long long), cudaMemcpyHostToDevice, b->stream));
    GS_CUDA_TRY(cudaMemcpyAsync(&b->d_ctrl->cur, &h.cur, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->ctrl_dirty = false;
    return GS_OK;
}

static void drop_graphs(gs_batch* b)
{
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Arguments, grid and (for a new grid) the tail-split item table of the
// single-step kernel for an n-step run.  Runs before a capture begins.
template <typename T, bool NOISE>
static int plain_prepare(gs_batch* b, int64_t n, BArgs<T>& a, size_t& smem)
{
    a.arena = (T*)b->arena;
    a.inst = b->d_inst;
    a.maps = b->d_maps;
    a.ctrl = b->d_ctrl;
    a.tz = b->tz;
    a.stages = b->stages;
    a.main_elems = b->main_elems;
    a.row_elems = b->row_elems;
    a.field_elems = b->field_elems;
    a.nsteps = n;
    GsCoef<T> c = gs_make_coef<T>(b->Du, b->Dv, 0.0, 0.0, b->dt, b->noise);
    a.Du6 = c.Du6;
    a.Dv6 = c.Dv6;
    a.dt = c.dt;
    a.noise24 = c.noise24;
    a.timeout_ns = b->timeout_ns;
    a.fault = b->fault;
    a.dynamic = 1;
    smem = (size_t)2 * b->field_elems * sizeof(T) * b->stages;
    auto kern = gs_batch_kernel<T, NOISE>;
    GS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, smem));
    if (per_sm < 1) return fail(GS_EINVAL, "batch kernel does not fit on an SM");
    const int grid = std::min(per_sm * num_sms(), (int)b->base_items.size());
    if (b->items_grid != grid) {
        // cut the last items for this grid (once per plan)
        std::vector<int4> items;
        split_last(b->base_items, grid / 2, 4, true, items);
        GS_CUDA_TRY(cudaStreamSynchronize(b->stream));  // no launch still reads the old table
        const int rc = upload_items(b, items);
        if (rc) return rc;
        b->items_grid = grid;
        drop_graphs(b);  // graphs captured with the old table
    }
    b->grid = grid;
    a.items = b->d_items;
    a.nitems = b->nitems;
    return GS_OK;
}

// The same for the temporally blocked kernel (npasses passes of D steps).
template <bool NOISE, int D>
static int tb_prepare(gs_batch* b, int64_t npasses, BtbArgs& a, size_t& smem)
{
    a.arena = (float*)b->arena;
    a.inst = b->d_inst;
    a.rows = b->d_tb_rows;
    a.ctrl = b->d_ctrl;
    a.pe = b->tb_pe;
    a.npasses = npasses;
    GsCoef<float> c = gs_make_coef<float>(b->Du, b->Dv, 0.0, 0.0, b->dt, b->noise);
    a.Du6 = c.Du6;
    a.Dv6 = c.Dv6;
    a.dt = c.dt;
    a.noise24 = c.noise24;
    a.timeout_ns = b->timeout_ns;
    a.fault = b->fault;
    smem = btb_smem_bytes(b->tb_pe, D);
    auto kern = gs_batch_tb_kernel<NOISE, D>;
    GS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBtbThreads, smem));
    if (per_sm < 1) return fail(GS_EINVAL, "blocked batch kernel does not fit on an SM");
    const int grid = std::min(per_sm * num_sms(), (int)b->tb_base_items.size());
    if (b->tb_items_grid != grid) {
        std::vector<int4> items;
        split_last(b->tb_base_items, grid / 2, 4, false, items);  // the blocked item marches up only
        GS_CUDA_TRY(cudaStreamSynchronize(b->stream));
        const int rc = upload_tb_items(b, items);
        if (rc) return rc;
        b->tb_items_grid = grid;
        drop_graphs(b);
    }
    b->tb_grid = grid;
    a.items = b->d_tb_items;
    a.nitems = b->tb_nitems;
    return GS_OK;
}

// one persistent launch inside a capture: barrier and ticket counters reset + kernel
template <typename K, typename A>
static cudaError_t capture_persistent(gs_batch* b, K kern, const A& args, int grid, int threads, size_t smem)
{
    cudaError_t e = cudaMemsetAsync(&b->d_ctrl->bar, 0, 2 * sizeof(unsigned), b->cap);  // bar and next
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b->cap;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = b->cooperative ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args);
}

// An n-step run as one graph: n / D blocked passes (D > 1), then the
// remaining steps on the single-step kernel (which reads the step counter
// and buffer set the blocked kernel leaves in the control block).
template <typename T, bool NOISE, int D>
static int batch_capture_t(gs_batch* b, int64_t n, cudaGraphExec_t* exec)
{
    const int64_t npasses = D > 1 ? n / D : 0;
    const int64_t rem = n - npasses * D;
    BArgs<T> pa{};
    size_t psmem = 0;
    BtbArgs ta{};
    size_t tsmem = 0;
    if constexpr (D > 1) {
        if (npasses) {
            const int rc = tb_prepare<NOISE, D>(b, npasses, ta, tsmem);
            if (rc) return rc;
        }
    }
    if (rem) {
        const int rc = plain_prepare<T, NOISE>(b, rem, pa, psmem);
        if (rc) return rc;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        cudaGraph_t g = nullptr;
        GS_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e2 = cudaSuccess;
        if constexpr (D > 1) {
            if (npasses) e2 = capture_persistent(b, gs_batch_tb_kernel<NOISE, D>, ta, b->tb_grid, kBtbThreads, tsmem);
        }
        if (e2 == cudaSuccess && rem)
            e2 = capture_persistent(b, gs_batch_kernel<T, NOISE>, pa, b->grid, kBatchThreads, psmem);
        cudaError_t e3 = cudaStreamEndCapture(b->cap, &g);
        cudaError_t e4 = cudaErrorUnknown;
        if (e2 == cudaSuccess && e3 == cudaSuccess) e4 = cudaGraphInstantiate(exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e2 == cudaSuccess && e3 == cudaSuccess && e4 == cudaSuccess) return GS_OK;
        cudaGetLastError();
        if (!b->cooperative) {
            cudaError_t e = e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4);
            return cuda_fail(e, "capturing the batched persistent launch");
        }
        b->cooperative = false;  // retry without the cooperative attribute (grids are sized to be co-resident)
    }
    return fail(GS_ECUDA, "capturing the batched persistent launch failed");
}

static int batch_capture(gs_batch* b, int64_t n, cudaGraphExec_t* exec)
{
    const bool noise = b->noise != 0.0;
    if (b->dtype != GS_F32)
        return noise ? batch_capture_t<double, true, 1>(b, n, exec) : batch_capture_t<double, false, 1>(b, n, exec);
    switch (b->depth) {
    case 2: return noise ? batch_capture_t<float, true, 2>(b, n, exec) : batch_capture_t<float, false, 2>(b, n, exec);
    case 3: return noise ? batch_capture_t<float, true, 3>(b, n, exec) : batch_capture_t<float, false, 3>(b, n, exec);
    case 4: return noise ? batch_capture_t<float, true, 4>(b, n, exec) : batch_capture_t<float, false, 4>(b, n, exec);
    default: return noise ? batch_capture_t<float, true, 1>(b, n, exec) : batch_capture_t<float, false, 1>(b, n, exec);
    }
}

// buffer flips of an n-step run: one per blocked pass, one per single step
static int batch_flips(const gs_batch* b, int64_t n)
{
    const int64_t passes = b->depth > 1 ? n / b->depth : 0;
    return (int)((passes + (n - passes * b->depth)) & 1);
}

static int batch_check_inst(gs_batch* b, int i, int field)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (i < 0 || i >= b->n) return fail(GS_EINVAL, "instance %d out of range [0, %d)", i, b->n);
    if (field != GS_U && field != GS_V) return fail(GS_EINVAL, "field=%d must be GS_U or GS_V", field);
    return GS_OK;
}

extern "C" {

int gs_batch_destroy(gs_batch* b)
{
    if (!b) return GS_OK;
    drop_graphs(b);
    guarded_free(b->arena);
    guarded_free(b->d_inst);
    guarded_free(b->d_items);
    guarded_free(b->d_maps);
    guarded_free(b->d_ctrl);
    guarded_free(b->d_tb_rows);
    guarded_free(b->d_tb_items);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return GS_OK;
}

int gs_batch_create(int n, const int* L, const double* F, const double* k, double Du, double Dv, double dt,
                    double noise, uint64_t seed, int dtype, gs_batch** out)
{
    if (!out) return fail(GS_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (n < 1) return fail(GS_EINVAL, "n=%d must be >= 1", n);
    if (!L || !F || !k) return fail(GS_EINVAL, "L, F, k must not be NULL");
    if (dtype != GS_F32 && dtype != GS_F64) return fail(GS_EINVAL, "dtype=%d must be GS_F32 or GS_F64", dtype);
    const int V = dtype == GS_F32 ? 4 : 2;
    const int esz = dtype == GS_F32 ? 4 : 8;
    int maxL = 0;
    for (int i = 0; i < n; ++i) {
        if (L[i] < V || L[i] > 256 || L[i] % V)
            return fail(GS_EINVAL, "instance %d: L=%d must be a multiple of %d in [%d, 256]", i, L[i], V, V);
        if (!std::isfinite(F[i]) || !std::isfinite(k[i])) return fail(GS_EINVAL, "instance %d: F, k must be finite", i);
        maxL = std::max(maxL, L[i]);
    }
    if (!std::isfinite(Du) || !std::isfinite(Dv) || !std::isfinite(dt) || !std::isfinite(noise))
        return fail(GS_EINVAL, "parameters must be finite");
    gs_batch* b = new (std::nothrow) gs_batch();
    if (!b) return fail(GS_ENOMEM, "host allocation failed");
    b->n = n;
    b->dtype = dtype;
    b->Du = Du;
    b->Dv = Dv;
    b->dt = dt;
    b->noise = noise;
    b->seed = seed;
    b->L.assign(L, L + n);
    b->F.assign(F, F + n);
    b->k.assign(k, k + n);
    // shared-memory layout per stage and field: the tile box (the largest
    // box of any instance, whole rows) then two halo rows, each 128-byte aligned
    const int a128 = 128 / esz;
    const int tile_cells = kBatchConsumers * V;
    int box_elems = 0;
    // instance table, arena offsets, work items
    int nit = 0;
    long long off = 0;
    const long long align = 256 / esz;
    for (int i = 0; i < n; ++i) {
        BInst I{};
        I.L = L[i];
        I.ty = run_box_rows(L[i], tile_cells);
        I.nty = run_tiles(L[i], tile_cells);
        box_elems = std::max(box_elems, I.ty * L[i]);
        I.ntz = (L[i] + b->tz - 1) / b->tz;
        I.item0 = nit;
        I.nitems = I.nty * I.ntz;
        nit += I.nitems;
        const uint64_t si = seed + (uint64_t)i;
        I.seed_lo = (uint32_t)si;
        I.seed_hi = (uint32_t)(si >> 32);
        I.F = F[i];
        I.Fk = F[i] + k[i];
        const long long cells = (long long)L[i] * L[i] * L[i];
        for (int s = 0; s < 2; ++s)
            for (int f = 0; f < 2; ++f) {
                I.off[s][f] = off;
                off += (cells + align - 1) / align * align;
            }
        b->h_inst.push_back(I);
    }
    b->main_elems = (box_elems + a128 - 1) / a128 * a128;
    b->row_elems = (maxL + a128 - 1) / a128 * a128;
    b->field_elems = b->main_elems + 2 * b->row_elems;
    plain_items(b->h_inst.data(), n, b->tz, tile_cells, b->base_items);
    b->nitems = (int)b->base_items.size();
    int rc = GS_OK;
    cudaError_t e;
    b->arena_bytes = (size_t)off * esz;
    if ((e = guarded_malloc((void**)&b->arena, (size_t)off * esz)) != cudaSuccess ||
        (e = guarded_malloc((void**)&b->d_inst, sizeof(BInst) * n)) != cudaSuccess ||
        (e = guarded_malloc((void**)&b->d_maps, sizeof(CUtensorMap) * (size_t)n * 8)) != cudaSuccess ||
        (e = guarded_malloc((void**)&b->d_ctrl, sizeof(BCtrl))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        rc = cuda_fail(e, "allocating the batch");
        gs_batch_destroy(b);
        return rc;
    }
    // tensor maps: persistent kernel (boxes of the rows a tile touches) and the sequential baseline (z-march plans)
    std::vector<CUtensorMap> maps((size_t)n * 8);
    b->zplan.resize(n);
    b->zmaps[0].resize(n);
    b->zmaps[1].resize(n);
    for (int i = 0; i < n && rc == GS_OK; ++i) {
        const BInst& I = b->h_inst[i];
        for (int s = 0; s < 2 && rc == GS_OK; ++s)
            for (int f = 0; f < 2 && rc == GS_OK; ++f) {
                void* base = (char*)b->arena + (size_t)I.off[s][f] * esz;
                CUtensorMap* m = &maps[((size_t)i * 2 + s) * 2 * 2 + f * 2];
                if (encode_tiled_3d(&m[0], dtype, base, I.L, I.L, I.ty) != CUDA_SUCCESS ||
                    encode_tiled_3d(&m[1], dtype, base, I.L, I.L, 1) != CUDA_SUCCESS)
                    rc = fail(GS_ECUDA, "cuTensorMapEncodeTiled failed for instance %d (L=%d)", i, I.L);
            }
        ZPlan pl;
        pl.tx = std::min(dtype == GS_F32 ? 128 : 64, I.L);
        pl.ty = std::min(8, I.L);
        pl.tz = std::min(32, I.L);
        pl.stages = 4;
        pl.depth = 1;
        if (rc == GS_OK) rc = zmarch_validate(dtype, I.L, pl);
        b->zplan[i] = pl;
        for (int s = 0; s < 2 && rc == GS_OK; ++s)
            rc = zmarch_encode(dtype, I.L, pl, (char*)b->arena + (size_t)I.off[s][0] * esz,
                               (char*)b->arena + (size_t)I.off[s][1] * esz, &b->zmaps[s][i]);
    }
    if (rc == GS_OK) {
        if ((e = cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMemset(b->d_ctrl, 0, sizeof(BCtrl))) != cudaSuccess)
            rc = cuda_fail(e, "uploading the batch tables");
    }
    if (rc == GS_OK) rc = upload_items(b, b->base_items);
    if (rc == GS_OK) rc = gs_batch_init(b);
    if (rc != GS_OK) {
        gs_batch_destroy(b);
        return rc;
    }
    *out = b;
    return GS_OK;
}

int gs_batch_set_stream(gs_batch* b, void* stream)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    // the work already issued finishes first: the next launch must not
    // overlap it (they share the arena and the control block)
    if ((cudaStream_t)stream != b->stream) GS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->stream = (cudaStream_t)stream;
    return GS_OK;
}

int gs_batch_init(gs_batch* b)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    const int esz = elem_size(b->dtype);
    for (int i = 0; i < b->n; ++i) {
        const BInst& I = b->h_inst[i];
        int rc = launch_init(b->dtype, I.L, (char*)b->arena + (size_t)I.off[0][0] * esz,
                             (char*)b->arena + (size_t)I.off[0][1] * esz, b->stream);
        if (rc) return rc;
        b->launches += 1;
    }
    b->t = 0;
    b->cur = 0;
    GS_CUDA_TRY(cudaMemsetAsync(&b->d_ctrl->err, 0, sizeof(int), b->stream));
    return batch_upload_ctrl(b);
}

int gs_batch_step(gs_batch* b, int64_t n)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (n < 0) return fail(GS_EINVAL, "n must be >= 0");
    if (n == 0) return GS_OK;
    if (b->ctrl_dirty) {
        int rc = batch_upload_ctrl(b);
        if (rc) return rc;
    }
    auto it = b->graphs.find(n);
    cudaGraphExec_t exec = nullptr;
    if (it == b->graphs.end()) {
        int rc = batch_capture(b, n, &exec);
        if (rc) return rc;
        b->graphs[n] = exec;
    } else {
        exec = it->second;
    }
    GS_CUDA_TRY(cudaGraphLaunch(exec, b->stream));
    b->launches += 1;
    b->t += n;
    b->cur = (b->cur + batch_flips(b, n)) & 1;
    return GS_OK;
}

int gs_batch_step_sequential(gs_batch* b, int64_t n)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (n < 0) return fail(GS_EINVAL, "n must be >= 0");
    const int esz = elem_size(b->dtype);
    for (int64_t s = 0; s < n; ++s) {
        const int in = b->cur, out = 1 - b->cur;
        for (int i = 0; i < b->n; ++i) {
            const BInst& I = b->h_inst[i];
            Params p{b->Du, b->Dv, b->F[i], b->k[i], b->dt, b->noise, b->seed + (uint64_t)i};
            int rc = launch_zmarch(b->dtype, I.L, b->zplan[i], b->zmaps[in][i],
                                   (char*)b->arena + (size_t)I.off[out][0] * esz,
                                   (char*)b->arena + (size_t)I.off[out][1] * esz, p, b->t, &b->d_ctrl->err,
                                   b->timeout_ns, 0, nullptr, b->stream);
            if (rc) return rc;
            b->launches += 1;
        }
        b->cur = out;
        b->t += 1;
    }
    b->ctrl_dirty = true;
    return GS_OK;
}

int gs_batch_autotune(gs_batch* b, int steps_per_trial, int* best_tile_z, int* best_stages, double* best_us,
                      int* best_depth)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (steps_per_trial < 1) return fail(GS_EINVAL, "steps_per_trial must be >= 1");
    // whole passes at every depth: the trial length is a multiple of 12
    const int trial = (steps_per_trial + 11) / 12 * 12;
    const int tz0 = b->tz, st0 = b->stages, d0 = b->depth;
    const int64_t t0 = b->t;
    const int cur0 = b->cur;
    void* saved = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    int rc = GS_OK;
    if ((e = cudaMalloc(&saved, b->arena_bytes)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
        (e = cudaEventCreate(&e1)) != cudaSuccess)
        rc = cuda_fail(e, "batch autotune set-up");
    if (!rc && (e = cudaMemcpyAsync(saved, b->arena, b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream)) != cudaSuccess)
        rc = cuda_fail(e, "batch autotune save");
    int win_tz = tz0, win_st = st0, win_d = d0;
    double win_us = -1.0;
    for (int depth = 1; depth <= kBtbMaxDepth && !rc; ++depth) {
        if (depth > 1 && b->dtype != GS_F32) break;
        for (int tz : {16, 32, 64, 128}) {
            for (int st : {4, 6, 8}) {
                if (rc) break;
                if (depth == 1 && tz > 64) continue;  // one step per pass: longer chunks only lengthen the tail
                if (depth > 1 && st != 4) continue;   // the blocked form has no TMA ring
                if (gs_batch_set_plan(b, tz, st) != GS_OK) continue;  // a ring that does not fit
                if (gs_batch_set_depth(b, depth) != GS_OK) continue;  // no blocked tile for some instance
                int r = gs_batch_step(b, trial);                      // captures the graph, warms up
                if (!r) r = gs_batch_sync(b);
                if (!r && (e = cudaEventRecord(e0, b->stream)) != cudaSuccess) r = cuda_fail(e, "event");
                if (!r) r = gs_batch_step(b, trial);
                if (!r && (e = cudaEventRecord(e1, b->stream)) != cudaSuccess) r = cuda_fail(e, "event");
                if (!r) r = gs_batch_sync(b);
                float ms = 0.f;
                if (!r && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) r = cuda_fail(e, "event");
                if (r) {
                    rc = r;
                    break;
                }
                const double us = 1e3 * ms / trial;
                if (win_us < 0 || us < win_us) {
                    win_us = us;
                    win_tz = tz;
                    win_st = depth > 1 ? st0 : st;
                    win_d = depth;
                }
            }
        }
    }
    // restore the state, keep the winner (the previous plan on failure)
    if (saved) {
        cudaMemcpyAsync(b->arena, saved, b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream);
        cudaStreamSynchronize(b->stream);
        cudaFree(saved);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->t = t0;
    b->cur = cur0;
    b->ctrl_dirty = true;
    int rc2 = rc ? gs_batch_set_plan(b, tz0, st0) : gs_batch_set_plan(b, win_tz, win_st);
    if (!rc2) rc2 = gs_batch_set_depth(b, rc ? d0 : win_d);
    if (rc) return rc;
    if (rc2) return rc2;
    if (best_tile_z) *best_tile_z = win_tz;
    if (best_stages) *best_stages = win_st;
    if (best_us) *best_us = win_us;
    if (best_depth) *best_depth = win_d;
    return GS_OK;
}

int gs_batch_sync(gs_batch* b)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    int err = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&err, &b->d_ctrl->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (err == GS_DERR_TIMEOUT) return fail(GS_ETIMEOUT, "a device-side wait timed out");
    if (err) return fail(GS_ECUDA, "device error code %d", err);
    return GS_OK;
}

int gs_batch_read(gs_batch* b, int i, int field, void* dst, size_t bytes)
{
    int rc = batch_check_inst(b, i, field);
    if (rc) return rc;
    const BInst& I = b->h_inst[i];
    const size_t need = (size_t)I.L * I.L * I.L * elem_size(b->dtype);
    if (bytes != need) return fail(GS_EINVAL, "bytes=%zu, instance %d field holds %zu", bytes, i, need);
    if (!dst) return fail(GS_EINVAL, "dst is NULL");
    GS_CUDA_TRY(cudaMemcpyAsync(dst, (char*)b->arena + (size_t)I.off[b->cur][field] * elem_size(b->dtype), bytes,
                                cudaMemcpyDeviceToHost, b->stream));
    return gs_batch_sync(b);
}

int gs_batch_write(gs_batch* b, int i, int field, const void* src, size_t bytes)
{
    int rc = batch_check_inst(b, i, field);
    if (rc) return rc;
    const BInst& I = b->h_inst[i];
    const size_t need = (size_t)I.L * I.L * I.L * elem_size(b->dtype);
    if (bytes != need) return fail(GS_EINVAL, "bytes=%zu, instance %d field holds %zu", bytes, i, need);
    if (!src) return fail(GS_EINVAL, "src is NULL");
    GS_CUDA_TRY(cudaMemcpyAsync((char*)b->arena + (size_t)I.off[b->cur][field] * elem_size(b->dtype), src, bytes,
                                cudaMemcpyHostToDevice, b->stream));
    return gs_batch_sync(b);
}

int gs_batch_get_step(gs_batch* b, int64_t* t)
{
    if (!b || !t) return fail(GS_EINVAL, "NULL argument");
    *t = b->t;
    return GS_OK;
}

int gs_batch_set_step(gs_batch* b, int64_t t)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (t < 0) return fail(GS_EINVAL, "t must be >= 0");
    b->t = t;
    b->ctrl_dirty = true;
    return GS_OK;
}

int gs_batch_set_fault(gs_batch* b, int mode, uint64_t timeout_ns)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (mode < 0 || mode > 2) return fail(GS_EINVAL, "fault mode %d must be 0, 1 or 2", mode);
    if (timeout_ns == 0) return fail(GS_EINVAL, "timeout_ns must be > 0");
    if (mode != b->fault || timeout_ns != b->timeout_ns) drop_graphs(b);
    b->fault = mode;
    b->timeout_ns = timeout_ns;
    if (mode == 0) {
        // clear a recorded failure so the batch can be used again
        GS_CUDA_TRY(cudaMemsetAsync(&b->d_ctrl->err, 0, sizeof(int), b->stream));
    }
    return GS_OK;
}

int gs_batch_set_plan(gs_batch* b, int tile_z, int stages)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (tile_z < 1 || tile_z > 256) return fail(GS_EINVAL, "tile_z=%d must be in [1, 256]", tile_z);
    if (stages < 3 || stages > 8) return fail(GS_EINVAL, "stages=%d must be in [3, 8]", stages);
    const size_t esz = elem_size(b->dtype);
    if ((size_t)2 * b->field_elems * esz * stages > 200 * 1024) return fail(GS_EINVAL, "ring too large");
    // rebuild the work-item tables for the new z-chunk (the tail is cut again
    // at the next capture, when the grid is known)
    int nit = 0;
    for (int i = 0; i < b->n; ++i) {
        BInst& I = b->h_inst[i];
        I.ntz = (I.L + tile_z - 1) / tile_z;
        I.item0 = nit;
        I.nitems = I.nty * I.ntz;
        nit += I.nitems;
    }
    plain_items(b->h_inst.data(), b->n, tile_z, kBatchConsumers * (b->dtype == GS_F32 ? 4 : 2), b->base_items);
    GS_CUDA_TRY(cudaStreamSynchronize(b->stream));  // no launch still reads the old table
    {
        const int rc = upload_items(b, b->base_items);
        if (rc) return rc;
    }
    b->items_grid = -1;
    GS_CUDA_TRY(cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(BInst) * b->n, cudaMemcpyHostToDevice));
    b->tz = tile_z;
    b->stages = stages;
    drop_graphs(b);
    if (b->depth > 1) return build_tb_tables(b, b->depth);  // the blocked items follow the z-chunk
    return GS_OK;
}

int gs_batch_set_depth(gs_batch* b, int depth)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (depth < 1 || depth > kBtbMaxDepth) return fail(GS_EINVAL, "depth=%d must be in [1, %d]", depth, kBtbMaxDepth);
    if (depth > 1 && b->dtype != GS_F32) return fail(GS_EINVAL, "the temporally blocked batch is FP32 only");
    if (depth > 1) {
        const int rc = build_tb_tables(b, depth);
        if (rc) return rc;
    }
    b->depth = depth;
    drop_graphs(b);
    return GS_OK;
}

int gs_batch_guard_check(gs_batch* b, int64_t* bad)
{
    if (!b || !bad) return fail(GS_EINVAL, "NULL argument");
    GS_CUDA_TRY(cudaStreamSynchronize(b->stream));
    int64_t n = 0;
    for (const void* p : {(const void*)b->arena, (const void*)b->d_inst, (const void*)b->d_items, (const void*)b->d_maps,
                          (const void*)b->d_ctrl, (const void*)b->d_tb_rows, (const void*)b->d_tb_items}) {
        const int64_t r = guarded_check(p);
        if (r < 0) return fail(GS_ECUDA, "reading a guard band failed");
        n += r;
    }
    *bad = n;
    return GS_OK;
}

int gs_batch_info(gs_batch* b, int* grid, int* items, int* cooperative, int64_t* launches, int* depth)
{
    if (!b) return fail(GS_EINVAL, "batch is NULL");
    if (depth) *depth = b->depth;
    if (grid) *grid = b->depth > 1 ? b->tb_grid : b->grid;
    if (items) *items = b->depth > 1 ? b->tb_nitems : b->nitems;
    if (cooperative) *cooperative = b->cooperative ? 1 : 0;
    if (launches) *launches = b->launches;
    return GS_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free batched step.
//
// Everything gs_batch_create would allocate besides the fields (control
// block, instance table, work-item table, TMA descriptors) lives instead in
// one file-scope device array of fixed size, which the driver reserves on
// every GPU that loads this library for as long as the process runs.  The
// caller supplies the field arena and the step state; nothing is allocated
// per call.
// ===========================================================================
namespace gs {

constexpr int kNoAllocMaxInst = 256;
constexpr int kNoAllocMaxItems = 8192;
constexpr size_t kNaCtrlOff = 0;
constexpr size_t kNaInstOff = 256;
constexpr size_t kNaItemOff = kNaInstOff + (kNoAllocMaxInst * sizeof(BInst) + 255) / 256 * 256;
constexpr size_t kNaMapOff = kNaItemOff + (kNoAllocMaxItems * sizeof(int4) + 255) / 256 * 256;
constexpr size_t kNaBytes = kNaMapOff + (size_t)kNoAllocMaxInst * 8 * sizeof(CUtensorMap);
constexpr int kNaMaxDevices = 64;
// 256 B control block + 20,480 B instance table + 131,072 B work items +
// 262,144 B TMA descriptors (quoted in the public header)
static_assert(sizeof(BInst) == 80 && sizeof(CUtensorMap) == 128, "scratch layout");
static_assert(kNaBytes == 413952, "allocation-free scratch size");

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: the device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

static std::mutex g_na_mutex;
static void* g_na_addr[kNaMaxDevices] = {};
static BInst g_na_inst[kNoAllocMaxInst];
static int4 g_na_items[kNoAllocMaxItems];
static CUtensorMap g_na_maps[(size_t)kNoAllocMaxInst * 8];

template <typename T, bool NOISE>
static int noalloc_launch_t(char* scratch, void* arena, int n, int nitems, int main_elems, int row_elems,
                            double Du, double Dv, double dt, double noise, int64_t nsteps, cudaStream_t s)
{
    BArgs<T> a;
    a.arena = (T*)arena;
    a.inst = (const BInst*)(scratch + kNaInstOff);
    a.items = (const int4*)(scratch + kNaItemOff);
    a.maps = (const CUtensorMap*)(scratch + kNaMapOff);
    a.ctrl = (BCtrl*)(scratch + kNaCtrlOff);
    a.nitems = nitems;
    a.tz = 32;
    a.stages = 4;
    a.main_elems = main_elems;
    a.row_elems = row_elems;
    a.field_elems = main_elems + 2 * row_elems;
    a.nsteps = nsteps;
    GsCoef<T> c = gs_make_coef<T>(Du, Dv, 0.0, 0.0, dt, noise);
    a.Du6 = c.Du6;
    a.Dv6 = c.Dv6;
    a.dt = c.dt;
    a.noise24 = c.noise24;
    a.timeout_ns = 2000000000ull;
    a.fault = 0;
    a.dynamic = 0;
    (void)n;
    const size_t smem = (size_t)2 * a.field_elems * sizeof(T) * a.stages;
    auto kern = gs_batch_kernel<T, NOISE>;
    GS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, smem));
    if (per_sm < 1) return fail(GS_EINVAL, "batch kernel does not fit on an SM");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(per_sm * num_sms(), nitems));
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, a) != cudaSuccess) {
        cudaGetLastError();
        cfg.numAttrs = 0;  // the grid is sized to be co-resident; the barrier waits are bounded
        GS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
    }
    return GS_OK;
}

}  // namespace gs

extern "C" int gs_batch_step_noalloc(int n, const int* L, const double* F, const double* k, double Du,
                                     double Dv, double dt, double noise, uint64_t seed, int dtype, void* arena,
                                     int64_t t, int cur, int64_t nsteps, void* stream)
{
    if (n < 1 || n > kNoAllocMaxInst)
        return fail(GS_EINVAL, "n=%d instances: the allocation-free step takes 1 to %d", n, kNoAllocMaxInst);
    if (!L || !F || !k) return fail(GS_EINVAL, "L, F, k must not be NULL");
    if (dtype != GS_F32 && dtype != GS_F64) return fail(GS_EINVAL, "dtype=%d must be GS_F32 or GS_F64", dtype);
    if (!arena || reinterpret_cast<uintptr_t>(arena) % 256) return fail(GS_EINVAL, "arena must be a 256-byte aligned device pointer");
    if (t < 0 || (cur != 0 && cur != 1) || nsteps < 0) return fail(GS_EINVAL, "need t >= 0, cur in {0, 1}, nsteps >= 0");
    if (!std::isfinite(Du) || !std::isfinite(Dv) || !std::isfinite(dt) || !std::isfinite(noise))
        return fail(GS_EINVAL, "parameters must be finite");
    const int V = dtype == GS_F32 ? 4 : 2;
    const int esz = dtype == GS_F32 ? 4 : 8;
    int maxL = 0;
    long long items = 0;
    for (int i = 0; i < n; ++i) {
        if (L[i] < V || L[i] > 256 || L[i] % V)
            return fail(GS_EINVAL, "instance %d: L=%d must be a multiple of %d in [%d, 256]", i, L[i], V, V);
        if (!std::isfinite(F[i]) || !std::isfinite(k[i])) return fail(GS_EINVAL, "instance %d: F, k must be finite", i);
        maxL = std::max(maxL, L[i]);
        items += (long long)run_tiles(L[i], kBatchConsumers * V) * ((L[i] + 31) / 32);
    }
    if (items > kNoAllocMaxItems)
        return fail(GS_EINVAL, "%lld work items: the allocation-free step takes at most %d", items, kNoAllocMaxItems);
    if (nsteps == 0) return GS_OK;

    std::lock_guard<std::mutex> lock(g_na_mutex);
    int dev = 0;
    GS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return fail(GS_EINVAL, "device %d beyond the supported %d", dev, kNaMaxDevices);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(allocation-free scratch)");
        g_na_addr[dev] = p;
    }
    char* scratch = (char*)g_na_addr[dev];

    // same tables as gs_batch_create, built in static host staging
    const int a128 = 128 / esz;
    const int tile_cells = kBatchConsumers * V;
    int box_elems = 0;
    for (int i = 0; i < n; ++i) box_elems = std::max(box_elems, run_box_rows(L[i], tile_cells) * L[i]);
    const int main_elems = (box_elems + a128 - 1) / a128 * a128;
    const int row_elems = (maxL + a128 - 1) / a128 * a128;
    const long long align = 256 / esz;
    long long off = 0;
    int nit = 0;
    for (int i = 0; i < n; ++i) {
        BInst I{};
        I.L = L[i];
        I.ty = run_box_rows(L[i], tile_cells);
        I.nty = run_tiles(L[i], tile_cells);
        I.ntz = (L[i] + 31) / 32;
        I.item0 = nit;
        I.nitems = I.nty * I.ntz;
        const uint64_t si = seed + (uint64_t)i;
        I.seed_lo = (uint32_t)si;
        I.seed_hi = (uint32_t)(si >> 32);
        I.F = F[i];
        I.Fk = F[i] + k[i];
        const long long cells = (long long)L[i] * L[i] * L[i];
        for (int s = 0; s < 2; ++s)
            for (int f = 0; f < 2; ++f) {
                I.off[s][f] = off;
                off += (cells + align - 1) / align * align;
            }
        for (int j = 0; j < I.nitems; ++j) {
            const int c0 = (j % I.nty) * tile_cells, zc = j / I.nty, z0 = zc * 32;
            g_na_items[nit++] = march_item(i, c0, z0, std::min(32, I.L - z0), zc);
        }
        g_na_inst[i] = I;
        for (int s = 0; s < 2; ++s)
            for (int f = 0; f < 2; ++f) {
                void* base = (char*)arena + (size_t)I.off[s][f] * esz;
                CUtensorMap* m = &g_na_maps[((size_t)i * 2 + s) * 2 * 2 + f * 2];
                if (encode_tiled_3d(&m[0], dtype, base, I.L, I.L, I.ty) != CUDA_SUCCESS ||
                    encode_tiled_3d(&m[1], dtype, base, I.L, I.L, 1) != CUDA_SUCCESS)
                    return fail(GS_ECUDA, "cuTensorMapEncodeTiled failed for instance %d (L=%d)", i, I.L);
            }
    }
    BCtrl h{};
    h.t = t;
    h.cur = cur;
    cudaStream_t s = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemcpyAsync(scratch + kNaCtrlOff, &h, sizeof(BCtrl), cudaMemcpyHostToDevice, s));
    GS_CUDA_TRY(cudaMemcpyAsync(scratch + kNaInstOff, g_na_inst, sizeof(BInst) * n, cudaMemcpyHostToDevice, s));
    GS_CUDA_TRY(cudaMemcpyAsync(scratch + kNaItemOff, g_na_items, sizeof(int4) * nit, cudaMemcpyHostToDevice, s));
    GS_CUDA_TRY(cudaMemcpyAsync(scratch + kNaMapOff, g_na_maps, sizeof(CUtensorMap) * (size_t)n * 8,
                                cudaMemcpyHostToDevice, s));
    const bool nz = noise != 0.0;
    int rc;
    if (dtype == GS_F32)
        rc = nz ? noalloc_launch_t<float, true>(scratch, arena, n, nit, main_elems, row_elems, Du, Dv, dt, noise, nsteps, s)
                : noalloc_launch_t<float, false>(scratch, arena, n, nit, main_elems, row_elems, Du, Dv, dt, noise, nsteps, s);
    else
        rc = nz ? noalloc_launch_t<double, true>(scratch, arena, n, nit, main_elems, row_elems, Du, Dv, dt, noise, nsteps, s)
                : noalloc_launch_t<double, false>(scratch, arena, n, nit, main_elems, row_elems, Du, Dv, dt, noise, nsteps, s);
    if (rc) return rc;
    int err = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&err, scratch + kNaCtrlOff + offsetof(BCtrl, err), sizeof(int),
                                cudaMemcpyDeviceToHost, s));
    GS_CUDA_TRY(cudaStreamSynchronize(s));
    if (err == GS_DERR_TIMEOUT) return fail(GS_ETIMEOUT, "a device-side wait timed out");
    if (err) return fail(GS_ECUDA, "device error code %d", err);
    return GS_OK;
}
