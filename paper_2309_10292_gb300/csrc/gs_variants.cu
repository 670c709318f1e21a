// Variants of the paper's own kernel, for its bandwidth study (Listing 2;
// Section 5.1, Tables 2-3):
//
//  * held outer layer: the paper's kernel returns early for cells on the
//    first or last layer of any axis (ghost faces filled by MPI on the full
//    domain).  On one grid those cells keep their values.  The stencil
//    kernels compute every cell; after each step gs_hold_faces_kernel copies
//    the six faces of the input state over the output, which leaves interior
//    cells exact (they read only the input state and never wrap);
//
//  * one field without noise ("1-variable no random"):
//      f' = f + dt (D lap f),  lap f = (s - 6 f) / 6  (Eq. 3),
//    periodic or held, with its own single-field z-marching kernel (TMA
//    producer warp, register z-queue, x neighbours by warp shuffle).
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {

// ---------------------------------------------------------------------------
// Held outer layer: copy the six faces of (iu, iv) into (ou, ov)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void gs_hold_faces_kernel(const T* __restrict__ iu, const T* __restrict__ iv, T* __restrict__ ou,
                                     T* __restrict__ ov, int L)
{
    const long long LL = (long long)L * L;
    const long long n = 6 * LL;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int face = (int)(i / LL);
        const long long r = i - face * LL;
        const int a = (int)(r / L), b = (int)(r % L);
        const int e = (face & 1) ? L - 1 : 0;
        long long c;
        if (face < 2)
            c = e * LL + (long long)a * L + b;  // z = e, (y, x) = (a, b)
        else if (face < 4)
            c = (long long)a * LL + (long long)e * L + b;  // y = e, (z, x) = (a, b)
        else
            c = (long long)a * LL + (long long)b * L + e;  // x = e, (z, y) = (a, b)
        ou[c] = iu[c];
        if (iv) ov[c] = iv[c];
    }
}

int launch_hold_faces(int dtype, int L, const void* iu, const void* iv, void* ou, void* ov, cudaStream_t s)
{
    const long long n = 6LL * L * L;
    const int block = 256;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + block - 1) / block, 8LL * num_sms()));
    if (dtype == GS_F32)
        gs_hold_faces_kernel<float><<<grid, block, 0, s>>>((const float*)iu, (const float*)iv, (float*)ou, (float*)ov, L);
    else
        gs_hold_faces_kernel<double><<<grid, block, 0, s>>>((const double*)iu, (const double*)iv, (double*)ou,
                                                            (double*)ov, L);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------------------
// One field: z-marching kernel
// ---------------------------------------------------------------------------
// Shared-memory stage (one field), each block 128-B aligned:
//   main [ty][tx], top [tx], bot [tx], left [ty][V], right [ty][V]
struct Z1Layout {
    int main_off, top_off, bot_off, left_off, right_off;  // elements
    int stage_elems;   // padded
    int tx_bytes;      // bytes TMA writes per stage
};

static inline int round_up1(int a, int b) { return (a + b - 1) / b * b; }

static Z1Layout make_layout1(int esz, int V, int tx, int ty)
{
    const int a = 128 / esz;
    Z1Layout l;
    l.main_off = 0;
    l.top_off = round_up1(tx * ty, a);
    l.bot_off = l.top_off + round_up1(tx, a);
    l.left_off = l.bot_off + round_up1(tx, a);
    l.right_off = l.left_off + round_up1(V * ty, a);
    l.stage_elems = l.right_off + round_up1(V * ty, a);
    l.tx_bytes = (tx * ty + 2 * tx + 2 * V * ty) * esz;
    return l;
}

template <typename T>
struct Z1Args {
    T* fn;
    int L;
    int tx, ty, tz;
    int ntx, nty, ntiles;
    int stages;
    Z1Layout lay;
    T D6, dt;            // D / 6 and the time step
    int* err;
    uint64_t timeout_ns;
};

// f' = f + dt * (D/6) * (s - 6 f), s in the order x-, x+, y-, y+, z-, z+
template <typename T>
GS_D T gs_diffuse_cell(T D6, T dt, T c, T s)
{
    return gs_fma(gs_mul(D6, gs_fma((T)-6, c, s)), dt, c);
}

template <typename T>
__global__ void gs_zmarch1_kernel(const __grid_constant__ ZMaps maps, const Z1Args<T> a)
{
    constexpr int V = GsVec<T>::N;
    using VT = typename GsVec<T>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2 * 8];
    __shared__ volatile int abort_flag;

    const int S = a.stages;
    uint64_t* full = bars;
    uint64_t* empty = bars + S;
    const int nxv = a.tx / V;
    const int cons_threads = (nxv * a.ty + 31) & ~31;
    const int cons_warps = cons_threads >> 5;
    const int tid = threadIdx.x;
    const int L = a.L;
    T* ring = reinterpret_cast<T*>(smem);
    const int SE = a.lay.stage_elems;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            gs_mbar_init(&full[s], 1);
            gs_mbar_init(&empty[s], cons_warps);
        }
        abort_flag = 0;
        gs_fence_mbar_init();
    }
    __syncthreads();

    if (tid >= cons_threads) {
        // ------------------------------ producer warp ------------------------------
        if (tid != cons_threads) return;
        for (int m = 0; m < 3; ++m) gs_prefetch_tmap(&maps.m[0][m]);
        uint32_t seq = 0;
        int ps = 0;
        uint32_t pph = 0;
        bool wrapped = false;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
            const int txi = tile % a.ntx;
            const int tyi = (tile / a.ntx) % a.nty;
            const int tzi = tile / (a.ntx * a.nty);
            const int x0 = txi * a.tx, y0 = tyi * a.ty, z0 = tzi * a.tz;
            const int nvx = min(a.tx, L - x0), nvy = min(a.ty, L - y0), nz = min(a.tz, L - z0);
            const int ytop = (y0 - 1 + L) % L, ybot = (y0 + nvy) % L;
            const int xl = (x0 - V + L) % L, xr = (x0 + nvx) % L;
            int zp = (z0 - 1 + L) % L;
            for (int j = 0; j < nz + 2; ++j) {
                if (wrapped && !gs_mbar_wait(&empty[ps], pph ^ 1u, a.timeout_ns)) {
                    gs_report(a.err, GS_DERR_TIMEOUT);
                    abort_flag = 1;
                    goto drain;
                }
                if (abort_flag) goto drain;
                gs_mbar_arrive_expect_tx(&full[ps], a.lay.tx_bytes);
                {
                    T* b = ring + (size_t)ps * SE;
                    gs_tma_load_3d(b + a.lay.main_off, &maps.m[0][0], &full[ps], x0, y0, zp);
                    gs_tma_load_3d(b + a.lay.top_off, &maps.m[0][1], &full[ps], x0, ytop, zp);
                    gs_tma_load_3d(b + a.lay.bot_off, &maps.m[0][1], &full[ps], x0, ybot, zp);
                    gs_tma_load_3d(b + a.lay.left_off, &maps.m[0][2], &full[ps], xl, y0, zp);
                    gs_tma_load_3d(b + a.lay.right_off, &maps.m[0][2], &full[ps], xr, y0, zp);
                }
                ++seq;
                if (++ps == S) { ps = 0; pph ^= 1u; wrapped = true; }
                zp = zp + 1 == L ? 0 : zp + 1;
            }
        }
        return;
    drain:
        for (uint32_t q = (seq > (uint32_t)S ? seq - S : 0); q < seq; ++q)
            gs_mbar_wait(&full[q % S], (q / S) & 1, 2000000000ull);
        return;
    }

    // ------------------------------- consumer warps --------------------------------
    const int xv = tid % nxv;
    const int row = tid / nxv;
    const int lane = tid & 31;
    const int64_t LL = (int64_t)L * L;
    int cs = 0;
    uint32_t cph = 0;
    auto advance = [&]() {
        if (++cs == S) { cs = 0; cph ^= 1u; }
    };
    auto release = [&](int s) {
        __syncwarp();
        if (lane == 0) gs_mbar_arrive(&empty[s]);
    };
    auto wait_full = [&]() -> bool {
        if (gs_mbar_wait(&full[cs], cph, a.timeout_ns)) return true;
        gs_report(a.err, GS_DERR_TIMEOUT);
        abort_flag = 1;
        return false;
    };

    T q[3][V];
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int txi = tile % a.ntx;
        const int tyi = (tile / a.ntx) % a.nty;
        const int tzi = tile / (a.ntx * a.nty);
        const int x0 = txi * a.tx, y0 = tyi * a.ty, z0 = tzi * a.tz;
        const int nvx = min(a.tx, L - x0), nvy = min(a.ty, L - y0), nz = min(a.tz, L - z0);
        const bool active = row < nvy && xv * V < nvx;
        const int rr = row < a.ty ? row : 0;
        const int moff = a.lay.main_off + rr * a.tx + xv * V;
        const int om = row > 0 ? a.lay.main_off + (row - 1) * a.tx + xv * V : a.lay.top_off + xv * V;
        const int op = row + 1 < nvy ? a.lay.main_off + (row + 1) * a.tx + xv * V : a.lay.bot_off + xv * V;
        const bool has_r = xv * V + V < nvx;
        const bool l_smem = xv == 0 || lane == 0;
        const bool r_smem = !has_r || lane == 31;
        const int oxl = xv > 0 ? moff - 1 : a.lay.left_off + rr * V + (V - 1);
        const int oxr = has_r ? moff + V : a.lay.right_off + rr * V;
        int64_t gidx = (int64_t)z0 * LL + (int64_t)(y0 + row) * L + x0 + xv * V;
        int sc = 0;

        auto load_centre = [&](T (&f)[V]) {
            gs_unpack<T>(*reinterpret_cast<const VT*>(ring + (size_t)cs * SE + moff), f);
        };
        auto plane = [&](T (&p)[V], T (&c)[V], T (&n)[V]) -> bool {
            const int sn = cs;
            if (!wait_full()) return false;
            load_centre(n);
            const T shl = __shfl_up_sync(0xffffffffu, c[V - 1], 1);
            const T shr = __shfl_down_sync(0xffffffffu, c[0], 1);
            if (active) {
                const T* b = ring + (size_t)sc * SE;
                T ym[V], yp[V], out[V];
                gs_unpack<T>(*reinterpret_cast<const VT*>(b + om), ym);
                gs_unpack<T>(*reinterpret_cast<const VT*>(b + op), yp);
                const T xl = l_smem ? b[oxl] : shl;
                const T xr = r_smem ? b[oxr] : shr;
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const T s = gs_nsum(e > 0 ? c[e - 1] : xl, e < V - 1 ? c[e + 1] : xr, ym[e], yp[e], p[e], n[e]);
                    out[e] = gs_diffuse_cell<T>(a.D6, a.dt, c[e], s);
                }
                *reinterpret_cast<VT*>(a.fn + gidx) = gs_pack<T>(out);
            }
            release(sc);
            sc = sn;
            advance();
            gidx += LL;
            return true;
        };

        if (!wait_full()) return;
        load_centre(q[0]);
        release(cs);
        advance();
        sc = cs;
        if (!wait_full()) return;
        load_centre(q[1]);
        advance();
        int zi = 0;
        for (; zi + 3 <= nz; zi += 3) {
            if (!plane(q[0], q[1], q[2])) return;
            if (!plane(q[1], q[2], q[0])) return;
            if (!plane(q[2], q[0], q[1])) return;
        }
        if (zi < nz && !plane(q[0], q[1], q[2])) return;
        if (zi + 1 < nz && !plane(q[1], q[2], q[0])) return;
        release(sc);
        if (abort_flag) return;
    }
}

// plain one-thread-per-cell version (any L)
template <typename T>
__global__ void gs_naive1_kernel(const T* __restrict__ f, T* __restrict__ fn, int L, T D6, T dt)
{
    const long long n = (long long)L * L * L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((long long)L * L));
        const long long LL = (long long)L * L;
        const int xm = x == 0 ? L - 1 : x - 1, xp = x == L - 1 ? 0 : x + 1;
        const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
        const int zm = z == 0 ? L - 1 : z - 1, zp = z == L - 1 ? 0 : z + 1;
        const long long r = (long long)z * LL + (long long)y * L;
        const T s = gs_nsum(f[r + xm], f[r + xp], f[(long long)z * LL + (long long)ym * L + x],
                            f[(long long)z * LL + (long long)yp * L + x], f[(long long)zm * LL + (long long)y * L + x],
                            f[(long long)zp * LL + (long long)y * L + x]);
        fn[i] = gs_diffuse_cell<T>(D6, dt, f[i], s);
    }
}

}  // namespace gs

using namespace gs;

// ---------------------------------------------------------------------------
// gs_single: one field, f' = f + dt (D lap f)
// ---------------------------------------------------------------------------
struct gs_single {
    int L = 0, dtype = GS_F32, boundary = GS_BOUNDARY_PERIODIC;
    double D = 0, dt = 0;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t t = 0;
    cudaStream_t stream = nullptr;
    int* d_err = nullptr;
    bool zmarch = false;
    ZPlan pl{256, 4, 64, 4, 1};
    ZMaps maps[2];
    int64_t launches = 0;
};

static int single_encode(gs_single* s)
{
    const int V = s->dtype == GS_F32 ? 4 : 2;
    for (int i = 0; i < 2; ++i) {
        CUresult r0 = encode_tiled_3d(&s->maps[i].m[0][0], s->dtype, s->buf[i], s->L, s->pl.tx, s->pl.ty);
        CUresult r1 = encode_tiled_3d(&s->maps[i].m[0][1], s->dtype, s->buf[i], s->L, s->pl.tx, 1);
        CUresult r2 = encode_tiled_3d(&s->maps[i].m[0][2], s->dtype, s->buf[i], s->L, V, s->pl.ty);
        if (r0 != CUDA_SUCCESS || r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
            return fail(GS_ECUDA, "cuTensorMapEncodeTiled failed for the single-field maps");
    }
    return GS_OK;
}

int gs_single_create(int L, double D, double dt, int dtype, int boundary, gs_single** out)
{
    if (!out) return fail(GS_EINVAL, "out is NULL");
    *out = nullptr;
    if (L < 1 || L > GS_MAX_L) return fail(GS_EINVAL, "L=%d must be in [1, %d]", L, GS_MAX_L);
    if (dtype != GS_F32 && dtype != GS_F64) return fail(GS_EINVAL, "dtype=%d", dtype);
    if (boundary != GS_BOUNDARY_PERIODIC && boundary != GS_BOUNDARY_HELD)
        return fail(GS_EINVAL, "boundary=%d", boundary);
    if (!std::isfinite(D) || !std::isfinite(dt)) return fail(GS_EINVAL, "D and dt must be finite");
    gs_single* s = new gs_single();
    s->L = L;
    s->dtype = dtype;
    s->boundary = boundary;
    s->D = D;
    s->dt = dt;
    const size_t bytes = (size_t)L * L * L * elem_size(dtype);
    cudaError_t e = cudaMalloc(&s->buf[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->buf[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(s->buf[0], 0, bytes);
    if (e != cudaSuccess) {
        cudaFree(s->buf[0]);
        cudaFree(s->buf[1]);
        cudaFree(s->d_err);
        delete s;
        return e == cudaErrorMemoryAllocation ? fail(GS_ENOMEM, "gs_single_create: %s", cudaGetErrorString(e))
                                              : cuda_fail(e, "gs_single_create");
    }
    // the z-marching kernel needs 16-byte rows (L a multiple of the vector
    // width); partial tiles at the grid's edge are handled in the kernel
    const int V = dtype == GS_F32 ? 4 : 2;
    if (L % V == 0) {
        s->pl.tx = std::min(L, 256);
        s->pl.ty = std::min(L, 4);
        s->pl.tz = std::min(L, 64);
        if (single_encode(s) == GS_OK) s->zmarch = true;
    }
    *out = s;
    return GS_OK;
}

int gs_single_set_stream(gs_single* s, void* stream)
{
    if (!s) return fail(GS_EINVAL, "single is NULL");
    s->stream = (cudaStream_t)stream;
    return GS_OK;
}

int gs_single_write(gs_single* s, const void* src, size_t bytes)
{
    if (!s || !src) return fail(GS_EINVAL, "NULL argument");
    const size_t want = (size_t)s->L * s->L * s->L * elem_size(s->dtype);
    if (bytes != want) return fail(GS_EINVAL, "bytes=%zu, expected %zu", bytes, want);
    GS_CUDA_TRY(cudaMemcpyAsync(s->buf[s->cur], src, bytes, cudaMemcpyHostToDevice, s->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GS_OK;
}

int gs_single_read(gs_single* s, void* dst, size_t bytes)
{
    if (!s || !dst) return fail(GS_EINVAL, "NULL argument");
    const size_t want = (size_t)s->L * s->L * s->L * elem_size(s->dtype);
    if (bytes != want) return fail(GS_EINVAL, "bytes=%zu, expected %zu", bytes, want);
    GS_CUDA_TRY(cudaMemcpyAsync(dst, s->buf[s->cur], bytes, cudaMemcpyDeviceToHost, s->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    int err = 0;
    GS_CUDA_TRY(cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) return fail(GS_ETIMEOUT, "a device-side wait of the single-field kernel expired");
    return GS_OK;
}

template <typename T>
static int single_step_t(gs_single* s)
{
    constexpr int V = GsVec<T>::N;
    const int in = s->cur, out = 1 - s->cur;
    const T D6 = (T)(s->D / 6.0), dt = (T)s->dt;
    if (s->zmarch) {
        Z1Args<T> a;
        a.fn = (T*)s->buf[out];
        a.L = s->L;
        a.tx = s->pl.tx;
        a.ty = s->pl.ty;
        a.tz = s->pl.tz;
        a.ntx = (s->L + a.tx - 1) / a.tx;
        a.nty = (s->L + a.ty - 1) / a.ty;
        a.ntiles = a.ntx * a.nty * ((s->L + a.tz - 1) / a.tz);
        a.stages = s->pl.stages;
        a.lay = make_layout1(sizeof(T), V, a.tx, a.ty);
        a.D6 = D6;
        a.dt = dt;
        a.err = s->d_err;
        a.timeout_ns = 2000000000ull;
        const int threads = (((a.tx / V) * a.ty + 31) & ~31) + 32;
        const size_t smem = (size_t)a.lay.stage_elems * sizeof(T) * a.stages;
        auto kern = gs_zmarch1_kernel<T>;
        GS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        if (per_sm < 1) return fail(GS_EINVAL, "single-field tile does not fit on an SM");
        kern<<<std::min(a.ntiles, per_sm * num_sms()), threads, smem, s->stream>>>(s->maps[in], a);
    } else {
        const long long n = (long long)s->L * s->L * s->L;
        const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * num_sms()));
        gs_naive1_kernel<T><<<grid, 256, 0, s->stream>>>((const T*)s->buf[in], (T*)s->buf[out], s->L, D6, dt);
    }
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    if (s->boundary == GS_BOUNDARY_HELD) {
        const int rc = launch_hold_faces(s->dtype, s->L, s->buf[in], nullptr, s->buf[out], nullptr, s->stream);
        if (rc) return rc;
        s->launches += 1;
    }
    s->cur = out;
    s->t += 1;
    return GS_OK;
}

int gs_single_step(gs_single* s, int64_t n)
{
    if (!s) return fail(GS_EINVAL, "single is NULL");
    if (n < 0) return fail(GS_EINVAL, "n=%lld must be >= 0", (long long)n);
    for (int64_t i = 0; i < n; ++i) {
        const int rc = s->dtype == GS_F32 ? single_step_t<float>(s) : single_step_t<double>(s);
        if (rc) return rc;
    }
    return GS_OK;
}

int gs_single_info(gs_single* s, int* zmarch, int64_t* steps, int64_t* launches)
{
    if (!s) return fail(GS_EINVAL, "single is NULL");
    if (zmarch) *zmarch = s->zmarch ? 1 : 0;
    if (steps) *steps = s->t;
    if (launches) *launches = s->launches;
    return GS_OK;
}

int gs_single_sync(gs_single* s)
{
    if (!s) return fail(GS_EINVAL, "single is NULL");
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GS_OK;
}

int gs_single_destroy(gs_single* s)
{
    if (!s) return GS_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->buf[0]);
    cudaFree(s->buf[1]);
    cudaFree(s->d_err);
    delete s;
    return GS_OK;
}
