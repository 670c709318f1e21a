// z-slab decomposition of one periodic L^3 grid (the paper's domain
// decomposition with face exchange, Section 3.3 and Listing 3, cut along z
// only).
//
// A slab holds the global planes z0 .. z0+nz-1 of the grid plus `depth` = D
// ghost planes on each side: local plane zl (0 .. nz+2D-1) is global plane
// (z0 - D + zl) mod L.  One pass advances the slab by D steps without any
// exchange: sub-step s (0 .. D-1) updates local planes s+1 .. nz+2D-s-2 from
// their neighbours, so after D sub-steps the nz interior planes hold the
// state D steps later and the ghosts are stale.  Each exchange then copies a
// neighbour's D interior planes next to the face into the ghost planes (into
// the receiving slab's own memory).  Every cell update calls gs_update with
// the single grid's neighbour order, step index and global cell index for
// the noise draw, so slabs reproduce the single-grid run bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {

// Cells of local planes [zlo, zhi) of a slab; x and y are periodic in L,
// z neighbours are the adjacent local planes (zlo >= 1, zhi <= planes - 1).
// zg0 = global plane of local plane 0 (mod L), used for the noise index.
template <typename T, bool NOISE>
__global__ void __launch_bounds__(256) gs_slab_kernel(const T* __restrict__ u, const T* __restrict__ v,
                                                      T* __restrict__ un, T* __restrict__ vn, int L, int zlo, int zhi,
                                                      int zg0, GsCoef<T> c, GsKeys k)
{
    const int64_t LL = (int64_t)L * L;
    const int64_t n = (int64_t)(zhi - zlo) * LL;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(j % L);
        const int64_t r = j / L;
        const int y = (int)(r % L);
        const int zl = zlo + (int)(r / L);
        const int64_t i = (int64_t)zl * LL + (int64_t)y * L + x;  // local index
        const int64_t row = i - x;
        const int64_t pl = i - (int64_t)y * L;
        const int64_t ixm = row + (x == 0 ? L - 1 : x - 1);
        const int64_t ixp = row + (x == L - 1 ? 0 : x + 1);
        const int64_t iym = pl + (int64_t)(y == 0 ? L - 1 : y - 1) * L;
        const int64_t iyp = pl + (int64_t)(y == L - 1 ? 0 : y + 1) * L;
        const T uc = u[i], vc = v[i];
        const T su = gs_nsum(u[ixm], u[ixp], u[iym], u[iyp], u[i - LL], u[i + LL]);
        const T sv = gs_nsum(v[ixm], v[ixp], v[iym], v[iyp], v[i - LL], v[i + LL]);
        T rn = (T)0;
        if (NOISE) {
            const int zg = (zg0 + zl) % L;
            rn = (T)gs_noise_num((uint32_t)(x + L * (y + (int64_t)L * zg)), k);
        }
        T a, b;
        gs_update<T, NOISE>(c, uc, vc, su, sv, rn, a, b);
        un[i] = a;
        vn[i] = b;
    }
}

// centred-cube initial state on every local plane (ghosts included)
template <typename T>
__global__ void gs_slab_init_kernel(T* __restrict__ u, T* __restrict__ v, int L, int planes, int zg0)
{
    const int64_t LL = (int64_t)L * L;
    const int64_t n = (int64_t)planes * LL;
    const int lo = L / 2 - 3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L);
        const int y = (int)((i / L) % L);
        const int z = (int)((zg0 + i / LL) % L);
        const bool in = x >= lo && x < lo + 6 && y >= lo && y < lo + 6 && z >= lo && z < lo + 6;
        u[i] = in ? (T)0.25 : (T)1.0;
        v[i] = in ? (T)0.33 : (T)0.0;
    }
}

}  // namespace gs

using namespace gs;

struct gs_slab {
    int L = 0, z0 = 0, nz = 0, D = 0, dtype = GS_F32;
    Params p{};
    void* f[2][2] = {};  // [buffer set][field], caller-owned
    int cur = 0;
    int64_t t = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_done = nullptr, ev_copied = nullptr;
    int64_t launches = 0;
    int planes() const { return nz + 2 * D; }
    size_t plane_bytes() const { return (size_t)L * L * elem_size(dtype); }
};

namespace {

int slab_grid(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16));
}

template <typename T>
int slab_pass_t(gs_slab* s)
{
    const GsCoef<T> c = gs_make_coef<T>(s->p.Du, s->p.Dv, s->p.F, s->p.k, s->p.dt, s->p.noise);
    const bool nz = s->p.noise != 0.0;
    const int zg0 = ((s->z0 - s->D) % s->L + s->L) % s->L;
    for (int sub = 0; sub < s->D; ++sub) {
        const int zlo = sub + 1, zhi = s->planes() - sub - 1;
        const GsKeys k = gs_step_keys(s->p.seed, s->t + sub);
        const T* u = (const T*)s->f[s->cur][0];
        const T* v = (const T*)s->f[s->cur][1];
        T* un = (T*)s->f[s->cur ^ 1][0];
        T* vn = (T*)s->f[s->cur ^ 1][1];
        const int64_t n = (int64_t)(zhi - zlo) * s->L * s->L;
        if (nz)
            gs_slab_kernel<T, true><<<slab_grid(n), 256, 0, s->stream>>>(u, v, un, vn, s->L, zlo, zhi, zg0, c, k);
        else
            gs_slab_kernel<T, false><<<slab_grid(n), 256, 0, s->stream>>>(u, v, un, vn, s->L, zlo, zhi, zg0, c, k);
        GS_CUDA_TRY(cudaGetLastError());
        s->launches += 1;
        s->cur ^= 1;
    }
    s->t += s->D;
    return GS_OK;
}

int check_slab(const gs_slab* s) { return s ? GS_OK : fail(GS_EINVAL, "slab is NULL"); }

}  // namespace

extern "C" {

int gs_slab_create_on(int L, int z0, int nz, int depth, double Du, double Dv, double F, double k, double dt,
                      double noise, uint64_t seed, int dtype, void* u0, void* v0, void* u1, void* v1, gs_slab** out)
{
    if (!out) return fail(GS_EINVAL, "out is NULL");
    *out = nullptr;
    if (L < 1 || L > 1625) return fail(GS_EINVAL, "L=%d must be in [1, 1625]", L);
    if (depth < 1) return fail(GS_EINVAL, "depth=%d must be >= 1", depth);
    if (nz < depth || nz > L) return fail(GS_EINVAL, "nz=%d must be in [depth=%d, L=%d]", nz, depth, L);
    if (z0 < 0 || z0 >= L) return fail(GS_EINVAL, "z0=%d must be in [0, L)", z0);
    if (dtype != GS_F32 && dtype != GS_F64) return fail(GS_EINVAL, "dtype=%d must be GS_F32 or GS_F64", dtype);
    if (!u0 || !v0 || !u1 || !v1) return fail(GS_EINVAL, "the four field buffers must not be NULL");
    const double pv[6] = {Du, Dv, F, k, dt, noise};
    for (double x : pv)
        if (!std::isfinite(x)) return fail(GS_EINVAL, "parameters must be finite");
    gs_slab* s = new (std::nothrow) gs_slab();
    if (!s) return fail(GS_ENOMEM, "host allocation failed");
    s->L = L;
    s->z0 = z0;
    s->nz = nz;
    s->D = depth;
    s->dtype = dtype;
    s->p.Du = Du;
    s->p.Dv = Dv;
    s->p.F = F;
    s->p.k = k;
    s->p.dt = dt;
    s->p.noise = noise;
    s->p.seed = seed;
    s->f[0][0] = u0;
    s->f[0][1] = v0;
    s->f[1][0] = u1;
    s->f[1][1] = v1;
    cudaError_t e = cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_copied, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (s->ev_done) cudaEventDestroy(s->ev_done);
        delete s;
        return cuda_fail(e, "slab events");
    }
    *out = s;
    return GS_OK;
}

int gs_slab_set_stream(gs_slab* s, void* stream)
{
    if (int rc = check_slab(s)) return rc;
    s->stream = (cudaStream_t)stream;
    return GS_OK;
}

int gs_slab_init(gs_slab* s)
{
    if (int rc = check_slab(s)) return rc;
    const int64_t n = (int64_t)s->planes() * s->L * s->L;
    const int zg0 = ((s->z0 - s->D) % s->L + s->L) % s->L;
    if (s->dtype == GS_F32)
        gs_slab_init_kernel<float><<<slab_grid(n), 256, 0, s->stream>>>((float*)s->f[0][0], (float*)s->f[0][1], s->L,
                                                                        s->planes(), zg0);
    else
        gs_slab_init_kernel<double><<<slab_grid(n), 256, 0, s->stream>>>((double*)s->f[0][0], (double*)s->f[0][1],
                                                                         s->L, s->planes(), zg0);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    s->cur = 0;
    s->t = 0;
    return GS_OK;
}

int gs_slab_pass(gs_slab* s)
{
    if (int rc = check_slab(s)) return rc;
    return s->dtype == GS_F32 ? slab_pass_t<float>(s) : slab_pass_t<double>(s);
}

int gs_slab_state(gs_slab* s, int64_t* t, int* cur)
{
    if (int rc = check_slab(s)) return rc;
    if (t) *t = s->t;
    if (cur) *cur = s->cur;
    return GS_OK;
}

int gs_slab_set_state(gs_slab* s, int64_t t, int cur)
{
    if (int rc = check_slab(s)) return rc;
    if (t < 0 || (cur != 0 && cur != 1)) return fail(GS_EINVAL, "need t >= 0 and cur in {0, 1}");
    s->t = t;
    s->cur = cur;
    return GS_OK;
}

int gs_slab_exchange(gs_slab** slabs, int n)
{
    if (!slabs || n < 1) return fail(GS_EINVAL, "need n >= 1 slabs");
    for (int i = 0; i < n; ++i) {
        if (!slabs[i]) return fail(GS_EINVAL, "slab %d is NULL", i);
        const gs_slab* a = slabs[i];
        const gs_slab* b = slabs[(i + 1) % n];
        if (a->L != b->L || a->D != b->D || a->dtype != b->dtype || a->t != b->t)
            return fail(GS_EINVAL, "slabs %d and %d differ in L, depth, dtype or step", i, (i + 1) % n);
        if ((a->z0 + a->nz) % a->L != b->z0)
            return fail(GS_EINVAL, "slab %d ends at plane %d, slab %d starts at %d", i, (a->z0 + a->nz) % a->L,
                        (i + 1) % n, b->z0);
    }
    // every slab's pass has finished before anything reads its planes
    for (int i = 0; i < n; ++i) GS_CUDA_TRY(cudaEventRecord(slabs[i]->ev_done, slabs[i]->stream));
    for (int i = 0; i < n; ++i) {
        gs_slab* r = slabs[i];
        const gs_slab* lo = slabs[(i + n - 1) % n];
        const gs_slab* hi = slabs[(i + 1) % n];
        GS_CUDA_TRY(cudaStreamWaitEvent(r->stream, lo->ev_done, 0));
        GS_CUDA_TRY(cudaStreamWaitEvent(r->stream, hi->ev_done, 0));
        const size_t pb = r->plane_bytes(), bytes = pb * r->D;
        for (int f = 0; f < 2; ++f) {
            char* dst = (char*)r->f[r->cur][f];
            // low ghosts <- the lower slab's last D interior planes
            GS_CUDA_TRY(cudaMemcpyAsync(dst, (const char*)lo->f[lo->cur][f] + pb * lo->nz, bytes,
                                        cudaMemcpyDeviceToDevice, r->stream));
            // high ghosts <- the upper slab's first D interior planes
            GS_CUDA_TRY(cudaMemcpyAsync(dst + pb * (r->nz + r->D), (const char*)hi->f[hi->cur][f] + pb * hi->D, bytes,
                                        cudaMemcpyDeviceToDevice, r->stream));
        }
        GS_CUDA_TRY(cudaEventRecord(r->ev_copied, r->stream));
    }
    // no slab overwrites planes a neighbour is still copying
    for (int i = 0; i < n; ++i) {
        GS_CUDA_TRY(cudaStreamWaitEvent(slabs[i]->stream, slabs[(i + n - 1) % n]->ev_copied, 0));
        GS_CUDA_TRY(cudaStreamWaitEvent(slabs[i]->stream, slabs[(i + 1) % n]->ev_copied, 0));
    }
    return GS_OK;
}

int gs_slab_sync(gs_slab* s)
{
    if (int rc = check_slab(s)) return rc;
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GS_OK;
}

int gs_slab_launch_count(gs_slab* s, int64_t* count)
{
    if (int rc = check_slab(s)) return rc;
    if (!count) return fail(GS_EINVAL, "count is NULL");
    *count = s->launches;
    return GS_OK;
}

int gs_slab_destroy(gs_slab* s)
{
    if (!s) return GS_OK;
    cudaEventDestroy(s->ev_done);
    cudaEventDestroy(s->ev_copied);
    delete s;
    return GS_OK;
}

}  // extern "C"
