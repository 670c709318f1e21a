// C-ABI of libgs: object lifetime, argument checks, plan selection, stream
// handling and error reporting around the stencil kernels (include/gs.h).
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <map>
#include <mutex>
#include <vector>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {

static thread_local char g_msg[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    const int code = e == cudaErrorMemoryAllocation ? GS_ENOMEM : GS_ECUDA;
    return fail(code, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

int elem_size(int dtype) { return dtype == GS_F32 ? 4 : 8; }

namespace {
std::mutex g_guard_mutex;
size_t g_guard_bytes = 0;
struct GuardRec {
    char* base;
    size_t bytes, guard;
};
std::map<const void*, GuardRec> g_guarded;
}  // namespace

cudaError_t guarded_malloc(void** p, size_t bytes)
{
    size_t g;
    {
        std::lock_guard<std::mutex> lk(g_guard_mutex);
        g = g_guard_bytes;
    }
    if (g == 0) return cudaMalloc(p, bytes);
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes + 2 * g);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemset(base, 0xFF, bytes + 2 * g)) != cudaSuccess) {
        cudaFree(base);
        return e;
    }
    *p = base + g;
    std::lock_guard<std::mutex> lk(g_guard_mutex);
    g_guarded[*p] = GuardRec{base, bytes, g};
    return cudaSuccess;
}

void guarded_free(void* p)
{
    if (!p) return;
    char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_guard_mutex);
        auto it = g_guarded.find(p);
        if (it != g_guarded.end()) {
            base = it->second.base;
            g_guarded.erase(it);
        }
    }
    cudaFree(base ? (void*)base : p);
}

int64_t guarded_check(const void* p)
{
    GuardRec r{};
    {
        std::lock_guard<std::mutex> lk(g_guard_mutex);
        auto it = g_guarded.find(p);
        if (it == g_guarded.end()) return 0;
        r = it->second;
    }
    std::vector<unsigned char> h(r.guard);
    int64_t bad = 0;
    for (int side = 0; side < 2; ++side) {
        const char* src = side == 0 ? r.base : r.base + r.guard + r.bytes;
        if (cudaMemcpy(h.data(), src, r.guard, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
        for (unsigned char c : h) bad += c != 0xFF;
    }
    return bad;
}

int num_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode;
}

CUresult encode_tiled_3d(CUtensorMap* map, int dtype, void* base, int L, int box_x, int box_y)
{
    auto enc = tensor_map_encoder();
    if (!enc) return CUDA_ERROR_NOT_FOUND;
    const size_t esz = elem_size(dtype);
    cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)L, (cuuint64_t)L};
    cuuint64_t strides[2] = {(cuuint64_t)L * esz, (cuuint64_t)L * L * esz};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, dtype == GS_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
               3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

CUresult encode_act_4d(CUtensorMap* map, const void* base, int C, int L, long long planes, int box_c, int box_x,
                       int swizzle)
{
    if (swizzle != 0 && swizzle != 32 && swizzle != 64) return CUDA_ERROR_INVALID_VALUE;
    auto enc = tensor_map_encoder();
    if (!enc) return CUDA_ERROR_NOT_FOUND;
    cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)L, (cuuint64_t)L, (cuuint64_t)planes};
    cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)L * C * 2, (cuuint64_t)L * L * C * 2};
    cuuint32_t box[4] = {(cuuint32_t)box_c, (cuuint32_t)box_x, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE,
               swizzle == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : (swizzle == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE),
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

}  // namespace gs

using namespace gs;


static bool finite_params(double a, double b, double c, double d, double e, double f)
{
    return std::isfinite(a) && std::isfinite(b) && std::isfinite(c) && std::isfinite(d) &&
           std::isfinite(e) && std::isfinite(f);
}

static int default_plan(gs_sim* s)
{
    if (zmarch_supported(s->dtype, s->L)) {
        ZPlan pl;
        const int V = s->dtype == GS_F32 ? 4 : 2;
        pl.tx = std::min(s->dtype == GS_F32 ? 128 : 64, s->L);
        pl.tx -= pl.tx % V;
        pl.ty = std::min(8, s->L);
        pl.tz = std::min(32, s->L);
        pl.stages = 4;
        pl.depth = 1;
        if (zmarch_validate(s->dtype, s->L, pl) == GS_OK) {
            s->zp = pl;
            s->kernel = GS_KERNEL_ZMARCH;
            return GS_OK;
        }
    }
    s->kernel = GS_KERNEL_NAIVE;
    return GS_OK;
}

static int encode_maps(gs_sim* s)
{
    s->maps_ok = false;
    if (s->kernel == GS_KERNEL_NAIVE || !zmarch_supported(s->dtype, s->L)) return GS_OK;
    for (int set = 0; set < 2; ++set) {
        int rc = zmarch_encode(s->dtype, s->L, s->zp, s->buf[set][0], s->buf[set][1], &s->maps[set]);
        if (rc) return rc;
    }
    s->maps_ok = true;
    return GS_OK;
}

static int check_common(int L, double Du, double Dv, double F, double k, double dt, double noise,
                        int dtype, gs_sim** out)
{
    if (!out) return fail(GS_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (L < 1 || L > GS_MAX_L) return fail(GS_EINVAL, "L=%d must be in [1, %d]", L, GS_MAX_L);
    if (dtype != GS_F32 && dtype != GS_F64) return fail(GS_EINVAL, "dtype=%d must be GS_F32 or GS_F64", dtype);
    if (!finite_params(Du, Dv, F, k, dt, noise)) return fail(GS_EINVAL, "parameters must be finite");
    return GS_OK;
}

static int finish_create(gs_sim* s, gs_sim** out)
{
    // the device error word, a pad word and the z-march kernel's two ticket words
    GS_CUDA_TRY(cudaMalloc(&s->d_err, 4 * sizeof(int)));
    GS_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, 4 * sizeof(int), s->stream));
    int rc = default_plan(s);
    if (!rc) rc = encode_maps(s);
    if (!rc) rc = launch_init(s->dtype, s->L, s->buf[0][0], s->buf[0][1], s->stream);
    if (rc) return rc;
    s->launches += 1;
    *out = s;
    return GS_OK;
}

extern "C" {

const char* gs_last_error(void) { return g_msg; }

int gs_create(int L, double Du, double Dv, double F, double k, double dt, double noise, uint64_t seed,
              int dtype, gs_sim** out)
{
    int rc = check_common(L, Du, Dv, F, k, dt, noise, dtype, out);
    if (rc) return rc;
    gs_sim* s = new (std::nothrow) gs_sim();
    if (!s) return fail(GS_ENOMEM, "host allocation failed");
    s->L = L;
    s->dtype = dtype;
    s->p = Params{Du, Dv, F, k, dt, noise, seed};
    s->owns = true;
    const size_t bytes = (size_t)L * L * L * elem_size(dtype);
    for (int set = 0; set < 2; ++set)
        for (int f = 0; f < 2; ++f) {
            cudaError_t e = cudaMalloc(&s->buf[set][f], bytes);
            if (e != cudaSuccess) {
                gs_destroy(s);
                return cuda_fail(e, "cudaMalloc(field)");
            }
        }
    rc = finish_create(s, out);
    if (rc) {
        gs_destroy(s);
        *out = nullptr;
    }
    return rc;
}

int gs_create_on(int L, double Du, double Dv, double F, double k, double dt, double noise, uint64_t seed,
                 int dtype, void* u0, void* v0, void* u1, void* v1, void* stream, gs_sim** out)
{
    int rc = check_common(L, Du, Dv, F, k, dt, noise, dtype, out);
    if (rc) return rc;
    void* b[4] = {u0, v0, u1, v1};
    for (int i = 0; i < 4; ++i) {
        if (!b[i]) return fail(GS_EINVAL, "device buffer %d is NULL", i);
        if (reinterpret_cast<uintptr_t>(b[i]) % 256) return fail(GS_EINVAL, "device buffer %d not 256-byte aligned", i);
    }
    gs_sim* s = new (std::nothrow) gs_sim();
    if (!s) return fail(GS_ENOMEM, "host allocation failed");
    s->L = L;
    s->dtype = dtype;
    s->p = Params{Du, Dv, F, k, dt, noise, seed};
    s->owns = false;
    s->buf[0][0] = u0;
    s->buf[0][1] = v0;
    s->buf[1][0] = u1;
    s->buf[1][1] = v1;
    s->stream = (cudaStream_t)stream;
    rc = finish_create(s, out);
    if (rc) {
        gs_destroy(s);
        *out = nullptr;
    }
    return rc;
}

int gs_set_stream(gs_sim* s, void* stream)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    // the work already issued finishes first: the next step's kernels must
    // not overlap it (they share the fields and the work-unit counter)
    if ((cudaStream_t)stream != s->stream) GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->stream = (cudaStream_t)stream;
    return GS_OK;
}

int gs_get_stream(gs_sim* s, void** stream)
{
    if (!s || !stream) return fail(GS_EINVAL, "NULL argument");
    *stream = (void*)s->stream;
    return GS_OK;
}

int gs_sim_shape(gs_sim* s, int* L, int* dtype)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (L) *L = s->L;
    if (dtype) *dtype = s->dtype;
    return GS_OK;
}

int gs_init(gs_sim* s)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    s->cur = 0;
    s->t = 0;
    GS_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, 4 * sizeof(int), s->stream));  // error word and tickets
    int rc = launch_init(s->dtype, s->L, s->buf[0][0], s->buf[0][1], s->stream);
    if (!rc) s->launches += 1;
    return rc;
}

int gs_step(gs_sim* s, int64_t n)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (n < 0) return fail(GS_EINVAL, "n=%lld must be >= 0", (long long)n);
    int64_t i = 0;
    if (s->kernel == GS_KERNEL_TBLOCK) {
        const int D = s->tp.depth;
        for (; i + D <= n; i += D) {
            const int in = s->cur, outs = 1 - s->cur;
            int rc = launch_tblock(s->L, s->tp, s->buf[in][0], s->buf[in][1], s->buf[outs][0], s->buf[outs][1],
                                   s->p, s->t, (unsigned*)(s->d_err + 2), s->stream);
            if (rc) return rc;
            s->launches += 1;
            s->cur = outs;
            s->t += D;
        }
    }
    const int64_t first = i;
    for (; i < n; ++i) {
        const int in = s->cur, outs = 1 - s->cur;
        // the FP64 arithmetics other than IEEE keep the fields in their own
        // packed form between the steps of this call (periodic grids): the
        // first step reads FP64, the last writes FP64
        Params p = s->p;
        if (p.arith != GS_ARITH_IEEE && s->boundary == GS_BOUNDARY_PERIODIC)
            p.io = (i > first ? 1 : 0) | (i + 1 < n ? 2 : 0);
        int rc;
        if (s->kernel != GS_KERNEL_NAIVE) {
            if (!s->maps_ok) return fail(GS_ESTATE, "tensor maps not encoded");
            rc = launch_zmarch(s->dtype, s->L, s->zp, s->maps[in], s->buf[outs][0], s->buf[outs][1], p, s->t,
                               s->d_err, s->timeout_ns, s->fault, (unsigned*)(s->d_err + 2), s->stream);
        } else {
            rc = launch_naive(s->dtype, s->L, s->buf[in][0], s->buf[in][1], s->buf[outs][0], s->buf[outs][1], p,
                              s->t, s->d_err, s->stream);
        }
        if (rc) return rc;
        s->launches += 1;
        if (s->boundary == GS_BOUNDARY_HELD) {
            rc = launch_hold_faces(s->dtype, s->L, s->buf[in][0], s->buf[in][1], s->buf[outs][0], s->buf[outs][1],
                                   s->stream);
            if (rc) return rc;
            s->launches += 1;
        }
        s->cur = outs;
        s->t += 1;
    }
    return GS_OK;
}

static int check_field(gs_sim* s, int field, size_t bytes)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (field != GS_U && field != GS_V) return fail(GS_EINVAL, "field=%d must be GS_U or GS_V", field);
    const size_t need = (size_t)s->L * s->L * s->L * elem_size(s->dtype);
    if (bytes != need) return fail(GS_EINVAL, "bytes=%zu, field holds %zu", bytes, need);
    return GS_OK;
}

int gs_sync(gs_sim* s)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    int err = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (err == GS_DERR_TIMEOUT) return fail(GS_ETIMEOUT, "a device-side wait timed out");
    if (err == GS_DERR_RANGE) {
        // reported once: the steps since the last check met a value outside
        // the fixed-point range (the fields are unreliable from there on)
        GS_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
        return fail(GS_EINVAL, "a field value left the fixed-point range (|u|, |v| < %s) of %s",
                    s->p.arith == GS_ARITH_FXF ? "4" : "1024", s->p.arith == GS_ARITH_FXF ? "GS_ARITH_FXF" : "GS_ARITH_FX");
    }
    if (err) return fail(GS_ECUDA, "device error code %d", err);
    return GS_OK;
}

int gs_read(gs_sim* s, int field, void* dst, size_t bytes)
{
    int rc = check_field(s, field, bytes);
    if (rc) return rc;
    if (!dst) return fail(GS_EINVAL, "dst is NULL");
    GS_CUDA_TRY(cudaMemcpyAsync(dst, s->buf[s->cur][field], bytes, cudaMemcpyDeviceToHost, s->stream));
    return gs_sync(s);
}

int gs_write(gs_sim* s, int field, const void* src, size_t bytes)
{
    int rc = check_field(s, field, bytes);
    if (rc) return rc;
    if (!src) return fail(GS_EINVAL, "src is NULL");
    GS_CUDA_TRY(cudaMemcpyAsync(s->buf[s->cur][field], src, bytes, cudaMemcpyHostToDevice, s->stream));
    return gs_sync(s);
}

int gs_read_async(gs_sim* s, int field, void* dst, size_t bytes)
{
    int rc = check_field(s, field, bytes);
    if (rc) return rc;
    if (!dst) return fail(GS_EINVAL, "dst is NULL");
    GS_CUDA_TRY(cudaMemcpyAsync(dst, s->buf[s->cur][field], bytes, cudaMemcpyDeviceToHost, s->stream));
    return GS_OK;
}

int gs_write_async(gs_sim* s, int field, const void* src, size_t bytes)
{
    int rc = check_field(s, field, bytes);
    if (rc) return rc;
    if (!src) return fail(GS_EINVAL, "src is NULL");
    GS_CUDA_TRY(cudaMemcpyAsync(s->buf[s->cur][field], src, bytes, cudaMemcpyHostToDevice, s->stream));
    return GS_OK;
}

int gs_device_ptr(gs_sim* s, int field, void** p)
{
    if (!s || !p) return fail(GS_EINVAL, "NULL argument");
    if (field != GS_U && field != GS_V) return fail(GS_EINVAL, "field=%d must be GS_U or GS_V", field);
    *p = s->buf[s->cur][field];
    return GS_OK;
}

int gs_get_step(gs_sim* s, int64_t* t)
{
    if (!s || !t) return fail(GS_EINVAL, "NULL argument");
    *t = s->t;
    return GS_OK;
}

int gs_set_step(gs_sim* s, int64_t t)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (t < 0) return fail(GS_EINVAL, "t must be >= 0");
    s->t = t;
    return GS_OK;
}

static int apply_plan(gs_sim* s, int kernel, int tile_x, int tile_y, int tile_z, int depth, int stages)
{
    if (kernel == GS_KERNEL_AUTO) {
        int rc = default_plan(s);
        return rc ? rc : encode_maps(s);
    }
    if (kernel == GS_KERNEL_NAIVE) {
        s->kernel = GS_KERNEL_NAIVE;
        s->maps_ok = false;
        return GS_OK;
    }
    if (kernel == GS_KERNEL_ZMARCH) {
        if (depth > 1) return fail(GS_EINVAL, "GS_KERNEL_ZMARCH takes depth 1");
        ZPlan pl = s->zp;
        const int V = s->dtype == GS_F32 ? 4 : 2;
        pl.tx = tile_x > 0 ? tile_x : std::min(s->dtype == GS_F32 ? 128 : 64, s->L - s->L % V);
        pl.ty = tile_y > 0 ? tile_y : std::min(8, s->L);
        pl.tz = tile_z > 0 ? tile_z : std::min(32, s->L);
        pl.stages = stages > 0 ? stages : 4;
        pl.depth = 1;
        int rc = zmarch_validate(s->dtype, s->L, pl);
        if (rc) return rc;
        const int old_kernel = s->kernel;
        const ZPlan old = s->zp;
        s->kernel = GS_KERNEL_ZMARCH;
        s->zp = pl;
        rc = encode_maps(s);
        if (rc) {
            s->kernel = old_kernel;
            s->zp = old;
            encode_maps(s);
        }
        return rc;
    }
    if (kernel == GS_KERNEL_TBLOCK) {
        if (s->boundary != GS_BOUNDARY_PERIODIC)
            return fail(GS_EINVAL, "temporal blocking supports the periodic boundary only");
        ZPlan pl = s->tp;
        pl.tx = tile_x > 0 ? tile_x : 64;
        pl.ty = tile_y > 0 ? tile_y : 16;
        pl.tz = tile_z > 0 ? tile_z : 64;
        pl.depth = depth > 0 ? depth : 2;
        pl.stages = 5;
        int rc = tblock_validate(s->dtype, s->L, pl);
        if (rc) return rc;
        if (!zmarch_supported(s->dtype, s->L)) return fail(GS_EINVAL, "L=%d not supported by the z-march kernel", s->L);
        const int old_kernel = s->kernel;
        s->kernel = GS_KERNEL_TBLOCK;
        s->tp = pl;
        if (!s->maps_ok) {
            rc = encode_maps(s);
            if (rc) {
                s->kernel = old_kernel;
                return rc;
            }
        }
        return GS_OK;
    }
    return fail(GS_EINVAL, "kernel=%d not available", kernel);
}

int gs_set_plan(gs_sim* s, int kernel, int tile_x, int tile_y, int tile_z, int depth)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    const int rc = apply_plan(s, kernel, tile_x, tile_y, tile_z, depth, 0);
    if (!rc) s->plan_us = 0.0;
    return rc;
}

int gs_set_plan_full(gs_sim* s, const gs_plan* p)
{
    if (!s || !p) return fail(GS_EINVAL, "NULL argument");
    const int rc = apply_plan(s, p->kernel, p->tile_x, p->tile_y, p->tile_z, p->depth, p->stages);
    if (!rc) s->plan_us = 0.0;
    return rc;
}

static gs_plan current_plan(gs_sim* s)
{
    gs_plan p{};
    p.kernel = s->kernel;
    if (s->kernel == GS_KERNEL_ZMARCH) {
        p.tile_x = s->zp.tx; p.tile_y = s->zp.ty; p.tile_z = s->zp.tz; p.depth = 1; p.stages = s->zp.stages;
    } else if (s->kernel == GS_KERNEL_TBLOCK) {
        p.tile_x = s->tp.tx; p.tile_y = s->tp.ty; p.tile_z = s->tp.tz; p.depth = s->tp.depth; p.stages = s->tp.stages;
    } else {
        p.depth = 1;
    }
    return p;
}

int gs_autotune(gs_sim* s, int steps_per_trial, gs_plan* results, int max_results, int* n_results, gs_plan* best)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (steps_per_trial < 1) return fail(GS_EINVAL, "steps_per_trial must be >= 1");
    if (max_results < 0 || (max_results > 0 && !results)) return fail(GS_EINVAL, "bad results buffer");
    const int n = (steps_per_trial + 11) / 12 * 12;
    // candidate plans
    std::vector<gs_plan> cand;
    cand.push_back(gs_plan{GS_KERNEL_NAIVE, 0, 0, 0, 1, 0, 0.0});
    const int zt[][2] = {{128, 8}, {256, 4}, {64, 16}, {128, 4}, {64, 8}, {256, 8}, {128, 16}, {32, 16}, {128, 10},
                         {128, 12}, {256, 6}};
    for (auto& t : zt)
        for (int tz : {32, 64, 128})
            for (int st : {4, 6, 8}) cand.push_back(gs_plan{GS_KERNEL_ZMARCH, t[0], t[1], tz, 1, st, 0.0});
    const int bt[][2] = {{64, 16}, {128, 8}, {64, 8}, {32, 16}, {128, 4}, {32, 32}};
    for (int d = 2; d <= 4; ++d)
        for (auto& t : bt)
            for (int tz : {64, 128}) cand.push_back(gs_plan{GS_KERNEL_TBLOCK, t[0], t[1], tz, d, 5, 0.0});
    const int dtl[][2] = {{16, 8}, {16, 16}, {32, 8}};  // depths 5-8: small tiles (shared memory)
    for (int d = 5; d <= 8; ++d)
        for (auto& t : dtl)
            for (int tz : {64, 128}) cand.push_back(gs_plan{GS_KERNEL_TBLOCK, t[0], t[1], tz, d, 5, 0.0});
    // save the state
    const size_t bytes = (size_t)s->L * s->L * s->L * elem_size(s->dtype);
    const gs_plan saved_plan = current_plan(s);
    const int64_t t0 = s->t;
    const int cur0 = s->cur;
    void* bu = nullptr;
    void* bv = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GS_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&bu, bytes)) != cudaSuccess || (e = cudaMalloc(&bv, bytes)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        rc = cuda_fail(e, "autotune set-up");
    }
    if (!rc) {
        if ((e = cudaMemcpyAsync(bu, s->buf[cur0][0], bytes, cudaMemcpyDeviceToDevice, s->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(bv, s->buf[cur0][1], bytes, cudaMemcpyDeviceToDevice, s->stream)) != cudaSuccess)
            rc = cuda_fail(e, "autotune save");
    }
    gs_plan win{};
    win.us_per_step = -1.0;
    int count = 0;
    for (size_t i = 0; i < cand.size() && !rc; ++i) {
        gs_plan& c = cand[i];
        if (apply_plan(s, c.kernel, c.tile_x, c.tile_y, c.tile_z, c.depth, c.stages) != GS_OK) continue;
        c = current_plan(s);
        // a whole number of passes of this plan's depth
        const int nc = c.kernel == GS_KERNEL_TBLOCK ? (n + c.depth - 1) / c.depth * c.depth : n;
        int r = gs_step(s, c.kernel == GS_KERNEL_TBLOCK ? 2 * c.depth : 2);
        // a plan that validates but cannot be launched on this GPU (its block
        // does not fit an SM) is skipped; the state is restored at the end
        if (r == GS_EINVAL) continue;
        if (!r && (e = cudaEventRecord(e0, s->stream)) != cudaSuccess) r = cuda_fail(e, "event");
        if (!r) r = gs_step(s, nc);
        if (!r && (e = cudaEventRecord(e1, s->stream)) != cudaSuccess) r = cuda_fail(e, "event");
        if (!r) r = gs_sync(s);
        float ms = 0.f;
        if (!r && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) r = cuda_fail(e, "event");
        if (r) {
            rc = r;
            break;
        }
        c.us_per_step = 1e3 * ms / nc;
        if (results && count < max_results) results[count] = c;
        ++count;
        if (win.us_per_step < 0 || c.us_per_step < win.us_per_step) win = c;
    }
    // restore the state and keep the winner (or the previous plan on failure)
    if (bu && bv) {
        cudaMemcpyAsync(s->buf[cur0][0], bu, bytes, cudaMemcpyDeviceToDevice, s->stream);
        cudaMemcpyAsync(s->buf[cur0][1], bv, bytes, cudaMemcpyDeviceToDevice, s->stream);
        cudaStreamSynchronize(s->stream);
    }
    s->cur = cur0;
    s->t = t0;
    const gs_plan keep = (!rc && win.us_per_step >= 0) ? win : saved_plan;
    int rc2 = apply_plan(s, keep.kernel, keep.tile_x, keep.tile_y, keep.tile_z, keep.depth, keep.stages);
    if (!rc && !rc2) s->plan_us = keep.us_per_step;
    if (bu) cudaFree(bu);
    if (bv) cudaFree(bv);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    if (rc2) return rc2;
    if (n_results) *n_results = count;
    if (best) *best = keep;
    return GS_OK;
}

// Plan cache: one text line per tuned configuration,
//   gs-plan-v1 <key> <kernel> <tile_x> <tile_y> <tile_z> <depth> <stages> <us_per_step>
// with key = <device name>/sm<major><minor>/L<L>/<f32|f64>/<ieee|ds>/<periodic|held>/<noise|still>
// (spaces and '/' in the device name written as '_').
static int plan_key(gs_sim* s, char* key, size_t n)
{
    int dev = 0;
    GS_CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp pr;
    GS_CUDA_TRY(cudaGetDeviceProperties(&pr, dev));
    char name[sizeof(pr.name) + 1];
    size_t i = 0;
    for (; i < sizeof(pr.name) && pr.name[i]; ++i) name[i] = (pr.name[i] == ' ' || pr.name[i] == '/') ? '_' : pr.name[i];
    name[i] = 0;
    snprintf(key, n, "%s/sm%d%d/L%d/%s/%s/%s/%s", name, pr.major, pr.minor, s->L, s->dtype == GS_F32 ? "f32" : "f64",
             s->p.arith == GS_ARITH_DS ? "ds" : s->p.arith == GS_ARITH_FX ? "fx" : s->p.arith == GS_ARITH_FXF ? "fxf" : "ieee",
             s->boundary == GS_BOUNDARY_HELD ? "held" : "periodic",
             s->p.noise != 0.0 ? "noise" : "still");
    return GS_OK;
}

int gs_autotune_cached(gs_sim* s, int steps_per_trial, const char* path, gs_plan* best, int* hit)
{
    if (!s || !path) return fail(GS_EINVAL, "sim and path must not be NULL");
    if (steps_per_trial < 1) return fail(GS_EINVAL, "steps_per_trial must be >= 1");
    char key[512];
    int rc = plan_key(s, key, sizeof key);
    if (rc) return rc;
    // the last line with this key wins; lines that do not parse are skipped
    gs_plan found{};
    bool have = false;
    if (FILE* f = fopen(path, "r")) {
        char line[1024];
        while (fgets(line, sizeof line, f)) {
            char k[512];
            gs_plan q{};
            if (sscanf(line, "gs-plan-v1 %511s %d %d %d %d %d %d %lf", k, &q.kernel, &q.tile_x, &q.tile_y, &q.tile_z,
                       &q.depth, &q.stages, &q.us_per_step) == 8 &&
                strcmp(k, key) == 0) {
                found = q;
                have = true;
            }
        }
        fclose(f);
    }
    if (have) {
        const gs_plan before = current_plan(s);
        if (apply_plan(s, found.kernel, found.tile_x, found.tile_y, found.tile_z, found.depth, found.stages) == GS_OK) {
            s->plan_us = found.us_per_step;
            if (best) {
                *best = current_plan(s);
                best->us_per_step = found.us_per_step;
            }
            if (hit) *hit = 1;
            return GS_OK;
        }
        // a plan this build or GPU no longer accepts: tune afresh
        apply_plan(s, before.kernel, before.tile_x, before.tile_y, before.tile_z, before.depth, before.stages);
    }
    gs_plan b{};
    if ((rc = gs_autotune(s, steps_per_trial, nullptr, 0, nullptr, &b))) return rc;
    FILE* w = fopen(path, "a");
    if (!w) return fail(GS_EIO, "cannot append to the plan cache %s", path);
    const int n = fprintf(w, "gs-plan-v1 %s %d %d %d %d %d %d %.17g\n", key, b.kernel, b.tile_x, b.tile_y, b.tile_z,
                          b.depth, b.stages, b.us_per_step);
    if (fclose(w) != 0 || n < 0) return fail(GS_EIO, "writing the plan cache %s failed", path);
    if (best) *best = b;
    if (hit) *hit = 0;
    return GS_OK;
}

int gs_get_plan(gs_sim* s, int* kernel, int* tx, int* ty, int* tz, int* depth)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (kernel) *kernel = s->kernel;
    const bool z = s->kernel != GS_KERNEL_NAIVE;
    const ZPlan& pl = s->kernel == GS_KERNEL_TBLOCK ? s->tp : s->zp;
    if (tx) *tx = z ? pl.tx : 0;
    if (ty) *ty = z ? pl.ty : 0;
    if (tz) *tz = z ? pl.tz : 0;
    if (depth) *depth = z ? pl.depth : 1;
    return GS_OK;
}

int gs_set_boundary(gs_sim* s, int boundary)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (boundary != GS_BOUNDARY_PERIODIC && boundary != GS_BOUNDARY_HELD)
        return fail(GS_EINVAL, "boundary=%d must be GS_BOUNDARY_PERIODIC or GS_BOUNDARY_HELD", boundary);
    if (boundary == GS_BOUNDARY_HELD && s->kernel == GS_KERNEL_TBLOCK)
        return fail(GS_EINVAL, "temporal blocking supports the periodic boundary only; choose another plan first");
    s->boundary = boundary;
    return GS_OK;
}

int gs_set_arith(gs_sim* s, int arith)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (arith != GS_ARITH_IEEE && arith != GS_ARITH_DS && arith != GS_ARITH_FX && arith != GS_ARITH_FXF)
        return fail(GS_EINVAL, "arith=%d must be GS_ARITH_IEEE, GS_ARITH_DS, GS_ARITH_FX or GS_ARITH_FXF", arith);
    if (arith != GS_ARITH_IEEE && s->dtype != GS_F64)
        return fail(GS_EINVAL, "double-single and fixed-point arithmetic apply to FP64 fields only");
    s->p.arith = arith;
    return GS_OK;
}

int gs_get_arith(gs_sim* s, int* arith)
{
    if (!s || !arith) return fail(GS_EINVAL, "sim or arith is NULL");
    *arith = s->p.arith;
    return GS_OK;
}

int gs_get_boundary(gs_sim* s, int* boundary)
{
    if (!s || !boundary) return fail(GS_EINVAL, "sim or boundary is NULL");
    *boundary = s->boundary;
    return GS_OK;
}

int gs_get_plan_full(gs_sim* s, gs_plan* out)
{
    if (!s || !out) return fail(GS_EINVAL, "sim or out is NULL");
    *out = current_plan(s);
    out->us_per_step = s->plan_us;
    return GS_OK;
}

int gs_set_fault(gs_sim* s, int mode, uint64_t timeout_ns)
{
    if (!s) return fail(GS_EINVAL, "sim is NULL");
    if (mode != 0 && mode != 1) return fail(GS_EINVAL, "fault mode %d must be 0 or 1", mode);
    if (timeout_ns == 0) return fail(GS_EINVAL, "timeout_ns must be > 0");
    s->fault = mode;
    s->timeout_ns = timeout_ns;
    return GS_OK;
}

int gs_launch_count(gs_sim* s, int64_t* count)
{
    if (!s || !count) return fail(GS_EINVAL, "NULL argument");
    *count = s->launches;
    return GS_OK;
}

int gs_destroy(gs_sim* s)
{
    if (!s) return GS_OK;
    if (s->owns)
        for (int set = 0; set < 2; ++set)
            for (int f = 0; f < 2; ++f)
                if (s->buf[set][f]) cudaFree(s->buf[set][f]);
    if (s->d_err) cudaFree(s->d_err);
    delete s;
    return GS_OK;
}

int gs_noise_field(uint64_t seed, int64_t t, int64_t n, int dtype, void* dev_out, void* stream)
{
    if (n < 0) return fail(GS_EINVAL, "n must be >= 0");
    if (dtype != GS_F32 && dtype != GS_F64) return fail(GS_EINVAL, "dtype=%d must be GS_F32 or GS_F64", dtype);
    if (n > 0 && !dev_out) return fail(GS_EINVAL, "dev_out is NULL");
    return launch_noise_field(dtype, seed, t, n, dev_out, (cudaStream_t)stream);
}

}  // extern "C"

extern "C" int gs_set_alloc_guard(size_t bytes)
{
    if (bytes % 256) return fail(GS_EINVAL, "guard bytes=%zu must be a multiple of 256", bytes);
    std::lock_guard<std::mutex> lk(g_guard_mutex);
    g_guard_bytes = bytes;
    return GS_OK;
}
