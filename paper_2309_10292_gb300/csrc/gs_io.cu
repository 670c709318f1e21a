// Output stage of the workflow: field statistics and slices, a snapshot
// writer that overlaps with the stencil, and checkpoints.
//
// The paper stores U and V every few steps together with a provenance
// record of the run's parameters and each field's minimum and maximum
// (Section 3.4, Listing 1; ADIOS2 BP files on Lustre, Section 5.3).  Here a
// snapshot is a device-to-device copy of the state on the simulation's
// stream (so the stencil may overwrite its buffers right away), then, on a
// separate copy stream, a min/max/sum reduction and a device-to-host copy
// into one of two pinned host slots, and finally a native writer thread
// appends the record to a single self-describing file.
//
// File layout (little-endian):
//   header  : 8-byte magic ("GSSNAP01", or "GSCKPT01" for a checkpoint),
//             uint32 n, n bytes of JSON provenance (L, dtype, layout, the
//             model parameters Du, Dv, F, k, dt, noise, seed, boundary)
//   record  : 8-byte magic "GSREC001", int64 step, 4 x float64 (U min,
//             U max, V min, V max), U then V (L^3 elements each, [z][y][x],
//             x fastest, in the simulation's dtype)
#include <condition_variable>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gs_internal.h"

namespace gs {

// ---------------------------------------------------------------------------
// Reductions: min, max, sum, sum of squares, NaN count (FP64 accumulation)
// ---------------------------------------------------------------------------
constexpr int kStatThreads = 256;
constexpr int kStatVals = 5;

struct StatAcc {
    double mn, mx, s, s2, nan;
};

__device__ __forceinline__ void stat_merge(StatAcc& a, const StatAcc& b)
{
    a.mn = fmin(a.mn, b.mn);
    a.mx = fmax(a.mx, b.mx);
    a.s += b.s;
    a.s2 += b.s2;
    a.nan += b.nan;
}

__device__ __forceinline__ StatAcc stat_block_reduce(StatAcc a)
{
    __shared__ double red[kStatThreads / 32][kStatVals];
    for (int o = 16; o > 0; o >>= 1) {
        StatAcc b;
        b.mn = __shfl_xor_sync(0xffffffffu, a.mn, o);
        b.mx = __shfl_xor_sync(0xffffffffu, a.mx, o);
        b.s = __shfl_xor_sync(0xffffffffu, a.s, o);
        b.s2 = __shfl_xor_sync(0xffffffffu, a.s2, o);
        b.nan = __shfl_xor_sync(0xffffffffu, a.nan, o);
        stat_merge(a, b);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[w][0] = a.mn;
        red[w][1] = a.mx;
        red[w][2] = a.s;
        red[w][3] = a.s2;
        red[w][4] = a.nan;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kStatThreads / 32; ++i) stat_merge(a, StatAcc{red[i][0], red[i][1], red[i][2], red[i][3], red[i][4]});
    }
    return a;
}

template <typename T>
__global__ void __launch_bounds__(kStatThreads) gs_stats_partial_kernel(const T* __restrict__ f, long long n,
                                                                        double* __restrict__ partial)
{
    StatAcc a{INFINITY, -INFINITY, 0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = (double)f[i];
        if (isnan(x)) {
            a.nan += 1.0;
        } else {
            a.mn = fmin(a.mn, x);
            a.mx = fmax(a.mx, x);
            a.s += x;
            a.s2 += x * x;
        }
    }
    a = stat_block_reduce(a);
    if (threadIdx.x == 0) {
        double* p = partial + (size_t)blockIdx.x * kStatVals;
        p[0] = a.mn;
        p[1] = a.mx;
        p[2] = a.s;
        p[3] = a.s2;
        p[4] = a.nan;
    }
}

__global__ void __launch_bounds__(kStatThreads) gs_stats_final_kernel(const double* __restrict__ partial, int nblocks,
                                                                      double* __restrict__ out)
{
    StatAcc a{INFINITY, -INFINITY, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double* p = partial + (size_t)b * kStatVals;
        stat_merge(a, StatAcc{p[0], p[1], p[2], p[3], p[4]});
    }
    a = stat_block_reduce(a);
    if (threadIdx.x == 0) {
        out[0] = a.mn;
        out[1] = a.mx;
        out[2] = a.s;
        out[3] = a.s2;
        out[4] = a.nan;
    }
}

static int stats_blocks() { return 4 * num_sms(); }

// Enqueue the reduction of n elements of `f` into out[5] (device) on stream s.
static int launch_stats(int dtype, const void* f, long long n, double* partial, double* out, cudaStream_t s)
{
    const int nb = stats_blocks();
    if (dtype == GS_F32)
        gs_stats_partial_kernel<float><<<nb, kStatThreads, 0, s>>>((const float*)f, n, partial);
    else
        gs_stats_partial_kernel<double><<<nb, kStatThreads, 0, s>>>((const double*)f, n, partial);
    GS_CUDA_TRY(cudaGetLastError());
    gs_stats_final_kernel<<<1, kStatThreads, 0, s>>>(partial, nb, out);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------------------
// Provenance header
// ---------------------------------------------------------------------------
static std::string provenance_json(const gs_sim* s)
{
    char buf[1024];
    std::snprintf(buf, sizeof buf,
                  "{\"format\": \"gs-snapshot\", \"version\": 1, \"L\": %d, \"dtype\": \"%s\", "
                  "\"layout\": \"[z][y][x], x fastest, little-endian\", \"boundary\": \"%s\", "
                  "\"Du\": %.17g, \"Dv\": %.17g, \"F\": %.17g, \"k\": %.17g, \"dt\": %.17g, \"noise\": %.17g, "
                  "\"seed\": %llu, \"arithmetic\": \"%s\", \"variables\": [\"U\", \"V\"], "
                  "\"record\": \"GSREC001, int64 step, float64 Umin Umax Vmin Vmax, U, V\"}",
                  s->L, s->dtype == GS_F32 ? "f32" : "f64", s->boundary == GS_BOUNDARY_HELD ? "held" : "periodic",
                  s->p.Du, s->p.Dv, s->p.F, s->p.k, s->p.dt, s->p.noise, (unsigned long long)s->p.seed,
                  s->p.arith == GS_ARITH_DS    ? "double-single"
                  : s->p.arith == GS_ARITH_FX  ? "fixed-point"
                  : s->p.arith == GS_ARITH_FXF ? "fixed-point-remainder"
                                               : "ieee");
    return buf;
}

static bool write_header(FILE* f, const char* magic, const std::string& json)
{
    const uint32_t n = (uint32_t)json.size();
    return std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&n, sizeof n, 1, f) == 1 &&
           std::fwrite(json.data(), 1, n, f) == n;
}

static bool write_record(FILE* f, int64_t step, const double mm[4], const void* u, const void* v, size_t bytes)
{
    return std::fwrite("GSREC001", 1, 8, f) == 8 && std::fwrite(&step, sizeof step, 1, f) == 1 &&
           std::fwrite(mm, sizeof(double), 4, f) == 4 && std::fwrite(u, 1, bytes, f) == bytes &&
           std::fwrite(v, 1, bytes, f) == bytes;
}

// value of "key" in our own JSON header (numbers only)
static bool json_number(const std::string& js, const char* key, double* out)
{
    const std::string k = std::string("\"") + key + "\": ";
    const size_t at = js.find(k);
    if (at == std::string::npos) return false;
    char* end = nullptr;
    const double v = std::strtod(js.c_str() + at + k.size(), &end);
    if (end == js.c_str() + at + k.size()) return false;
    *out = v;
    return true;
}

// value of "key" as an unsigned 64-bit integer (exact, for the seed)
static bool json_u64(const std::string& js, const char* key, uint64_t* out)
{
    const std::string k = std::string("\"") + key + "\": ";
    const size_t at = js.find(k);
    if (at == std::string::npos) return false;
    char* end = nullptr;
    const unsigned long long v = std::strtoull(js.c_str() + at + k.size(), &end, 10);
    if (end == js.c_str() + at + k.size()) return false;
    *out = (uint64_t)v;
    return true;
}

}  // namespace gs

using namespace gs;

// ---------------------------------------------------------------------------
// Statistics and slices
// ---------------------------------------------------------------------------
int gs_stats(gs_sim* s, int field, double* out, int64_t* nan_count)
{
    if (!s || !out) return fail(GS_EINVAL, "sim or out is NULL");
    if (field != GS_U && field != GS_V) return fail(GS_EINVAL, "field=%d must be GS_U or GS_V", field);
    const long long n = (long long)s->L * s->L * s->L;
    double* d = nullptr;
    const size_t nbytes = ((size_t)stats_blocks() * kStatVals + kStatVals) * sizeof(double);
    GS_CUDA_TRY(cudaMallocAsync((void**)&d, nbytes, s->stream));
    int rc = launch_stats(s->dtype, s->buf[s->cur][field], n, d + kStatVals, d, s->stream);
    double h[kStatVals] = {};
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(d, s->stream);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "gs_stats");
    s->launches += 2;
    const double valid = (double)n - h[4];
    out[0] = h[0];
    out[1] = h[1];
    out[2] = valid > 0 ? h[2] / valid : NAN;
    out[3] = valid > 0 ? std::sqrt(h[3] / valid) : NAN;
    if (nan_count) *nan_count = (int64_t)h[4];
    return GS_OK;
}

int gs_slice(gs_sim* s, int field, int axis, int index, void* dst, size_t bytes)
{
    if (!s || !dst) return fail(GS_EINVAL, "sim or dst is NULL");
    if (field != GS_U && field != GS_V) return fail(GS_EINVAL, "field=%d must be GS_U or GS_V", field);
    if (axis < 0 || axis > 2) return fail(GS_EINVAL, "axis=%d must be 0 (x), 1 (y) or 2 (z)", axis);
    if (index < 0 || index >= s->L) return fail(GS_EINVAL, "index=%d outside [0, %d)", index, s->L);
    const size_t esz = elem_size(s->dtype), L = (size_t)s->L;
    if (bytes != L * L * esz) return fail(GS_EINVAL, "bytes=%zu, expected L*L*%zu=%zu", bytes, esz, L * L * esz);
    const char* f = (const char*)s->buf[s->cur][field];
    cudaError_t e;
    if (axis == 2)  // plane z = index: contiguous [y][x]
        e = cudaMemcpyAsync(dst, f + (size_t)index * L * L * esz, bytes, cudaMemcpyDeviceToHost, s->stream);
    else if (axis == 1)  // [z][x]: one row of L elements per z
        e = cudaMemcpy2DAsync(dst, L * esz, f + (size_t)index * L * esz, L * L * esz, L * esz, L,
                              cudaMemcpyDeviceToHost, s->stream);
    else  // [z][y]: one element per row
        e = cudaMemcpy2DAsync(dst, esz, f + (size_t)index * esz, L * esz, esz, L * L, cudaMemcpyDeviceToHost,
                              s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gs_slice");
    return GS_OK;
}

// ---------------------------------------------------------------------------
// Snapshot writer
// ---------------------------------------------------------------------------
struct gs_snap {
    gs_sim* sim = nullptr;
    FILE* file = nullptr;
    size_t field_bytes = 0;
    void* staging[2] = {nullptr, nullptr};          // device copy of U, V
    void* pinned[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [slot][field]
    double* d_red = nullptr;                        // partials + 2 x 5 results (device)
    double* h_stats[2] = {nullptr, nullptr};        // [slot] 10 values (pinned)
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_state = nullptr;                 // state copied to staging (sim stream)
    cudaEvent_t ev_staging_free = nullptr;          // staging read by the last copy (copy stream)
    cudaEvent_t ev_slot[2] = {nullptr, nullptr};    // slot filled (copy stream)
    std::thread writer;
    std::mutex m;
    std::condition_variable cv;
    struct Job {
        int slot;
        int64_t step;
    };
    std::deque<Job> queue;
    bool slot_busy[2] = {false, false};
    int next_slot = 0;
    bool stop = false;
    bool writing = false;
    int error = GS_OK;
    std::string error_msg;
    int64_t written = 0;
    double bytes = 0.0;
};

static void snap_writer_loop(gs_snap* w)
{
    for (;;) {
        gs_snap::Job job;
        {
            std::unique_lock<std::mutex> lk(w->m);
            w->cv.wait(lk, [&] { return w->stop || !w->queue.empty(); });
            if (w->queue.empty()) return;  // stop requested and nothing left
            job = w->queue.front();
            w->queue.pop_front();
            w->writing = true;
        }
        int err = GS_OK;
        std::string msg;
        const cudaError_t e = cudaEventSynchronize(w->ev_slot[job.slot]);
        if (e != cudaSuccess) {
            err = GS_ECUDA;
            msg = std::string("snapshot copy failed: ") + cudaGetErrorString(e);
        } else {
            const double* st = w->h_stats[job.slot];
            const double mm[4] = {st[0], st[1], st[5], st[6]};
            if (!write_record(w->file, job.step, mm, w->pinned[job.slot][0], w->pinned[job.slot][1], w->field_bytes)) {
                err = GS_EIO;
                msg = "snapshot write failed (disk full?)";
            }
        }
        {
            std::lock_guard<std::mutex> lk(w->m);
            w->slot_busy[job.slot] = false;
            w->writing = false;
            if (err && !w->error) {
                w->error = err;
                w->error_msg = msg;
            }
            if (!err) {
                w->written += 1;
                w->bytes += 2.0 * (double)w->field_bytes + 48.0;
            }
        }
        w->cv.notify_all();
    }
}

static void snap_free(gs_snap* w)
{
    if (w->writer.joinable()) {
        {
            std::lock_guard<std::mutex> lk(w->m);
            w->stop = true;
        }
        w->cv.notify_all();
        w->writer.join();
    }
    if (w->copy) cudaStreamSynchronize(w->copy);
    for (int i = 0; i < 2; ++i) {
        if (w->staging[i]) cudaFree(w->staging[i]);
        for (int j = 0; j < 2; ++j)
            if (w->pinned[i][j]) cudaFreeHost(w->pinned[i][j]);
        if (w->h_stats[i]) cudaFreeHost(w->h_stats[i]);
        if (w->ev_slot[i]) cudaEventDestroy(w->ev_slot[i]);
    }
    if (w->d_red) cudaFree(w->d_red);
    if (w->ev_state) cudaEventDestroy(w->ev_state);
    if (w->ev_staging_free) cudaEventDestroy(w->ev_staging_free);
    if (w->copy) cudaStreamDestroy(w->copy);
    if (w->file) std::fclose(w->file);
    delete w;
}

int gs_snap_open(gs_sim* s, const char* path, gs_snap** out)
{
    if (!s || !path || !out) return fail(GS_EINVAL, "NULL argument");
    *out = nullptr;
    gs_snap* w = new gs_snap();
    w->sim = s;
    w->field_bytes = (size_t)s->L * s->L * s->L * elem_size(s->dtype);
    w->file = std::fopen(path, "wb");
    if (!w->file) {
        delete w;
        return fail(GS_EIO, "cannot open %s for writing", path);
    }
    if (!write_header(w->file, "GSSNAP01", provenance_json(s))) {
        snap_free(w);
        return fail(GS_EIO, "cannot write the header of %s", path);
    }
    cudaError_t e = cudaSuccess;
    const size_t red = ((size_t)stats_blocks() * kStatVals + 2 * kStatVals) * sizeof(double);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMalloc(&w->staging[i], w->field_bytes);
        for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaMallocHost(&w->pinned[i][j], w->field_bytes);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&w->h_stats[i], 2 * kStatVals * sizeof(double));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->ev_slot[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&w->d_red, red);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->ev_state, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->ev_staging_free, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(w->ev_staging_free, w->copy);
    if (e != cudaSuccess) {
        snap_free(w);
        return e == cudaErrorMemoryAllocation ? fail(GS_ENOMEM, "snapshot buffers: %s", cudaGetErrorString(e))
                                              : cuda_fail(e, "gs_snap_open");
    }
    w->writer = std::thread(snap_writer_loop, w);
    *out = w;
    return GS_OK;
}

int gs_snap_write(gs_snap* w)
{
    if (!w) return fail(GS_EINVAL, "snap is NULL");
    gs_sim* s = w->sim;
    int slot;
    {
        // a free pinned slot (the writer thread releases them)
        std::unique_lock<std::mutex> lk(w->m);
        if (w->error) return fail(w->error, "%s", w->error_msg.c_str());
        slot = w->next_slot;
        w->cv.wait(lk, [&] { return !w->slot_busy[slot] || w->error; });
        if (w->error) return fail(w->error, "%s", w->error_msg.c_str());
        w->slot_busy[slot] = true;
        w->next_slot ^= 1;
    }
    const int64_t step = s->t;
    cudaError_t e;
    // 1. on the simulation's stream: state -> staging (once the previous
    //    snapshot has left the staging buffer)
    e = cudaStreamWaitEvent(s->stream, w->ev_staging_free, 0);
    for (int f = 0; f < 2 && e == cudaSuccess; ++f)
        e = cudaMemcpyAsync(w->staging[f], s->buf[s->cur][f], w->field_bytes, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(w->ev_state, s->stream);
    // 2. on the copy stream: statistics, staging -> pinned slot
    if (e == cudaSuccess) e = cudaStreamWaitEvent(w->copy, w->ev_state, 0);
    int rc = GS_OK;
    const long long n = (long long)s->L * s->L * s->L;
    double* res = w->d_red + (size_t)stats_blocks() * kStatVals;
    for (int f = 0; f < 2 && e == cudaSuccess && !rc; ++f)
        rc = launch_stats(s->dtype, w->staging[f], n, w->d_red, res + f * kStatVals, w->copy);
    for (int f = 0; f < 2 && e == cudaSuccess && !rc; ++f)
        e = cudaMemcpyAsync(w->pinned[slot][f], w->staging[f], w->field_bytes, cudaMemcpyDeviceToHost, w->copy);
    if (e == cudaSuccess && !rc)
        e = cudaMemcpyAsync(w->h_stats[slot], res, 2 * kStatVals * sizeof(double), cudaMemcpyDeviceToHost, w->copy);
    if (e == cudaSuccess && !rc) e = cudaEventRecord(w->ev_staging_free, w->copy);
    if (e == cudaSuccess && !rc) e = cudaEventRecord(w->ev_slot[slot], w->copy);
    if (e != cudaSuccess || rc) {
        std::lock_guard<std::mutex> lk(w->m);
        w->slot_busy[slot] = false;
        return rc ? rc : cuda_fail(e, "gs_snap_write");
    }
    s->launches += 4;
    {
        std::lock_guard<std::mutex> lk(w->m);
        w->queue.push_back(gs_snap::Job{slot, step});
    }
    w->cv.notify_all();
    return GS_OK;
}

int gs_snap_flush(gs_snap* w)
{
    if (!w) return fail(GS_EINVAL, "snap is NULL");
    std::unique_lock<std::mutex> lk(w->m);
    w->cv.wait(lk, [&] { return (w->queue.empty() && !w->writing) || w->error; });
    if (w->error) return fail(w->error, "%s", w->error_msg.c_str());
    if (std::fflush(w->file) != 0) return fail(GS_EIO, "snapshot flush failed");
    return GS_OK;
}

int gs_snap_info(gs_snap* w, int64_t* records, double* bytes)
{
    if (!w) return fail(GS_EINVAL, "snap is NULL");
    std::lock_guard<std::mutex> lk(w->m);
    if (records) *records = w->written;
    if (bytes) *bytes = w->bytes;
    return GS_OK;
}

int gs_snap_close(gs_snap* w)
{
    if (!w) return GS_OK;
    const int rc = gs_snap_flush(w);
    snap_free(w);
    return rc;
}

// ---------------------------------------------------------------------------
// Checkpoints
// ---------------------------------------------------------------------------
int gs_checkpoint_save(gs_sim* s, const char* path)
{
    if (!s || !path) return fail(GS_EINVAL, "NULL argument");
    const size_t bytes = (size_t)s->L * s->L * s->L * elem_size(s->dtype);
    std::vector<char> u(bytes), v(bytes);
    int rc = gs_read(s, GS_U, u.data(), bytes);
    if (!rc) rc = gs_read(s, GS_V, v.data(), bytes);
    if (rc) return rc;
    double su[4], sv[4];
    if ((rc = gs_stats(s, GS_U, su, nullptr)) || (rc = gs_stats(s, GS_V, sv, nullptr))) return rc;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(GS_EIO, "cannot open %s for writing", path);
    const double mm[4] = {su[0], su[1], sv[0], sv[1]};
    const bool ok = write_header(f, "GSCKPT01", provenance_json(s)) && write_record(f, s->t, mm, u.data(), v.data(), bytes);
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) return fail(GS_EIO, "cannot write checkpoint %s", path);
    return GS_OK;
}

int gs_checkpoint_load(gs_sim* s, const char* path)
{
    if (!s || !path) return fail(GS_EINVAL, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(GS_EIO, "cannot open %s", path);
    char magic[8];
    uint32_t n = 0;
    int rc = GS_OK;
    std::string js;
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, "GSCKPT01", 8) != 0 || std::fread(&n, sizeof n, 1, f) != 1 ||
        n > (1u << 20)) {
        rc = fail(GS_EINVAL, "%s is not a checkpoint", path);
    } else {
        js.resize(n);
        if (std::fread(&js[0], 1, n, f) != n) rc = fail(GS_EIO, "truncated checkpoint header in %s", path);
    }
    if (!rc) {
        // the checkpoint must describe this simulation
        double L = 0;
        const bool dt32 = js.find("\"dtype\": \"f32\"") != std::string::npos;
        if (!json_number(js, "L", &L) || (int)L != s->L || dt32 != (s->dtype == GS_F32))
            rc = fail(GS_EINVAL, "checkpoint %s holds another grid (L or dtype differ)", path);
        const char* keys[6] = {"Du", "Dv", "F", "k", "dt", "noise"};
        const double mine[6] = {s->p.Du, s->p.Dv, s->p.F, s->p.k, s->p.dt, s->p.noise};
        for (int i = 0; i < 6 && !rc; ++i) {
            double x;
            if (!json_number(js, keys[i], &x) || x != mine[i])
                rc = fail(GS_EINVAL, "checkpoint %s was written with %s=%g (this run: %g)", path, keys[i], x, mine[i]);
        }
        uint64_t seed = 0;
        if (!rc && (!json_u64(js, "seed", &seed) || seed != s->p.seed))
            rc = fail(GS_EINVAL, "checkpoint %s was written with another seed", path);
    }
    const size_t bytes = (size_t)s->L * s->L * s->L * elem_size(s->dtype);
    std::vector<char> u, v;
    int64_t step = 0;
    if (!rc) {
        double mm[4];
        u.resize(bytes);
        v.resize(bytes);
        if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, "GSREC001", 8) != 0 ||
            std::fread(&step, sizeof step, 1, f) != 1 || std::fread(mm, sizeof(double), 4, f) != 4 ||
            std::fread(u.data(), 1, bytes, f) != bytes || std::fread(v.data(), 1, bytes, f) != bytes)
            rc = fail(GS_EIO, "truncated checkpoint record in %s", path);
    }
    std::fclose(f);
    if (rc) return rc;
    if ((rc = gs_write(s, GS_U, u.data(), bytes)) || (rc = gs_write(s, GS_V, v.data(), bytes))) return rc;
    return gs_set_step(s, step);
}
