// Host-side declarations shared by the libgs translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/gs.h"

namespace gs {

// Model parameters in double; each kernel converts to its own type once.
struct Params {
    double Du, Dv, F, k, dt, noise;
    uint64_t seed;
    int arith = GS_ARITH_IEEE;  // GS_ARITH_DS: FP64 fields in double-single arithmetic
    // FP64 fields in GS_ARITH_DS, _FX or _FXF: bit 0 = the input fields hold
    // that arithmetic's packed values instead of FP64 values, bit 1 = write
    // packed values (the steps inside one gs_step call keep the fields
    // packed; the call's first step reads FP64 and its last writes FP64)
    int io = 0;
};

// Thread-local error message + status helper.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
#define GS_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return ::gs::cuda_fail(_e, #expr); \
    } while (0)

int elem_size(int dtype);
int num_sms();

// Library-owned device allocations that honour the guard-band checking aid
// (gs_set_alloc_guard): with a guard of G bytes the buffer sits between two
// G-byte bands of 0xFF bytes (and its own bytes start as 0xFF too).
cudaError_t guarded_malloc(void** p, size_t bytes);
void guarded_free(void* p);
// guard bytes of p that no longer hold 0xFF (0 for an unguarded buffer);
// -1 if the check itself failed
int64_t guarded_check(const void* p);

// Tensor-map encoder obtained from the driver at first use.
CUresult encode_tiled_3d(CUtensorMap* map, int dtype, void* base, int L, int box_x, int box_y);
// channels-last bf16 activations [planes][L][L][C] (planes = N * L): boxes of
// box_c channels x box_x cells x 1 row x 1 plane, with the 32- or 64-byte
// swizzle (swizzle = 32: box_c = 16; 64: box_c = 32) or none (0)
CUresult encode_act_4d(CUtensorMap* map, const void* base, int C, int L, long long planes, int box_c, int box_x,
                       int swizzle);

// ---------------------------------------------------------------------------
// Stencil kernels (gs_stencil.cu)
// ---------------------------------------------------------------------------
int launch_init(int dtype, int L, void* u, void* v, cudaStream_t s);
int launch_noise_field(int dtype, uint64_t seed, int64_t t, int64_t n, void* out, cudaStream_t s);
int launch_naive(int dtype, int L, const void* u, const void* v, void* un, void* vn,
                 const Params& p, int64_t t, int* err, cudaStream_t s);

// Three tensor maps per field for the z-marching kernels (main tile, one
// halo row, one halo column block), for the two fields u, v.
struct ZMaps {
    CUtensorMap m[2][3];
};

struct ZPlan {
    int tx, ty, tz;   // tile in cells
    int stages;       // TMA ring depth
    int depth;        // fused steps per pass (1 = plain z-march)
};

bool zmarch_supported(int dtype, int L);
int zmarch_validate(int dtype, int L, const ZPlan& pl);
int zmarch_encode(int dtype, int L, const ZPlan& pl, void* u, void* v, ZMaps* maps);
// tickets: two zeroed words of device memory the launch leaves zeroed (the
// CTAs take work units from it as they become free), or null for a static
// round robin
int launch_zmarch(int dtype, int L, const ZPlan& pl, const ZMaps& maps, void* un, void* vn,
                  const Params& p, int64_t t, int* d_err, uint64_t timeout_ns, int stall,
                  unsigned* tickets, cudaStream_t s);

// Held outer layer (gs_variants.cu): copy the six faces of the input state
// over the output state (iv/ov may be NULL for one field).
int launch_hold_faces(int dtype, int L, const void* iu, const void* iv, void* ou, void* ov, cudaStream_t s);

// Temporally blocked kernel (gs_tblock.cu): `depth` steps per pass, FP32.
int tblock_validate(int dtype, int L, const ZPlan& pl);
// tickets: as for launch_zmarch (the same two words serve both kernels)
int launch_tblock(int L, const ZPlan& pl, const void* u, const void* v, void* un, void* vn, const Params& p,
                  int64_t t, unsigned* tickets, cudaStream_t s);

}  // namespace gs

// The single-grid simulation object (gs_api.cu owns its life cycle; the
// output stage in gs_io.cu reads its fields and stream).
struct gs_sim {
    using Params = gs::Params;
    using ZPlan = gs::ZPlan;
    using ZMaps = gs::ZMaps;
    int L = 0;
    int dtype = GS_F32;
    Params p{};
    void* buf[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [set][field]
    bool owns = false;
    int cur = 0;       // set holding the current state
    int64_t t = 0;     // step counter
    cudaStream_t stream = nullptr;
    int* d_err = nullptr;  // 4 words: the error word, a pad word, the z-march kernel's two ticket words
    int kernel = GS_KERNEL_NAIVE;
    ZPlan zp{128, 8, 32, 4, 1};   // z-march plan (also runs the steps a blocked pass leaves over)
    ZPlan tp{64, 16, 64, 5, 2};   // temporal-blocking plan (kernel GS_KERNEL_TBLOCK)
    ZMaps maps[2];     // tensor maps reading set 0 / set 1
    bool maps_ok = false;
    int64_t launches = 0;
    uint64_t timeout_ns = 2000000000ull;
    int fault = 0;
    double plan_us = 0.0;  // the tuner's time for the current plan (0: set by hand)
    int boundary = GS_BOUNDARY_PERIODIC;  // or GS_BOUNDARY_HELD (gs_set_boundary)
};
