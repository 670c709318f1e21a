// FP64 pipe throughput (a measurement aid, not part of the method): the
// denominator of the FP64 stencil's ALU roofline.  Each thread runs eight
// independent chains of fused multiply-adds a = a * b + c, so the FP64 pipe,
// not the instruction latency, sets the rate; the chains stay finite
// (|b| < 1) and their sum is stored only under a condition that never holds,
// which keeps them alive without a memory write per thread.
#include <algorithm>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {

constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(256) gs_dfma_rate_kernel(double* __restrict__ sink, int iters, double b, double c)
{
    double a[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) a[j] = 1e-3 * (threadIdx.x + 1) + j;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < kPeakChains; ++j) a[j] = __fma_rn(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += a[j];
    if (s == -1.0) sink[0] = s;  // the chains are positive: never taken
}

}  // namespace gs

using namespace gs;

extern "C" int gs_measure_fp64_fma(void* stream, double* fma_per_s)
{
    if (!fma_per_s) return fail(GS_EINVAL, "fma_per_s is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    double* sink = nullptr;
    GS_CUDA_TRY(cudaMalloc(&sink, sizeof(double)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = num_sms() * 8, threads = 256, iters = 2048;
    const double fmas = (double)blocks * threads * iters * 4 * kPeakChains;
    float best = 0.f;
    int rc = GS_OK;
    for (int rep = 0; rep < 4 && rc == GS_OK; ++rep) {  // the first is a warm-up
        cudaEventRecord(e0, s);
        gs_dfma_rate_kernel<<<blocks, threads, 0, s>>>(sink, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "FP64 rate kernel");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc) return rc;
    *fma_per_s = fmas / (best * 1e-3);
    return GS_OK;
}
