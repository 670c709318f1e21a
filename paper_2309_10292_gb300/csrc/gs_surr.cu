// Learned surrogate of the Gray-Scott stencil (not in the paper): a 6-layer
// 3D residual convolution network advancing (u, v) by K = 16 steps.
//
//   x0  = bf16(u - 1, v, 20 F, 20 k)             4 channels (padded to 16)
//   h1  = relu(conv0(x0))                        4 -> 32
//   h_l = h_{l-1} + relu(conv_l(h_{l-1}))        32 -> 32, l = 2..5
//   out = (u, v) + conv5(h5)                     32 -> 2 (padded to 8)
//
// conv = circular 3x3x3 convolution with bias, weights [tap][Cin][Cout],
// tap = 9 (dz+1) + 3 (dy+1) + (dx+1).  Activations are bf16, channels-last
// [n][z][y][x][c]; every contraction runs on the tensor cores (bf16 x bf16 ->
// fp32, mma.sync m16n8k16) as an implicit GEMM over M = cells, N = output
// channels, K = 27 taps x input channels:
//
//   gs_conv_kernel    forward (epilogues: first / residual hidden / final
//                     state update) and data gradient (the same convolution
//                     with tap-flipped, transposed weights; epilogue adds the
//                     residual-path gradient and applies the ReLU mask of the
//                     layer below)
//   gs_wgrad_kernel   weight gradient: per tap, [Cin x cells] x [cells x Cout]
//   + packing, bias-gradient, MSE-loss, Adam and weight-layout kernels.
//
// A CTA stages 4 output rows (y0..y0+3) of a 128-cell x segment: 6 x 3 input
// rows with a one-cell periodic halo, and the layer's weights, in shared
// memory with a 16-byte XOR swizzle so every ldmatrix is conflict-free.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {

typedef __nv_bfloat16 bf16;

constexpr int kSurrLayers = 6;
constexpr int kChan[kSurrLayers + 1] = {4, 32, 32, 32, 32, 32, 2};
constexpr int kCinP[kSurrLayers] = {16, 32, 32, 32, 32, 32};
constexpr int kCoutP[kSurrLayers] = {32, 32, 32, 32, 32, 8};
constexpr float kFkScale = 20.f;
constexpr int kRows = 4;          // output rows per CTA work item
constexpr int kConvThreads = 512; // 16 warps: 4 rows x 4 segments of 32 cells

enum { EPI_FIRST = 0, EPI_HIDDEN = 1, EPI_LAST = 2, EPI_DGRAD = 3 };

// byte offset of 16-byte chunk j of row `r` in a swizzled [rows][nch * 16 B] buffer
GS_D uint32_t swz(int r, int j, int nch)
{
    const int x = nch >= 4 ? ((r >> 1) & 3) : (nch == 2 ? ((r >> 2) & 1) : 0);
    return (uint32_t)(r * nch * 16 + ((j ^ x) * 16));
}

GS_D void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
GS_D void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
GS_D void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
GS_D void ldsm_x2_t(uint32_t addr, uint32_t& r0, uint32_t& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
GS_D void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
GS_D void cp16(uint32_t smem, const void* g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(g) : "memory");
}
GS_D void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct ConvArgs {
    const bf16* in;     // [N][L^3][CINP]
    const bf16* w;      // [27][COUTP][CINP] (n-major rows of k)
    const float* bias;  // [COUTP] or null
    int N, L;
    const bf16* res;    // EPI_HIDDEN: residual h_in [..][32]
    bf16* out;          // EPI_FIRST / EPI_HIDDEN: h_out [..][32]
    uint32_t* zmask;    // forward (training): ReLU mask, bit c = (pre-activation c > 0), one word a cell (or null)
    const float* su;    // EPI_LAST: state in, u and v planes [N][L^3]
    const float* sv;
    float* ou;          // EPI_LAST: state out
    float* ov;
    bf16* gh;           // EPI_DGRAD: residual-path gradient [..][32], bf16, in / out
    int gh_acc;         // EPI_DGRAD: 1 -> gh += acc, 0 -> gh = acc
    const uint32_t* mprev;  // EPI_DGRAD: ReLU mask words of the layer below
    bf16* gz;           // EPI_DGRAD: gz = gh * mask
};

// Work item: (n, z, y-group of 4 rows, x segment).
template <int CINP, int COUTP, int EPI>
__global__ void __launch_bounds__(kConvThreads, 1) gs_conv_kernel(const ConvArgs a)
{
    constexpr int NCH = CINP / 8;  // 16-byte chunks per input cell
    constexpr int NT = COUTP / 8;  // n8 tiles
    extern __shared__ __align__(128) unsigned char smem[];
    const int L = a.L;
    const int SEG = L < 128 ? L : 128;
    const int HC = SEG + 2;
    const int nseg = L / SEG;
    const long long L3 = (long long)L * L * L;
    unsigned char* wsm = smem;                                      // weights
    unsigned char* hsm = smem + 27 * COUTP * CINP * 2;              // halo [18 rows][HC cells]
    const uint32_t wbase = gs_smem_addr(wsm), hbase = gs_smem_addr(hsm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // weights once per CTA
    for (int i = tid; i < 27 * COUTP * NCH; i += kConvThreads) {
        const int r = i / NCH, j = i % NCH;
        cp16(wbase + swz(r, j, NCH), a.w + (size_t)r * CINP + j * 8);
    }

    const int wrow = warp >> 2;           // output row within the item
    const int wseg = (warp & 3) * 32;     // first cell of this warp's 32
    const bool wact = wseg < SEG;
    const int nmt = SEG - wseg >= 32 ? 2 : 1;  // m16 tiles of this warp
    const int g = lane >> 2, t = lane & 3;

    const long long items = (long long)a.N * L * (L / kRows) * nseg;
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int seg = (int)(item % nseg);
        long long r = item / nseg;
        const int yg = (int)(r % (L / kRows));
        r /= (L / kRows);
        const int z = (int)(r % L);
        const int n = (int)(r / L);
        const int x0 = seg * SEG, y0 = yg * kRows;
        __syncthreads();  // previous item's reads of the halo are done
        // halo rows: yi = 0..5 -> y0 - 1 + yi, zi = 0..2 -> z - 1 + zi
        const int hchunks = 18 * HC * NCH;
        for (int i = tid; i < hchunks; i += kConvThreads) {
            const int j = i % NCH;
            const int c = (i / NCH) % HC;
            const int hr = i / (NCH * HC);
            const int yy = (y0 - 1 + hr % 6 + L) % L;
            const int zz = (z - 1 + hr / 6 + L) % L;
            const int xx = (x0 + c - 1 + L) % L;
            const bf16* src = a.in + ((size_t)n * L3 + ((size_t)zz * L + yy) * L + xx) * CINP + j * 8;
            cp16(hbase + swz(hr * HC + c, j, NCH), src);
        }
        cp_wait_all();
        __syncthreads();
        if (!wact) continue;

        float acc[2][NT][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.f;

#pragma unroll 1
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            const int hr = (wrow + 1 + dy) + 6 * (1 + dz);
#pragma unroll
            for (int kc = 0; kc < CINP / 16; ++kc) {
                uint32_t b[NT][2];
                if constexpr (NT == 1) {
                    const int m = (lane >> 3) & 1;
                    const int co = lane & 7;
                    ldsm_x2(wbase + swz(tap * COUTP + co, kc * 2 + m, NCH), b[0][0], b[0][1]);
                } else {
#pragma unroll
                    for (int np = 0; np < NT; np += 2) {
                        const int m = lane >> 3;
                        const int co = (np + (m >> 1)) * 8 + (lane & 7);
                        ldsm_x4(wbase + swz(tap * COUTP + co, kc * 2 + (m & 1), NCH), b[np][0], b[np][1],
                                b[np + 1][0], b[np + 1][1]);
                    }
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    if (mt >= nmt) break;
                    const int m = lane >> 3;
                    const int cell = wseg + mt * 16 + (lane & 7) + (m & 1) * 8;
                    uint32_t af[4];
                    ldsm_x4(hbase + swz(hr * HC + 1 + dx + cell, kc * 2 + (m >> 1), NCH), af[0], af[1], af[2], af[3]);
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], af, b[nt][0], b[nt][1]);
                }
            }
        }

        // epilogue
        const int y = y0 + wrow;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            if (mt >= nmt) break;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int x = x0 + wseg + mt * 16 + g + hh * 8;
                const size_t cell = (size_t)n * L3 + ((size_t)z * L + y) * L + x;
                uint32_t bits = 0;  // this thread's channels of the cell's ReLU mask
                uint32_t mw = 0;
                if constexpr (EPI == EPI_DGRAD) mw = a.gz ? a.mprev[cell] : 0u;
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int ch = nt * 8 + 2 * t;
                    float v0 = acc[mt][nt][2 * hh], v1 = acc[mt][nt][2 * hh + 1];
                    if constexpr (EPI == EPI_FIRST || EPI == EPI_HIDDEN) {
                        v0 += a.bias[ch];
                        v1 += a.bias[ch + 1];
                        bits |= (v0 > 0.f ? 1u : 0u) << ch;
                        bits |= (v1 > 0.f ? 1u : 0u) << (ch + 1);
                        float h0 = fmaxf(v0, 0.f), h1 = fmaxf(v1, 0.f);
                        if constexpr (EPI == EPI_HIDDEN) {
                            const __nv_bfloat162 rr = *reinterpret_cast<const __nv_bfloat162*>(a.res + cell * 32 + ch);
                            h0 = __bfloat162float(rr.x) + h0;
                            h1 = __bfloat162float(rr.y) + h1;
                        }
                        *reinterpret_cast<__nv_bfloat162*>(a.out + cell * 32 + ch) = __floats2bfloat162_rn(h0, h1);
                    } else if constexpr (EPI == EPI_LAST) {
                        if (ch == 0) {
                            a.ou[cell] = a.su[cell] + (v0 + a.bias[0]);
                            a.ov[cell] = a.sv[cell] + (v1 + a.bias[1]);
                        }
                    } else {  // EPI_DGRAD
                        __nv_bfloat162* gp = reinterpret_cast<__nv_bfloat162*>(a.gh + cell * 32 + ch);
                        if (a.gh_acc) {
                            const __nv_bfloat162 old = *gp;
                            v0 = __bfloat162float(old.x) + v0;
                            v1 = __bfloat162float(old.y) + v1;
                        }
                        const __nv_bfloat162 gn = __floats2bfloat162_rn(v0, v1);
                        *gp = gn;
                        if (a.gz) {
                            __nv_bfloat162 m = gn;
                            if (!((mw >> ch) & 1u)) m.x = __float2bfloat16_rn(0.f);
                            if (!((mw >> (ch + 1)) & 1u)) m.y = __float2bfloat16_rn(0.f);
                            *reinterpret_cast<__nv_bfloat162*>(a.gz + cell * 32 + ch) = m;
                        }
                    }
                }
                if constexpr (EPI == EPI_FIRST || EPI == EPI_HIDDEN) {
                    // the four threads of a quad hold the cell's 32 channels
                    bits |= __shfl_xor_sync(0xffffffffu, bits, 1);
                    bits |= __shfl_xor_sync(0xffffffffu, bits, 2);
                    if (a.zmask && t == 0) a.zmask[cell] = bits;
                }
            }
        }
    }
    cp_wait_all();
}

// Weight gradient: dW[tap][ci][co] += sum over cells of in[cell + d(tap)][ci] * g[cell][co]
struct WgArgs {
    const bf16* in;  // [N][L^3][CINP]
    const bf16* g;   // [N][L^3][GST] (first NP channels used)
    float* dw;       // [27][cin][cout] (fp32, accumulated with atomics)
    int N, L, GST, cin, cout;
};

constexpr int kWgThreads = 288;  // 9 warps x 3 taps

template <int CINP, int NP>
__global__ void __launch_bounds__(kWgThreads, 1) gs_wgrad_kernel(const WgArgs a)
{
    constexpr int NCH = CINP / 8, GCH = NP / 8;
    constexpr int MT = CINP / 16, NT = NP / 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int L = a.L;
    const int SEG = L < 128 ? L : 128;
    const int HC = SEG + 2;
    const int nseg = L / SEG;
    const long long L3 = (long long)L * L * L;
    unsigned char* hsm = smem;                      // 18 halo rows of `in`
    unsigned char* gsm = smem + 18 * HC * CINP * 2; // 4 rows of g
    const uint32_t hbase = gs_smem_addr(hsm), gbase = gs_smem_addr(gsm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g8 = lane >> 2, t4 = lane & 3;

    float acc[3][MT][NT][4];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[q][mt][nt][i] = 0.f;

    const long long items = (long long)a.N * L * (L / kRows) * nseg;
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int seg = (int)(item % nseg);
        long long r = item / nseg;
        const int yg = (int)(r % (L / kRows));
        r /= (L / kRows);
        const int z = (int)(r % L);
        const int n = (int)(r / L);
        const int x0 = seg * SEG, y0 = yg * kRows;
        __syncthreads();
        for (int i = tid; i < 18 * HC * NCH; i += kWgThreads) {
            const int j = i % NCH;
            const int c = (i / NCH) % HC;
            const int hr = i / (NCH * HC);
            const int yy = (y0 - 1 + hr % 6 + L) % L;
            const int zz = (z - 1 + hr / 6 + L) % L;
            const int xx = (x0 + c - 1 + L) % L;
            cp16(hbase + swz(hr * HC + c, j, NCH), a.in + ((size_t)n * L3 + ((size_t)zz * L + yy) * L + xx) * CINP + j * 8);
        }
        for (int i = tid; i < kRows * SEG * GCH; i += kWgThreads) {
            const int j = i % GCH;
            const int c = (i / GCH) % SEG;
            const int rr = i / (GCH * SEG);
            cp16(gbase + swz(rr * SEG + c, j, GCH),
                 a.g + ((size_t)n * L3 + ((size_t)z * L + (y0 + rr)) * L + x0 + c) * a.GST + j * 8);
        }
        cp_wait_all();
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int tap = warp * 3 + q;
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
#pragma unroll 1
            for (int rr = 0; rr < kRows; ++rr) {
                const int hr = (rr + 1 + dy) + 6 * (1 + dz);
                for (int k0 = 0; k0 < SEG; k0 += 16) {
                    // B (cells x co) from g, transposed load
                    uint32_t b[NT][2];
                    if constexpr (NT == 1) {
                        const int m = (lane >> 3) & 1;
                        const int cell = k0 + (lane & 7) + m * 8;
                        ldsm_x2_t(gbase + swz(rr * SEG + cell, 0, GCH), b[0][0], b[0][1]);
                    } else {
#pragma unroll
                        for (int np = 0; np < NT; np += 2) {
                            const int m = lane >> 3;
                            const int cell = k0 + (lane & 7) + (m & 1) * 8;
                            ldsm_x4_t(gbase + swz(rr * SEG + cell, np + (m >> 1), GCH), b[np][0], b[np][1],
                                      b[np + 1][0], b[np + 1][1]);
                        }
                    }
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt) {
                        // A (ci x cells) from the shifted input row, transposed load
                        const int m = lane >> 3;
                        const int cell = k0 + (lane & 7) + (m >> 1) * 8;
                        uint32_t af[4];
                        ldsm_x4_t(hbase + swz(hr * HC + 1 + dx + cell, mt * 2 + (m & 1), NCH), af[0], af[1], af[2],
                                  af[3]);
#pragma unroll
                        for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[q][mt][nt], af, b[nt][0], b[nt][1]);
                    }
                }
            }
        }
    }
    // accumulate this CTA's partial sums
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int tap = warp * 3 + q;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int ci = mt * 16 + g8 + (i >= 2 ? 8 : 0);
                    const int co = nt * 8 + 2 * t4 + (i & 1);
                    if (ci < a.cin && co < a.cout) atomicAdd(a.dw + ((size_t)tap * a.cin + ci) * a.cout + co, acc[q][mt][nt][i]);
                }
    }
}

// 32-byte global store / load (p 32-byte aligned): one whole sector per thread
GS_D void gs_st_v8(void* p, const uint4& a, const uint4& b)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a.x), "r"(a.y), "r"(a.z),
                 "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
                 : "memory");
}

GS_D void gs_ld_v8(const void* p, uint4& a, uint4& b)
{
    asm volatile("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(p));
}

// x0 = bf16(u - 1, v, 20 F, 20 k, 0, ...) : [N][L^3][16].  With xtaps set
// (the tensor-core inference path), channels 4 d + c hold channel c of the x
// neighbour x + d - 1 (d = 0, 1, 2; periodic in x) and 12..15 are zero, so one
// 16-deep K step of the first layer covers its three dx taps.
__global__ void gs_pack_kernel(const float* __restrict__ u, const float* __restrict__ v, const float* __restrict__ Fk,
                               bf16* __restrict__ x0, long long L3, int N, int L, int xtaps)
{
    const long long total = L3 * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(i / L3);
        const bf16 f = __float2bfloat16_rn(Fk[2 * n] * kFkScale);
        const bf16 k = __float2bfloat16_rn(Fk[2 * n + 1] * kFkScale);
        __align__(16) bf16 c[16];
        for (int j = 0; j < 16; ++j) c[j] = __float2bfloat16_rn(0.f);
        if (xtaps) {
            const int x = (int)(i % L);
            for (int d = 0; d < 3; ++d) {
                const long long src = i - x + (x + d - 1 + L) % L;
                c[4 * d] = __float2bfloat16_rn(u[src] - 1.f);
                c[4 * d + 1] = __float2bfloat16_rn(v[src]);
                c[4 * d + 2] = f;
                c[4 * d + 3] = k;
            }
        } else {
            c[0] = __float2bfloat16_rn(u[i] - 1.f);  // zero on the u = 1 background
            c[1] = __float2bfloat16_rn(v[i]);
            c[2] = f;
            c[3] = k;
        }
        // one 32-byte store: the cell's whole sector
        gs_st_v8(x0 + i * 16, reinterpret_cast<const uint4*>(c)[0], reinterpret_cast<const uint4*>(c)[1]);
    }
}

// fp32 master weights [27][cin][cout] -> bf16 forward layout [27][COUTP][CINP]
// (and, for dgrad, [27][cin][COUTP'] with taps flipped: entry (tap, ci, co) =
// W[26 - tap][ci][co], i.e. the forward layout of the transposed conv).
__global__ void gs_wprep_kernel(const float* __restrict__ w, int cin, int cout, bf16* __restrict__ wf, int coutp,
                                int cinp, bf16* __restrict__ wd, int dcoutp_k)
{
    const int total = 27 * coutp * cinp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int ci = i % cinp, co = (i / cinp) % coutp, tap = i / (cinp * coutp);
        const float val = (ci < cin && co < cout) ? w[((size_t)tap * cin + ci) * cout + co] : 0.f;
        wf[i] = __float2bfloat16_rn(val);
    }
    if (!wd) return;
    // dgrad layout: rows n = ci (cin, = 32), k = co (padded to dcoutp_k)
    const int total2 = 27 * cin * dcoutp_k;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total2; i += gridDim.x * blockDim.x) {
        const int co = i % dcoutp_k, ci = (i / dcoutp_k) % cin, tap = i / (dcoutp_k * cin);
        const float val = co < cout ? w[((size_t)(26 - tap) * cin + ci) * cout + co] : 0.f;
        wd[i] = __float2bfloat16_rn(val);
    }
}

// loss = sum (out - tgt)^2 / count;  gd[cell][0..1] = 2 (out - tgt) / count, rest 0;
// db[0..1] += sum over cells of the stored (bf16) gd[cell][0..1] (the last
// layer's bias gradient; db may be null)
//
// With L > 0 the stored gradient is x-tap packed for the tensor-core path:
// channels 2 d + c (d < 3) hold channel c of the x neighbour x + d - 1
// (periodic in each row of L cells), the rest 0; db stays the cells' own sums.
__global__ void gs_mse_kernel(const float* __restrict__ ou, const float* __restrict__ ov, const float* __restrict__ tu,
                              const float* __restrict__ tv, long long total, double inv_count, bf16* __restrict__ gd,
                              double* __restrict__ loss, float* __restrict__ db, int L)
{
    // FP32 arithmetic per cell (GB300's FP64 pipe is narrow); 2 / count is a
    // power of two whenever the cell count is, and the per-thread partial
    // losses are added in FP64
    float lf = 0.f, su = 0.f, sv = 0.f;
    const float scale = (float)(2.0 * inv_count);
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const float du = ou[i] - tu[i], dv = ov[i] - tv[i];
        lf = fmaf(du, du, fmaf(dv, dv, lf));
        __nv_bfloat162 c01;
        c01.x = __float2bfloat16_rn(du * scale);
        c01.y = __float2bfloat16_rn(dv * scale);
        su += __bfloat162float(c01.x);
        sv += __bfloat162float(c01.y);
        uint4 first = zero;
        if (L > 0) {
            const int x = (int)(i % L);
            const long long row = i - x;
            const long long il = row + (x == 0 ? L - 1 : x - 1), ir = row + (x == L - 1 ? 0 : x + 1);
            __nv_bfloat162 l01, r01;
            l01.x = __float2bfloat16_rn((ou[il] - tu[il]) * scale);
            l01.y = __float2bfloat16_rn((ov[il] - tv[il]) * scale);
            r01.x = __float2bfloat16_rn((ou[ir] - tu[ir]) * scale);
            r01.y = __float2bfloat16_rn((ov[ir] - tv[ir]) * scale);
            first.x = *reinterpret_cast<const uint32_t*>(&l01);
            first.y = *reinterpret_cast<const uint32_t*>(&c01);
            first.z = *reinterpret_cast<const uint32_t*>(&r01);
        } else {
            first.x = *reinterpret_cast<const uint32_t*>(&c01);
        }
        gs_st_v8(gd + i * 16, first, zero);  // 32 bytes: the whole cell
    }
    double local = lf;
    for (int o = 16; o > 0; o >>= 1) {
        local += __shfl_xor_sync(0xffffffffu, local, o);
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    __shared__ double red[32];
    __shared__ float reds[32][2];
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = local;
        reds[threadIdx.x >> 5][0] = su;
        reds[threadIdx.x >> 5][1] = sv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        float a0 = 0.f, a1 = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += red[w];
            a0 += reds[w][0];
            a1 += reds[w][1];
        }
        atomicAdd(loss, t * inv_count);
        if (db) {
            atomicAdd(db, a0);
            atomicAdd(db + 1, a1);
        }
    }
}

// db[co] += sum over cells of g[cell][co] (co < cout)
__global__ void gs_bias_grad_kernel(const bf16* __restrict__ g, long long cells, int gst, int cout, float* __restrict__ db)
{
    __shared__ float part[32];
    if (threadIdx.x < 32) part[threadIdx.x] = 0.f;
    __syncthreads();
    const int co = threadIdx.x % 32;
    float s = 0.f;
    if (co < cout)
        for (long long i = blockIdx.x * (long long)(blockDim.x / 32) + threadIdx.x / 32; i < cells;
             i += (long long)gridDim.x * (blockDim.x / 32))
            s += __bfloat162float(g[i * gst + co]);
    atomicAdd(&part[co], s);
    __syncthreads();
    if (threadIdx.x < cout) atomicAdd(db + threadIdx.x, part[threadIdx.x]);
}

__global__ void gs_bf16_to_f32_kernel(const bf16* __restrict__ a, long long n, float* __restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(a[i]);
}

// Adam (Kingma & Ba 2015, Algorithm 1) on fp32 master parameters.
__global__ void gs_adam_kernel(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                               float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                               float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float g = gr[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// max |a - b| and sum (a - b)^2 over n values
__global__ void gs_diff_kernel(const float* __restrict__ a, const float* __restrict__ b, long long n,
                               unsigned int* __restrict__ maxbits, double* __restrict__ sumsq)
{
    float mx = 0.f;
    double ss = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float d = fabsf(a[i] - b[i]);
        if (!(d <= 3.402823466e38f)) d = __int_as_float(0x7f800000);  // NaN or inf counts as +inf
        mx = fmaxf(mx, d);
        ss += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxbits, __float_as_uint(mx));  // non-negative floats order like their bits
        atomicAdd(sumsq, ss);
    }
}

}  // namespace gs

namespace gs {

// ===========================================================================
// 5th-generation tensor-core forward convolution (tcgen05, TMEM accumulators)
// ===========================================================================
//
// One persistent CTA per SM, three warp roles: a TMA warp stages input
// planes, one elected lane of the MMA warp issues tcgen05.mma (M = 128, K =
// 16, bf16 x bf16 -> fp32 in TMEM), four epilogue warps drain the
// accumulators (tcgen05.ld, 32 TMEM lanes each).  A work unit is a column of
// 4 output rows (y0..y0+3) by 128 cells (x0..x0+127) of one grid, marched
// over a z-chunk.  Input planes (each: 6 rows y0-1..y0+4 by the 128 cells
// plus an x halo, periodic) sit in a shared ring of slabs, K-major with one
// cell per row of the A operand:
//   - 32 channels: 64-byte rows with the 64-byte swizzle (one TMA line a cell);
//   - the first layer's 16-channel x-tap input (inference): 32-byte rows with
//     the 32-byte swizzle, no x halo (its channels already hold x +- 1);
//   - otherwise (16 channels, training): 16-byte chunk planes, no swizzle.
// The A operand of tap (dz, dy, dx) for output row r is 128 consecutive cells
// from (row r+1+dy, cell 1+dx) of the dz slab: a descriptor offset, no data
// movement.  Weights (B) stay in shared memory, K-major.  In the hidden and
// first layers the three dy taps of a (dz, dx) sit side by side along N and
// the 4 output rows' accumulators are adjacent in TMEM, so one input slab
// row feeds up to three output rows in one MMA (N = NT .. 3 NT); the first
// MMAs into a fresh accumulator set (slab rows 5 and 2, which together touch
// every row once) overwrite, the rest accumulate, and two sets alternate
// between output planes.  The last layer (2 channels) instead stacks the
// three dz taps along N: each input plane is one group of MMAs into z-chunk
// accumulators that the epilogue zeroes (see EPI_LAST below).  Slabs are
// released by tcgen05.commit as soon as their last MMA is issued.  Every wait
// is bounded; on a timeout the CTA records it, lets its own MMAs and copies
// finish and frees its TMEM.

// Warp roles: epilogue warps 0 .. E-1 (warp w reads TMEM lanes 32 (w % 4) ..
// 32 (w % 4) + 31), then the MMA warp and the TMA warp.  E = 4, except for the
// x-tap first layer, whose few MMAs per plane leave the epilogue as the
// longer role: it runs on E = 8 warps, two per SM sub-partition, each taking
// 2 of the 4 rows (measured slower for the MMA-bound hidden layers).
GS_HD constexpr int tc_epi_warps(int epi, bool xt) { return (xt || epi == EPI_DGRAD) ? 8 : 4; }
GS_HD constexpr int tc_threads(int epi, bool xt) { return 32 * (tc_epi_warps(epi, xt) + 2); }
constexpr int kTcRows = 4;
constexpr int kTcCells = 128;
constexpr int kTcSlabRows = kTcRows + 2;  // rows per slab
constexpr int kTcZChunk = 16;
// A slab row holds cells x0-8 .. x0+135 (144 cells of 16, 32 or 64 bytes):
// TMA boxes of 8, 128 and 8 cells, each landing on a 128-byte (swizzled:
// atom) boundary.  Input cell x0 - 1 + c is row cell kTcRowX0 - 1 + c.
constexpr int kTcRowCells = kTcCells + 16;
constexpr int kTcRowX0 = 8;

struct ConvTcArgs {
    CUtensorMap map_main;  // a.in, boxes of 8 channels (or all 16 / 32, swizzled) x 128 cells
    CUtensorMap map_halo;  // a.in, the same x 8 cells
    const bf16* in;     // [N][L^3][CINP]
    const bf16* w;      // B operands: gs_wprep_tc_kernel's layout, or the x-tap first
                        // layer's (gs_wprep_tc_xtaps_kernel) or the last layer's
                        // (gs_wprep_tc_last_kernel)
    const float* bias;  // fp32, the layer's output channels (NT, or 2 for the last layer)
    int N, L;
    const bf16* res;    // unused (the residual comes from the centre slab)
    bf16* out;
    uint32_t* zmask;    // training: ReLU mask words (bit c = pre-activation c > 0), or null
    const float* su;
    const float* sv;
    float* ou;
    float* ov;
    // EPI_DGRAD (data gradient: the convolution of gz_l with the tap-flipped,
    // transposed weights of layer l): gh = bf16(acc (+ gh when gh_acc)),
    // [..][32]; gz = gh * mask for the layer below, [..][32], with the mask
    // words the layer below's forward pass stored
    bf16* gh;
    int gh_acc;
    const uint32_t* mprev;
    bf16* gz;
    int* err;
    uint64_t timeout_ns;
};

GS_D uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // shared-memory matrix descriptor, no swizzle: start, LBO, SBO (all >> 4),
    // bits 46-48 = 0b001, base offset 0, layout type 0
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

GS_D uint64_t tc_desc_sw64(uint32_t saddr, uint32_t sbo)
{
    // the same with the 64-byte swizzle (layout type 4 at bits 61-63): K-major
    // rows of 64 bytes in 8-row, 512-byte atoms; LBO unused (16 B)
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) |
           (4ull << 61);
}

GS_D uint64_t tc_desc_sw32(uint32_t saddr, uint32_t sbo)
{
    // the 32-byte swizzle (layout type 6): K-major rows of 32 bytes in
    // 8-row, 256-byte atoms; LBO unused (16 B)
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) |
           (6ull << 61);
}

GS_HD uint32_t tc_idesc(int n)
{
    // kind::f16 instruction descriptor: D fp32 (bits 4-5 = 1), A bf16 (7-9 = 1),
    // B bf16 (10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Warp-uniform issue: the whole warp runs the issuing code (so descriptors
// and coordinates stay warp-uniform) and one elected lane executes the
// instruction.
GS_D uint32_t tc_elect_one()
{
    uint32_t is_leader;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(is_leader));
    return is_leader;
}

GS_D void tc_mma_if(uint32_t leader, uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "setp.ne.b32 e, %5, 0;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum), "r"(leader)
        : "memory");
}

GS_D void tc_commit_if(uint32_t leader, uint64_t* bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "setp.ne.b32 e, %1, 0;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
            gs_smem_addr(bar)),
        "r"(leader)
        : "memory");
}

GS_D void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
GS_D void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int NCOL>
GS_D void tc_ld(uint32_t taddr, float (&v)[NCOL]);

template <>
GS_D void tc_ld<32>(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
GS_D void tc_ld<16>(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
GS_D void tc_ld<8>(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// zero 32 consecutive columns of this warp's 32 TMEM lanes (and wait for it)
GS_D void tc_st_zero32(uint32_t taddr)
{
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(z)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 4D tiled TMA load (channels, x, y, plane) -> shared, completion on `bar`;
// the channel coordinate is a multiple of 8 (16 bytes) by construction.
GS_D void tc_tma_load_4d_if(uint32_t leader, uint32_t dst, const CUtensorMap* map, uint64_t* bar, int c, int x, int y,
                            int zp)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "setp.ne.b32 e, %7, 0;\n\t"
        "@e cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n\t}" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(zp), "r"(gs_smem_addr(bar)), "r"(leader)
        : "memory");
}

GS_D void tc_arrive_expect_tx_if(uint32_t leader, uint64_t* bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "setp.ne.b32 e, %2, 0;\n\t"
        "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t}" ::"r"(gs_smem_addr(bar)),
        "r"(bytes), "r"(leader)
        : "memory");
}

template <int CINP, int NT, int EPI, bool XT>
__global__ void __launch_bounds__(tc_threads(EPI, XT), 1) gs_conv_tc_kernel(const __grid_constant__ ConvTcArgs a)
{
    constexpr int EPIW = tc_epi_warps(EPI, XT), MMAW = EPIW, PRODW = EPIW + 1, NTHR = tc_threads(EPI, XT);
    constexpr int EROWS = kTcRows * 4 / EPIW;  // output rows drained by one epilogue warp
    // XT: the input is x-tap packed (gs_pack_kernel with xtaps), so the three
    // dx taps are one K step: one MMA per (dz, slab row), no x halo boxes
    static_assert(!XT || CINP == 16, "x-tap packing is for the 16-channel first layer");
    constexpr int NCH = CINP / 8;
    constexpr uint32_t ROWB = kTcRowCells * 16;           // bytes of one slab row of one chunk
    constexpr uint32_t PLANE = kTcSlabRows * ROWB;         // bytes of one chunk plane of a slab
    constexpr uint32_t SLAB = NCH * PLANE;
    // 32 input channels: a slab row is [cell][32 channels] (64 bytes a cell)
    // with the 64-byte swizzle, one TMA line per cell instead of four
    constexpr bool SW = CINP == 32;
    constexpr uint32_t SROWB = kTcRowCells * 64;          // bytes of one swizzled slab row
    static_assert(!SW || kTcSlabRows * SROWB == SLAB, "swizzled slab size");
    // x-tap input: a slab row is [cell][16 channels] (32 bytes a cell) with the
    // 32-byte swizzle, one TMA line per cell instead of two 16-byte ones
    constexpr uint32_t XROWB = kTcRowCells * 32;          // bytes of one 32-byte-swizzled slab row
    static_assert(!XT || kTcSlabRows * XROWB == SLAB, "x-tap slab size");
    // EPI_LAST (2 output channels): the dz taps side by side along N, each
    // block holding the 4 output rows x 2 channels (8 columns, padded to 16),
    // so each input plane is read by one group of MMAs (N = 48, fewer at the
    // ends of a z-chunk) that adds into the accumulators of the three output
    // planes it feeds; an accumulator set holds a whole z-chunk (16 columns a
    // plane), zeroed by the epilogue before use
    constexpr bool ZS = EPI == EPI_LAST;
    static_assert(!ZS || (CINP == 32 && kTcRows == 4 && kTcSlabRows == 6), "dz-stacked last layer");
    constexpr uint32_t ZS_SETC = kTcZChunk * 16;
    constexpr uint32_t ZS_WB = 2 * 48 * 16;  // bytes of B per (slab row, dx, K step)
    constexpr uint32_t WBYTES = ZS ? kTcSlabRows * 3 * 2 * ZS_WB : (XT ? 9 : 27) * NCH * NT * 16;
    // bytes the TMA delivers per slab (x-tap input: the 128 cells of each row only)
    constexpr uint32_t SLAB_TX = XT ? NCH * kTcSlabRows * kTcCells * 16 : SLAB;
    // slab ring depth: the x-tap first layer does little MMA work per plane,
    // so its small slabs are prefetched further ahead to cover the copy latency
    constexpr uint32_t NSLAB = XT ? 6 : 3;
    constexpr uint32_t ACC_COLS = kTcRows * NT;            // one accumulator set (4 output rows)
    constexpr uint32_t TMEM_COLS = ZS ? 512 : (2 * ACC_COLS <= 64 ? 64 : (2 * ACC_COLS <= 128 ? 128 : 256));
    static_assert(!ZS || 2 * ZS_SETC <= TMEM_COLS, "accumulator sets fit in TMEM");
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    // slab_full: the producer's expect-tx arrival, completed by the TMA bytes;
    // slab_empty: the MMA commit after the plane's last tap; acc_full: the
    // commit after an item's last MMA; acc_empty: one arrival per epilogue warp
    __shared__ __align__(8) uint64_t slab_full[NSLAB], slab_empty[NSLAB], acc_full[2], acc_empty[2], bar_fin;
    __shared__ uint32_t tmem_base_s;
    __shared__ float bias_s[NT];
    __shared__ volatile int abort_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = a.L;
    const long long L3 = (long long)L * L * L;
    const uint32_t sbase = gs_smem_addr(smem_tc);
    const uint32_t wbase = sbase + NSLAB * SLAB;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gs_smem_addr(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (uint32_t i = 0; i < NSLAB; ++i) {
            gs_mbar_init(&slab_full[i], 1);
            gs_mbar_init(&slab_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            gs_mbar_init(&acc_full[i], 1);
            gs_mbar_init(&acc_empty[i], EPIW);
        }
        gs_mbar_init(&bar_fin, 1);
        abort_s = 0;
        gs_fence_mbar_init();
    }
    if (tid < NT) bias_s[tid] = (EPI == EPI_DGRAD || (EPI == EPI_LAST && tid >= 2)) ? 0.f : a.bias[tid];
    for (uint32_t i = tid; i < WBYTES / 16; i += NTHR) cp16(wbase + i * 16, a.w + (size_t)i * 8);
    cp_wait_all();
    gs_fence_proxy_async();  // cp.async (generic) writes -> visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const int nseg = L / kTcCells;
    const int nyg = L / kTcRows;
    const int nzc = (L + kTcZChunk - 1) / kTcZChunk;
    const long long nunits = (long long)a.N * nyg * nseg * nzc;
    struct Unit {
        int n, x0, y0, z0, nz;
    };
    auto decode_unit = [&](long long unit) {
        Unit u;
        const int zc = (int)(unit % nzc);
        long long r0 = unit / nzc;
        const int seg = (int)(r0 % nseg);
        r0 /= nseg;
        u.y0 = (int)(r0 % nyg) * kTcRows;
        u.n = (int)(r0 / nyg);
        u.x0 = seg * kTcCells;
        u.z0 = zc * kTcZChunk;
        u.nz = min(kTcZChunk, L - u.z0);
        return u;
    };
    // CTAs take units round robin; the units of a partial last round are cut
    // along z into up to 4 pieces, so that round ends after a fraction of a
    // unit.  Every role walks the same sequence: index v < full is unit v,
    // beyond it piece (v - full) % nsplit of unit full + (v - full) / nsplit.
    const long long full = nunits / gridDim.x * gridDim.x;
    const long long rem = nunits - full;
    const int fsplit = (full > 0 && rem > 0) ? (int)min(4LL, (long long)gridDim.x / rem) : 1;
    const int nsplit = fsplit >= 2 ? fsplit : 1;
    const long long units = full + rem * nsplit;
    auto decode = [&](long long v) -> Unit {
        if (v < full) return decode_unit(v);
        const long long p = v - full;
        Unit u = decode_unit(full + p / nsplit);
        const int part = (int)(p % nsplit);
        const int za = u.nz * part / nsplit, zb = u.nz * (part + 1) / nsplit;
        u.z0 += za;
        u.nz = zb - za;
        return u;
    };
    // bounded wait that also gives up once another role has aborted
    auto bwait = [&](uint64_t* bar, uint32_t parity) -> bool {
        if (gs_mbar_try_wait(bar, parity)) return true;
        const uint64_t t0 = gs_globaltimer();
        for (;;) {
#pragma unroll 1
            for (int i = 0; i < 32; ++i)
                if (gs_mbar_try_wait(bar, parity)) return true;
            if (abort_s) return false;
            if (gs_globaltimer() - t0 > a.timeout_ns) {
                abort_s = 1;
                gs_report(a.err, GS_DERR_TIMEOUT);
                return false;
            }
        }
    };

    // warp-uniform bounded wait (lane 0 polls; the result is broadcast)
    auto wwait = [&](uint64_t* bar, uint32_t parity) -> bool {
        int r = 0;
        if (lane == 0) r = bwait(bar, parity) ? 1 : 0;
        r = __shfl_sync(0xffffffffu, r, 0);
        return r != 0;
    };

    if (warp == PRODW) {
        // ------------------------ producer (TMA, one elected lane) ------------------------
        // plane z0 - 1 + i of a unit (i = 0 .. nz+1) is global plane g, slot g % NSLAB;
        // per plane and channel chunk, each of the 6 rows is three boxes (left
        // halo, 128 cells, right halo), wrapped periodically by their start
        // coordinates (L is a multiple of 128, so no box straddles the wrap)
        const uint32_t leader = tc_elect_one();
        if ((sbase & (SW ? 511u : (XT ? 255u : 127u))) == 0) {
            if (leader) {
                gs_prefetch_tmap(&a.map_main);
                gs_prefetch_tmap(&a.map_halo);
            }
            __syncwarp();
            uint32_t g = 0;
            bool ok = true;
            for (long long unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
                const Unit u = decode(unit);
                const int xl = (u.x0 - kTcRowX0 + L) % L, xr = (u.x0 + kTcCells) % L;
                int yrow[kTcSlabRows];
#pragma unroll
                for (int yi = 0; yi < kTcSlabRows; ++yi) yrow[yi] = (u.y0 - 1 + yi + L) % L;
                for (int i = 0; i < u.nz + 2; ++i, ++g) {
                    const int slot = (int)(g % NSLAB);
                    if (g >= NSLAB && !wwait(&slab_empty[slot], ((g / NSLAB) - 1u) & 1u)) {
                        ok = false;
                        break;
                    }
                    const int zp = u.n * L + (u.z0 - 1 + i + L) % L;
                    tc_arrive_expect_tx_if(leader, &slab_full[slot], SLAB_TX);
                    const uint32_t dst0 = sbase + slot * SLAB;
                    if constexpr (XT) {
                        // one 16-channel box of the 128 cells per row, at cell
                        // slot 8 (a 256-byte boundary); no halo boxes
#pragma unroll
                        for (int yi = 0; yi < kTcSlabRows; ++yi)
                            tc_tma_load_4d_if(leader, dst0 + yi * XROWB + kTcRowX0 * 32, &a.map_main, &slab_full[slot],
                                              0, u.x0, yrow[yi], zp);
                    } else if constexpr (SW) {
                        // three boxes of 32 channels per row, each landing on a
                        // 512-byte boundary (cell slots 0, 8 and 136 of 64 bytes)
#pragma unroll
                        for (int yi = 0; yi < kTcSlabRows; ++yi) {
                            const uint32_t row = dst0 + yi * SROWB;
                            tc_tma_load_4d_if(leader, row, &a.map_halo, &slab_full[slot], 0, xl, yrow[yi], zp);
                            tc_tma_load_4d_if(leader, row + kTcRowX0 * 64, &a.map_main, &slab_full[slot], 0, u.x0,
                                              yrow[yi], zp);
                            tc_tma_load_4d_if(leader, row + (kTcRowX0 + kTcCells) * 64, &a.map_halo, &slab_full[slot],
                                              0, xr, yrow[yi], zp);
                        }
                    } else
#pragma unroll
                    for (int j = 0; j < NCH; ++j)
#pragma unroll
                        for (int yi = 0; yi < kTcSlabRows; ++yi) {
                            const uint32_t row = dst0 + j * PLANE + yi * ROWB;
                            tc_tma_load_4d_if(leader, row, &a.map_halo, &slab_full[slot], j * 8, xl, yrow[yi], zp);
                            tc_tma_load_4d_if(leader, row + kTcRowX0 * 16, &a.map_main, &slab_full[slot], j * 8, u.x0,
                                              yrow[yi], zp);
                            tc_tma_load_4d_if(leader, row + (kTcRowX0 + kTcCells) * 16, &a.map_halo, &slab_full[slot],
                                              j * 8, xr, yrow[yi], zp);
                        }
                }
            }
            if (!ok && lane == 0) {
                // let the copies in flight land (fixed budget)
                for (uint32_t q = g > NSLAB ? g - NSLAB : 0u; q < g; ++q)
                    gs_mbar_wait(&slab_full[q % NSLAB], (q / NSLAB) & 1u, 2000000000ull);
            }
        } else if (lane == 0) {
            abort_s = 1;  // unaligned shared memory: refuse to issue TMA
            gs_report(a.err, GS_DERR_BADARG);
        }
    } else if (warp == MMAW) {
        // ------------------------ MMA issuer (one elected lane) ------------------------
        const uint32_t leader = tc_elect_one();
        // the MMAs of one dz group of an item into accumulator set `set`,
        // operand A from the slab in `slot`.  Descriptors: the start address is
        // the low 14 bits, so a descriptor plus (byte offset >> 4) addresses
        // the shifted operand.
        auto issue_group = [&](int set, int dzi, int slot) {
            constexpr uint32_t WCH = 3 * NT * 16;  // bytes of one weight chunk plane
            constexpr int kOrder[kTcSlabRows] = {5, 2, 0, 1, 3, 4};
            const uint32_t dset = tmem + (uint32_t)(set * ACC_COLS);
            const uint32_t idn[3] = {tc_idesc(NT), tc_idesc(2 * NT), tc_idesc(3 * NT)};
            // A: no swizzle (LBO = one chunk plane, SBO = 8 cells), or the
            // 64-byte swizzle (SBO = one 8-cell atom; K steps of 32 bytes)
            const uint64_t adz = SW   ? tc_desc_sw64(sbase + slot * SLAB, 512)
                                 : XT ? tc_desc_sw32(sbase + slot * SLAB, 256)
                                      : tc_desc(sbase + slot * SLAB, PLANE, 128);
            constexpr uint32_t AROW = SW ? SROWB : (XT ? XROWB : ROWB);  // bytes between slab rows
            constexpr int DX0 = XT ? 1 : 0, DX1 = XT ? 2 : 3;  // x-tap input: the unshifted operand only
#pragma unroll
            for (int dxi = DX0; dxi < DX1; ++dxi)
#pragma unroll
                for (int kk = 0; kk < CINP / 16; ++kk) {
                    const int wplane = XT ? dzi * NCH + 2 * kk : (dzi * 3 + dxi) * NCH + 2 * kk;
                    const uint64_t bk = tc_desc(wbase + (uint32_t)wplane * WCH, WCH, 128);
                    // output cell i of tap dx reads input cell x0 + i + dx - 1
                    // (x-tap input: dxi = 1 and kk = 0 only, an atom-aligned start)
                    const uint64_t ak = SW   ? adz + (uint64_t)((kk * 32) >> 4) + (uint64_t)(((kTcRowX0 - 1 + dxi) * 64) >> 4)
                                        : XT ? adz + (uint64_t)(((kTcRowX0 - 1 + dxi) * 32) >> 4)
                                             : adz + (uint64_t)((2 * kk * PLANE) >> 4) + (uint64_t)(kTcRowX0 - 1 + dxi);
                    // slab rows 5 and 2 first: together they touch every output row once
#pragma unroll
                    for (int q = 0; q < kTcSlabRows; ++q) {
                        const int sr = kOrder[q];
                        const int rlo = sr - 2 > 0 ? sr - 2 : 0;
                        const int rhi = sr < kTcRows - 1 ? sr : kTcRows - 1;
                        const int b0 = 2 - sr + rlo;  // first dy block (dy = +1 - block)
                        const bool fresh = dzi == 0 && dxi == DX0 && kk == 0 && q < 2;
                        tc_mma_if(leader, dset + (uint32_t)(rlo * NT), ak + (uint64_t)(sr * (AROW >> 4)),
                                  bk + (uint64_t)((b0 * NT * 16) >> 4), idn[rhi - rlo], fresh ? 0u : 1u);
                    }
                }
        };
        // EPI_LAST: all MMAs of input plane i (i = 0 .. nz+1, plane z0 - 1 + i)
        // of a unit.  It feeds output planes i - 2, i - 1, i (dz blocks 0-2);
        // those inside the unit, plo .. phi, are one N window at column
        // 16 plo of the set, B rows from block plo - (i - 2) on
        auto issue_zs = [&](int set, int i, int slot, int nz) {
            const int plo = i - 2 > 0 ? i - 2 : 0, phi = i < nz - 1 ? i : nz - 1;
            const uint32_t dcol = tmem + (uint32_t)(set * ZS_SETC + plo * 16);
            const uint32_t boff = (uint32_t)(plo - (i - 2)) * 16 * 16;
            const uint64_t adz = tc_desc_sw64(sbase + slot * SLAB, 512);
            const uint32_t idz = tc_idesc((phi - plo + 1) * 16);
#pragma unroll
            for (int sr = 0; sr < kTcSlabRows; ++sr)
#pragma unroll
                for (int dxi = 0; dxi < 3; ++dxi)
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t ak = adz + (uint64_t)((kk * 32) >> 4) +
                                            (uint64_t)(((kTcRowX0 - 1 + dxi) * 64) >> 4) +
                                            (uint64_t)(sr * (SROWB >> 4));
                        const uint64_t bk =
                            tc_desc(wbase + (uint32_t)((sr * 3 + dxi) * 2 + kk) * ZS_WB + boff, 48 * 16, 128);
                        tc_mma_if(leader, dcol, ak, bk, idz, 1u);
                    }
        };
        bool ok = true;
        if constexpr (ZS) {
            uint32_t g = 0, k = 0;  // planes and units seen by this CTA
            for (long long unit = blockIdx.x; unit < units && ok; unit += gridDim.x, ++k) {
                const Unit u = decode(unit);
                const int set = (int)(k & 1u);
                // completion 0 of acc_empty is the epilogue's initial zeroing
                if (!wwait(&acc_empty[set], (k / 2u) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int i = 0; i < u.nz + 2; ++i, ++g) {
                    const int slot = (int)(g % NSLAB);
                    if (!wwait(&slab_full[slot], (g / NSLAB) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    issue_zs(set, i, slot, u.nz);
                    tc_commit_if(leader, &slab_empty[slot]);  // each plane has one group of MMAs
                }
                if (!ok) break;
                tc_commit_if(leader, &acc_full[set]);
            }
        } else {
            uint32_t g = 0, k = 0;  // planes and items seen by this CTA
            for (long long unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
                const Unit u = decode(unit);
                const uint32_t gb = g;
                for (int q = 0; q < u.nz && ok; ++q, ++k) {
                    const int set = (int)(k & 1u);
                    if (k >= 2 && !wwait(&acc_empty[set], ((k / 2u) - 1u) & 1u)) {
                        ok = false;
                        break;
                    }
                    for (int d = 0; d < 3; ++d) {
                        // item q reads planes q, q+1, q+2 of the unit (dz = d - 1)
                        const uint32_t gp = gb + (uint32_t)(q + d);
                        const int slot = (int)(gp % NSLAB);
                        if ((q == 0 || d == 2) && !wwait(&slab_full[slot], (gp / NSLAB) & 1u)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        issue_group(set, d, slot);
                        // last MMA use of plane q (its dz=-1 taps); of the unit's
                        // last two planes, the last item's dz = 0 and +1 taps
                        if (d == 0 || q == u.nz - 1) tc_commit_if(leader, &slab_empty[slot]);
                    }
                    if (!ok) break;
                    tc_commit_if(leader, &acc_full[set]);
                }
                g = gb + (uint32_t)(u.nz + 2);
            }
        }
        if (!ok) {
            // one more commit tracks every MMA issued (fixed budget: issued
            // MMAs always complete)
            tc_commit_if(leader, &bar_fin);
            if (lane == 0) gs_mbar_wait(&bar_fin, 0, 2000000000ull);
        }
    } else {
        // --------------------- epilogue warps (0 .. EPIW-1) ----------------------
        static_assert(!ZS || EPIW == 4, "the last layer drains all 4 rows per warp");
        const int x_in_seg = tid & 127;      // this thread's cell in the 128-cell segment
        const int r0 = (warp >> 2) * EROWS;  // its first output row
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const float* bias_r = bias_s;  // shared memory: same-address reads broadcast
        // per-item inputs of the epilogue that do not depend on the MMAs (the
        // residual of the hidden layers, the state of the last one), loaded one
        // item ahead so their latency overlaps the wait for the accumulators
        constexpr int NRES = EPI == EPI_HIDDEN ? NT / 8 : 1;
        uint4 rv[EROWS][NRES];
        float sres[EROWS][2];
        // EPI_DGRAD: the layer below's ReLU mask word one item ahead; the
        // incoming residual-path gradient (bf16) is loaded in the epilogue
        // itself (registers)
        constexpr bool DG = EPI == EPI_DGRAD;
        static_assert(!DG || NT == 32, "the data gradient has 32 output channels");
        uint32_t pm[DG ? EROWS : 1];
        auto cell_of = [&](const Unit& u, int q, int r) -> size_t {
            return (size_t)u.n * L3 + ((size_t)(u.z0 + q) * L + (u.y0 + r)) * L + (u.x0 + x_in_seg);
        };
        auto prefetch = [&](const Unit& u, int q) {
#pragma unroll
            for (int rr = 0; rr < EROWS; ++rr) {
                const size_t cell = cell_of(u, q, r0 + rr);
                if constexpr (EPI == EPI_HIDDEN) {
                    // 32-byte loads: each a whole sector of the cell's 64 bytes
#pragma unroll
                    for (int j = 0; j < NRES; j += 2) gs_ld_v8(a.in + cell * CINP + j * 8, rv[rr][j], rv[rr][j + 1]);
                } else if constexpr (EPI == EPI_LAST) {
                    sres[rr][0] = a.su[cell];
                    sres[rr][1] = a.sv[cell];
                } else if constexpr (DG) {
                    pm[rr] = a.mprev[cell];
                }
            }
        };
        auto epilogue = [&](int set, const Unit& u, int q) {
            // EPI_DGRAD: the incoming gh (bf16) of all this warp's rows, issued
            // before the first TMEM load so their latencies overlap
            uint4 gin[DG ? EROWS : 1][DG ? 4 : 1];
            if constexpr (DG) {
                if (a.gh_acc) {
#pragma unroll
                    for (int rr = 0; rr < EROWS; ++rr) {
                        const size_t cell = cell_of(u, q, r0 + rr);
#pragma unroll
                        for (int j = 0; j < 4; j += 2) gs_ld_v8(a.gh + cell * 32 + j * 8, gin[rr][j], gin[rr][j + 1]);
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < EROWS; ++rr) {
                const int r = r0 + rr;
                const size_t cell = cell_of(u, q, r);
                float acc[NT];
                tc_ld<NT>(lane_base + (uint32_t)(set * ACC_COLS + r * NT), acc);
                if constexpr (DG) {
                    // gh = bf16(gh + acc); gz = gh * mask (exact in bf16)
                    uint4 gout[4], zo[4];
                    const uint32_t mw = pm[rr];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const __nv_bfloat162* gi = reinterpret_cast<const __nv_bfloat162*>(&gin[rr][j]);
                        __nv_bfloat162* go = reinterpret_cast<__nv_bfloat162*>(&gout[j]);
                        __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&zo[j]);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c = j * 8 + 2 * e;
                            float g0 = acc[c], g1 = acc[c + 1];
                            if (a.gh_acc) {
                                g0 = __bfloat162float(gi[e].x) + g0;
                                g1 = __bfloat162float(gi[e].y) + g1;
                            }
                            go[e] = __floats2bfloat162_rn(g0, g1);
                            const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
                            ob[e].x = (mw >> c) & 1u ? go[e].x : zero;
                            ob[e].y = (mw >> (c + 1)) & 1u ? go[e].y : zero;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; j += 2) gs_st_v8(a.gh + cell * 32 + j * 8, gout[j], gout[j + 1]);
#pragma unroll
                    for (int j = 0; j < 4; j += 2) gs_st_v8(a.gz + cell * 32 + j * 8, zo[j], zo[j + 1]);
                } else if constexpr (EPI != EPI_LAST) {  // (the last layer drains in its own loop below)
                    static_assert(NT % 16 == 0, "the epilogue stores 16 channels (32 bytes) at a time");
                    static_assert(NT <= 32, "one mask word a cell");
                    uint4 ho[NT / 8];
                    uint32_t bits = 0;
#pragma unroll
                    for (int j = 0; j < NT / 8; ++j) {
                        float h[8], zv[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            zv[e] = acc[j * 8 + e] + bias_r[j * 8 + e];
                            h[e] = fmaxf(zv[e], 0.f);
                            bits |= (zv[e] > 0.f ? 1u : 0u) << (j * 8 + e);
                        }
                        if constexpr (EPI == EPI_HIDDEN) {
                            const __nv_bfloat162* rb = reinterpret_cast<const __nv_bfloat162*>(&rv[rr][j]);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                h[2 * e] = __bfloat162float(rb[e].x) + h[2 * e];
                                h[2 * e + 1] = __bfloat162float(rb[e].y) + h[2 * e + 1];
                            }
                        }
                        __nv_bfloat162* hb = reinterpret_cast<__nv_bfloat162*>(&ho[j]);
#pragma unroll
                        for (int e = 0; e < 4; ++e) hb[e] = __floats2bfloat162_rn(h[2 * e], h[2 * e + 1]);
                    }
                    // 32-byte stores: each writes a whole sector of the cell's 64 bytes
#pragma unroll
                    for (int j = 0; j < NT / 8; j += 2) gs_st_v8(a.out + cell * 32 + j * 8, ho[j], ho[j + 1]);
                    if (a.zmask) a.zmask[cell] = bits;
                }
            }
        };
        if constexpr (ZS) {
            // this warp's 32 lanes of a set's columns
            const uint32_t lanes = lane_base;
            auto zero_set = [&](int set) {
#pragma unroll
                for (int c = 0; c < (int)ZS_SETC; c += 32) tc_st_zero32(lanes + (uint32_t)(set * ZS_SETC + c));
            };
            zero_set(0);
            zero_set(1);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                gs_mbar_arrive(&acc_empty[0]);
                gs_mbar_arrive(&acc_empty[1]);
            }
            uint32_t k = 0;
            bool ok = true;
            if (blockIdx.x < units) prefetch(decode(blockIdx.x), 0);
            for (long long unit = blockIdx.x; unit < units && ok; unit += gridDim.x, ++k) {
                const Unit u = decode(unit);
                const int set = (int)(k & 1u);
                if (!wwait(&acc_full[set], (k / 2u) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int q = 0; q < u.nz; ++q) {
                    float st[kTcRows][2];
#pragma unroll
                    for (int r = 0; r < kTcRows; ++r) {
                        st[r][0] = sres[r][0];
                        st[r][1] = sres[r][1];
                    }
                    if (q + 1 < u.nz) prefetch(u, q + 1);
                    else if (unit + gridDim.x < units) prefetch(decode(unit + gridDim.x), 0);
                    float acc[8];  // (row, channel) pairs of output plane q
                    tc_ld<8>(lanes + (uint32_t)(set * ZS_SETC + q * 16), acc);
#pragma unroll
                    for (int r = 0; r < kTcRows; ++r) {
                        const size_t cell = cell_of(u, q, r);
                        a.ou[cell] = st[r][0] + (acc[2 * r] + bias_r[0]);
                        a.ov[cell] = st[r][1] + (acc[2 * r + 1] + bias_r[1]);
                    }
                }
                zero_set(set);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) gs_mbar_arrive(&acc_empty[set]);
            }
        } else {
            uint32_t k = 0;
            bool ok = true;
            if (blockIdx.x < units) prefetch(decode(blockIdx.x), 0);
            for (long long unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
                const Unit u = decode(unit);
                for (int q = 0; q < u.nz; ++q, ++k) {
                    const int set = (int)(k & 1u);
                    if (!wwait(&acc_full[set], (k / 2u) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    epilogue(set, u, q);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) gs_mbar_arrive(&acc_empty[set]);
                    // the next item's inputs (this unit's next plane, or the next unit's first)
                    if (q + 1 < u.nz) prefetch(u, q + 1);
                    else if (unit + gridDim.x < units) prefetch(decode(unit + gridDim.x), 0);
                }
            }
        }
    }
    // nothing of this CTA may be in flight when its TMEM and shared memory go
    cp_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ===========================================================================
// 5th-generation tensor-core weight gradient (tcgen05, TMEM accumulators)
// ===========================================================================
//
//   dW[tap][ci][co] = sum over cells c of h[c + d(tap)][ci] * g[c][co]
//
// is a contraction over cells (K), so both operands are read MN-major from
// channels-last slabs: a row of 128 cells of HC (or GC) channels staged with
// the 64-byte (32 channels) or 32-byte (16 channels) swizzle is, read with
// K = cells, one swizzle atom column of an MN-major operand.  A work unit is
// 2 output rows (y0, y0+1) x 128 cells x a z-chunk of 8 planes.
//   A (M = 128): MB = 128 / HC consecutive rows of an input slab (rows y0-1
//     .. y0+2 of input plane p, with an x halo), starting at row i for output
//     row i, so M block j holds dy = j - 1 (blocks j >= 3 are never used:
//     their products land in TMEM lanes that are not read); the dx tap is a
//     start offset of dx cells.
//   B (N = 3 GC at most): the gradient planes p-1, p, p+1 of the unit (dz =
//     +1, 0, -1), row i, clipped to the unit's planes.  They sit in a ring of
//     4 slots whose first two are mirrored after the fourth, so any three
//     consecutive planes are at a uniform stride.
// Every MMA accumulates into one of 3 (dx) x 3 (dz) column blocks of GC
// columns; the CTA keeps all 27 taps in TMEM for its whole life (zeroed
// first), and its epilogue warps drain them once into per-CTA partial sums
// that gs_wgrad_reduce_kernel adds up in a fixed order.  While the MMAs run,
// the epilogue warps add up every gradient plane the ring receives (once per
// unit, so once per cell) per channel: the layer's bias gradient, reduced
// the same way.  Three warp roles as in gs_conv_tc_kernel (TMA producer, MMA
// issuer, 4 epilogue warps); every wait is bounded.
constexpr int kWgRows = 2;     // output rows per unit
constexpr int kWgZChunk = 8;   // planes per unit
constexpr int kWgHSlabs = 3;   // input-slab ring depth
constexpr int kWgGSlots = 4;   // gradient-plane ring depth (+ 2 mirrored slots)
constexpr int kWgTcThreads = 192;

struct WgTcArgs {
    CUtensorMap map_hmain;  // h: HC channels x 128 cells
    CUtensorMap map_hhalo;  // h: HC channels x 8 cells
    CUtensorMap map_g;      // g: GC channels x 128 cells
    float* part;            // [gridDim.x][27 HC GC + GC] partial sums (weights, then biases)
    int N, L;
    int* err;
    uint64_t timeout_ns;
};

GS_D uint64_t tc_desc_lay(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout)
{
    // shared-memory matrix descriptor with an explicit LBO and layout type
    // (4: 64-byte swizzle, 6: 32-byte swizzle)
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}

GS_HD uint32_t tc_idesc_mn(int n)
{
    // kind::f16, D fp32, A and B bf16, both MN-major (bits 15, 16), M = 128
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// XTS (x-tap packed operands; one MMA per K step covers the three dx taps):
//   0  none;
//   1  A is the first layer's packed input: channel 4 d + c of cell x holds
//      channel c of cell x + d - 1 (d < 3), so M row 16 j + 4 d + c is
//      (dy = j - 1, dx = d - 1, ci = c);
//   2  B is the last layer's packed dL/dout: channel 2 d + c of cell x holds
//      channel c of cell x + d - 1, so N column 2 d + c pairs input cell x
//      with gradient cell x + d - 1, i.e. dx = 1 - d.
template <int HC, int GC, int XTS>
__global__ void __launch_bounds__(kWgTcThreads, 1) gs_wgrad_tc_kernel(const __grid_constant__ WgTcArgs a)
{
    static_assert((HC == 32 || HC == 16) && (GC == 32 || GC == 16), "16 or 32 channels");
    static_assert(XTS == 0 || (XTS == 1 && HC == 16) || (XTS == 2 && GC == 16), "x-tap packing of a 16-channel operand");
    constexpr int NDX = XTS ? 1 : 3;  // dx column blocks in TMEM (one when a packed operand carries dx)
    constexpr int MB = 128 / HC;                          // M blocks (slab rows) per MMA
    constexpr uint32_t HROWB = kTcRowCells * HC * 2;     // bytes of one input-slab row
    constexpr uint32_t HSLAB = (kWgRows + 2) * HROWB;
    constexpr uint32_t GROWB = kTcCells * GC * 2;         // bytes of one gradient row
    constexpr uint32_t GSLOT = kWgRows * GROWB;
    constexpr uint32_t HLAY = HC == 32 ? 4u : 6u, GLAY = GC == 32 ? 4u : 6u;
    constexpr uint32_t HATOM = HC == 32 ? 512u : 256u, GATOM = GC == 32 ? 512u : 256u;
    constexpr uint32_t ACOLS = NDX * 3 * GC;              // accumulator columns (dx blocks x 3 dz x GC)
    constexpr uint32_t TMEM_COLS = ACOLS <= 256 ? 256 : 512;
    constexpr int MMAW = 4, PRODW = 5;
    // blocks j >= 3 of the last slab read up to MB - 3 rows past it: the
    // gradient ring that follows is larger
    static_assert((MB - 3) * HROWB <= (kWgGSlots + 2) * GSLOT, "A reads stay in shared memory");
    static_assert(HSLAB % 1024 == 0 && GSLOT % 1024 == 0, "slabs keep the swizzle atoms aligned");
    extern __shared__ __align__(1024) unsigned char smem_wg[];
    __shared__ __align__(8) uint64_t h_full[kWgHSlabs], h_empty[kWgHSlabs], g_full[kWgGSlots], g_empty[kWgGSlots];
    __shared__ __align__(8) uint64_t zero_bar, done_bar, fin_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = a.L;
    const uint32_t hbase = gs_smem_addr(smem_wg);
    const uint32_t gbase = hbase + kWgHSlabs * HSLAB;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gs_smem_addr(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kWgHSlabs; ++i) {
            gs_mbar_init(&h_full[i], 1);
            gs_mbar_init(&h_empty[i], 1);
        }
        for (int i = 0; i < kWgGSlots; ++i) {
            gs_mbar_init(&g_full[i], 1);
            gs_mbar_init(&g_empty[i], 1 + 4);  // the MMA commit and the 4 epilogue warps
        }
        gs_mbar_init(&zero_bar, 4);
        gs_mbar_init(&done_bar, 1);
        gs_mbar_init(&fin_bar, 1);
        abort_s = 0;
        gs_fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const int nseg = L / kTcCells, nyg = L / kWgRows, nzc = (L + kWgZChunk - 1) / kWgZChunk;
    const long long units = (long long)a.N * nyg * nseg * nzc;
    struct Unit {
        int n, x0, y0, z0, nz;
    };
    auto decode = [&](long long unit) {
        Unit u;
        const int zc = (int)(unit % nzc);
        long long r0 = unit / nzc;
        const int seg = (int)(r0 % nseg);
        r0 /= nseg;
        u.y0 = (int)(r0 % nyg) * kWgRows;
        u.n = (int)(r0 / nyg);
        u.x0 = seg * kTcCells;
        u.z0 = zc * kWgZChunk;
        u.nz = min(kWgZChunk, L - u.z0);
        return u;
    };
    auto bwait = [&](uint64_t* bar, uint32_t parity) -> bool {
        if (gs_mbar_try_wait(bar, parity)) return true;
        const uint64_t t0 = gs_globaltimer();
        for (;;) {
#pragma unroll 1
            for (int i = 0; i < 32; ++i)
                if (gs_mbar_try_wait(bar, parity)) return true;
            if (abort_s) return false;
            if (gs_globaltimer() - t0 > a.timeout_ns) {
                abort_s = 1;
                gs_report(a.err, GS_DERR_TIMEOUT);
                return false;
            }
        }
    };
    auto wwait = [&](uint64_t* bar, uint32_t parity) -> bool {
        int r = 0;
        if (lane == 0) r = bwait(bar, parity) ? 1 : 0;
        r = __shfl_sync(0xffffffffu, r, 0);
        return r != 0;
    };

    if (warp == PRODW) {
        // ------------------------ producer (TMA, one elected lane) ------------------------
        // per unit, for pi = 0 .. nz+1: gradient plane z0 + pi (if pi < nz; into
        // slot G % 4, and also slot G % 4 + 4 when G % 4 < 2), then input plane
        // z0 - 1 + pi (rows y0-1 .. y0+2, each as halo / 128-cell / halo boxes)
        const uint32_t leader = tc_elect_one();
        if ((hbase & 1023u) == 0) {
            if (leader) {
                gs_prefetch_tmap(&a.map_hmain);
                gs_prefetch_tmap(&a.map_hhalo);
                gs_prefetch_tmap(&a.map_g);
            }
            __syncwarp();
            uint32_t H = 0, G = 0;
            bool ok = true;
            for (long long unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
                const Unit u = decode(unit);
                const int xl = (u.x0 - kTcRowX0 + L) % L, xr = (u.x0 + kTcCells) % L;
                for (int pi = 0; pi < u.nz + 2 && ok; ++pi) {
                    if (pi < u.nz) {
                        const uint32_t gs = G % kWgGSlots;
                        if (G >= (uint32_t)kWgGSlots && !wwait(&g_empty[gs], ((G / kWgGSlots) - 1u) & 1u)) {
                            ok = false;
                            break;
                        }
                        const bool mirror = gs < 2;
                        tc_arrive_expect_tx_if(leader, &g_full[gs], GSLOT * (mirror ? 2u : 1u));
                        const int zq = u.n * L + u.z0 + pi;
#pragma unroll
                        for (int r = 0; r < kWgRows; ++r) {
                            const uint32_t dst = gbase + gs * GSLOT + r * GROWB;
                            tc_tma_load_4d_if(leader, dst, &a.map_g, &g_full[gs], 0, u.x0, u.y0 + r, zq);
                            if (mirror)
                                tc_tma_load_4d_if(leader, dst + kWgGSlots * GSLOT, &a.map_g, &g_full[gs], 0, u.x0,
                                                  u.y0 + r, zq);
                        }
                        ++G;
                    }
                    const uint32_t hs = H % kWgHSlabs;
                    if (H >= (uint32_t)kWgHSlabs && !wwait(&h_empty[hs], ((H / kWgHSlabs) - 1u) & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_arrive_expect_tx_if(leader, &h_full[hs], HSLAB);
                    const int zp = u.n * L + (u.z0 - 1 + pi + L) % L;
#pragma unroll
                    for (int r = 0; r < kWgRows + 2; ++r) {
                        const int yy = (u.y0 - 1 + r + L) % L;
                        const uint32_t row = hbase + hs * HSLAB + r * HROWB;
                        tc_tma_load_4d_if(leader, row, &a.map_hhalo, &h_full[hs], 0, xl, yy, zp);
                        tc_tma_load_4d_if(leader, row + kTcRowX0 * HC * 2, &a.map_hmain, &h_full[hs], 0, u.x0, yy, zp);
                        tc_tma_load_4d_if(leader, row + (kTcRowX0 + kTcCells) * HC * 2, &a.map_hhalo, &h_full[hs], 0,
                                          xr, yy, zp);
                    }
                    ++H;
                }
            }
            if (!ok && lane == 0) {
                // let the copies in flight land (fixed budget)
                for (uint32_t q = H > (uint32_t)kWgHSlabs ? H - kWgHSlabs : 0u; q < H; ++q)
                    gs_mbar_wait(&h_full[q % kWgHSlabs], (q / kWgHSlabs) & 1u, 2000000000ull);
                for (uint32_t q = G > (uint32_t)kWgGSlots ? G - kWgGSlots : 0u; q < G; ++q)
                    gs_mbar_wait(&g_full[q % kWgGSlots], (q / kWgGSlots) & 1u, 2000000000ull);
            }
        } else if (lane == 0) {
            abort_s = 1;  // unaligned shared memory: refuse to issue TMA
            gs_report(a.err, GS_DERR_BADARG);
        }
    } else if (warp == MMAW) {
        // ------------------------ MMA issuer (one elected lane) ------------------------
        const uint32_t leader = tc_elect_one();
        bool ok = wwait(&zero_bar, 0);
        tc_fence_after();
        uint32_t H = 0, G = 0;
        for (long long unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
            const Unit u = decode(unit);
            const uint32_t Gb = G;
            for (int pi = 0; pi < u.nz + 2; ++pi) {
                // gradient plane z0 + pi is first needed now
                if (pi < u.nz && !wwait(&g_full[(Gb + pi) % kWgGSlots], ((Gb + pi) / kWgGSlots) & 1u)) {
                    ok = false;
                    break;
                }
                const uint32_t hs = H % kWgHSlabs;
                if (!wwait(&h_full[hs], (H / kWgHSlabs) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // gradient planes q = p - 1 + b (b = 0, 1, 2 <-> dz = +1, 0, -1) inside the unit
                const int b_lo = max(0, 2 - pi), b_hi = min(2, u.nz + 1 - pi);
                const uint32_t gslot = (Gb + (uint32_t)(pi - 2 + b_lo)) % kWgGSlots;
                const uint32_t idesc = tc_idesc_mn((b_hi - b_lo + 1) * GC);
#pragma unroll 1
                for (int i = 0; i < kWgRows; ++i) {
                    const uint32_t arow = hbase + hs * HSLAB + i * HROWB;
                    const uint32_t brow = gbase + gslot * GSLOT + i * GROWB;
#pragma unroll
                    for (int dxc = 0; dxc < NDX; ++dxc) {
                        // with a packed operand the input cell is not shifted (dx in the channels)
                        const int shift = XTS ? 0 : dxc - 1;
                        const uint32_t dcol = tmem + (uint32_t)(dxc * 3 * GC + b_lo * GC);
#pragma unroll
                        for (int ks = 0; ks < kTcCells / 16; ++ks) {
                            // output cell x0 + 16 ks + k reads input cell x0 + 16 ks + k + dx
                            const uint64_t ad = tc_desc_lay(arow + (uint32_t)(kTcRowX0 + 16 * ks + shift) * HC * 2,
                                                            HROWB, 8 * HC * 2, HLAY);
                            const uint64_t bd = tc_desc_lay(brow + (uint32_t)(16 * ks) * GC * 2, GSLOT, 8 * GC * 2, GLAY);
                            tc_mma_if(leader, dcol, ad, bd, idesc, 1u);
                        }
                    }
                }
                tc_commit_if(leader, &h_empty[hs]);
                // gradient plane z0 + pi - 2 (= p - 1) had its last use
                if (pi >= 2) tc_commit_if(leader, &g_empty[(Gb + pi - 2) % kWgGSlots]);
                ++H;
            }
            G = Gb + (uint32_t)u.nz;
        }
        if (ok) {
            tc_commit_if(leader, &done_bar);
        } else {
            tc_commit_if(leader, &fin_bar);
            if (lane == 0) gs_mbar_wait(&fin_bar, 0, 2000000000ull);
        }
        (void)HATOM;
        (void)GATOM;
    } else {
        // --------------------- epilogue warps 0..3 ----------------------
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (uint32_t c = 0; c < ACOLS; c += 32) tc_st_zero32(lane_base + c);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) gs_mbar_arrive(&zero_bar);
        // bias gradient: thread t sums channel pair t % (GC/2) over the cells
        // t / (GC/2), + 128/(GC/2), ... of every gradient plane (2 rows x 128
        // cells, channels-last with the TMA's 64- or 32-byte swizzle: the
        // 16-byte chunk index is XORed with address bits 7-8, resp. bit 7)
        constexpr int NPAIR = GC / 2, NGRP = 128 / NPAIR;
        const int cp = tid % NPAIR, cg = tid / NPAIR;
        float db0 = 0.f, db1 = 0.f;
        bool ok = true;
        {
            uint32_t G = 0;
            for (long long unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
                const Unit u = decode(unit);
                for (int pi = 0; pi < u.nz; ++pi, ++G) {
                    const uint32_t gs = G % kWgGSlots;
                    if (!wwait(&g_full[gs], (G / kWgGSlots) & 1u)) {
                        ok = false;
                        break;
                    }
                    const unsigned char* slot = smem_wg + kWgHSlabs * HSLAB + gs * GSLOT;
#pragma unroll 4
                    for (int c = cg; c < kWgRows * kTcCells; c += NGRP) {
                        const uint32_t off = (uint32_t)c * GC * 2 + (uint32_t)cp * 4;
                        const uint32_t sw = GC == 32 ? ((off >> 7) & 3u) : ((off >> 7) & 1u);
                        const __nv_bfloat162 v2 =
                            *reinterpret_cast<const __nv_bfloat162*>(slot + (off ^ (sw << 4)));
                        db0 += __bfloat162float(v2.x);
                        db1 += __bfloat162float(v2.y);
                    }
                    __syncwarp();
                    if (lane == 0) gs_mbar_arrive(&g_empty[gs]);
                }
            }
        }
        if (ok && wwait(&done_bar, 0)) {
            tc_fence_after();
            // TMEM lane m = 32 warp + lane is M row m: block j = m / HC (dy = j - 1), channel ci = m % HC
            const int m = warp * 32 + lane;
            const int j = m / HC, ci = m % HC;
            float* const part = a.part + (size_t)blockIdx.x * (27 * HC * GC + GC);
#pragma unroll 1
            for (int dxc = 0; dxc < NDX; ++dxc)
#pragma unroll 1
                for (int b = 0; b < 3; ++b) {
                    float v[GC];
                    tc_ld<GC>(lane_base + (uint32_t)(dxc * 3 * GC + b * GC), v);
                    if (j > 2) continue;
                    if constexpr (XTS == 0) {
                        const int tap = 9 * (2 - b) + 3 * j + dxc;  // dz = 1 - b, dy = j - 1, dx = dxc - 1
                        float* dst = part + ((size_t)tap * HC + ci) * GC;
#pragma unroll
                        for (int e = 0; e < GC; e += 8) {
                            uint4 lo, hi;
                            lo.x = __float_as_uint(v[e]);
                            lo.y = __float_as_uint(v[e + 1]);
                            lo.z = __float_as_uint(v[e + 2]);
                            lo.w = __float_as_uint(v[e + 3]);
                            hi.x = __float_as_uint(v[e + 4]);
                            hi.y = __float_as_uint(v[e + 5]);
                            hi.z = __float_as_uint(v[e + 6]);
                            hi.w = __float_as_uint(v[e + 7]);
                            gs_st_v8(dst + e, lo, hi);
                        }
                    } else if constexpr (XTS == 1) {
                        // packed input channel ci = 4 d + c: dx = d - 1, input channel c
                        const int d = ci / 4, c = ci % 4;
                        if (d < 3) {
                            float* dst = part + ((size_t)(9 * (2 - b) + 3 * j + d) * HC + c) * GC;
#pragma unroll
                            for (int e = 0; e < GC; ++e) dst[e] = v[e];
                        }
                    } else {
                        // packed gradient column 2 d + co: dx = 1 - d, output channel co
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            float* dst = part + ((size_t)(9 * (2 - b) + 3 * j + (2 - d)) * HC + ci) * GC;
                            dst[0] = v[2 * d];
                            dst[1] = v[2 * d + 1];
                        }
                    }
                }
        }
        // bias partial sums: the cell groups of a channel pair, in a fixed order
        __shared__ float dbs[128][2];
        dbs[tid][0] = db0;
        dbs[tid][1] = db1;
        asm volatile("bar.sync 1, 128;" ::: "memory");  // the 4 epilogue warps only
        if (tid < NPAIR) {
            float s0 = 0.f, s1 = 0.f;
            for (int g = 0; g < NGRP; ++g) {
                s0 += dbs[g * NPAIR + tid][0];
                s1 += dbs[g * NPAIR + tid][1];
            }
            float* dst = a.part + (size_t)blockIdx.x * (27 * HC * GC + GC) + 27 * HC * GC;
            if constexpr (XTS == 2) {
                // the packed dL/dout holds each cell's own values in channels 2, 3 (d = 1)
                if (tid == 1) {
                    dst[0] = s0;
                    dst[1] = s1;
                }
            } else {
                dst[2 * tid] = s0;
                dst[2 * tid + 1] = s1;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// dW[tap][ci][co] and db[co] = sums over the CTAs' partial sums (ci < cin,
// co < cout); part is [nblk][27 HC GC + GC].  A block takes 32 consecutive
// outputs; its 8 thread groups sum every 8th CTA's partials (several loads in
// flight per thread), then the 8 sums are added in a fixed order (the result
// does not depend on timing).
constexpr int kWgRedOut = 32, kWgRedGrp = 8;
__global__ void __launch_bounds__(kWgRedOut * kWgRedGrp) gs_wgrad_reduce_kernel(const float* __restrict__ part, int nblk,
                                                                                int HC, int GC, int cin, int cout,
                                                                                float* __restrict__ dw,
                                                                                float* __restrict__ db)
{
    __shared__ float red[kWgRedGrp][kWgRedOut];
    const int nw = 27 * cin * cout;
    const int o = threadIdx.x % kWgRedOut, grp = threadIdx.x / kWgRedOut;
    const int i = blockIdx.x * kWgRedOut + o;
    float acc = 0.f;
    if (i < nw + cout) {
        size_t off;
        if (i < nw) {
            const int co = i % cout, ci = (i / cout) % cin, tap = i / (cout * cin);
            off = ((size_t)tap * HC + ci) * GC + co;
        } else {
            off = (size_t)27 * HC * GC + (i - nw);
        }
        const float* p = part + off;
        const size_t stride = (size_t)27 * HC * GC + GC;
#pragma unroll 4
        for (int b = grp; b < nblk; b += kWgRedGrp) acc += p[(size_t)b * stride];
    }
    red[grp][o] = acc;
    __syncthreads();
    if (grp == 0 && i < nw + cout) {
        float v = 0.f;
#pragma unroll
        for (int g = 0; g < kWgRedGrp; ++g) v += red[g][o];
        if (i < nw) dw[i] = v;
        else db[i - nw] = v;
    }
}

// fp32 master weights [27][cin][cout] (tap = 9 dz + 3 dy + dx, each + 1) ->
// tcgen05 B layout [3 dz][3 dx][cinp/8][3 nt][8], n = (2 - (dy + 1)) * nt + cout
// (zero padded)
__global__ void gs_wprep_tc_kernel(const float* __restrict__ w, int cin, int cout, int cinp, int nt, bf16* __restrict__ wt)
{
    const int nn = 3 * nt;
    const int total = 9 * cinp * nn;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i % 8;
        const int n = (i / 8) % nn;
        const int j = (i / (8 * nn)) % (cinp / 8);
        const int dxi = (i / (8 * nn * (cinp / 8))) % 3;
        const int dzi = i / (8 * nn * (cinp / 8) * 3);
        const int dyi = 2 - n / nt;
        const int co = n % nt;
        const int tap = dzi * 9 + dyi * 3 + dxi;
        const int ci = j * 8 + e;
        const float val = (ci < cin && co < cout) ? w[((size_t)tap * cin + ci) * cout + co] : 0.f;
        wt[i] = __float2bfloat16_rn(val);
    }
}

// the data gradient's weights in the same B layout: the convolution of gz
// (K = the forward layer's output channels, padded to kp) with tap-flipped,
// transposed weights, W'[tap][k][n] = W[26 - tap][n][k] (n = the forward
// layer's input channels, padded to nt)
__global__ void gs_wprep_tc_dgrad_kernel(const float* __restrict__ w, int cin, int cout, int kp, int nt,
                                         bf16* __restrict__ wt)
{
    const int nn = 3 * nt;
    const int total = 9 * kp * nn;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i % 8;
        const int n = (i / 8) % nn;
        const int j = (i / (8 * nn)) % (kp / 8);
        const int dxi = (i / (8 * nn * (kp / 8))) % 3;
        const int dzi = i / (8 * nn * (kp / 8) * 3);
        const int dyi = 2 - n / nt;
        const int ci = n % nt;     // forward input channel (this convolution's output)
        const int co = j * 8 + e;  // forward output channel (this convolution's input)
        const int tap = dzi * 9 + dyi * 3 + dxi;
        const float val = (ci < cin && co < cout) ? w[((size_t)(26 - tap) * cin + ci) * cout + co] : 0.f;
        wt[i] = __float2bfloat16_rn(val);
    }
}

// the last layer's data-gradient weights for x-tap packed dL/dout (channels
// 2 d + c hold channel c of cell x + d - 1): [3 dz][2 chunks][3 nt][8], K
// index k = 2 d + c (k < 6), the three dy taps side by side along N
__global__ void gs_wprep_tc_dgrad_xtaps_kernel(const float* __restrict__ w, int cin, int cout, int nt,
                                               bf16* __restrict__ wt)
{
    const int nn = 3 * nt;
    const int total = 3 * 2 * nn * 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i % 8;
        const int n = (i / 8) % nn;
        const int j = (i / (8 * nn)) % 2;
        const int dzi = i / (8 * nn * 2);
        const int kx = j * 8 + e, d = kx / 2, co = kx % 2;
        const int dyi = 2 - n / nt;
        const int ci = n % nt;
        const int tap = dzi * 9 + dyi * 3 + d;
        const float val = (kx < 6 && ci < cin && co < cout) ? w[((size_t)(26 - tap) * cin + ci) * cout + co] : 0.f;
        wt[i] = __float2bfloat16_rn(val);
    }
}

// the last layer's weights for its dz-stacked schedule (EPI_LAST in
// gs_conv_tc_kernel): [6 slab rows][3 dx][2 K steps][2 chunks][48][8], row
// n = 16 b + 2 r + co (2 r + co < 8, the rest zero): block b feeds output
// plane z' - 1 + b from input plane z' (dz = 1 - b), and slab row sr feeds
// output row r through dy = sr - 1 - r (zero where |dy| > 1)
__global__ void gs_wprep_tc_last_kernel(const float* __restrict__ w, int cin, int cout, bf16* __restrict__ wt)
{
    const int total = 6 * 3 * 2 * 2 * 48 * 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i % 8;
        const int n = (i / 8) % 48;
        const int j = (i / (8 * 48)) % 2;
        const int kk = (i / (8 * 48 * 2)) % 2;
        const int dxi = (i / (8 * 48 * 4)) % 3;
        const int sr = i / (8 * 48 * 12);
        const int b = n / 16, rc = n % 16, r = rc / 2, co = rc % 2;
        const int dzi = 2 - b, dyi = sr - r;
        const int ci = kk * 16 + j * 8 + e;
        const bool on = rc < 8 && dyi >= 0 && dyi <= 2 && ci < cin && co < cout;
        const float val = on ? w[((size_t)(dzi * 9 + dyi * 3 + dxi) * cin + ci) * cout + co] : 0.f;
        wt[i] = __float2bfloat16_rn(val);
    }
}

// the first layer's weights for x-tap packed input (gs_pack_kernel with
// xtaps): [3 dz][2 chunks][3 NT][8], K index k = 4 dx + ci (k < 12), the three
// dy taps side by side along N as in gs_wprep_tc_kernel
__global__ void gs_wprep_tc_xtaps_kernel(const float* __restrict__ w, int cin, int cout, int nt, bf16* __restrict__ wt)
{
    const int nn = 3 * nt;
    const int total = 3 * 2 * nn * 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i % 8;
        const int n = (i / 8) % nn;
        const int j = (i / (8 * nn)) % 2;
        const int dzi = i / (8 * nn * 2);
        const int kx = j * 8 + e, dxi = kx / 4, ci = kx % 4;
        const int dyi = 2 - n / nt;
        const int co = n % nt;
        const int tap = dzi * 9 + dyi * 3 + dxi;
        const float val = (kx < 12 && ci < cin && co < cout) ? w[((size_t)tap * cin + ci) * cout + co] : 0.f;
        wt[i] = __float2bfloat16_rn(val);
    }
}

}  // namespace gs

// ===========================================================================
// Host side
// ===========================================================================
using namespace gs;

struct gs_surr {
    float* params = nullptr;  // fp32 master: per layer W [27][cin][cout] then b [cout]
    float* grads = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    size_t np = 0;
    size_t woff[kSurrLayers] = {}, boff[kSurrLayers] = {};
    bf16* wf[kSurrLayers] = {};  // forward layout
    bf16* wd[kSurrLayers] = {};  // data-gradient layout (layers 1..5)
    bf16* wt[kSurrLayers] = {};  // tcgen05 B layout [3 dz][3 dx][CINP/8][3 NT][8]
    bf16* wt0x = nullptr;        // the first layer's for x-tap packed input [3 dz][2][3 NT][8]
    bf16* wdt[kSurrLayers] = {}; // tcgen05 B layout of the data gradient (layers 1..5)
    bf16* wdt5x = nullptr;       // the last layer's, for x-tap packed dL/dout [3 dz][2][3 NT][8]
    unsigned wdirty = 3;        // bit 0: mma.sync weight layouts stale, bit 1: tcgen05 layouts stale
    int backend = 0;             // 0 auto (tcgen05 when L % 128 == 0), 1 mma.sync, 2 tcgen05
    int* d_err = nullptr;
    // workspace
    int N = 0, L = 0;
    bool train_ws = false;
    bf16* x0 = nullptr;
    bf16* h[kSurrLayers] = {};  // h[1..5] (training) / h[1], h[2] ping-pong (inference)
    uint32_t* zm[kSurrLayers - 1] = {};  // training: ReLU mask words of layers 0..4
    bf16* gh = nullptr;  // training: the residual-path gradient dL/dh_l, bf16 [cells][32]
    bf16* gz[2] = {};
    bf16* gd = nullptr;
    float* ou = nullptr;
    float* ov = nullptr;
    float* fk = nullptr;
    float* wpart = nullptr;  // per-CTA weight-gradient partial sums (tensor-core path)
    double* d_loss = nullptr;
    unsigned* d_max = nullptr;
    double* d_ss = nullptr;
    cudaStream_t stream = nullptr;
    int64_t adam_t = 0;
    int64_t launches = 0;
    float* trace_dh = nullptr;  // checking aid: caller's array for dL/dh_l, l = 1..5
    size_t trace_count = 0;
};

namespace {

constexpr char kSurrMagic[8] = {'G', 'S', 'S', 'U', 'R', 'R', '0', '1'};

int surr_valid_L(int L)
{
    if (L < 16 || L % 16 || (L > 128 && L % 128))
        return fail(GS_EINVAL, "surrogate grid L=%d must be a multiple of 16 (and of 128 above 128)", L);
    return GS_OK;
}

void free_ws(gs_surr* s)
{
    guarded_free(s->x0);
    for (auto& p : s->h) { guarded_free(p); p = nullptr; }
    for (auto& p : s->zm) { guarded_free(p); p = nullptr; }
    guarded_free(s->gh);
    guarded_free(s->gz[0]);
    guarded_free(s->gz[1]);
    guarded_free(s->gd);
    guarded_free(s->ou);
    guarded_free(s->ov);
    guarded_free(s->fk);
    guarded_free(s->wpart);
    s->wpart = nullptr;
    s->x0 = nullptr; s->gh = nullptr; s->gz[0] = s->gz[1] = nullptr; s->gd = nullptr;
    s->ou = s->ov = nullptr; s->fk = nullptr;
    s->N = s->L = 0;
}

int ensure_ws(gs_surr* s, int N, int L, bool train)
{
    if (s->N == N && s->L == L && (s->train_ws || !train)) return GS_OK;
    free_ws(s);
    const size_t cells = (size_t)N * L * L * L;
    cudaError_t e;
#define ALLOC(p, bytes) if ((e = guarded_malloc((void**)&(p), (bytes))) != cudaSuccess) { free_ws(s); return cuda_fail(e, "surrogate workspace"); }
    ALLOC(s->x0, cells * 16 * sizeof(bf16));
    ALLOC(s->fk, (size_t)N * 2 * sizeof(float));
    const int nh = train ? 5 : 2;
    for (int l = 1; l <= nh; ++l) ALLOC(s->h[l], cells * 32 * sizeof(bf16));
    if (train) {
        for (int l = 0; l < 5; ++l) ALLOC(s->zm[l], cells * sizeof(uint32_t));
        ALLOC(s->gh, cells * 32 * sizeof(bf16));
        ALLOC(s->gz[0], cells * 32 * sizeof(bf16));
        ALLOC(s->gz[1], cells * 32 * sizeof(bf16));
        ALLOC(s->gd, cells * 16 * sizeof(bf16));
        ALLOC(s->ou, cells * sizeof(float));
        ALLOC(s->ov, cells * sizeof(float));
        ALLOC(s->wpart, (size_t)num_sms() * (27 * 32 * 32 + 32) * sizeof(float));
    }
#undef ALLOC
    s->N = N;
    s->L = L;
    s->train_ws = train;
    return GS_OK;
}

template <int CINP, int COUTP, int EPI>
int conv_launch(gs_surr* s, ConvArgs a)
{
    const int SEG = a.L < 128 ? a.L : 128;
    const size_t smem = (size_t)27 * COUTP * CINP * 2 + (size_t)18 * (SEG + 2) * CINP * 2;
    auto k = gs_conv_kernel<CINP, COUTP, EPI>;
    GS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kConvThreads, smem));
    if (per_sm < 1) return fail(GS_EINVAL, "convolution tile does not fit on an SM");
    const long long items = (long long)a.N * a.L * (a.L / kRows) * (a.L / SEG);
    const int grid = (int)std::min<long long>(items, (long long)per_sm * num_sms());
    k<<<grid, kConvThreads, smem, s->stream>>>(a);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    return GS_OK;
}

template <int CINP, int NP>
int wgrad_launch(gs_surr* s, WgArgs a)
{
    const int SEG = a.L < 128 ? a.L : 128;
    const size_t smem = (size_t)18 * (SEG + 2) * CINP * 2 + (size_t)kRows * SEG * NP * 2;
    auto k = gs_wgrad_kernel<CINP, NP>;
    GS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWgThreads, smem));
    if (per_sm < 1) return fail(GS_EINVAL, "weight-gradient tile does not fit on an SM");
    const long long items = (long long)a.N * a.L * (a.L / kRows) * (a.L / SEG);
    const int grid = (int)std::min<long long>(items, (long long)per_sm * num_sms());
    k<<<grid, kWgThreads, smem, s->stream>>>(a);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    return GS_OK;
}

// weight and bias gradients on the tensor cores: h (HC channels), g (GC
// channels) -> dw [27][cin][cout], db [cout] (overwritten)
template <int HC, int GC, int XTS>
int wgrad_tc_launch(gs_surr* s, int N, int L, const bf16* h, const bf16* g, int cin, int cout, float* dw, float* db)
{
    constexpr uint32_t HSLAB = (kWgRows + 2) * kTcRowCells * HC * 2;
    constexpr uint32_t GSLOT = kWgRows * kTcCells * GC * 2;
    const size_t smem = (size_t)kWgHSlabs * HSLAB + (size_t)(kWgGSlots + 2) * GSLOT;
    if (L % kTcCells) return fail(GS_EINVAL, "the tcgen05 path needs L %% %d == 0 (L=%d)", kTcCells, L);
    WgTcArgs a{};
    a.N = N;
    a.L = L;
    if (encode_act_4d(&a.map_hmain, h, HC, L, (long long)N * L, HC, kTcCells, HC == 32 ? 64 : 32) != CUDA_SUCCESS ||
        encode_act_4d(&a.map_hhalo, h, HC, L, (long long)N * L, HC, 8, HC == 32 ? 64 : 32) != CUDA_SUCCESS ||
        encode_act_4d(&a.map_g, g, GC, L, (long long)N * L, GC, kTcCells, GC == 32 ? 64 : 32) != CUDA_SUCCESS)
        return fail(GS_ECUDA, "cuTensorMapEncodeTiled failed for the weight-gradient maps");
    auto k = gs_wgrad_tc_kernel<HC, GC, XTS>;
    GS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWgTcThreads, smem));
    if (per_sm < 1) return fail(GS_EINVAL, "tensor-core weight gradient does not fit on an SM");
    const long long units = (long long)N * (L / kWgRows) * (L / kTcCells) * ((L + kWgZChunk - 1) / kWgZChunk);
    const int grid = (int)std::min<long long>(units, (long long)num_sms());
    a.part = s->wpart;
    a.err = s->d_err;
    a.timeout_ns = 2000000000ull;
    k<<<grid, kWgTcThreads, smem, s->stream>>>(a);
    GS_CUDA_TRY(cudaGetLastError());
    gs_wgrad_reduce_kernel<<<(27 * cin * cout + cout + kWgRedOut - 1) / kWgRedOut, kWgRedOut * kWgRedGrp, 0, s->stream>>>(
        s->wpart, grid, HC, GC, cin, cout, dw, db);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 2;
    return GS_OK;
}

template <int CINP, int NT, int EPI, bool XT = false>
int tc_launch(gs_surr* s, ConvTcArgs a)
{
    constexpr uint32_t SLAB = (CINP / 8) * kTcSlabRows * kTcRowCells * 16;
    const size_t wbytes = EPI == EPI_LAST ? (size_t)6 * 3 * 2 * 2 * 48 * 16 : (size_t)(XT ? 9 : 27) * (CINP / 8) * NT * 16;
    const size_t smem = (XT ? 6 : 3) * (size_t)SLAB + wbytes;  // the kernel's slab ring depth
    if (a.L % kTcCells) return fail(GS_EINVAL, "the tcgen05 path needs L %% %d == 0 (L=%d)", kTcCells, a.L);
    // see gs_conv_tc_kernel: 32 channels with the 64-byte swizzle, x-tap
    // input (16 channels) with the 32-byte swizzle, else 16-byte chunks
    constexpr int SWZ = CINP == 32 ? 64 : (XT ? 32 : 0);
    const int box_c = SWZ ? CINP : 8;
    if (encode_act_4d(&a.map_main, a.in, CINP, a.L, (long long)a.N * a.L, box_c, kTcCells, SWZ) != CUDA_SUCCESS ||
        encode_act_4d(&a.map_halo, a.in, CINP, a.L, (long long)a.N * a.L, box_c, 8, SWZ) != CUDA_SUCCESS)
        return fail(GS_ECUDA, "cuTensorMapEncodeTiled failed for the activation maps");
    auto k = gs_conv_tc_kernel<CINP, NT, EPI, XT>;
    GS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, tc_threads(EPI, XT), smem));
    if (per_sm < 1) return fail(GS_EINVAL, "tensor-core convolution does not fit on an SM");
    per_sm = std::min(per_sm, EPI == EPI_LAST ? 1 : 2);  // TMEM: 512 columns a CTA (last layer), else <= 256
    a.err = s->d_err;
    a.timeout_ns = 2000000000ull;
    const long long units = (long long)a.N * (a.L / kTcRows) * (a.L / kTcCells) * ((a.L + kTcZChunk - 1) / kTcZChunk);
    const int grid = (int)std::min<long long>(units, (long long)per_sm * num_sms());
    k<<<grid, tc_threads(EPI, XT), smem, s->stream>>>(a);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    return GS_OK;
}

int grid1d(long long n, int block) { return (int)std::max<long long>(1, std::min<long long>((n + block - 1) / block, 8LL * num_sms())); }

// bf16 weight layouts of the path about to run (mma.sync: forward and data
// gradient; tcgen05: forward, x-tap first layer, data gradient, x-tap last
// layer), redone after the parameters change
int prep_weights(gs_surr* s, bool tc)
{
    const unsigned need = tc ? 2u : 1u;
    if (!(s->wdirty & need)) return GS_OK;
    for (int l = 0; l < kSurrLayers; ++l) {
        const int cin = kChan[l], cout = kChan[l + 1];
        if (!tc) {
            gs_wprep_kernel<<<64, 256, 0, s->stream>>>(s->params + s->woff[l], cin, cout, s->wf[l], kCoutP[l],
                                                      kCinP[l], l >= 1 ? s->wd[l] : nullptr, l == 5 ? 16 : 32);
        } else if (l == 5) {
            gs_wprep_tc_last_kernel<<<64, 256, 0, s->stream>>>(s->params + s->woff[l], cin, cout, s->wt[l]);
        } else {
            if (l >= 1)
                gs_wprep_tc_kernel<<<64, 256, 0, s->stream>>>(s->params + s->woff[l], cin, cout, kCinP[l], 32,
                                                             s->wt[l]);
            if (l >= 1)
                gs_wprep_tc_dgrad_kernel<<<64, 256, 0, s->stream>>>(s->params + s->woff[l], cin, cout, 32, 32,
                                                                   s->wdt[l]);
        }
        GS_CUDA_TRY(cudaGetLastError());
        s->launches += (tc && l >= 1 && l <= 4) ? 2 : (tc && l == 0 ? 0 : 1);
    }
    if (tc) {
        gs_wprep_tc_xtaps_kernel<<<16, 256, 0, s->stream>>>(s->params + s->woff[0], kChan[0], kChan[1], 32, s->wt0x);
        GS_CUDA_TRY(cudaGetLastError());
        gs_wprep_tc_dgrad_xtaps_kernel<<<16, 256, 0, s->stream>>>(s->params + s->woff[5], kChan[5], kChan[6], 32,
                                                                  s->wdt5x);
        GS_CUDA_TRY(cudaGetLastError());
        s->launches += 2;
    }
    s->wdirty &= ~need;
    return GS_OK;
}

int upload_fk(gs_surr* s, int N, const double* F, const double* k)
{
    std::vector<float> h((size_t)N * 2);
    for (int n = 0; n < N; ++n) {
        h[2 * n] = (float)F[n];
        h[2 * n + 1] = (float)k[n];
    }
    GS_CUDA_TRY(cudaMemcpyAsync(s->fk, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream));
    return GS_OK;
}

// forward pass; train: keep h1..h5 and z0..z4, write (ou, ov); else ping-pong
int forward(gs_surr* s, int N, int L, const float* u, const float* v, float* uo, float* vo, bool train)
{
    const long long cells = (long long)N * L * L * L;
    const bool tc = s->backend != 1 && L % kTcCells == 0;
    int rc = prep_weights(s, tc);
    if (rc) return rc;
    if (s->backend == 2 && !tc) return fail(GS_EINVAL, "the tcgen05 path needs L %% 128 == 0 (L=%d)", L);
    // the tensor-core path packs the x taps into the first layer's input
    // (its weight gradient reads the packed form too); mma.sync keeps the
    // plain layout
    const bool xtaps = tc;
    gs_pack_kernel<<<grid1d(cells, 256), 256, 0, s->stream>>>(u, v, s->fk, s->x0, (long long)L * L * L, N, L,
                                                              xtaps ? 1 : 0);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    if (tc) {
        ConvTcArgs t{};
        t.N = N;
        t.L = L;
        t.in = s->x0;
        t.w = xtaps ? s->wt0x : s->wt[0];
        t.bias = s->params + s->boff[0];
        t.out = s->h[1];
        t.zmask = train ? s->zm[0] : nullptr;
        if ((rc = xtaps ? tc_launch<16, 32, EPI_FIRST, true>(s, t) : tc_launch<16, 32, EPI_FIRST>(s, t))) return rc;
        for (int l = 1; l <= 4; ++l) {
            t.in = train ? s->h[l] : s->h[1 + ((l - 1) & 1)];
            t.out = train ? s->h[l + 1] : s->h[1 + (l & 1)];
            t.w = s->wt[l];
            t.bias = s->params + s->boff[l];
            t.zmask = train ? s->zm[l] : nullptr;
            if ((rc = tc_launch<32, 32, EPI_HIDDEN>(s, t))) return rc;
        }
        ConvTcArgs b{};
        b.N = N;
        b.L = L;
        b.in = train ? s->h[5] : s->h[1];
        b.w = s->wt[5];
        b.bias = s->params + s->boff[5];
        b.su = u;
        b.sv = v;
        b.ou = uo;
        b.ov = vo;
        return tc_launch<32, 16, EPI_LAST>(s, b);
    }
    ConvArgs a{};
    a.N = N;
    a.L = L;
    // layer 0
    a.in = s->x0;
    a.w = s->wf[0];
    a.bias = s->params + s->boff[0];
    a.out = s->h[1];
    a.zmask = train ? s->zm[0] : nullptr;
    if ((rc = conv_launch<16, 32, EPI_FIRST>(s, a))) return rc;
    // layers 1..4
    for (int l = 1; l <= 4; ++l) {
        bf16* hin = train ? s->h[l] : s->h[1 + ((l - 1) & 1)];
        bf16* hout = train ? s->h[l + 1] : s->h[1 + (l & 1)];
        a.in = hin;
        a.res = hin;
        a.w = s->wf[l];
        a.bias = s->params + s->boff[l];
        a.out = hout;
        a.zmask = train ? s->zm[l] : nullptr;
        if ((rc = conv_launch<32, 32, EPI_HIDDEN>(s, a))) return rc;
    }
    // layer 5: state update
    ConvArgs b{};
    b.N = N;
    b.L = L;
    b.in = train ? s->h[5] : s->h[1];
    b.w = s->wf[5];
    b.bias = s->params + s->boff[5];
    b.su = u;
    b.sv = v;
    b.ou = uo;
    b.ov = vo;
    return conv_launch<32, 8, EPI_LAST>(s, b);
}

// checking aid: copy the residual-path gradient gh = dL/dh_l (bf16) as FP32
// into slot l - 1 of the caller's trace array
int trace_dh(gs_surr* s, int l, long long cells)
{
    if (!s->trace_dh) return GS_OK;
    const long long n = cells * 32;
    gs_bf16_to_f32_kernel<<<grid1d(n, 256), 256, 0, s->stream>>>(s->gh, n, s->trace_dh + (size_t)(l - 1) * n);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

// gradients of the MSE loss into s->grads (zeroed first); loss into *loss
int backward(gs_surr* s, int N, int L, const float* tu, const float* tv, double* loss)
{
    const long long cells = (long long)N * L * L * L;
    // the tensor-core path (as in forward()) also takes the data and weight
    // gradients; the weight-gradient kernel also sums the bias gradients
    const bool tc = s->backend != 1 && L % kTcCells == 0;
    GS_CUDA_TRY(cudaMemsetAsync(s->grads, 0, s->np * sizeof(float), s->stream));
    GS_CUDA_TRY(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
    gs_mse_kernel<<<grid1d(cells, 256), 256, 0, s->stream>>>(s->ou, s->ov, tu, tv, cells, 1.0 / (2.0 * cells), s->gd,
                                                            s->d_loss, tc ? nullptr : s->grads + s->boff[5],
                                                            tc ? L : 0);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    int rc;
    auto bias_grad = [&](const bf16* g, int gst, int cout, float* db) -> int {
        gs_bias_grad_kernel<<<grid1d(cells, 32), 256, 0, s->stream>>>(g, cells, gst, cout, db);
        GS_CUDA_TRY(cudaGetLastError());
        s->launches += 1;
        return GS_OK;
    };
    // data gradient of layer l (input g, 16 or 32 channels): gh (+)= conv^T, gz
    // for the layer below (on the mma.sync path also db of the layer below; the
    // tensor-core weight gradient sums the bias gradients itself)
    auto dgrad = [&](int l, const bf16* g, int gh_acc, bf16* gz) -> int {
        if (tc) {
            ConvTcArgs t{};
            t.N = N;
            t.L = L;
            t.in = g;
            t.w = s->wdt[l];
            t.gh = s->gh;
            t.gh_acc = gh_acc;
            t.mprev = s->zm[l - 1];
            t.gz = gz;
            if (l == 5) {
                t.w = s->wdt5x;  // dL/dout is x-tap packed on this path
                return tc_launch<16, 32, EPI_DGRAD, true>(s, t);
            }
            return tc_launch<32, 32, EPI_DGRAD>(s, t);
        }
        ConvArgs d{};
        d.N = N;
        d.L = L;
        d.in = g;
        d.w = s->wd[l];
        d.gh = s->gh;
        d.gh_acc = gh_acc;
        d.mprev = s->zm[l - 1];
        d.gz = gz;
        int r = l == 5 ? conv_launch<16, 32, EPI_DGRAD>(s, d) : conv_launch<32, 32, EPI_DGRAD>(s, d);
        if (r) return r;
        return bias_grad(gz, 32, 32, s->grads + s->boff[l - 1]);
    };
    // layer 5
    WgArgs w{};
    w.N = N;
    w.L = L;
    w.in = s->h[5];
    w.g = s->gd;
    w.GST = 16;
    w.cin = 32;
    w.cout = 2;
    w.dw = s->grads + s->woff[5];
    if ((rc = tc ? wgrad_tc_launch<32, 16, 2>(s, N, L, s->h[5], s->gd, 32, 2, w.dw, s->grads + s->boff[5]) : wgrad_launch<32, 8>(s, w))) return rc;
    if ((rc = dgrad(5, s->gd, 0, s->gz[0]))) return rc;
    if ((rc = trace_dh(s, 5, cells))) return rc;
    int cur = 0;
    for (int l = 4; l >= 1; --l) {
        w.in = s->h[l];
        w.g = s->gz[cur];
        w.GST = 32;
        w.cin = 32;
        w.cout = 32;
        w.dw = s->grads + s->woff[l];
        if ((rc = tc ? wgrad_tc_launch<32, 32, 0>(s, N, L, s->h[l], s->gz[cur], 32, 32, w.dw, s->grads + s->boff[l]) : wgrad_launch<32, 32>(s, w)))
            return rc;
        if ((rc = dgrad(l, s->gz[cur], 1, s->gz[cur ^ 1]))) return rc;
        if ((rc = trace_dh(s, l, cells))) return rc;
        cur ^= 1;
    }
    // layer 0
    w.in = s->x0;
    w.g = s->gz[cur];
    w.GST = 32;
    w.cin = 4;
    w.cout = 32;
    w.dw = s->grads + s->woff[0];
    if ((rc = tc ? wgrad_tc_launch<16, 32, 1>(s, N, L, s->x0, s->gz[cur], 4, 32, w.dw, s->grads + s->boff[0]) : wgrad_launch<16, 32>(s, w)))
        return rc;
    if (loss) GS_CUDA_TRY(cudaMemcpyAsync(loss, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    return gs_surr_sync(s);
}

int diff(gs_surr* s, const float* a, const float* b, long long n, double* maxabs, double* rms)
{
    GS_CUDA_TRY(cudaMemsetAsync(s->d_max, 0, sizeof(unsigned), s->stream));
    GS_CUDA_TRY(cudaMemsetAsync(s->d_ss, 0, sizeof(double), s->stream));
    gs_diff_kernel<<<grid1d(n, 256), 256, 0, s->stream>>>(a, b, n, s->d_max, s->d_ss);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    unsigned mb = 0;
    double ss = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&mb, s->d_max, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    GS_CUDA_TRY(cudaMemcpyAsync(&ss, s->d_ss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    float mx;
    memcpy(&mx, &mb, sizeof(float));
    if (maxabs) *maxabs = mx;
    if (rms) *rms = sqrt(ss / (double)n);
    return GS_OK;
}

int check_fields(int N, int L, const void* u, const void* v)
{
    if (N < 1) return fail(GS_EINVAL, "N=%d must be >= 1", N);
    int rc = surr_valid_L(L);
    if (rc) return rc;
    if (!u || !v) return fail(GS_EINVAL, "field pointers must not be NULL");
    return GS_OK;
}

}  // namespace

extern "C" {

int gs_surr_param_count(size_t* count)
{
    if (!count) return fail(GS_EINVAL, "count is NULL");
    size_t n = 0;
    for (int l = 0; l < kSurrLayers; ++l) n += (size_t)27 * kChan[l] * kChan[l + 1] + kChan[l + 1];
    *count = n;
    return GS_OK;
}

int gs_surr_destroy(gs_surr* s)
{
    if (!s) return GS_OK;
    free_ws(s);
    guarded_free(s->params);
    guarded_free(s->grads);
    guarded_free(s->m);
    guarded_free(s->v);
    for (int l = 0; l < kSurrLayers; ++l) {
        guarded_free(s->wf[l]);
        guarded_free(s->wd[l]);
        guarded_free(s->wt[l]);
        guarded_free(s->wdt[l]);
    }
    guarded_free(s->wt0x);
    guarded_free(s->wdt5x);
    guarded_free(s->d_err);
    guarded_free(s->d_loss);
    guarded_free(s->d_max);
    guarded_free(s->d_ss);
    delete s;
    return GS_OK;
}

int gs_surr_create(gs_surr** out)
{
    if (!out) return fail(GS_EINVAL, "out is NULL");
    *out = nullptr;
    gs_surr* s = new (std::nothrow) gs_surr();
    if (!s) return fail(GS_ENOMEM, "host allocation failed");
    size_t off = 0;
    for (int l = 0; l < kSurrLayers; ++l) {
        s->woff[l] = off;
        off += (size_t)27 * kChan[l] * kChan[l + 1];
        s->boff[l] = off;
        off += kChan[l + 1];
    }
    s->np = off;
    cudaError_t e = cudaSuccess;
    if ((e = guarded_malloc((void**)&s->params, off * 4)) != cudaSuccess || (e = guarded_malloc((void**)&s->grads, off * 4)) != cudaSuccess ||
        (e = guarded_malloc((void**)&s->m, off * 4)) != cudaSuccess || (e = guarded_malloc((void**)&s->v, off * 4)) != cudaSuccess ||
        (e = guarded_malloc((void**)&s->d_loss, sizeof(double))) != cudaSuccess ||
        (e = guarded_malloc((void**)&s->d_max, sizeof(unsigned))) != cudaSuccess ||
        (e = guarded_malloc((void**)&s->d_ss, sizeof(double))) != cudaSuccess ||
        (e = guarded_malloc((void**)&s->d_err, sizeof(int))) != cudaSuccess || (e = cudaMemset(s->d_err, 0, sizeof(int))) != cudaSuccess) {
        int rc = cuda_fail(e, "surrogate allocation");
        gs_surr_destroy(s);
        return rc;
    }
    for (int l = 0; l < kSurrLayers && e == cudaSuccess; ++l) {
        e = guarded_malloc((void**)&s->wf[l], (size_t)27 * kCoutP[l] * kCinP[l] * sizeof(bf16));
        if (e == cudaSuccess)
            e = guarded_malloc((void**)&s->wt[l], (l == 5 ? (size_t)6 * 3 * 2 * 2 * 48 * 8 : (size_t)27 * kCinP[l] * 32) * sizeof(bf16));
        if (e == cudaSuccess && l >= 1) e = guarded_malloc((void**)&s->wd[l], (size_t)27 * 32 * (l == 5 ? 16 : 32) * sizeof(bf16));
        if (e == cudaSuccess && l >= 1) e = guarded_malloc((void**)&s->wdt[l], (size_t)27 * 32 * (l == 5 ? 16 : 32) * sizeof(bf16));
    }
    if (e == cudaSuccess) e = guarded_malloc((void**)&s->wt0x, (size_t)9 * kCinP[0] * 32 * sizeof(bf16));
    if (e == cudaSuccess) e = guarded_malloc((void**)&s->wdt5x, (size_t)9 * 16 * 32 * sizeof(bf16));
    if (e != cudaSuccess || (e = cudaMemset(s->params, 0, off * 4)) != cudaSuccess ||
        (e = cudaMemset(s->m, 0, off * 4)) != cudaSuccess || (e = cudaMemset(s->v, 0, off * 4)) != cudaSuccess) {
        int rc = cuda_fail(e, "surrogate allocation");
        gs_surr_destroy(s);
        return rc;
    }
    *out = s;
    return GS_OK;
}

int gs_surr_set_stream(gs_surr* s, void* stream)
{
    if (!s) return fail(GS_EINVAL, "surrogate is NULL");
    s->stream = (cudaStream_t)stream;
    return GS_OK;
}

int gs_surr_set_params(gs_surr* s, const float* host, size_t count)
{
    if (!s || !host) return fail(GS_EINVAL, "NULL argument");
    if (count != s->np) return fail(GS_EINVAL, "count=%zu, the network has %zu parameters", count, s->np);
    GS_CUDA_TRY(cudaMemcpyAsync(s->params, host, count * 4, cudaMemcpyHostToDevice, s->stream));
    GS_CUDA_TRY(cudaMemsetAsync(s->m, 0, count * 4, s->stream));
    GS_CUDA_TRY(cudaMemsetAsync(s->v, 0, count * 4, s->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->adam_t = 0;
    s->wdirty = 3;
    return GS_OK;
}

int gs_surr_get_params(gs_surr* s, float* host, size_t count)
{
    if (!s || !host) return fail(GS_EINVAL, "NULL argument");
    if (count != s->np) return fail(GS_EINVAL, "count=%zu, the network has %zu parameters", count, s->np);
    GS_CUDA_TRY(cudaMemcpyAsync(host, s->params, count * 4, cudaMemcpyDeviceToHost, s->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GS_OK;
}

int gs_surr_get_grads(gs_surr* s, float* host, size_t count)
{
    if (!s || !host) return fail(GS_EINVAL, "NULL argument");
    if (count != s->np) return fail(GS_EINVAL, "count=%zu, the network has %zu parameters", count, s->np);
    GS_CUDA_TRY(cudaMemcpyAsync(host, s->grads, count * 4, cudaMemcpyDeviceToHost, s->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GS_OK;
}

int gs_surr_forward(gs_surr* s, int N, int L, const float* u, const float* v, const double* F, const double* k,
                    float* u_out, float* v_out)
{
    if (!s || !F || !k || !u_out || !v_out) return fail(GS_EINVAL, "NULL argument");
    int rc = check_fields(N, L, u, v);
    if (rc) return rc;
    if ((rc = ensure_ws(s, N, L, false))) return rc;
    if ((rc = upload_fk(s, N, F, k))) return rc;
    return forward(s, N, L, u, v, u_out, v_out, false);
}

int gs_surr_grad(gs_surr* s, int N, int L, const float* u, const float* v, const double* F, const double* k,
                 const float* u_tgt, const float* v_tgt, double* loss)
{
    if (!s || !F || !k || !u_tgt || !v_tgt) return fail(GS_EINVAL, "NULL argument");
    int rc = check_fields(N, L, u, v);
    if (rc) return rc;
    if (s->trace_dh && s->trace_count != (size_t)5 * N * L * L * L * 32)
        return fail(GS_EINVAL, "gradient trace holds %zu floats, this call needs 5 x N x L^3 x 32", s->trace_count);
    if ((rc = ensure_ws(s, N, L, true))) return rc;
    if ((rc = upload_fk(s, N, F, k))) return rc;
    if ((rc = forward(s, N, L, u, v, s->ou, s->ov, true))) return rc;
    return backward(s, N, L, u_tgt, v_tgt, loss);
}

int gs_surr_save(gs_surr* s, const char* path)
{
    if (!s || !path) return fail(GS_EINVAL, "NULL argument");
    std::vector<float> h(s->np);
    int rc = gs_surr_get_params(s, h.data(), h.size());
    if (rc) return rc;
    FILE* f = fopen(path, "wb");
    if (!f) return fail(GS_EIO, "cannot create %s", path);
    const uint32_t n = (uint32_t)s->np;
    bool ok = fwrite(kSurrMagic, 1, 8, f) == 8 && fwrite(&n, sizeof(n), 1, f) == 1 &&
              fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? GS_OK : fail(GS_EIO, "writing %s failed", path);
}

int gs_surr_load(gs_surr* s, const char* path)
{
    if (!s || !path) return fail(GS_EINVAL, "NULL argument");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(GS_EIO, "cannot open %s", path);
    char magic[8] = {};
    uint32_t n = 0;
    std::vector<float> h(s->np);
    const bool head = fread(magic, 1, 8, f) == 8 && fread(&n, sizeof(n), 1, f) == 1;
    const bool body = head && memcmp(magic, kSurrMagic, 8) == 0 && n == (uint32_t)s->np &&
                      fread(h.data(), sizeof(float), h.size(), f) == h.size();
    char extra;
    const bool at_end = body && fread(&extra, 1, 1, f) == 0;
    fclose(f);
    if (!head) return fail(GS_EIO, "%s: truncated header", path);
    if (memcmp(magic, kSurrMagic, 8) != 0) return fail(GS_EINVAL, "%s is not a surrogate weights file", path);
    if (n != (uint32_t)s->np) return fail(GS_EINVAL, "%s holds %u parameters, the network has %zu", path, n, s->np);
    if (!body) return fail(GS_EIO, "%s: truncated parameters", path);
    if (!at_end) return fail(GS_EINVAL, "%s: trailing bytes after the parameters", path);
    return gs_surr_set_params(s, h.data(), h.size());
}

int gs_surr_trace_grads(gs_surr* s, float* dh, size_t count)
{
    if (!s) return fail(GS_EINVAL, "surrogate is NULL");
    if (dh && count == 0) return fail(GS_EINVAL, "count must be > 0 with a trace array");
    s->trace_dh = dh;
    s->trace_count = dh ? count : 0;
    return GS_OK;
}

int gs_surr_get_train_output(gs_surr* s, float* u_out, float* v_out, size_t cells)
{
    if (!s || !u_out || !v_out) return fail(GS_EINVAL, "NULL argument");
    if (!s->train_ws || !s->ou) return fail(GS_ESTATE, "no gradient computation has run yet");
    const size_t have = (size_t)s->N * s->L * s->L * s->L;
    if (cells != have) return fail(GS_EINVAL, "cells=%zu, the last gradient computation had %zu", cells, have);
    GS_CUDA_TRY(cudaMemcpyAsync(u_out, s->ou, cells * 4, cudaMemcpyDeviceToDevice, s->stream));
    GS_CUDA_TRY(cudaMemcpyAsync(v_out, s->ov, cells * 4, cudaMemcpyDeviceToDevice, s->stream));
    return gs_surr_sync(s);
}

int gs_surr_adam(gs_surr* s, double lr, double beta1, double beta2, double eps)
{
    if (!s) return fail(GS_EINVAL, "surrogate is NULL");
    if (!(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return fail(GS_EINVAL, "bad Adam hyper-parameters");
    s->adam_t += 1;
    const float c1 = (float)(1.0 - pow(beta1, (double)s->adam_t));
    const float c2 = (float)(1.0 - pow(beta2, (double)s->adam_t));
    gs_adam_kernel<<<grid1d((long long)s->np, 256), 256, 0, s->stream>>>(s->params, s->grads, s->m, s->v,
                                                                         (long long)s->np, (float)lr, (float)beta1,
                                                                         (float)beta2, (float)eps, c1, c2);
    GS_CUDA_TRY(cudaGetLastError());
    s->launches += 1;
    s->wdirty = 3;
    return GS_OK;
}

int gs_surr_train_step(gs_surr* s, int N, int L, const float* u, const float* v, const double* F, const double* k,
                       const float* u_tgt, const float* v_tgt, double lr, double* loss)
{
    int rc = gs_surr_grad(s, N, L, u, v, F, k, u_tgt, v_tgt, loss);
    if (rc) return rc;
    return gs_surr_adam(s, lr, 0.9, 0.999, 1e-8);
}

int gs_surr_diff(gs_surr* s, const float* a, const float* b, int64_t n, double* maxabs, double* rms)
{
    if (!s || !a || !b || n < 1) return fail(GS_EINVAL, "bad argument");
    return diff(s, a, b, n, maxabs, rms);
}

int gs_surr_run(gs_surr* s, gs_sim* sim, double F, double k, int64_t nsteps, int check_every, double tol,
                gs_surr_report* rep)
{
    if (!s || !sim) return fail(GS_EINVAL, "NULL argument");
    if (nsteps < 0 || check_every < 16 || check_every % 16) return fail(GS_EINVAL, "check_every must be a positive multiple of 16");
    if (!(tol > 0)) return fail(GS_EINVAL, "tol must be > 0");
    int kernel = 0;
    int rc = gs_get_plan(sim, &kernel, nullptr, nullptr, nullptr, nullptr);
    if (rc) return rc;
    int L = 0, dtype = 0;
    if ((rc = gs_sim_shape(sim, &L, &dtype))) return rc;
    if (dtype != GS_F32) return fail(GS_EINVAL, "the surrogate runs on FP32 simulations");
    if ((rc = surr_valid_L(L))) return rc;
    // run the network on the simulation's stream so both stay ordered
    void* sim_stream = nullptr;
    if ((rc = gs_get_stream(sim, &sim_stream))) return rc;
    cudaStream_t saved_stream = s->stream;
    s->stream = (cudaStream_t)sim_stream;
    if ((rc = ensure_ws(s, 1, L, false)) || (rc = upload_fk(s, 1, &F, &k))) {
        s->stream = saved_stream;
        return rc;
    }
    const size_t cells = (size_t)L * L * L;
    float* tu = nullptr;
    float* tv = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&tu, cells * 4)) != cudaSuccess || (e = cudaMalloc(&tv, cells * 4)) != cudaSuccess) {
        cudaFree(tu);
        s->stream = saved_stream;
        return cuda_fail(e, "surrogate run buffers");
    }
    gs_surr_report r{};
    bool fallback = false;
    int64_t done = 0;
    while (done < nsteps && !rc) {
        const int64_t seg = std::min<int64_t>(check_every, nsteps - done);
        if (fallback || seg < 16) {
            rc = gs_step(sim, seg);
            r.stencil_steps += seg;
            done += seg;
            fallback = false;  // try the surrogate again on the next segment
            continue;
        }
        // surrogate for all but the last 16 steps of the segment
        const int64_t napp = seg / 16 - 1;
        for (int64_t a = 0; a < napp && !rc; ++a) {
            void* cu;
            void* cv;
            gs_device_ptr(sim, GS_U, &cu);
            gs_device_ptr(sim, GS_V, &cv);
            rc = forward(s, 1, L, (const float*)cu, (const float*)cv, tu, tv, false);
            if (!rc) {
                cudaMemcpyAsync(cu, tu, cells * 4, cudaMemcpyDeviceToDevice, s->stream);
                cudaMemcpyAsync(cv, tv, cells * 4, cudaMemcpyDeviceToDevice, s->stream);
                int64_t t;
                gs_get_step(sim, &t);
                gs_set_step(sim, t + 16);
                r.surrogate_applications += 1;
                r.surrogate_steps += 16;
            }
        }
        if (rc) break;
        // check: one application against 16 stencil steps from the same state; keep the stencil's
        void* cu;
        void* cv;
        gs_device_ptr(sim, GS_U, &cu);
        gs_device_ptr(sim, GS_V, &cv);
        if ((rc = forward(s, 1, L, (const float*)cu, (const float*)cv, tu, tv, false))) break;
        if ((rc = gs_step(sim, 16))) break;
        r.stencil_steps += 16;
        gs_device_ptr(sim, GS_U, &cu);
        gs_device_ptr(sim, GS_V, &cv);
        double mu = 0, ru = 0, mv = 0, rv = 0;
        if ((rc = diff(s, tu, (const float*)cu, (long long)cells, &mu, &ru))) break;
        if ((rc = diff(s, tv, (const float*)cv, (long long)cells, &mv, &rv))) break;
        if ((rc = gs_surr_sync(s))) break;
        const double err = (std::isnan(mu) || std::isnan(mv)) ? INFINITY : std::max(mu, mv);
        r.checks += 1;
        r.max_check_error = std::max(r.max_check_error, err);
        r.last_check_error = err;
        if (err > tol) {
            r.fallbacks += 1;
            fallback = true;
        }
        done += seg;
    }
    cudaStreamSynchronize(s->stream);
    cudaFree(tu);
    cudaFree(tv);
    s->stream = saved_stream;
    if (rep) *rep = r;
    return rc;
}

int gs_surr_guard_check(gs_surr* s, int64_t* bad)
{
    if (!s || !bad) return fail(GS_EINVAL, "NULL argument");
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    std::vector<const void*> bufs = {s->params, s->grads, s->m, s->v, s->wt0x, s->wdt5x, s->d_err, s->d_loss, s->d_max, s->d_ss,
                                     s->x0, s->gh, s->gz[0], s->gz[1], s->gd, s->ou, s->ov, s->fk, s->wpart};
    for (int l = 0; l < kSurrLayers; ++l) {
        bufs.push_back(s->wf[l]);
        bufs.push_back(s->wd[l]);
        bufs.push_back(s->wt[l]);
        bufs.push_back(s->wdt[l]);
        bufs.push_back(s->h[l]);
        if (l < kSurrLayers - 1) bufs.push_back(s->zm[l]);
    }
    int64_t n = 0;
    for (const void* p : bufs) {
        if (!p) continue;
        const int64_t r = guarded_check(p);
        if (r < 0) return fail(GS_ECUDA, "reading a guard band failed");
        n += r;
    }
    *bad = n;
    return GS_OK;
}

int gs_surr_set_backend(gs_surr* s, int backend)
{
    if (!s) return fail(GS_EINVAL, "surrogate is NULL");
    if (backend < 0 || backend > 2) return fail(GS_EINVAL, "backend=%d must be 0, 1 or 2", backend);
    s->backend = backend;
    return GS_OK;
}

int gs_surr_sync(gs_surr* s)
{
    if (!s) return fail(GS_EINVAL, "surrogate is NULL");
    int err = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    GS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (err == GS_DERR_TIMEOUT) return fail(GS_ETIMEOUT, "a device-side wait timed out");
    if (err) return fail(GS_ECUDA, "device error code %d", err);
    return GS_OK;
}

int gs_surr_launch_count(gs_surr* s, int64_t* count)
{
    if (!s || !count) return fail(GS_EINVAL, "NULL argument");
    *count = s->launches;
    return GS_OK;
}

}  // extern "C"
