#pragma once
// The proposal network on the tensor cores (sm_103a): bfloat16 operands,
// float accumulation, 128 rows at a time.
//
// x = (a, b, T, n/s, q_L, q_R) -> Linear(6,128) -> GELU -> Linear(128,128)
// -> GELU -> Linear(128,128) -> GELU -> Linear(128,2) = (shift, log-scale),
// GELU(v) = v (1 + erf(v/sqrt 2))/2.  Host weights: one float vector
// (W1[128][6], b1, W2[128][128], b2, W3[128][128], b3, W4[2][128], b4),
// matrices stored [out][in].
//
// On the device the weights form one blob whose layout is the shared-memory
// layout: bfloat16 matrices [out][in] with rows padded to 24 or 136 elements
// (48 / 272 bytes, so the eight rows an ldmatrix reads fall into distinct
// 16-byte bank groups), the 2-row output matrix padded to 8 zero rows, then
// the float biases.  A CTA copies the blob once and keeps it resident.
//
// Layer GEMMs use mma.sync m16n8k16 (bf16 x bf16 -> f32): warp w of 8 owns
// rows 16w..16w+15 of the 128-row tile and all output columns.
#include <cuda_bf16.h>
#include <cstdint>

namespace su {
namespace mlp {

constexpr int kIn = 6, kHid = 128, kOut = 2;
constexpr int kParams = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kOut * kHid + kOut;   // 34178
constexpr int kS1 = 24;    // row stride (elements) of W1 and of the input tile
constexpr int kSH = 136;   // row stride of W2, W3, W4 and of the hidden tile
constexpr int kRows = 128; // rows per tile
constexpr int kThreads = 256;

// blob layout, byte offsets
constexpr int kOffW1 = 0;
constexpr int kOffW2 = kOffW1 + kHid * kS1 * 2;
constexpr int kOffW3 = kOffW2 + kHid * kSH * 2;
constexpr int kOffW4 = kOffW3 + kHid * kSH * 2;
constexpr int kOffB = kOffW4 + 8 * kSH * 2;
constexpr int kBlobBytes = kOffB + (3 * kHid + 8) * 4;   // 79520
static_assert(kBlobBytes % 16 == 0, "blob copies in 16-byte pieces");

// tile buffers (shared memory, byte sizes)
constexpr int kX0Bytes = kRows * kS1 * 2;
constexpr int kHBytes = kRows * kSH * 2;

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t &r0, uint32_t &r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float v) { return 0.5f * v * (1.0f + erff(v * 0.70710678118654752f)); }

// acc[16 n-tiles][4] of warp w (rows 16w..16w+15, columns 0..127) from the
// input tile A (row stride sa elements, K = 16 * ksteps) and the matrix W
// ([128][sw]), both in shared memory
__device__ __forceinline__ void tile_gemm_128(float (&acc)[16][4], const __nv_bfloat16 *A, int sa,
                                              const __nv_bfloat16 *W, int sw, int ksteps) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 16; ++t)
        acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    const int arow = 16 * warp + (lane & 15);
    const int acol = (lane >> 4) * 8;
    const int brow = (lane & 7) + ((lane >> 4) << 3);
    const int bcol = ((lane >> 3) & 1) * 8;
    for (int ks = 0; ks < ksteps; ++ks) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(smem_u32(A + arow * sa + ks * 16 + acol), a0, a1, a2, a3);
#pragma unroll
        for (int np = 0; np < 8; ++np) {   // two n8 tiles per ldmatrix.x4
            uint32_t b0, b1, b2, b3;
            ldsm_x4(smem_u32(W + (np * 16 + brow) * sw + ks * 16 + bcol), b0, b1, b2, b3);
            mma_bf16(acc[2 * np], a0, a1, a2, a3, b0, b1);
            mma_bf16(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
        }
    }
}

// bias + GELU, bfloat16, into the hidden tile H (row stride kSH)
__device__ __forceinline__ void tile_store_gelu(const float (&acc)[16][4], const float *bias, __nv_bfloat16 *H) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = 16 * warp + (lane >> 2);
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const int c = 8 * t + (lane & 3) * 2;
        const float b0 = bias[c], b1 = bias[c + 1];
        __nv_bfloat162 lo = __floats2bfloat162_rn(gelu(acc[t][0] + b0), gelu(acc[t][1] + b1));
        __nv_bfloat162 hi = __floats2bfloat162_rn(gelu(acc[t][2] + b0), gelu(acc[t][3] + b1));
        *reinterpret_cast<__nv_bfloat162 *>(H + r0 * kSH + c) = lo;
        *reinterpret_cast<__nv_bfloat162 *>(H + (r0 + 8) * kSH + c) = hi;
    }
}

// The whole network on one 128-row tile: inputs in X0 (bf16, [128][kS1],
// columns 6..15 zero), hidden tile H ([128][kSH]), outputs (shift, ls) into
// out[row * 2 + {0,1}].  All 256 threads of the CTA take part; contains
// __syncthreads.
__device__ __forceinline__ void tile_forward(const unsigned char *blob, const __nv_bfloat16 *X0,
                                             __nv_bfloat16 *H, float *out) {
    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(blob + kOffW1);
    const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(blob + kOffW2);
    const __nv_bfloat16 *W3 = reinterpret_cast<const __nv_bfloat16 *>(blob + kOffW3);
    const __nv_bfloat16 *W4 = reinterpret_cast<const __nv_bfloat16 *>(blob + kOffW4);
    const float *B = reinterpret_cast<const float *>(blob + kOffB);
    float acc[16][4];
    tile_gemm_128(acc, X0, kS1, W1, kS1, 1);
    tile_store_gelu(acc, B, H);
    __syncthreads();
    tile_gemm_128(acc, H, kSH, W2, kSH, 8);
    __syncthreads();                    // every warp has read H
    tile_store_gelu(acc, B + kHid, H);
    __syncthreads();
    tile_gemm_128(acc, H, kSH, W3, kSH, 8);
    __syncthreads();
    tile_store_gelu(acc, B + 2 * kHid, H);
    __syncthreads();
    // output layer: one n8 tile (rows 0, 1 of W4 are the network's, 2..7 zero)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const int arow = 16 * warp + (lane & 15);
    const int acol = (lane >> 4) * 8;
    const int brow = lane & 7;
    const int bcol = ((lane >> 3) & 1) * 8;
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {
        uint32_t a0, a1, a2, a3, b0, b1;
        ldsm_x4(smem_u32(H + arow * kSH + ks * 16 + acol), a0, a1, a2, a3);
        ldsm_x2(smem_u32(W4 + brow * kSH + ks * 16 + bcol), b0, b1);
        mma_bf16(d, a0, a1, a2, a3, b0, b1);
    }
    if ((lane & 3) == 0) {              // columns 0 and 1 live in lanes 0, 4, ..., 28
        const int r0 = 16 * warp + (lane >> 2);
        out[2 * r0] = d[0] + B[3 * kHid];
        out[2 * r0 + 1] = d[1] + B[3 * kHid + 1];
        out[2 * (r0 + 8)] = d[2] + B[3 * kHid];
        out[2 * (r0 + 8) + 1] = d[3] + B[3 * kHid + 1];
    }
    __syncthreads();
}
#endif

// host: float parameter vector -> device blob image (kBlobBytes)
void pack_blob(const float *theta, unsigned char *blob);

}  // namespace mlp
}  // namespace su
