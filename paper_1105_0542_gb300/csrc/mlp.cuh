#pragma once
// The proposal network on the 5th-generation tensor cores (sm_103a):
// tcgen05.mma with bfloat16 operands in shared memory and float accumulators
// in tensor memory, 128 rows (paths) at a time.
//
// x = (a, b, T, n/s, q_L, q_R) -> Linear(6,128) -> GELU -> Linear(128,128)
// -> GELU -> Linear(128,128) -> GELU -> Linear(128,2) = (shift, log-scale),
// GELU(v) = v (1 + erf(v/sqrt 2))/2.  Host weights: one float vector
// (W1[128][6], b1, W2[128][128], b2, W3[128][128], b3, W4[2][128], b4),
// matrices stored [out][in].
//
// Operand layout (A = activations [128 rows][K], B = weights [N rows][K],
// both K-major): core matrices of 8 rows x 16 bytes (8 bf16), stored
// contiguously; K-adjacent core matrices 128 bytes apart (the descriptor's
// leading byte offset), 8-row groups K/8 * 128 bytes apart (stride byte
// offset); no swizzle.  A CTA copies the weight blob (this layout, plus the
// float biases) once and keeps it resident.
//
// One layer = K/16 MMAs of M = 128, N = 128 (N = 16 for the output layer,
// rows 2..15 of W4 zero) issued by one thread into tensor-memory columns
// [0, 128) (outputs: [128, 144)), a commit to an mbarrier, and an epilogue
// in which warp w reads tensor-memory lanes 32 (w % 4) .. +31 (its rows) and
// a quarter of the columns of its quadrant's rows (16 warps: 32 columns each),
// adds the bias, applies GELU (erf by a polynomial, two values per packed
// multiply-add) and writes the bfloat16 activations back into the A tile for
// the next layer.
#include <cuda_bf16.h>
#include <cstdint>

#include "erf_poly.h"

namespace su {
namespace mlp {

constexpr int kIn = 6, kHid = 128, kOut = 2;
constexpr int kParams = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kOut * kHid + kOut;   // 34178
constexpr int kK1 = 16;        // layer-1 K: the 6 features, zero-padded
constexpr int kNOut = 16;      // output-layer N: 2 outputs, zero-padded
constexpr int kRows = 128;     // rows per tile = the MMA's M
constexpr int kThreads = 512;  // 16 warps: four per tensor-memory lane quadrant
constexpr int kColsPerWarp = kHid * 4 / (kThreads / 32);   // epilogue columns of a warp
constexpr int kTmemCols = 256; // [0, 128) hidden accumulator, [128, 144) outputs

// byte offset of element (r, k) of an operand with K columns
__host__ __device__ constexpr int cm_off(int r, int k, int K) {
    return (r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// blob layout (the shared-memory image), byte offsets
constexpr int kOffW1 = 0;                                 // [128][16]
constexpr int kOffW2 = kOffW1 + kHid * kK1 * 2;           // [128][128]
constexpr int kOffW3 = kOffW2 + kHid * kHid * 2;          // [128][128]
constexpr int kOffW4 = kOffW3 + kHid * kHid * 2;          // [16][128]
constexpr int kOffB = kOffW4 + kNOut * kHid * 2;          // b1, b2, b3 [128], b4 [2] (+ pad), float
constexpr int kBlobBytes = kOffB + (3 * kHid + 8) * 4;    // 75296
static_assert(kBlobBytes % 16 == 0, "blob copies in 16-byte pieces");

// tile buffers (shared memory, byte sizes)
constexpr int kX0Bytes = kRows * kK1 * 2;
constexpr int kHBytes = kRows * kHid * 2;

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// erf(v/sqrt 2) from the polynomial of erf_poly.h (one value)
__device__ __forceinline__ float erf_sqrt2(float v) {
    const float x = fminf(fmaxf(v, -kErfClamp), kErfClamp);
    const float z = x * x;
    float p = erf_poly(kErfTerms - 1);
#pragma unroll
    for (int k = kErfTerms - 2; k >= 0; --k) p = fmaf(p, z, erf_poly(k));
    return x * p;
}

// GELU of two values, v (1 + erf(v/sqrt 2))/2, with erf(v/sqrt 2) from the
// odd polynomial v Q(v^2) of erf_poly.h (v clamped to [-3 sqrt 2, 3 sqrt 2],
// error <= 1e-4, below the bfloat16 rounding the epilogue applies) evaluated
// on the pair by packed multiply-adds (fma.rn.f32x2): one instruction for
// both values.
__device__ __forceinline__ float2 gelu2(float2 v) {
    const float2 x = make_float2(fminf(fmaxf(v.x, -kErfClamp), kErfClamp), fminf(fmaxf(v.y, -kErfClamp), kErfClamp));
    const float2 z = __fmul2_rn(x, x);
    float2 p = make_float2(erf_poly(kErfTerms - 1), erf_poly(kErfTerms - 1));
#pragma unroll
    for (int k = kErfTerms - 2; k >= 0; --k) p = __ffma2_rn(p, z, make_float2(erf_poly(k), erf_poly(k)));
    const float2 e = __fmul2_rn(x, p);                                   // erf(v/sqrt 2)
    const float2 h = __fmul2_rn(v, make_float2(0.5f, 0.5f));
    return __ffma2_rn(h, e, h);                                           // v/2 + v/2 erf
}

// ---- tcgen05 plumbing
// shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: float accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

constexpr unsigned long long kWaitNs = 1000000000ull;   // a wait gives up after one second
constexpr int kWaitPolls = 1 << 28;                      // and after this many polls in any case

struct Tc {
    uint32_t tmem;     // tensor-memory base address (lane 0, first column)
    uint32_t mbar;     // shared address of the MMA-completion mbarrier
    uint32_t phase;    // parity of the next completion to wait for
    uint32_t ncols;    // allocated columns
};

// All threads: mbarrier init (thread 0), allocation of ncols tensor-memory
// columns (warp 0; a power of two >= 32).  slot and bar are shared-memory
// words of the CTA.
__device__ __forceinline__ Tc tc_begin(uint32_t *slot, uint64_t *bar, uint32_t ncols = kTmemCols) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    Tc t;
    t.tmem = *slot;
    t.mbar = smem_u32(bar);
    t.phase = 0;
    t.ncols = ncols;
    return t;
}

// All threads, after the last use: warp 0 frees the tensor memory.
__device__ __forceinline__ void tc_end(const Tc &t) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem), "r"(t.ncols));
}

// One layer's MMAs, D[:, col..col+N) = A[128][K] B[N][K]^T, issued by thread
// 0 after the other threads' shared-memory writes (fenced for the async
// proxy and synchronised by the caller), then committed to the mbarrier.
// withhold (fault injection): issue nothing, so the wait runs out.
__device__ __forceinline__ void tc_layer(const Tc &t, uint32_t a, uint32_t b, int K, int N, uint32_t col,
                                         bool withhold = false) {
    if (threadIdx.x == 0 && !withhold) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sbo = (uint32_t)(K / 8) * 128;
        const uint32_t id = instr_desc(kRows, N);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = smem_desc(a + ks * 256, 128, sbo);
            const uint64_t bd = smem_desc(b + ks * 256, 128, sbo);
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(t.tmem + col),
                "l"(ad), "l"(bd), "r"(id), "r"((uint32_t)(ks > 0)));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(t.mbar));
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    return v;
}

// All threads: wait (bounded: one second of the global timer) for the last
// commit; false if it never came.
__device__ __forceinline__ bool tc_wait(Tc &t) {
    uint32_t done = 0;
    const unsigned long long t0 = global_ns();
    for (int it = 0; it < kWaitPolls && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(t.mbar), "r"(t.phase));
        if (!done && (it & 255) == 255 && global_ns() - t0 > kWaitNs) break;
    }
    t.phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Epilogue of a hidden layer: bias + GELU of the accumulator, bfloat16, into
// the A tile H ([128][128], operand layout); then fenced for the next MMA.
__device__ __forceinline__ void tc_store_gelu(const Tc &t, const float *bias, unsigned char *H) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = 32 * (warp & 3) + lane;
    const int c0 = kColsPerWarp * (warp >> 2);
    const uint32_t base = t.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
#pragma unroll
    for (int cc = 0; cc < kColsPerWarp; cc += 16) {
        float v[16];
        tmem_ld16(base + (uint32_t)cc, v);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int c = c0 + cc + 8 * half;
            // the eight columns' biases (16-byte aligned: the blob's bias block is)
            const float4 b0 = *reinterpret_cast<const float4 *>(bias + c);
            const float4 b1 = *reinterpret_cast<const float4 *>(bias + c + 4);
            const float *u = v + 8 * half;
            const float2 g0 = gelu2(__fadd2_rn(make_float2(u[0], u[1]), make_float2(b0.x, b0.y)));
            const float2 g1 = gelu2(__fadd2_rn(make_float2(u[2], u[3]), make_float2(b0.z, b0.w)));
            const float2 g2 = gelu2(__fadd2_rn(make_float2(u[4], u[5]), make_float2(b1.x, b1.y)));
            const float2 g3 = gelu2(__fadd2_rn(make_float2(u[6], u[7]), make_float2(b1.z, b1.w)));
            uint4 w;
            w.x = pack_bf16(g0.x, g0.y);
            w.y = pack_bf16(g1.x, g1.y);
            w.z = pack_bf16(g2.x, g2.y);
            w.w = pack_bf16(g3.x, g3.y);
            *reinterpret_cast<uint4 *>(H + cm_off(row, c, kHid)) = w;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
}

// The whole network on one 128-row tile.  X0: the features in operand layout
// ([128][16], columns 6..15 zero), written and synchronised by the caller
// (fence.proxy.async by the writers, then __syncthreads); H: the hidden tile;
// out[row * 2 + {0, 1}] = (shift, ls).  All kThreads threads; returns false on
// all threads if an MMA never completed (the tile's outputs are then invalid
// and the caller must stop).  withhold: fault injection (see tc_layer).
__device__ __forceinline__ bool tile_forward(Tc &t, const unsigned char *blob, const unsigned char *X0,
                                             unsigned char *H, float *out, bool withhold = false) {
    const float *B = reinterpret_cast<const float *>(blob + kOffB);
    const uint32_t sb = smem_u32(blob), sx = smem_u32(X0), sh = smem_u32(H);
    // each wait's outcome agreed by the whole CTA before the epilogue reads
    tc_layer(t, sx, sb + kOffW1, kK1, kHid, 0, withhold);
    if (!__syncthreads_and(tc_wait(t) ? 1 : 0)) return false;
    tc_store_gelu(t, B, H);
    tc_layer(t, sh, sb + kOffW2, kHid, kHid, 0);
    if (!__syncthreads_and(tc_wait(t) ? 1 : 0)) return false;
    tc_store_gelu(t, B + kHid, H);
    tc_layer(t, sh, sb + kOffW3, kHid, kHid, 0);
    if (!__syncthreads_and(tc_wait(t) ? 1 : 0)) return false;
    tc_store_gelu(t, B + 2 * kHid, H);
    tc_layer(t, sh, sb + kOffW4, kHid, kNOut, kHid);
    if (!__syncthreads_and(tc_wait(t) ? 1 : 0)) return false;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {   // the output columns of the warp's 32 rows
        uint32_t r0, r1;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                     : "=r"(r0), "=r"(r1)
                     : "r"(t.tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)kHid));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const int row = 32 * warp + lane;
        out[2 * row] = __uint_as_float(r0) + B[3 * kHid];
        out[2 * row + 1] = __uint_as_float(r1) + B[3 * kHid + 1];
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    return true;
}

// features of one row into the X0 tile (operand layout): columns 0..5, the
// zero padding of columns 6..7 in the same 16-byte chunk
__device__ __forceinline__ void store_features(unsigned char *X0, int row, __nv_bfloat16 f0, __nv_bfloat16 f1,
                                               __nv_bfloat16 f2, __nv_bfloat16 f3, __nv_bfloat16 f4,
                                               __nv_bfloat16 f5) {
    __nv_bfloat162 p0 = __halves2bfloat162(f0, f1), p1 = __halves2bfloat162(f2, f3), p2 = __halves2bfloat162(f4, f5);
    uint4 w;
    w.x = *reinterpret_cast<uint32_t *>(&p0);
    w.y = *reinterpret_cast<uint32_t *>(&p1);
    w.z = *reinterpret_cast<uint32_t *>(&p2);
    w.w = 0u;
    *reinterpret_cast<uint4 *>(X0 + cm_off(row, 0, kK1)) = w;
}
#endif

// host: float parameter vector -> device blob image (kBlobBytes)
void pack_blob(const float *theta, unsigned char *blob);

}  // namespace mlp
}  // namespace su
