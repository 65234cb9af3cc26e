// Training of the proposal network on the tensor cores (sm_103a).
//
// The objective (weighted maximum likelihood of midpoints of plain-sampler
// paths): L = sum_r rw_r [ls_r + (u_r - shift_r)^2 e^{-2 ls_r} / 2] / sum_r rw_r,
// u_r = the midpoint's standardized offset (q - mu)/sigma_n.  One step on R
// rows (rows = the N-1 midpoints of each path of a minibatch):
//
//   forward   pre_l = H_{l-1} W_l^T + b_l, H_l = GELU(pre_l), Y = H_3 W_4^T + b_4
//   backward  dY = dL/dY; dH_3 = dY W_4; dPre_l = dH_l * GELU'(pre_l);
//             dW_l = dPre_l^T H_{l-1}; db_l = column sums of dPre_l;
//             dH_{l-1} = dPre_l W_l
//   update    Adam on the float master weights.
//
// Every product is one "NT" GEMM, C[M][N] = sum_k A[m][k] B[n][k], bf16
// operands with K contiguous, float accumulation on the 5th-generation tensor
// cores (tcgen05.mma, accumulator in tensor memory), so the activations and
// gradients are kept both row-major and transposed (bf16).  Products with
// K = R (the weight gradients) are split over K and summed with atomic adds.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mlp.cuh"
#include "philox.cuh"
#include "train.h"

namespace su {
namespace train {
namespace {

using mlp::kHid;
using mlp::kIn;
using mlp::kOut;
constexpr int kK1 = 32;        // padded input width (K of the first layer)
constexpr int kBM = 128, kBN = 128, kBK = 32;   // output tile; K granularity
constexpr int kTK = 128;                         // K staged per MMA round
// A and B stages (64 KB), reused for the 128 x (128 + 4) float output tile:
// 66 KB; 2 CTAs of 256 threads per SM (registers), 256 tensor-memory columns
constexpr int kGemmSmem = 128 * (kBN + 4) * 4 > 2 * 128 * kTK * 2 ? 128 * (kBN + 4) * 4 : 2 * 128 * kTK * 2;

// GELU and its derivative with erf(v/sqrt 2) from the polynomial the
// inference epilogue uses (mlp::erf_sqrt2): the same activations in training
// and in the proposal kernel
__device__ __forceinline__ float gelu(float v) { return 0.5f * v * (1.0f + mlp::erf_sqrt2(v)); }
__device__ __forceinline__ float gelu_grad(float v) {
    return 0.5f * (1.0f + mlp::erf_sqrt2(v)) + v * 0.39894228040143268f * __expf(-0.5f * v * v);
}

// What the GEMM's epilogue does with the accumulator tile acc[row][col]:
//   EP_STORE  C = acc (float)             EP_ADD  C += acc (atomic; split K)
//   EP_GELU   pre = acc + bias[col] (float), H = bf16(GELU(pre)) [M][N] and
//             HT = its transpose [N][M] (the forward layers)
//   EP_DGELU  P = bf16(acc * GELU'(pre)) [M][N] and PT = its transpose
//             (the backward layers: acc = dL/dH, P = dL/dpre)
enum Epilogue { EP_STORE = 0, EP_ADD = 1, EP_GELU = 2, EP_DGELU = 3 };
struct EpArgs {
    const float *bias;        // EP_GELU
    float *pre;               // EP_GELU: written; EP_DGELU: read ([M][ldc])
    __nv_bfloat16 *H, *HT;    // EP_GELU: H, HT; EP_DGELU: P, PT ([M][ldc], [N][M])
};

// C[M][N] (+)= sum_k A[m][k] B[n][k] over the K-range of blockIdx.z.
// A: [M][lda], B: [N][ldb] bf16 (lda, ldb multiples of 8); K and the K-range
// multiples of 32.  kGemmThreads = 256 threads: warp w reads tensor-memory lane
// quadrant w % 4, columns [64 (w / 4), 64 (w / 4) + 64) of the tile.
// Per K-step, 128 x 128 of A and min(N - n0, 128) x 128 of B are staged in the
// operand layout of mlp.cuh (zeros outside M, N and the K-range), thread 0
// issues K/16 MMAs (M = 128, N = the tile's width rounded up to 16) and
// commits them; all threads wait (bounded) before the next K-step overwrites
// the stage.  Epilogue: tcgen05.ld of each thread's row, stored or added.
// A wait that gives up sets *status.
constexpr int kGemmThreads = 256;
__global__ void __launch_bounds__(kGemmThreads, 2) gemm_nt(const __nv_bfloat16 *__restrict__ A, int lda,
                                                  const __nv_bfloat16 *__restrict__ B, int ldb,
                                                  float *__restrict__ C, int ldc, int M, int N, int K,
                                                  int kchunk, int mode, EpArgs ep, int *status) {
    extern __shared__ __align__(16) unsigned char gsm[];
    unsigned char *sA = gsm, *sB = gsm + 128 * kTK * 2;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mma_bar;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);
    const int nn = min(kBN, N - n0);
    const int NT = (nn + 15) & ~15;
    mlp::Tc tc = mlp::tc_begin(&tmem_slot, &mma_bar, 128);
    bool ok = true;
    for (int k0 = kb; k0 < ke; k0 += kTK) {
        const int kn = min(kTK, ke - k0);
        // 16-byte asynchronous copies, all in flight at once; a source size of
        // 0 fills the destination with zeros (rows past M or N, K past the range)
        for (int idx = tid; idx < 128 * (kTK / 8); idx += kGemmThreads) {
            const int r = idx / (kTK / 8), q = idx % (kTK / 8);
            const bool kin = 8 * q < kn;
            const bool ain = kin && m0 + r < M, bin = kin && r < nn;
            const __nv_bfloat16 *ga = ain ? A + (size_t)(m0 + r) * lda + k0 + 8 * q : A;
            const __nv_bfloat16 *gb = bin ? B + (size_t)(n0 + r) * ldb + k0 + 8 * q : B;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             mlp::smem_u32(sA + mlp::cm_off(r, 8 * q, kTK))),
                         "l"(ga), "r"(ain ? 16 : 0));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                             mlp::smem_u32(sB + mlp::cm_off(r, 8 * q, kTK))),
                         "l"(gb), "r"(bin ? 16 : 0));
        }
        asm volatile("cp.async.commit_group;");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = mlp::smem_u32(sA), b0 = mlp::smem_u32(sB);
            const uint32_t id = mlp::instr_desc(kBM, NT);
            for (int ks = 0; ks < kn / 16; ++ks) {
                const uint64_t ad = mlp::smem_desc(a0 + ks * 256, 128, (kTK / 8) * 128);
                const uint64_t bd = mlp::smem_desc(b0 + ks * 256, 128, (kTK / 8) * 128);
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tc.tmem),
                    "l"(ad), "l"(bd), "r"(id), "r"((uint32_t)(k0 > kb || ks > 0)));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tc.mbar));
        }
        ok &= mlp::tc_wait(tc);
        __syncthreads();
    }
    if (ke > kb) {
        // the accumulator tile through shared memory (the idle stage buffers,
        // rows of NT + 4 floats), then row-contiguous stores or adds to C
        float *Ts = reinterpret_cast<float *>(gsm);
        const int ts = NT + 4;
        const int quad = warp & 3, trow = 32 * quad + lane, c_lo = 64 * (warp >> 2);
        for (int c = c_lo; c < min(NT, c_lo + 64); c += 16) {
            float v[16];
            mlp::tmem_ld16(tc.tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4 *>(Ts + trow * ts + c + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        ok = __syncthreads_and(ok);   // one outcome for the whole CTA (the epilogue has a barrier)
        if (ok) {
            const int nq = NT / 4;
            for (int i = tid; i < 128 * nq; i += kGemmThreads) {
                const int r = i / nq, c = 4 * (i - r * nq);
                const int row = m0 + r, col = n0 + c;
                if (row >= M || col >= N) continue;
                float4 v = *reinterpret_cast<const float4 *>(Ts + r * ts + c);
                const int cnt = min(4, N - col);
                const size_t at = (size_t)row * ldc + col;
                if (mode == EP_GELU || mode == EP_DGELU) {   // N = ldc = 128: whole float4 groups
                    float e[4] = {v.x, v.y, v.z, v.w};
                    if (mode == EP_GELU) {
                        const float4 bb = *reinterpret_cast<const float4 *>(ep.bias + col);
                        const float b4[4] = {bb.x, bb.y, bb.z, bb.w};
                        float pr[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            pr[j] = e[j] + b4[j];
                            e[j] = gelu(pr[j]);
                        }
                        *reinterpret_cast<float4 *>(ep.pre + at) = make_float4(pr[0], pr[1], pr[2], pr[3]);
                    } else {
                        const float4 pv = *reinterpret_cast<const float4 *>(ep.pre + at);
                        const float p4[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) e[j] *= gelu_grad(p4[j]);
                    }
                    __nv_bfloat162 h2[2] = {__floats2bfloat162_rn(e[0], e[1]), __floats2bfloat162_rn(e[2], e[3])};
                    *reinterpret_cast<uint2 *>(ep.H + at) = *reinterpret_cast<const uint2 *>(h2);
                    *reinterpret_cast<float4 *>(Ts + r * ts + c) = make_float4(e[0], e[1], e[2], e[3]);
                    continue;
                }
                float *dst = C + at;
                const float e[4] = {v.x, v.y, v.z, v.w};
                if (mode == EP_ADD) {
                    for (int j = 0; j < cnt; ++j) atomicAdd(dst + j, e[j]);
                } else if (cnt == 4 && ((ldc | col) & 3) == 0) {
                    *reinterpret_cast<float4 *>(dst) = v;
                } else {
                    for (int j = 0; j < cnt; ++j) dst[j] = e[j];
                }
            }
            if (mode == EP_GELU || mode == EP_DGELU) {
                // the transpose: thread t takes column t % 128 of the tile's rows
                // 64 (t / 128) .. + 63, eight consecutive rows per 16-byte store
                // (M is a multiple of 32, so a group of eight rows is wholly
                // inside or outside; conflict-free reads of Ts)
                __syncthreads();
                const int c = tid & 127, rh = 64 * (tid >> 7);
                if (c < nn)
                    for (int r8 = rh; r8 < rh + 64 && m0 + r8 < M; r8 += 8) {
                        __nv_bfloat162 h[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            h[q] = __floats2bfloat162_rn(Ts[(r8 + 2 * q) * ts + c], Ts[(r8 + 2 * q + 1) * ts + c]);
                        *reinterpret_cast<uint4 *>(ep.HT + (size_t)(n0 + c) * M + m0 + r8) =
                            *reinterpret_cast<const uint4 *>(h);
                    }
            }
        }
    }
    if (!ok && tid == 0) atomicOr(status, 1);
    mlp::tc_end(tc);
}


// rows of a minibatch from stored paths: row r = path pb, heap index j
__global__ void rows_kernel(const float *__restrict__ paths, int np1, const int *__restrict__ ids, int nb,
                            float a, float b, float T, int S, const float *__restrict__ sig,
                            __nv_bfloat16 *X, __nv_bfloat16 *XT, int R, float *u) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int N = np1 - 1;
    const int pb = r / (N - 1), j = r - pb * (N - 1);
    const int n = 32 - __clz(j + 1);        // level: 2^(n-1) <= j + 1 < 2^n
    const int i = j - ((1 << (n - 1)) - 1);
    const int h = N >> n, k = (2 * i + 1) * h;
    const float *q = paths + (size_t)ids[pb] * np1;
    const float qL = q[k - h], qR = q[k + h];
    const float f[kIn] = {a, b, T, (float)n / (float)S, qL, qR};
    for (int c = 0; c < kK1; ++c) {
        const __nv_bfloat16 v = __float2bfloat16_rn(c < kIn ? f[c] : 0.f);
        X[(size_t)r * kK1 + c] = v;
        XT[(size_t)c * R + r] = v;
    }
    u[r] = (q[k] - 0.5f * (qL + qR)) / sig[n];
}

// loss and dL/dY per row; dY row-major padded to 32 columns and transposed [2][R]
__global__ void out_loss_kernel(const float *__restrict__ Y, const float *__restrict__ b4,
                                const float *__restrict__ u, const float *__restrict__ rw, double inv_norm,
                                __nv_bfloat16 *dYp, __nv_bfloat16 *dYT, int R, double *loss) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0;
    if (r < R) {
        const float sh = Y[2 * r] + b4[0], ls = Y[2 * r + 1] + b4[1];
        const float w = rw ? rw[r] : 1.f;
        const float d = u[r] - sh;
        const float e2 = __expf(-2.f * ls);
        l = (double)w * ((double)ls + 0.5 * (double)d * d * e2) * inv_norm;
        const float g0 = (float)(-(double)d * e2 * w * inv_norm);
        const float g1 = (float)((1.0 - (double)d * d * e2) * w * inv_norm);
        const __nv_bfloat16 h0 = __float2bfloat16_rn(g0), h1 = __float2bfloat16_rn(g1);
        dYp[(size_t)r * kK1] = h0;
        dYp[(size_t)r * kK1 + 1] = h1;
        dYT[r] = h0;
        dYT[R + r] = h1;
    }
    // block sum, one atomic per block
    __shared__ double sb[256];
    sb[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) sb[threadIdx.x] += sb[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sb[0]);
}

// out[row] = sum_r XT[row][r] (bias gradients from transposed gradients):
// one CTA of kRowsumThreads per row, 16-byte loads of eight bf16 (R is a
// multiple of 32, so every row starts 16-byte aligned), warp shuffles, then
// the warps in order: a fixed summation order.
constexpr int kRowsumThreads = 512;
__global__ void __launch_bounds__(kRowsumThreads) rowsum_kernel(const __nv_bfloat16 *__restrict__ XT, int R,
                                                                float *out) {
    const uint4 *row = reinterpret_cast<const uint4 *>(XT + (size_t)blockIdx.x * R);
    float s = 0.f;
    for (int i = threadIdx.x; i < R / 8; i += kRowsumThreads) {
        const uint4 v = row[i];
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(h[q]);
            s += f.x + f.y;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float sw[kRowsumThreads / 32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kRowsumThreads / 32; ++w) t += sw[w];
        out[blockIdx.x] = t;
    }
}

// float master weights -> the bf16 operands of one step
__global__ void prep_weights_kernel(const float *__restrict__ th, __nv_bfloat16 *W1p, __nv_bfloat16 *W2,
                                    __nv_bfloat16 *W3, __nv_bfloat16 *W4, __nv_bfloat16 *W2T,
                                    __nv_bfloat16 *W3T, __nv_bfloat16 *W4T) {
    const int o = blockIdx.x, i = threadIdx.x;   // 128 x 128
    const float *pW1 = th, *pW2 = pW1 + kHid * kIn + kHid, *pW3 = pW2 + kHid * kHid + kHid,
                *pW4 = pW3 + kHid * kHid + kHid;
    if (i < kK1) W1p[o * kK1 + i] = __float2bfloat16_rn(i < kIn ? pW1[o * kIn + i] : 0.f);
    W2[o * kHid + i] = __float2bfloat16_rn(pW2[o * kHid + i]);
    W3[o * kHid + i] = __float2bfloat16_rn(pW3[o * kHid + i]);
    W2T[i * kHid + o] = W2[o * kHid + i];
    W3T[i * kHid + o] = W3[o * kHid + i];
    if (o < kOut) W4[o * kHid + i] = __float2bfloat16_rn(pW4[o * kHid + i]);
    // W4T [in][32]: column o < 2 holds W4[o][in]
    if (i < kK1) W4T[o * kK1 + i] = __float2bfloat16_rn(i < kOut ? pW4[i * kHid + o] : 0.f);
}

// flat gradient (parameter order) from the GEMM outputs and the bias sums
__global__ void gather_grad_kernel(const float *dW1, const float *db1, const float *dW2, const float *db2,
                                   const float *dW3, const float *db3, const float *dW4, const float *db4,
                                   float *g) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int o = k;
    if (o < kHid * kIn) { g[k] = dW1[(o / kIn) * kK1 + o % kIn]; return; }
    o -= kHid * kIn;
    if (o < kHid) { g[k] = db1[o]; return; }
    o -= kHid;
    if (o < kHid * kHid) { g[k] = dW2[o]; return; }
    o -= kHid * kHid;
    if (o < kHid) { g[k] = db2[o]; return; }
    o -= kHid;
    if (o < kHid * kHid) { g[k] = dW3[o]; return; }
    o -= kHid * kHid;
    if (o < kHid) { g[k] = db3[o]; return; }
    o -= kHid;
    if (o < kOut * kHid) { g[k] = dW4[o]; return; }
    o -= kOut * kHid;
    if (o < kOut) g[k] = db4[o];
}

__global__ void adam_kernel(float *th, const float *__restrict__ g, float *m, float *v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    th[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

__global__ void features_kernel(const float *__restrict__ F, const float *__restrict__ uin,
                                const float *__restrict__ rwin, int n, int R, __nv_bfloat16 *X,
                                __nv_bfloat16 *XT, float *u, float *rw) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    for (int c = 0; c < kK1; ++c) {
        const __nv_bfloat16 v = __float2bfloat16_rn(r < n && c < kIn ? F[(size_t)r * kIn + c] : 0.f);
        X[(size_t)r * kK1 + c] = v;
        XT[(size_t)c * R + r] = v;
    }
    u[r] = r < n ? uin[r] : 0.f;
    rw[r] = r < n ? rwin[r] : 0.f;
}

__global__ void fill_kernel(float *p, float v, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = v;
}

// Minibatch path ids of step *step: draw k is the 53-bit uniform u of Philox
// call (*step, k, 0x7261696E, 0) under the key (seed lo, seed hi), and the id
// is the first index whose cumulative weight exceeds u * total (a draw in
// proportion to the weights).
__global__ void sample_ids_kernel(const double *__restrict__ cdf, int64_t n, double total, uint2 key,
                                  const int *__restrict__ step, int nb, int *ids) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)*step, (uint32_t)k, 0x7261696Eu, 0u), key);
    const double u = ((double)(((uint64_t)w.x << 21) | (w.y >> 11)) + 0.5) * 0x1p-53;
    const double x = u * total;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > x)
            hi = mid;
        else
            lo = mid + 1;
    }
    ids[k] = (int)(lo < n ? lo : n - 1);
}

// Adam with the step number t = *step + 1 read on the device
__global__ void adam_dev_kernel(float *th, const float *__restrict__ g, float *m, float *v, int n, float lr,
                                float b1, float b2, float eps, const int *__restrict__ step) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float t = (float)(*step + 1);
    const float c1 = 1.f - powf(b1, t), c2 = 1.f - powf(b2, t);
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    th[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// record the step's loss and advance the step counter
__global__ void step_tail_kernel(int *step, const double *__restrict__ loss, double *losses) {
    losses[*step] = *loss;
    *step += 1;
}

}  // namespace

cudaError_t rows_from_features(Workspace &ws, const float *X, const float *u, const float *rw, int n, int R,
                               cudaStream_t st) {
    features_kernel<<<(R + 255) / 256, 256, 0, st>>>(X, u, rw, n, R, ws.X, ws.XT, ws.u, ws.rw);
    return cudaGetLastError();
}

cudaError_t fill(float *p, float v, int n, cudaStream_t st) {
    fill_kernel<<<(n + 255) / 256, 256, 0, st>>>(p, v, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host

Workspace::~Workspace() { release(); }

void Workspace::release() {
    if (base) cudaFree(base);
    base = nullptr;
    cap_rows = 0;
}

cudaError_t Workspace::reserve(int R) {
    if (R <= cap_rows) return cudaSuccess;
    release();
    // byte layout (each piece 256-aligned)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t oX = take((size_t)R * kK1 * 2), oXT = take((size_t)kK1 * R * 2), ou = take((size_t)R * 4),
                 orw = take((size_t)R * 4);
    size_t opre[3], oH[3], oHT[3];
    for (int l = 0; l < 3; ++l) {
        opre[l] = take((size_t)R * kHid * 4);
        oH[l] = take((size_t)R * kHid * 2);
        oHT[l] = take((size_t)kHid * R * 2);
    }
    const size_t oY = take((size_t)R * 2 * 4), odYp = take((size_t)R * kK1 * 2), odYT = take((size_t)2 * R * 2),
                 odP = take((size_t)R * kHid * 2), odPT = take((size_t)kHid * R * 2),
                 odP2 = take((size_t)R * kHid * 2), odPT2 = take((size_t)kHid * R * 2);
    const size_t ow = take((size_t)(kHid * kK1 * 2 + 4 * kHid * kHid * 2 + kOut * kHid * 2 + kHid * kK1 * 2));
    const size_t og = take((size_t)(kHid * kK1 + 2 * kHid * kHid + kOut * kHid + 3 * kHid + kOut) * 4);
    const size_t oflat = take((size_t)mlp::kParams * 4 * 4);   // theta, grad, m, v
    const size_t oloss = take(8);
    const size_t ostatus = take(4);
    cudaError_t e = cudaFuncSetAttribute(gemm_nt, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&base, off);
    if (e != cudaSuccess) {
        base = nullptr;
        return e;
    }
    unsigned char *p = static_cast<unsigned char *>(base);
    X = (__nv_bfloat16 *)(p + oX);
    XT = (__nv_bfloat16 *)(p + oXT);
    u = (float *)(p + ou);
    rw = (float *)(p + orw);
    for (int l = 0; l < 3; ++l) {
        pre[l] = (float *)(p + opre[l]);
        H[l] = (__nv_bfloat16 *)(p + oH[l]);
        HT[l] = (__nv_bfloat16 *)(p + oHT[l]);
    }
    Y = (float *)(p + oY);
    dYp = (__nv_bfloat16 *)(p + odYp);
    dYT = (__nv_bfloat16 *)(p + odYT);
    dP = (__nv_bfloat16 *)(p + odP);
    dPT = (__nv_bfloat16 *)(p + odPT);
    dP2 = (__nv_bfloat16 *)(p + odP2);
    dPT2 = (__nv_bfloat16 *)(p + odPT2);
    __nv_bfloat16 *w = (__nv_bfloat16 *)(p + ow);
    W1p = w;
    W2 = W1p + kHid * kK1;
    W3 = W2 + kHid * kHid;
    W2T = W3 + kHid * kHid;
    W3T = W2T + kHid * kHid;
    W4 = W3T + kHid * kHid;
    W4T = W4 + kOut * kHid;
    float *g = (float *)(p + og);
    dW1 = g;
    dW2 = dW1 + kHid * kK1;
    dW3 = dW2 + kHid * kHid;
    dW4 = dW3 + kHid * kHid;
    db = dW4 + kOut * kHid;   // db1, db2, db3 (128 each), db4 (2)
    theta = (float *)(p + oflat);
    grad = theta + mlp::kParams;
    m = grad + mlp::kParams;
    v = m + mlp::kParams;
    loss = (double *)(p + oloss);
    status = (int *)(p + ostatus);
    e = cudaMemset(status, 0, sizeof(int));
    if (e != cudaSuccess) return e;
    grad_bytes = og;
    cap_rows = R;
    gbytes = (size_t)(kHid * kK1 + 2 * kHid * kHid + kOut * kHid + 3 * kHid + kOut) * 4;
    return cudaSuccess;
}

static int *g_status = nullptr;   // the workspace's timeout word, set by loss_grad

static cudaError_t gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, float *C, int ldc,
                        int M, int N, int K, cudaStream_t st, bool split, int mode = EP_STORE,
                        EpArgs ep = EpArgs{nullptr, nullptr, nullptr, nullptr}) {
    // weight gradients (K = R): split K over about one CTA per SM (chunks of
    // >= 256; 126 CTAs at 32 256 rows were 14 % faster for the whole training
    // step than 31 chunks of 1024)
    int splitk = 1, kchunk = K;
    if (split) {
        splitk = std::max(1, std::min(K / 256, 152));
        kchunk = ((K + splitk - 1) / splitk + kBK - 1) / kBK * kBK;
        splitk = (K + kchunk - 1) / kchunk;
    }
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, splitk);
    gemm_nt<<<grid, kGemmThreads, kGemmSmem, st>>>(A, lda, B, ldb, C, ldc, M, N, K, kchunk, split ? EP_ADD : mode,
                                                   ep, g_status);
    return cudaGetLastError();
}

cudaError_t loss_grad(Workspace &ws, int R, double inv_norm, bool use_rw, cudaStream_t st) {
    cudaGetLastError();
    g_status = ws.status;
    if (R % 32 != 0 || R > ws.cap_rows) return cudaErrorInvalidValue;
    const int Rp = R;   // K of the weight-gradient GEMMs
    const float *th = ws.theta;
    const float *b1 = th + kHid * kIn, *b2 = b1 + kHid + kHid * kHid, *b3 = b2 + kHid + kHid * kHid,
                *b4 = b3 + kHid + kOut * kHid;
    prep_weights_kernel<<<kHid, kHid, 0, st>>>(th, ws.W1p, ws.W2, ws.W3, ws.W4, ws.W2T, ws.W3T, ws.W4T);
    // forward: each hidden layer's GEMM adds the bias and applies GELU in its epilogue
    cudaError_t e = gemm(ws.X, kK1, ws.W1p, kK1, nullptr, kHid, R, kHid, kK1, st, false, EP_GELU,
                         EpArgs{b1, ws.pre[0], ws.H[0], ws.HT[0]});
    if (e) return e;
    if ((e = gemm(ws.H[0], kHid, ws.W2, kHid, nullptr, kHid, R, kHid, kHid, st, false, EP_GELU,
                  EpArgs{b2, ws.pre[1], ws.H[1], ws.HT[1]})))
        return e;
    if ((e = gemm(ws.H[1], kHid, ws.W3, kHid, nullptr, kHid, R, kHid, kHid, st, false, EP_GELU,
                  EpArgs{b3, ws.pre[2], ws.H[2], ws.HT[2]})))
        return e;
    if ((e = gemm(ws.H[2], kHid, ws.W4, kHid, ws.Y, 2, R, kOut, kHid, st, false))) return e;
    // loss and dY
    if ((e = cudaMemsetAsync(ws.loss, 0, 8, st))) return e;
    if ((e = cudaMemsetAsync(ws.dYp, 0, (size_t)R * kK1 * 2, st))) return e;
    out_loss_kernel<<<(R + 255) / 256, 256, 0, st>>>(ws.Y, b4, ws.u, use_rw ? ws.rw : nullptr, inv_norm, ws.dYp,
                                                     ws.dYT, R, ws.loss);
    // backward
    if ((e = cudaMemsetAsync(ws.dW1, 0, ws.gbytes, st))) return e;
    if ((e = gemm(ws.dYT, R, ws.HT[2], R, ws.dW4, kHid, kOut, kHid, Rp, st, true))) return e;
    rowsum_kernel<<<kOut, kRowsumThreads, 0, st>>>(ws.dYT, R, ws.db + 3 * kHid);
    // dL/dpre of the last hidden layer straight from the dL/dH GEMM's epilogue;
    // the layers' dP, dPT alternate between two buffers (one GEMM reads the
    // layer above's while writing the one below)
    __nv_bfloat16 *dP[2] = {ws.dP, ws.dP2}, *dPT[2] = {ws.dPT, ws.dPT2};
    if ((e = gemm(ws.dYp, kK1, ws.W4T, kK1, nullptr, kHid, R, kHid, kK1, st, false, EP_DGELU,
                  EpArgs{nullptr, ws.pre[2], dP[0], dPT[0]})))
        return e;
    const __nv_bfloat16 *WT[3] = {nullptr, ws.W2T, ws.W3T};
    float *dW[3] = {ws.dW1, ws.dW2, ws.dW3};
    for (int l = 2, cur = 0; l >= 0; --l, cur ^= 1) {
        rowsum_kernel<<<kHid, kRowsumThreads, 0, st>>>(dPT[cur], R, ws.db + l * kHid);
        if (l > 0) {
            if ((e = gemm(dPT[cur], R, ws.HT[l - 1], R, dW[l], kHid, kHid, kHid, Rp, st, true))) return e;
            if ((e = gemm(dP[cur], kHid, WT[l], kHid, nullptr, kHid, R, kHid, kHid, st, false, EP_DGELU,
                          EpArgs{nullptr, ws.pre[l - 1], dP[cur ^ 1], dPT[cur ^ 1]})))
                return e;
        } else {
            if ((e = gemm(dPT[cur], R, ws.XT, R, ws.dW1, kK1, kHid, kK1, Rp, st, true))) return e;
        }
    }
    gather_grad_kernel<<<(mlp::kParams + 255) / 256, 256, 0, st>>>(ws.dW1, ws.db, ws.dW2, ws.db + kHid, ws.dW3,
                                                                  ws.db + 2 * kHid, ws.dW4, ws.db + 3 * kHid,
                                                                  ws.grad);
    return cudaGetLastError();
}

cudaError_t adam_step(Workspace &ws, int t, float lr, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
    adam_kernel<<<(mlp::kParams + 255) / 256, 256, 0, st>>>(ws.theta, ws.grad, ws.m, ws.v, mlp::kParams, lr, b1, b2,
                                                           1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t sample_ids(const double *cdf, int64_t n, double total, uint64_t seed, const int *step, int nb,
                       int *ids, cudaStream_t st) {
    sample_ids_kernel<<<(nb + 127) / 128, 128, 0, st>>>(cdf, n, total,
                                                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), step,
                                                       nb, ids);
    return cudaGetLastError();
}

cudaError_t adam_step_dev(Workspace &ws, const int *step, float lr, cudaStream_t st) {
    adam_dev_kernel<<<(mlp::kParams + 255) / 256, 256, 0, st>>>(ws.theta, ws.grad, ws.m, ws.v, mlp::kParams, lr,
                                                               0.9f, 0.999f, 1e-8f, step);
    return cudaGetLastError();
}

cudaError_t step_tail(int *step, const double *loss, double *losses, cudaStream_t st) {
    step_tail_kernel<<<1, 1, 0, st>>>(step, loss, losses);
    return cudaGetLastError();
}

cudaError_t build_rows(Workspace &ws, const float *paths, int np1, const int *ids, int nb, float a, float b,
                       float T, int S, const float *sig, cudaStream_t st) {
    const int R = nb * (np1 - 2);
    if (R % 32 != 0 || R > ws.cap_rows) return cudaErrorInvalidValue;
    rows_kernel<<<(R + 255) / 256, 256, 0, st>>>(paths, np1, ids, nb, a, b, T, S, sig, ws.X, ws.XT, R, ws.u);
    return cudaGetLastError();
}

}  // namespace train
}  // namespace su
