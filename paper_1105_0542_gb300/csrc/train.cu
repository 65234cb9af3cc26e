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
// operands with K contiguous, float accumulation (mma.sync m16n8k16), so the
// activations and gradients are kept both row-major and transposed (bf16).
// Products with K = R (the weight gradients) are split over K and summed with
// atomic adds.
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
constexpr int kBM = 128, kBN = 128, kBK = 32, kLS = kBK + 8;   // smem row stride 40 elements

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                    uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C[M][N] (+)= sum_k A[m][k] B[n][k] over the K-range of blockIdx.z.
// A: [M][lda], B: [N][ldb] bf16 (lda, ldb multiples of 8); K multiple of 32.
// 256 threads: warp (wm, wn) of 4 x 2 owns rows 32 wm.., columns 64 wn..
__global__ void __launch_bounds__(256) gemm_nt(const __nv_bfloat16 *__restrict__ A, int lda,
                                               const __nv_bfloat16 *__restrict__ B, int ldb,
                                               float *__restrict__ C, int ldc, int M, int N, int K,
                                               int kchunk, int atomic) {
    __shared__ __align__(16) __nv_bfloat16 As[kBM * kLS];
    __shared__ __align__(16) __nv_bfloat16 Bs[kBN * kLS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);
    float acc[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;

    for (int k0 = kb; k0 < ke; k0 += kBK) {
        // 128 rows x 32 columns = 512 pieces of 8 elements per operand
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int idx = tid + it * 256;
            const int r = idx >> 2, c = (idx & 3) * 8;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + r < M) va = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + k0 + c);
            if (n0 + r < N) vb = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * ldb + k0 + c);
            *reinterpret_cast<uint4 *>(As + r * kLS + c) = va;
            *reinterpret_cast<uint4 *>(Bs + r * kLS + c) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kBK; ks += 16) {
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int row = wm * 32 + mt * 16 + (lane & 15);
                const int col = ks + (lane >> 4) * 8;
                ldsm_x4(mlp::smem_u32(As + row * kLS + col), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
            }
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                const int row = wn * 64 + np * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int col = ks + ((lane >> 3) & 1) * 8;
                uint32_t b0, b1, b2, b3;
                ldsm_x4(mlp::smem_u32(Bs + row * kLS + col), b0, b1, b2, b3);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                    mma(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int r = m0 + wm * 32 + mt * 16 + (lane >> 2);
            const int c = n0 + wn * 64 + nt * 8 + (lane & 3) * 2;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rr = r + 8 * h;
                if (rr >= M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (c + e >= N) continue;
                    float *dst = C + (size_t)rr * ldc + c + e;
                    if (atomic)
                        atomicAdd(dst, acc[mt][nt][2 * h + e]);
                    else
                        *dst = acc[mt][nt][2 * h + e];
                }
            }
        }
}

__device__ __forceinline__ float gelu(float v) { return 0.5f * v * (1.0f + erff(v * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float v) {
    return 0.5f * (1.0f + erff(v * 0.70710678118654752f)) + v * 0.39894228040143268f * __expf(-0.5f * v * v);
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

// pre += bias; H = GELU(pre) row-major and transposed (32 x 32 tiles through smem)
__global__ void bias_gelu_kernel(float *pre, const float *__restrict__ bias, __nv_bfloat16 *H,
                                 __nv_bfloat16 *HT, int R) {
    __shared__ float t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        float g = 0.f;
        if (r < R) {
            const float v = pre[(size_t)r * kHid + c] + bias[c];
            pre[(size_t)r * kHid + c] = v;
            g = gelu(v);
            H[(size_t)r * kHid + c] = __float2bfloat16_rn(g);
        }
        t[y][threadIdx.x] = g;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < R) HT[(size_t)c * R + r] = __float2bfloat16_rn(t[threadIdx.x][y]);
    }
}

// dPre = dH * GELU'(pre), row-major and transposed
__global__ void gelu_bwd_kernel(const float *__restrict__ dH, const float *__restrict__ pre,
                                __nv_bfloat16 *dP, __nv_bfloat16 *dPT, int R) {
    __shared__ float t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        float g = 0.f;
        if (r < R) {
            g = dH[(size_t)r * kHid + c] * gelu_grad(pre[(size_t)r * kHid + c]);
            dP[(size_t)r * kHid + c] = __float2bfloat16_rn(g);
        }
        t[y][threadIdx.x] = g;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < R) dPT[(size_t)c * R + r] = __float2bfloat16_rn(t[threadIdx.x][y]);
    }
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

// out[row] = sum_r XT[row][r] (bias gradients from transposed gradients)
__global__ void rowsum_kernel(const __nv_bfloat16 *__restrict__ XT, int R, float *out) {
    float s = 0.f;
    for (int r = threadIdx.x; r < R; r += blockDim.x) s += __bfloat162float(XT[(size_t)blockIdx.x * R + r]);
    __shared__ float sb[256];
    sb[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) sb[threadIdx.x] += sb[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sb[0];
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
                 odH = take((size_t)R * kHid * 4), odP = take((size_t)R * kHid * 2), odPT = take((size_t)kHid * R * 2);
    const size_t ow = take((size_t)(kHid * kK1 * 2 + 4 * kHid * kHid * 2 + kOut * kHid * 2 + kHid * kK1 * 2));
    const size_t og = take((size_t)(kHid * kK1 + 2 * kHid * kHid + kOut * kHid + 3 * kHid + kOut) * 4);
    const size_t oflat = take((size_t)mlp::kParams * 4 * 4);   // theta, grad, m, v
    const size_t oloss = take(8);
    cudaError_t e = cudaMalloc(&base, off);
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
    dH = (float *)(p + odH);
    dP = (__nv_bfloat16 *)(p + odP);
    dPT = (__nv_bfloat16 *)(p + odPT);
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
    grad_bytes = og;
    cap_rows = R;
    gbytes = (size_t)(kHid * kK1 + 2 * kHid * kHid + kOut * kHid + 3 * kHid + kOut) * 4;
    return cudaSuccess;
}

static cudaError_t gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, float *C, int ldc,
                        int M, int N, int K, cudaStream_t st, bool split) {
    // weight gradients (K = R): split K over enough CTAs to fill the GPU
    int splitk = 1, kchunk = K;
    if (split) {
        splitk = std::max(1, std::min(K / 1024, 64));
        kchunk = ((K + splitk - 1) / splitk + kBK - 1) / kBK * kBK;
        splitk = (K + kchunk - 1) / kchunk;
    }
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, splitk);
    gemm_nt<<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, kchunk, split ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t loss_grad(Workspace &ws, int R, double inv_norm, bool use_rw, cudaStream_t st) {
    cudaGetLastError();
    if (R % 32 != 0 || R > ws.cap_rows) return cudaErrorInvalidValue;
    const int Rp = R;   // K of the weight-gradient GEMMs
    const float *th = ws.theta;
    const float *b1 = th + kHid * kIn, *b2 = b1 + kHid + kHid * kHid, *b3 = b2 + kHid + kHid * kHid,
                *b4 = b3 + kHid + kOut * kHid;
    prep_weights_kernel<<<kHid, kHid, 0, st>>>(th, ws.W1p, ws.W2, ws.W3, ws.W4, ws.W2T, ws.W3T, ws.W4T);
    const dim3 tb(32, 8), tg((R + 31) / 32, kHid / 32);
    // forward
    cudaError_t e = gemm(ws.X, kK1, ws.W1p, kK1, ws.pre[0], kHid, R, kHid, kK1, st, false);
    if (e) return e;
    bias_gelu_kernel<<<tg, tb, 0, st>>>(ws.pre[0], b1, ws.H[0], ws.HT[0], R);
    if ((e = gemm(ws.H[0], kHid, ws.W2, kHid, ws.pre[1], kHid, R, kHid, kHid, st, false))) return e;
    bias_gelu_kernel<<<tg, tb, 0, st>>>(ws.pre[1], b2, ws.H[1], ws.HT[1], R);
    if ((e = gemm(ws.H[1], kHid, ws.W3, kHid, ws.pre[2], kHid, R, kHid, kHid, st, false))) return e;
    bias_gelu_kernel<<<tg, tb, 0, st>>>(ws.pre[2], b3, ws.H[2], ws.HT[2], R);
    if ((e = gemm(ws.H[2], kHid, ws.W4, kHid, ws.Y, 2, R, kOut, kHid, st, false))) return e;
    // loss and dY
    if ((e = cudaMemsetAsync(ws.loss, 0, 8, st))) return e;
    if ((e = cudaMemsetAsync(ws.dYp, 0, (size_t)R * kK1 * 2, st))) return e;
    out_loss_kernel<<<(R + 255) / 256, 256, 0, st>>>(ws.Y, b4, ws.u, use_rw ? ws.rw : nullptr, inv_norm, ws.dYp,
                                                     ws.dYT, R, ws.loss);
    // backward
    if ((e = cudaMemsetAsync(ws.dW1, 0, ws.gbytes, st))) return e;
    if ((e = gemm(ws.dYT, R, ws.HT[2], R, ws.dW4, kHid, kOut, kHid, Rp, st, true))) return e;
    rowsum_kernel<<<kOut, 256, 0, st>>>(ws.dYT, R, ws.db + 3 * kHid);
    if ((e = gemm(ws.dYp, kK1, ws.W4T, kK1, ws.dH, kHid, R, kHid, kK1, st, false))) return e;
    const __nv_bfloat16 *WT[3] = {nullptr, ws.W2T, ws.W3T};
    float *dW[3] = {ws.dW1, ws.dW2, ws.dW3};
    for (int l = 2; l >= 0; --l) {
        gelu_bwd_kernel<<<tg, tb, 0, st>>>(ws.dH, ws.pre[l], ws.dP, ws.dPT, R);
        rowsum_kernel<<<kHid, 256, 0, st>>>(ws.dPT, R, ws.db + l * kHid);
        if (l > 0) {
            if ((e = gemm(ws.dPT, R, ws.HT[l - 1], R, dW[l], kHid, kHid, kHid, Rp, st, true))) return e;
            if ((e = gemm(ws.dP, kHid, WT[l], kHid, ws.dH, kHid, R, kHid, kHid, st, false))) return e;
        } else {
            if ((e = gemm(ws.dPT, R, ws.XT, R, ws.dW1, kK1, kHid, kK1, Rp, st, true))) return e;
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
