// The learned bisection proposal on the device (single-precision path).
//
// proposal_kernel -- 128 paths per work item, one per thread of the first
// four warps; all eight warps evaluate the network.  For bisection level
// n = 1..S and midpoint index i, the 128 paths' features
// (a, b, T, n/S, q_L, q_R) form one 128-row tile; the network gives every
// path (shift, ls); the path's thread draws its normal z (the plain
// sampler's stream: normal j = 2^(n-1) - 1 + i) and places
//   q = (q_L + q_R)/2 + sigma_n (shift + e^ls z),
// adding z^2/2 - (shift + e^ls z)^2/2 + ls (log bridge density minus log
// proposal density) to the weight of every level >= n.  Then W_p is summed
// over every level of the path (Eq. SNp) and the item's weights are reduced
// as in the plain sampler.  Paths live in shared memory ([N+1][128] floats),
// so N <= 64.
//
// mlp_forward_kernel -- the network alone on rows of features in global
// memory (parity tests, diagnostics).
#include <cmath>
#include <cstdint>
#include <cstring>

#include "mlp.cuh"
#include "proposal.h"
#include "sampler_impl.cuh"

namespace su {

namespace mlp {

static uint16_t bf16_rn(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

void pack_blob(const float *theta, unsigned char *blob) {
    std::memset(blob, 0, kBlobBytes);
    // matrix [rows][cols] (row-major floats) into the operand layout with K
    // columns (cols <= K, the rest zero)
    auto put = [&](int off, int K, int rows, int cols, const float *src) {
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) {
                const uint16_t v = bf16_rn(src[r * cols + c]);
                std::memcpy(blob + off + cm_off(r, c, K), &v, 2);
            }
    };
    const float *p = theta;
    const float *W1 = p;
    p += kHid * kIn;
    const float *b1 = p;
    p += kHid;
    const float *W2 = p;
    p += kHid * kHid;
    const float *b2 = p;
    p += kHid;
    const float *W3 = p;
    p += kHid * kHid;
    const float *b3 = p;
    p += kHid;
    const float *W4 = p;
    p += kOut * kHid;
    const float *b4 = p;
    put(kOffW1, kK1, kHid, kIn, W1);
    put(kOffW2, kHid, kHid, kHid, W2);
    put(kOffW3, kHid, kHid, kHid, W3);
    put(kOffW4, kHid, kOut, kHid, W4);
    float *B = reinterpret_cast<float *>(blob + kOffB);
    std::memcpy(B, b1, kHid * 4);
    std::memcpy(B + kHid, b2, kHid * 4);
    std::memcpy(B + 2 * kHid, b3, kHid * 4);
    std::memcpy(B + 3 * kHid, b4, kOut * 4);
}

}  // namespace mlp

namespace {

using mlp::kBlobBytes;
using mlp::kX0Bytes;
using mlp::kHBytes;
using mlp::kRows;
using mlp::kIn;
using mlp::Tc;
using mlp::tile_forward;
constexpr int kT = mlp::kThreads;

__device__ __forceinline__ void copy16(void *dst, const void *src, int bytes, int tid, int nth) {
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = tid; i < bytes / 16; i += nth) d[i] = s[i];
}

// shared memory: blob | X0 | H | out[128][2] | qs[(N+1)][128] | tab[S][M] | sig[11] | corr[S+1][128] | sw[S][128]
template <int RING>
__global__ void __launch_bounds__(mlp::kThreads, 1) proposal_kernel(const __grid_constant__ ProposalParams Q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SamplerParams &P = Q.base;
    const int tid = threadIdx.x;
    const int S = P.S, N = 1 << S, L = P.levels;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mma_bar;
    unsigned char *blob = smem_raw;
    size_t off = kBlobBytes;
    unsigned char *X0 = smem_raw + off;
    off += kX0Bytes;
    unsigned char *H = smem_raw + off;
    off += kHBytes;
    float *out = reinterpret_cast<float *>(smem_raw + off);
    off += kRows * 2 * 4;
    float *qs = reinterpret_cast<float *>(smem_raw + off);
    off += (size_t)(N + 1) * kRows * 4;
    float *tab = reinterpret_cast<float *>(smem_raw + off);
    off += (size_t)S * P.M * 4;
    float *sig = reinterpret_cast<float *>(smem_raw + off);
    off += 16 * 4;
    float *corr = reinterpret_cast<float *>(smem_raw + off);
    off += (size_t)(S + 1) * kRows * 4;
    float *sw = reinterpret_cast<float *>(smem_raw + off);

    copy16(blob, Q.blob, kBlobBytes, tid, kT);
    {
        const float *g = reinterpret_cast<const float *>(P.tables);
        for (int i = tid; i < S * P.M; i += kT) tab[i] = g[i];
        for (int i = tid; i <= SU_MAX_S; i += kT) sig[i] = (float)P.sigma[i];
        for (int i = tid; i < kX0Bytes / 16; i += kT) reinterpret_cast<uint4 *>(X0)[i] = make_uint4(0, 0, 0, 0);
    }
    Tc tc = mlp::tc_begin(&tmem_slot, &mma_bar);   // contains __syncthreads
    bool alive = true;

    const float fa = (float)P.a, fb = (float)P.b, fT = (float)Q.T;
    const __nv_bfloat16 ba = __float2bfloat16_rn(fa), bb = __float2bfloat16_rn(fb), bT = __float2bfloat16_rn(fT);
    const float alpha = (float)P.alpha;
    const int warp = tid >> 5, lane = tid & 31;
    const bool owner = tid < kRows;
    Stream<float> st;
    st.key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    st.inst = P.instance;
    st.bm = nullptr;

    for (int64_t item = blockIdx.x; alive && item < P.n_items; item += gridDim.x) {
        const int64_t bk = item / P.items_per_block;
        const int64_t r = item - bk * P.items_per_block;
        const int64_t lo = bk * P.n_mc / P.n_blocks;
        const int64_t hi = (bk + 1) * P.n_mc / P.n_blocks;
        const int64_t start = lo + r * kRows;
        const int cnt = (int)max((int64_t)0, min((int64_t)kRows, hi - start));
        const int p = tid;
        const bool valid = owner && p < cnt;
        float quad[4] = {0.f, 0.f, 0.f, 0.f}, c = 0.f;
        if (owner) {
            const uint64_t smp = (uint64_t)(P.sample0 + start + p);
            st.slo = (uint32_t)smp;
            st.shi = (uint32_t)(smp >> 32);
            qs[p] = fa;
            qs[N * kRows + p] = fb;
            corr[p] = 0.f;
        }
        for (int n = 1; alive && n <= S; ++n) {
            const int h = N >> n;
            const __nv_bfloat16 bn = __float2bfloat16_rn((float)n / (float)S);
            for (int i = 0; alive && i < (1 << (n - 1)); ++i) {
                const int kL = 2 * i * h, kM = kL + h, kR = kL + 2 * h;
                if (owner)
                    mlp::store_features(X0, p, ba, bb, bT, bn, __float2bfloat16_rn(qs[kL * kRows + p]),
                                        __float2bfloat16_rn(qs[kR * kRows + p]));
                asm volatile("fence.proxy.async.shared::cta;");
                __syncthreads();
                if (!tile_forward(tc, blob, X0, H, out, Q.withhold != 0)) {
                    if (tid == 0) atomicOr(P.flags, 4);   // an MMA never completed
                    alive = false;
                    break;
                }
                if (owner) {
                    const uint32_t j = (1u << (n - 1)) - 1u + (uint32_t)i;
                    // the plain single-precision stream: slot j' & 3 of call j' >> 2, j' = j + 1
                    const uint32_t jp = j + 1;
                    if (j == 0 || (jp & 3u) == 0) st.quad(jp >> 2, quad);
                    const float z = pick4(quad, jp);
                    const float sh = out[2 * p], ls = out[2 * p + 1];
                    const float t = fmaf(__expf(ls), z, sh);
                    const float mid = 0.5f * (qs[kL * kRows + p] + qs[kR * kRows + p]);
                    qs[kM * kRows + p] = fmaf(sig[n], t, mid);
                    c += 0.5f * z * z - 0.5f * t * t + ls;
                    if (Q.outs && valid) {
                        float *o = Q.outs + ((start + p) * (int64_t)(N - 1) + j) * 2;
                        o[0] = sh;
                        o[1] = ls;
                    }
                }
            }
            if (owner) corr[n * kRows + p] = c;
        }
        if (!alive) break;
        // W_p on every level of the path, plus the proposal weight
        if (owner) {
            for (int d = 0; d < L; ++d) {
                const int n = S - d;
                const int stp = 1 << d;
                float s = 0.f;
                for (int k = 0; k < (1 << n); ++k)
                    s += slice<float, RING>(qs[k * stp * kRows + p], qs[(k + 1) * stp * kRows + p],
                                            tab + d * P.M, P, alpha);
                const float w = s + corr[n * kRows + p];
                sw[d * kRows + p] = w;
                if (valid && (isnan(w) || (isinf(w) && w > 0))) atomicOr(P.flags, 1);
                if (valid && P.w_out) P.w_out[(start + p) * (int64_t)S + (n - 1)] = (double)w;
            }
        }
        __syncthreads();
        if (!P.w_out) {
            for (int d = warp; d < L; d += kT / 32) {
                const float *v = sw + d * kRows;
                float m = -INFINITY;
                for (int t = lane; t < cnt; t += 32) m = fmaxf(m, v[t]);
                m = warp_max(m);
                double s = 0, q = 0;
                if (m > -INFINITY) {
                    for (int t = lane; t < cnt; t += 32) {
                        const double e = (double)__expf(v[t] - m);
                        s += e;
                        q = fma(e, e, q);
                    }
                }
                s = warp_sum(s);
                q = warp_sum(q);
                if (lane == 0) {
                    double *o = P.partial + 4 * (item * L + d);
                    o[0] = (double)m;
                    o[1] = s;
                    o[2] = q;
                    o[3] = (double)cnt;
                }
            }
        }
        __syncthreads();
    }
    mlp::tc_end(tc);
}

// rows of features X (n x 6 floats) -> Y (n x 2); a tile whose MMAs never
// complete gives NaN outputs and ends the CTA's work
__global__ void __launch_bounds__(mlp::kThreads, 1) mlp_forward_kernel(const unsigned char *gblob,
                                                                       const float *X, int64_t n,
                                                                       float *Y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mma_bar;
    unsigned char *blob = smem_raw;
    unsigned char *X0 = smem_raw + kBlobBytes;
    unsigned char *H = smem_raw + kBlobBytes + kX0Bytes;
    float *out = reinterpret_cast<float *>(smem_raw + kBlobBytes + kX0Bytes + kHBytes);
    const int tid = threadIdx.x;
    copy16(blob, gblob, kBlobBytes, tid, kT);
    for (int i = tid; i < kX0Bytes / 16; i += kT) reinterpret_cast<uint4 *>(X0)[i] = make_uint4(0, 0, 0, 0);
    Tc tc = mlp::tc_begin(&tmem_slot, &mma_bar);
    for (int64_t t0 = (int64_t)blockIdx.x * kRows; t0 < n; t0 += (int64_t)gridDim.x * kRows) {
        if (tid < kRows) {
            const int64_t r = t0 + tid;
            float f[kIn];
            for (int c = 0; c < kIn; ++c) f[c] = r < n ? X[r * kIn + c] : 0.f;
            mlp::store_features(X0, tid, __float2bfloat16_rn(f[0]), __float2bfloat16_rn(f[1]),
                                __float2bfloat16_rn(f[2]), __float2bfloat16_rn(f[3]), __float2bfloat16_rn(f[4]),
                                __float2bfloat16_rn(f[5]));
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        const bool ok = tile_forward(tc, blob, X0, H, out);
        if (tid < kRows && t0 + tid < n) {
            Y[(t0 + tid) * 2] = ok ? out[2 * tid] : NAN;
            Y[(t0 + tid) * 2 + 1] = ok ? out[2 * tid + 1] : NAN;
        }
        __syncthreads();
        if (!ok) break;
    }
    mlp::tc_end(tc);
}

const void *proposal_fn(int ring) {
    switch (ring) {
        case RING_EVEN: return (const void *)proposal_kernel<RING_EVEN>;
        case RING_X: return (const void *)proposal_kernel<RING_X>;
        default: return (const void *)proposal_kernel<RING_TANH2>;
    }
}

cudaError_t allow_smem(const void *fn, size_t smem) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

size_t proposal_smem_bytes(const ProposalParams &Q) {
    const SamplerParams &P = Q.base;
    const int N = 1 << P.S;
    size_t off = mlp::kBlobBytes + mlp::kX0Bytes + mlp::kHBytes + mlp::kRows * 2 * 4;
    off += (size_t)(N + 1) * mlp::kRows * 4;
    off += (size_t)P.S * P.M * 4 + 16 * 4;
    off += (size_t)(P.S + 1) * mlp::kRows * 4;
    off += (size_t)P.S * mlp::kRows * 4;
    return off;
}

int proposal_occupancy(const ProposalParams &Q, size_t smem) {
    const void *fn = proposal_fn(Q.base.ring);
    if (allow_smem(fn, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, mlp::kThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_proposal(const ProposalParams &Q, int grid, size_t smem, cudaStream_t st) {
    const void *fn = proposal_fn(Q.base.ring);
    cudaGetLastError();
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<ProposalParams *>(&Q)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(mlp::kThreads), args, smem, st);
}

cudaError_t launch_mlp_forward(const unsigned char *blob, const float *X, int64_t n, float *Y, int sms,
                               cudaStream_t st) {
    const size_t smem = mlp::kBlobBytes + mlp::kX0Bytes + mlp::kHBytes + mlp::kRows * 2 * 4;
    cudaGetLastError();
    cudaError_t e = allow_smem((const void *)mlp_forward_kernel, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + mlp::kRows - 1) / mlp::kRows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
    mlp_forward_kernel<<<grid, mlp::kThreads, smem, st>>>(blob, X, n, Y);
    return cudaGetLastError();
}

}  // namespace su
