// The amplitude estimator for systems of d = D x M coordinates (Sec. 2.2,
// Eq. EXP / Eq. MBrec): bisection paths of every coordinate (Sec. 4.1), the
// level-p effective potential W(x, xb; eps) of a polynomial potential per
// slice, per-sample log-weights of every level, per-item log-sum-exp tuples.
#include <cstdint>

#include "sampler_impl.cuh"

namespace su {
namespace {

// z[sym] with z in registers: a chain of selects on the integer pipes
// instead of a dynamically indexed local-memory load
template <typename R, int D>
__device__ __forceinline__ R pick(const R (&z)[2 * D], int sym) {
    R v = z[0];
#pragma unroll
    for (int i = 1; i < 2 * D; ++i) v = sym == i ? z[i] : v;
    return v;
}

// out[i] = in[i] * z[i][sym] for the B slices.  sym is the same for every
// thread (a node of the program): from three coordinates on a chain of
// uniform branches picks the register (2d - 1 selects per slice cost more:
// the 3D anharmonic oscillator in single precision 147 -> 135 ms); with one
// or two coordinates the selects are as fast.
template <typename R, int D, int B, int K = 0>
__device__ __forceinline__ void mul_sym(R (&out)[B], const R (&in)[B], const R (&z)[B][2 * D], int sym) {
    if constexpr (D < 3) {
#pragma unroll
        for (int i = 0; i < B; ++i) out[i] = in[i] * pick<R, D>(z[i], sym);
    } else if constexpr (K < 2 * D - 1) {
        if (sym == K) {
#pragma unroll
            for (int i = 0; i < B; ++i) out[i] = in[i] * z[i][K];
        } else {
            mul_sym<R, D, B, K + 1>(out, in, z, sym);
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) out[i] = in[i] * z[i][K];
    }
}

// One stack entry of B slices as one aligned vector (8 to 32 bytes: one or
// two 16-byte local accesses per node for all B slices).
template <typename R, int B>
struct alignas(sizeof(R) * B) Lanes {
    R v[B];
};

// -eps W for B slices at once, each with variables z = (x_1..x_D, xb_1..xb_D):
// the monomial program walked depth first (each prefix node its parent times
// one variable, the parent the top of the stack), each node's entries
// combined by Horner in z_H^G and added times its monomial; the B slices
// share every node and coefficient load.
template <typename R, int D, int B>
__device__ __forceinline__ void nd_multi(const R (&z)[B][2 * D], const R *__restrict__ coef, const NdParams &Q,
                                         R (&w)[B]) {
    Lanes<R, B> stk[kNdMaxDepth + 1];
    R Y[B], acc[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        stk[0].v[i] = 1;
        acc[i] = 0;
        Y[i] = 1;
    }
    for (int g = 0; g < Q.G; ++g) mul_sym<R, D, B>(Y, Y, z, Q.H);
    const GeneralNode *__restrict__ nodes = Q.nodes;
    for (int t = 0; t < Q.n_nodes; ++t) {
        const GeneralNode nd = nodes[t];
        Lanes<R, B> m;
        if (t) {
            const Lanes<R, B> par = stk[nd.depth - 1];
            mul_sym<R, D, B>(m.v, par.v, z, nd.sym);
            stk[nd.depth] = m;
        } else {
#pragma unroll
            for (int i = 0; i < B; ++i) m.v[i] = 1;
        }
        const int cnt = nd.count;
        if (cnt) {
            const R *c = coef + nd.first;
            R h[B];
            const R top = c[cnt - 1];
#pragma unroll
            for (int i = 0; i < B; ++i) h[i] = top;
#pragma unroll 4
            for (int e = cnt - 2; e >= 0; --e) {
                const R ce = c[e];
#pragma unroll
                for (int i = 0; i < B; ++i) h[i] = fma(h[i], Y[i], ce);
            }
#pragma unroll
            for (int i = 0; i < B; ++i) acc[i] = fma(h[i], m.v[i], acc[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < B; ++i) w[i] = acc[i];
}

// Slices k..k+B-1 of a level (points pt(k*stp) .. pt((k+B)*stp)), added to w
// two at a time in ascending order.
template <typename R, int D, int B, typename PT>
__device__ __forceinline__ void nd_block(const R *__restrict__ tab, const NdParams &Q, PT &&pt, int k, int stp,
                                         R &w) {
    R z[B][2 * D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        R pl = pt(k * stp, c);
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const R pr = pt((k + i + 1) * stp, c);
            z[i][c] = (R)0.5 * (pl + pr);
            z[i][D + c] = (R)0.5 * (pr - pl);
            pl = pr;
        }
    }
    R wv[B];
    nd_multi<R, D, B>(z, tab, Q, wv);
#pragma unroll
    for (int i = 0; i < B; i += 2) w += wv[i] + wv[i + 1];
}

// R = double or float (the path, W and the per-level sums; the item's
// log-sum-exp tuples in double either way).
// Shared memory: sw[levels][kThreads] (R, reduced runs) | Box-Muller node tables (double).
// Global scratch per slot: the 2^(S-F) + 1 segment endpoints (F = min(S, kNdSeg)).
template <typename R, int D>
__global__ void __launch_bounds__(kThreads, 4) nd_kernel(const __grid_constant__ NdParams Q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SamplerParams &P = Q.base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int L = P.levels, S = P.S;
    const bool per_sample = P.w_out != nullptr;
    R *sw = reinterpret_cast<R *>(smem_raw);
    size_t off = per_sample ? 0 : sizeof(R) * (size_t)L * kThreads;
    off = (off + 15) & ~(size_t)15;
    bm::Tables *bm_smem = reinterpret_cast<bm::Tables *>(smem_raw + off);
    if constexpr (sizeof(R) == 8) bm::tables_init(bm_smem, tid, kThreads);
    __syncthreads();

    Stream<R> st;
    st.key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    st.inst = P.instance;
    st.bm = sizeof(R) == 8 ? bm_smem : nullptr;
    const int64_t ps = Q.pstride;
    // the path in segments of 2^F slices: the C + 1 segment endpoints (the
    // coarse levels' points) in this slot of the global scratch, one
    // segment's points at a time in local memory
    const int F = min(S, kNdSeg), Cn = S - F, C = 1 << Cn, NF = 1 << F;
    R *q = reinterpret_cast<R *>(Q.paths) + (int64_t)blockIdx.x * kThreads + tid;
    auto co = [&](int i, int c) -> R & { return q[((int64_t)i * D + c) * ps]; };
    R seg[((1 << kNdSeg) + 1) * D];
    constexpr int kB = sizeof(R) == 8 ? 2 : 8;   // slices per pass of the program

    for (int64_t item = P.item0 + blockIdx.x; item < P.n_items; item += gridDim.x) {
        const int64_t b = item / P.items_per_block;
        const int64_t r = item - b * P.items_per_block;
        const int64_t lo = b * P.n_mc / P.n_blocks;
        const int64_t hi = (b + 1) * P.n_mc / P.n_blocks;
        const int64_t start = lo + r * kThreads;
        const int cnt = (int)max((int64_t)0, min((int64_t)kThreads, hi - start));
        if (tid < cnt) {
            const uint64_t sample = (uint64_t)(P.sample0 + start + tid);
            st.slo = (uint32_t)sample;
            st.shi = (uint32_t)(sample >> 32);
            // normal g of the sample's stream: double, branch g & 1 of the
            // Box-Muller pair of call g >> 1; float, slot (g + 1) & 3 of the
            // four normals of call (g + 1) >> 2 (the one-dimensional layouts)
            uint32_t have = 0xffffffffu;   // the call last drawn
            R zc[4] = {0, 0, 0, 0};
            auto normal = [&](uint32_t g) -> R {
                if constexpr (sizeof(R) == 8) {
                    if ((g >> 1) != have) {
                        double z0, z1;
                        st.pair(g >> 1, z0, z1);
                        zc[0] = z0;
                        zc[1] = z1;
                        have = g >> 1;
                    }
                    return (g & 1u) ? zc[1] : zc[0];
                } else {
                    if (((g + 1) >> 2) != have) {
                        st.quad((g + 1) >> 2, zc);
                        have = (g + 1) >> 2;
                    }
                    return pick4(zc, g + 1);
                }
            };
            // coarse levels n = 1..S-F: midpoint i at segment endpoint (2i+1) 2^(S-F-n)
            for (int c = 0; c < D; ++c) {
                co(0, c) = Q.a[c];
                co(C, c) = Q.b[c];
            }
            for (int n = 1; n <= Cn; ++n) {
                const R sg = (R)P.sigma[n];
                const int h = 1 << (Cn - n), j0 = (1 << (n - 1)) - 1;
                for (int i = 0; i < (1 << (n - 1)); ++i) {
                    const int idx = (2 * i + 1) * h;
                    for (int c = 0; c < D; ++c)
                        co(idx, c) = fma(sg, normal((uint32_t)((j0 + i) * D + c)), (R)0.5 * (co(idx - h, c) + co(idx + h, c)));
                }
            }
            // w_n = -eps_n sum_k W on the level-n subpath (level n = S - dl),
            // slices in ascending order, kB at a time (fewer on a level of two or four)
            R wloc[SU_MAX_S];
            for (int dl = 0; dl < L; ++dl) wloc[dl] = 0;
            auto slices = [&](const R *tab, auto &&pt, int stp, int ns, R &w) {
                if (ns < kB) {
                    if constexpr (kB > 4) {
                        if (ns == 4) {
                            nd_block<R, D, 4>(tab, Q, pt, 0, stp, w);
                            return;
                        }
                    }
                    nd_block<R, D, 2>(tab, Q, pt, 0, stp, w);
                    return;
                }
                for (int k = 0; k < ns; k += kB) nd_block<R, D, kB>(tab, Q, pt, k, stp, w);
            };
            const R *tabs = reinterpret_cast<const R *>(P.tables);
            for (int dl = F; dl < L; ++dl)   // coarse levels: between segment endpoints
                slices(tabs + (size_t)dl * P.M, co, 1 << (dl - F), 1 << (S - dl), wloc[dl]);
            // fine levels n = S-F+1..S, one segment at a time
            auto fp = [&](int i, int c) -> R & { return seg[i * D + c]; };
            for (int sgi = 0; sgi < C; ++sgi) {
                for (int c = 0; c < D; ++c) {
                    fp(0, c) = co(sgi, c);
                    fp(NF, c) = co(sgi + 1, c);
                }
                for (int n = Cn + 1; n <= S; ++n) {
                    const R sg = (R)P.sigma[n];
                    const int h = 1 << (S - n), m = 1 << (n - Cn - 1);
                    const int j0 = (1 << (n - 1)) - 1 + sgi * m;
                    for (int il = 0; il < m; ++il) {
                        const int idx = (2 * il + 1) * h;
                        for (int c = 0; c < D; ++c)
                            fp(idx, c) = fma(sg, normal((uint32_t)((j0 + il) * D + c)), (R)0.5 * (fp(idx - h, c) + fp(idx + h, c)));
                    }
                }
                for (int dl = 0; dl < min(F, L); ++dl)
                    slices(tabs + (size_t)dl * P.M, fp, 1 << dl, NF >> dl, wloc[dl]);
            }
            bool bad = false;
            for (int dl = 0; dl < L; ++dl) bad |= isnan(wloc[dl]) || (isinf(wloc[dl]) && wloc[dl] > 0);
            if (bad) atomicOr(P.flags, 1);
            if (per_sample) {
                double *dst = P.w_out + (start + tid) * (int64_t)S;
                for (int dl = 0; dl < L; ++dl) dst[S - dl - 1] = (double)wloc[dl];
            } else {
                for (int dl = 0; dl < L; ++dl) sw[(size_t)dl * kThreads + tid] = wloc[dl];
            }
        }
        if (per_sample) continue;
        __syncthreads();
        item_lse<R>(sw, L, kThreads, cnt, P.partial, item, warp, lane);
        __syncthreads();
    }
}

template <typename R>
const void *nd_fn_r(int D) {
    switch (D) {
        case 1: return (const void *)nd_kernel<R, 1>;
        case 2: return (const void *)nd_kernel<R, 2>;
        case 3: return (const void *)nd_kernel<R, 3>;
        default: return (const void *)nd_kernel<R, 4>;
    }
}

const void *nd_fn(int D, int precision) {
    return precision == SU_FP32 ? nd_fn_r<float>(D) : nd_fn_r<double>(D);
}

}  // namespace

size_t nd_smem_bytes(const NdParams &Q, int precision) {
    const size_t rs = precision == SU_FP32 ? sizeof(float) : sizeof(double);
    size_t off = Q.base.w_out ? 0 : rs * (size_t)Q.base.levels * kThreads;
    off = (off + 15) & ~(size_t)15;
    return off + (precision == SU_FP32 ? 0 : sizeof(bm::Tables));
}

int nd_occupancy(const NdParams &Q, int precision, size_t smem) {
    const void *fn = nd_fn(Q.D, precision);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_nd(const NdParams &Q, int precision, int grid, size_t smem, cudaStream_t st) {
    const void *fn = nd_fn(Q.D, precision);
    cudaGetLastError();
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<NdParams *>(&Q)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, smem, st);
}

}  // namespace su
