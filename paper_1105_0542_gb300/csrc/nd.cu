// The amplitude estimator for systems of d = D x M coordinates (Sec. 2.2,
// Eq. EXP / Eq. MBrec): bisection paths of every coordinate (Sec. 4.1), the
// level-p effective potential W(x, xb; eps) of a polynomial potential per
// slice, per-sample log-weights of every level, per-item log-sum-exp tuples.
#include <cstdint>

#include "sampler_impl.cuh"

namespace su {
namespace {

// -eps W of two slices with variables za, zb = (x_1..x_D, xb_1..xb_D): the
// monomial program walked depth first (each prefix its parent times one
// variable, the parent the top of a per-slice stack), each prefix's entries
// combined by Horner in z_H^G and added times the prefix; the two slices
// share every node and coefficient load.
// z[sym] with z in registers: a chain of selects on the integer pipes
// instead of a dynamically indexed local-memory load
template <typename R, int D>
__device__ __forceinline__ R pick(const R (&z)[2 * D], int sym) {
    R v = z[0];
#pragma unroll
    for (int i = 1; i < 2 * D; ++i) v = sym == i ? z[i] : v;
    return v;
}

template <typename R, int D>
__device__ __forceinline__ void nd_pair(const R (&za)[2 * D], const R (&zb)[2 * D], const R *__restrict__ coef,
                                        const NdParams &Q, R &wa, R &wb) {
    R sa[kNdMaxDepth + 1], sb[kNdMaxDepth + 1];
    sa[0] = 1;
    sb[0] = 1;
    R Ya = 1, Yb = 1;
    const R ha = pick<R, D>(za, Q.H), hb = pick<R, D>(zb, Q.H);
    for (int g = 0; g < Q.G; ++g) {
        Ya *= ha;
        Yb *= hb;
    }
    R acc_a = 0, acc_b = 0;
    const GeneralNode *__restrict__ nodes = Q.nodes;
    for (int t = 0; t < Q.n_nodes; ++t) {
        const GeneralNode nd = nodes[t];
        R ma = 1, mb = 1;
        if (t) {
            ma = sa[nd.depth - 1] * pick<R, D>(za, nd.sym);
            mb = sb[nd.depth - 1] * pick<R, D>(zb, nd.sym);
            sa[nd.depth] = ma;
            sb[nd.depth] = mb;
        }
        const int cnt = nd.count;
        if (cnt) {
            const R *c = coef + nd.first;
            R ha = c[cnt - 1], hb = ha;
#pragma unroll 4
            for (int e = cnt - 2; e >= 0; --e) {
                const R ce = c[e];
                ha = fma(ha, Ya, ce);
                hb = fma(hb, Yb, ce);
            }
            acc_a = fma(ha, ma, acc_a);
            acc_b = fma(hb, mb, acc_b);
        }
    }
    wa = acc_a;
    wb = acc_b;
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
    if constexpr (sizeof(R) == 8) {
        bm::tables_init(bm_smem, tid, kThreads);
        __syncthreads();
    }

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
            // slices in ascending order, two at a time
            R wloc[SU_MAX_S];
            for (int dl = 0; dl < L; ++dl) wloc[dl] = 0;
            auto slices = [&](const R *tab, auto &&pt, int stp, int ns, R &w) {
                for (int k = 0; k < ns; k += 2) {
                    R za[2 * D], zb[2 * D];
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        const R pl = pt(k * stp, c), pm = pt((k + 1) * stp, c), pr = pt((k + 2) * stp, c);
                        za[c] = (R)0.5 * (pl + pm);
                        za[D + c] = (R)0.5 * (pm - pl);
                        zb[c] = (R)0.5 * (pm + pr);
                        zb[D + c] = (R)0.5 * (pr - pm);
                    }
                    R wa, wb;
                    nd_pair<R, D>(za, zb, tab, Q, wa, wb);
                    w += wa + wb;
                }
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
