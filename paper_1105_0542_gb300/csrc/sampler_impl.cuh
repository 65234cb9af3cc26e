#pragma once
// Device code of the sampler (sm_103a); included once per (precision, ring)
// by sampler_inst.cu.
//
// sampler_kernel -- one bisection path per thread (Sec. 4.1):
//   Philox4x32-10 (Salmon et al., SC'11) -> Box-Muller -> bisection midpoints
//   -> W_p on every slice of every level of the hierarchy (Eq. SNp, Sec. 4.1)
//   -> per-sample log-weights -> per-item log-sum-exp tuples in double.
// combine_kernel -- merges the item tuples of each block in a fixed order.
//
// The hot path is ALU-bound (no HBM traffic per slice): paths live in
// registers, the coefficient tables in shared memory.  A path of N = 2^S
// slices is split into C = 2^(S-F) segments of 2^F slices (F = min(S, 5)):
// the C+1 segment endpoints (bisection levels 1..S-F) are generated first and
// parked in shared memory; each segment's 2^F - 1 interior points (levels
// S-F+1..S) are then generated in registers and all slices of the segment, at
// every level, are evaluated before the next segment starts.
//
// Normal j of a sample (heap order: level n, midpoint i -> j = 2^(n-1)-1+i)
// is Box-Muller branch (j & 1) of Philox call j >> 1.  Every call is computed
// once and its second normal carried to the midpoint that uses it, except the
// first midpoint of each in-register level in segment 0, whose call is shared
// with the last midpoint of the previous level (in the last segment) and is
// recomputed there (F-1 extra calls per path when C > 1).
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "boxmuller.cuh"
#include "generator.h"
#include "sampler.h"

namespace su {
namespace {

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// ------------------------------------------------------------ Box-Muller
template <typename R>
struct Normal;

template <>
struct Normal<double> {
    // 53-bit uniforms ((w0 2^21 + w1 >> 11) + 1/2) 2^-53 from (w0,w1) and (w2,w3),
    // through the table-driven routines of boxmuller.cuh
    static __device__ __forceinline__ void pair(uint4 w, const BMTables *t, double &z0, double &z1) {
        const uint64_t a = ((uint64_t)w.x << 21) | (w.y >> 11);
        const uint64_t b = ((uint64_t)w.z << 21) | (w.w >> 11);
        const double u1 = ((double)a + 0.5) * 0x1p-53;
        bm_rotate(bm_sqrt(bm_minus2log(u1, t)), b, t, z0, z1);
    }
};

template <>
struct Normal<float> {
    // 24-bit uniforms ((w >> 8) + 1/2) 2^-24 from w0 and w2
    static __device__ __forceinline__ void pair(uint4 w, const BMTables *, float &z0, float &z1) {
        const float u1 = ((float)(w.x >> 8) + 0.5f) * 0x1p-24f;
        const float u2 = ((float)(w.z >> 8) + 0.5f) * 0x1p-24f;
        const float r = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        z0 = r * cs;
        z1 = r * sn;
    }
};

template <typename R>
struct Stream {
    uint2 key;
    uint32_t inst, slo, shi;
    const BMTables *bm;   // shared-memory node tables (double path)
    __device__ __forceinline__ void pair(uint32_t call, R &z0, R &z1) const {
        Normal<R>::pair(philox4x32_10(make_uint4(call, inst, slo, shi), key), bm, z0, z1);
    }
};

// ------------------------------------------------------------------ W_p
template <typename R, int RING>
__device__ __forceinline__ R ring_var(R us, R alpha) {
    if constexpr (RING == RING_EVEN) {
        return us * us;
    } else if constexpr (RING == RING_X) {
        return us;
    } else {
        // tanh^2(alpha us / 2): tanh(y/2) = -em / (2 + em), em = expm1(-|y|),
        // accurate also where tanh is small
        const R em = expm1(-fabs(alpha * us));
        const R t = -em / ((R)2 + em);
        return t * t;
    }
}

// -eps W_p(x, xb; eps) of one slice, from the level's table in shared memory:
// sum_j (vs^2)^j sum_i T_ij Z^i, nested Horner (columns, then powers of vs^2).
template <typename R, int RING>
__device__ __forceinline__ R slice(R ql, R qr, const R *__restrict__ tab, const SamplerParams &P,
                                   R alpha) {
    const R us = ql + qr;
    const R vs = qr - ql;
    const R Y = vs * vs;
    const R Z = ring_var<R, RING>(us, alpha);
    int off = P.M;
    R acc = 0;
    for (int j = P.ncol - 1; j >= 0; --j) {
        const int L = P.len[j];
        off -= L;
        R h = tab[off + L - 1];
        for (int i = L - 2; i >= 0; --i) h = fma(h, Z, tab[off + i]);
        acc = fma(acc, Y, h);
    }
    return acc;
}

// Sum of -eps W_p over NS slices of one level of a segment, the slices taken
// between the points q[k STR] and q[(k+1) STR].  Slices are evaluated in
// batches of B side by side: each table entry is loaded once per batch (a
// broadcast shared-memory read) and feeds B independent multiply-add chains.
template <typename R>
struct Batch {
    static constexpr int B = sizeof(R) == 8 ? 4 : 8;
};

template <typename R, int RING, int NS, int STR, int NQ>
__device__ __forceinline__ R level_sum(const R (&q)[NQ], const R *__restrict__ tab,
                                       const SamplerParams &P, R alpha) {
    constexpr int B = NS < Batch<R>::B ? NS : Batch<R>::B;
    R total = 0;
#pragma unroll
    for (int k0 = 0; k0 < NS; k0 += B) {
        R Z[B], Y[B], acc[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const R ql = q[(k0 + b) * STR], qr = q[(k0 + b + 1) * STR];
            const R vs = qr - ql;
            Y[b] = vs * vs;
            Z[b] = ring_var<R, RING>(ql + qr, alpha);
        }
        int off = P.M;
        {   // last column starts the outer Horner in x-bar^2
            const int L = P.len[P.ncol - 1];
            off -= L;
            const R c = tab[off + L - 1];
#pragma unroll
            for (int b = 0; b < B; ++b) acc[b] = c;
            for (int i = L - 2; i >= 0; --i) {
                const R ci = tab[off + i];
#pragma unroll
                for (int b = 0; b < B; ++b) acc[b] = fma(acc[b], Z[b], ci);
            }
        }
        for (int j = P.ncol - 2; j >= 0; --j) {
            const int L = P.len[j];
            off -= L;
            R h[B];
            const R c = tab[off + L - 1];
#pragma unroll
            for (int b = 0; b < B; ++b) h[b] = c;
            for (int i = L - 2; i >= 0; --i) {
                const R ci = tab[off + i];
#pragma unroll
                for (int b = 0; b < B; ++b) h[b] = fma(h[b], Z[b], ci);
            }
#pragma unroll
            for (int b = 0; b < B; ++b) acc[b] = fma(acc[b], Y[b], h[b]);
        }
#pragma unroll
        for (int b = 0; b < B; ++b) total += acc[b];
    }
    return total;
}

// levels d = D..F of a segment (level n = S - d uses every 2^d-th point)
template <typename R, int RING, int F, int D>
__device__ __forceinline__ void segment_levels(R (&acc)[F + 1], const R (&q)[(1 << F) + 1],
                                               const R *__restrict__ tab, const SamplerParams &P,
                                               R alpha, int S) {
    if constexpr (D <= F) {
        if (D < S) {
            acc[D] += level_sum<R, RING, ((1 << F) >> D), (1 << D)>(q, tab + D * P.M, P, alpha);
            segment_levels<R, RING, F, D + 1>(acc, q, tab, P, alpha, S);
        }
    }
}

// --------------------------------------------------------------- a path
// This thread's shared-memory columns (stride kThreads): qc holds the C+1
// segment endpoints, zz the per-level sums of z^2 (width-factor weight only).
// Writes the log-weight of sampled level d (level n = S - d) to wout[d * wstride].
template <typename R, int RING, int F>
__device__ __forceinline__ void sample_path(const SamplerParams &P, const R *__restrict__ tab,
                                            R *__restrict__ qc, double *__restrict__ zz,
                                            const Stream<R> &st, double *__restrict__ wout,
                                            int wstride) {
    constexpr int NF = 1 << F;
    const int S = P.S;
    const int C = 1 << (S - F);
    const bool hier = P.levels > 1;
    const int M = P.M;
    const R alpha = (R)P.alpha;

    if (P.wf_on)
        for (int n = 0; n <= S; ++n) zz[n * kThreads] = 0.0;

    R cz[F + 1];
#pragma unroll
    for (int l = 0; l <= F; ++l) cz[l] = 0;

    // ---- segment endpoints: bisection levels 1..S-F, heap order j = 0..C-2
    if (C > 1) {
        qc[0] = (R)P.a;
        qc[C * kThreads] = (R)P.b;
        R carry = 0;
        uint32_t j = 0;
        for (int n = 1; n <= S - F; ++n) {
            const int hc = C >> n;
            const R sg = (R)P.sigma[n];
            for (int i = 0; i < (1 << (n - 1)); ++i, ++j) {
                R z;
                if ((j & 1u) == 0) {
                    R z0, z1;
                    st.pair(j >> 1, z0, z1);
                    z = z0;
                    carry = z1;
                } else {
                    z = carry;
                }
                if (P.wf_on) zz[n * kThreads] += (double)z * (double)z;
                const int idx = (2 * i + 1) * hc;
                qc[idx * kThreads] =
                    fma(sg, z, (R)0.5 * (qc[(idx - hc) * kThreads] + qc[(idx + hc) * kThreads]));
            }
        }
        cz[0] = carry;
    }

    // ---- segments: levels S-F+1..S in registers, all slices evaluated
    R acc[F + 1];
#pragma unroll
    for (int d = 0; d <= F; ++d) acc[d] = 0;

    for (int c = 0; c < C; ++c) {
        R q[NF + 1];
        q[0] = C > 1 ? qc[c * kThreads] : (R)P.a;
        q[NF] = C > 1 ? qc[(c + 1) * kThreads] : (R)P.b;
#pragma unroll
        for (int l = 1; l <= F; ++l) {
            const int n = S - F + l;
            const uint32_t jbase = (1u << (n - 1)) - 1u + ((uint32_t)c << (l - 1));
            const R sg = (R)P.sigma[n];
            constexpr int h0 = 1;
            const int h = h0 << (F - l);
#pragma unroll
            for (int il = 0; il < (1 << (l - 1)); ++il) {
                const uint32_t j = jbase + (uint32_t)il;
                R z;
                if ((j & 1u) == 0) {
                    R z0, z1;
                    st.pair(j >> 1, z0, z1);
                    z = z0;
                    cz[l] = z1;
                } else if (il == 0 && c == 0) {
                    if (C == 1) {
                        z = cz[l - 1];  // second normal of the previous level's last call
                    } else if (l == 1) {
                        z = cz[0];      // carried from the segment-endpoint levels
                    } else {
                        R z0, z1;       // shared with the last segment: recompute
                        st.pair(j >> 1, z0, z1);
                        z = z1;
                    }
                } else {
                    z = cz[l];
                }
                if (P.wf_on) zz[n * kThreads] += (double)z * (double)z;
                const int idx = (2 * il + 1) * h;
                q[idx] = fma(sg, z, (R)0.5 * (q[idx - h] + q[idx + h]));
            }
        }
        // top level: every slice of the segment; then the coarser levels
        acc[0] += level_sum<R, RING, NF, 1>(q, tab, P, alpha);
        if (hier) segment_levels<R, RING, F, 1>(acc, q, tab, P, alpha, S);
    }

    // ---- width-factor weight, cumulative over levels 1..n (stored in zz)
    if (P.wf_on) {
        double cum = 0;
        for (int n = 1; n <= S; ++n) {
            cum += (double)(1 << (n - 1)) * P.lwf + P.hcoef * zz[n * kThreads];
            zz[n * kThreads] = cum;
        }
    }
    auto corr = [&](int n) -> double { return P.wf_on ? zz[n * kThreads] : 0.0; };

    // ---- outputs, level n = S - d
#pragma unroll
    for (int d = 0; d <= F; ++d)
        if (d == 0 || (hier && d < S)) wout[d * wstride] = (double)acc[d] + corr(S - d);
    if (hier) {
        for (int n = 1; n < S - F; ++n) {
            const int d = S - n;
            const int stp = C >> n;
            R sum = 0;
            for (int k = 0; k < (1 << n); ++k)
                sum += slice<R, RING>(qc[k * stp * kThreads], qc[(k + 1) * stp * kThreads], tab + d * M,
                                      P, alpha);
            wout[d * wstride] = (double)sum + corr(n);
        }
    }
}

// -------------------------------------------------------- warp helpers
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ----------------------------------------------------------- the kernel
// Shared memory: sw[levels][chunk] (double) | tables[levels][M] (R) |
//                qc[(C+1)][kThreads] (R) | zz[S+1][kThreads] (double, if wf_on)
template <typename R, int RING>
__global__ void __launch_bounds__(kThreads) sampler_kernel(const __grid_constant__ SamplerParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int L = P.levels;
    const int chunk = kThreads * P.rounds;
    const bool per_sample = P.w_out != nullptr;
    const int C = 1 << (P.S - P.F);

    double *sw = reinterpret_cast<double *>(smem_raw);
    size_t off = per_sample ? 0 : sizeof(double) * (size_t)L * chunk;
    R *tab = reinterpret_cast<R *>(smem_raw + off);
    off += sizeof(R) * (size_t)P.S * P.M;
    off = (off + 15) & ~(size_t)15;
    R *qc = reinterpret_cast<R *>(smem_raw + off) + tid;
    off += sizeof(R) * (size_t)(C > 1 ? C + 1 : 0) * kThreads;
    off = (off + 15) & ~(size_t)15;
    double *zz = reinterpret_cast<double *>(smem_raw + off) + tid;
    off += P.wf_on ? sizeof(double) * (size_t)(P.S + 1) * kThreads : 0;
    BMTables *bm_smem = reinterpret_cast<BMTables *>(smem_raw + off);   // double path only

    // stage the coefficient tables of every sampled level (and the
    // Box-Muller node tables of the double path)
    {
        const R *g = reinterpret_cast<const R *>(P.tables);
        const int n = P.S * P.M;
        for (int i = tid; i < n; i += kThreads) tab[i] = g[i];
        if constexpr (sizeof(R) == 8) bm_tables_init(bm_smem, tid, kThreads);
    }
    __syncthreads();

    Stream<R> st;
    st.key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    st.inst = P.instance;
    st.bm = sizeof(R) == 8 ? bm_smem : nullptr;

    const int warp = tid >> 5, lane = tid & 31;
    for (int64_t item = blockIdx.x; item < P.n_items; item += gridDim.x) {
        const int64_t b = item / P.items_per_block;
        const int64_t r = item - b * P.items_per_block;
        const int64_t lo = b * P.n_mc / P.n_blocks;
        const int64_t hi = (b + 1) * P.n_mc / P.n_blocks;
        const int64_t start = lo + r * chunk;
        const int cnt = (int)max((int64_t)0, min((int64_t)chunk, hi - start));

        for (int rd = 0; rd < P.rounds; ++rd) {
            const int t = rd * kThreads + tid;
            if (t >= cnt) break;
            const uint64_t sample = (uint64_t)(P.sample0 + start + t);
            st.slo = (uint32_t)sample;
            st.shi = (uint32_t)(sample >> 32);
            double wloc[SU_MAX_S];
            double *wout;
            int wstride;
            if (per_sample) {
                wout = wloc;
                wstride = 1;
            } else {
                wout = sw + t;
                wstride = chunk;
            }
            switch (P.F) {
                case 1: sample_path<R, RING, 1>(P, tab, qc, zz, st, wout, wstride); break;
                case 2: sample_path<R, RING, 2>(P, tab, qc, zz, st, wout, wstride); break;
                case 3: sample_path<R, RING, 3>(P, tab, qc, zz, st, wout, wstride); break;
                case 4: sample_path<R, RING, 4>(P, tab, qc, zz, st, wout, wstride); break;
                default: sample_path<R, RING, 5>(P, tab, qc, zz, st, wout, wstride); break;
            }
            bool bad = false;
            for (int d = 0; d < L; ++d) {
                const double w = wout[d * wstride];
                bad |= isnan(w) || (isinf(w) && w > 0);
            }
            if (bad) atomicOr(P.flags, 1);
            if (per_sample) {
                double *dst = P.w_out + (start + t) * (int64_t)P.S;
                for (int d = 0; d < L; ++d) dst[P.S - d - 1] = wloc[d];
            }
        }
        if (per_sample) continue;

        // log-sum-exp tuple of this item, per level, in a fixed order
        __syncthreads();
        for (int d = warp; d < L; d += kThreads / 32) {
            const double *v = sw + (size_t)d * chunk;
            double m = -INFINITY;
            for (int t = lane; t < cnt; t += 32) m = fmax(m, v[t]);
            m = warp_max(m);
            double s = 0, q = 0;
            if (m > -INFINITY) {
                for (int t = lane; t < cnt; t += 32) {
                    const double e = exp(v[t] - m);
                    s += e;
                    q = fma(e, e, q);
                }
            }
            s = warp_sum(s);
            q = warp_sum(q);
            if (lane == 0) {
                double *o = P.partial + 4 * (item * L + d);
                o[0] = m;
                o[1] = s;
                o[2] = q;
                o[3] = (double)cnt;
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace su
