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
// slices is split into C = 2^(S-F) segments of 2^F slices (F <= min(S, 5),
// the launch shape's segment size):
// the C+1 segment endpoints (bisection levels 1..S-F) are generated first and
// parked in shared memory; each segment's 2^F - 1 interior points (levels
// S-F+1..S) are then generated in registers and all slices of the segment, at
// every level, are evaluated before the next segment starts.  The double path
// keeps the segment's points as scalars; the single path as pairs
// (q_m, q_{m+2^(F-1)}), so that two slices or two midpoints go through one
// packed instruction (level_sum_pairs), and with its table shape compiled in
// where the library has it (fixed_shapes.h).
//
// Normal j of a sample (heap order: level n, midpoint i -> j = 2^(n-1)-1+i).
// Double path: Box-Muller branch (j & 1) of Philox call j >> 1; every call is
// computed once and its second normal carried to the midpoint that uses it,
// except the first midpoint of each in-register level in segment 0, whose
// call is shared with the last midpoint of the previous level (in the last
// segment) and is recomputed there (F-1 extra calls per path when C > 1).
// Single path: slot (j+1) & 3 of call (j+1) >> 2 (four normals per call), so
// that from level 3 on a level's normals start on a call boundary; levels 1
// and 2 of the register segment keep their call across segments.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "boxmuller.cuh"
#include "fixed_shapes.h"
#include "philox.cuh"
#include "generator.h"
#include "sampler.h"

namespace su {
namespace {


// ------------------------------------------------------------ Box-Muller
template <typename R>
struct Normal;

template <>
struct Normal<double> {
    // 53-bit uniforms ((w0 2^21 + w1 >> 11) + 1/2) 2^-53 from (w0,w1) and (w2,w3),
    // through the table-driven routines of boxmuller.cuh
    static __device__ __forceinline__ void pair(uint4 w, const bm::Tables *t, double &z0, double &z1) {
        const uint64_t a = ((uint64_t)w.x << 21) | (w.y >> 11);
        const uint64_t b = ((uint64_t)w.z << 21) | (w.w >> 11);
        bm::rotate(bm::sqrt_pos(bm::minus2log(a, t)), b, t, z0, z1);
    }
};

template <>
struct Normal<float> {
    // four normals per call: (z0, z1) from the 24-bit uniforms
    // ((w >> 8) + 1/2) 2^-24 of (w0, w1), (z2, z3) from (w2, w3), through the
    // single-precision routine of boxmuller.cuh (hardware approximations)
    static __device__ __forceinline__ void quad(uint4 w, float (&z)[4]) {
        bm32::pair(w.x, w.y, z[0], z[1]);
        bm32::pair(w.z, w.w, z[2], z[3]);
    }
};

// Stream layout.  Double path: normal j (heap order of the bisection
// midpoints) is branch j & 1 of call j >> 1.  Single path: with j' = j + 1,
// normal j is slot j' & 3 of call j' >> 2, so that from level 3 on every
// level's normals start on a call boundary.
template <typename R>
struct Stream {
    uint2 key;
    uint32_t inst, slo, shi;
    const bm::Tables *bm;   // shared-memory node tables (double path)
    float4 *zq;             // single path: this thread's column (stride kThreads) of
                            // staged quads, levels 3..F of a segment (see sample_path)
    __device__ __forceinline__ uint4 words(uint32_t call) const {
        return philox4x32_10(make_uint4(call, inst, slo, shi), key);
    }
    __device__ __forceinline__ void pair(uint32_t call, double &z0, double &z1) const {
        Normal<double>::pair(words(call), bm, z0, z1);
    }
    __device__ __forceinline__ void quad(uint32_t call, float (&z)[4]) const {
        Normal<float>::quad(words(call), z);
    }
};

// v[s & 3] for a run-time slot
__device__ __forceinline__ float pick4(const float (&v)[4], uint32_t s) {
    const float lo = (s & 1u) ? v[1] : v[0];
    const float hi = (s & 1u) ? v[3] : v[2];
    return (s & 2u) ? hi : lo;
}

// ------------------------------------------------------------------ W_p
template <typename R, int RING>
__device__ __forceinline__ R ring_var(R us, R alpha) {
    if constexpr (RING == RING_EVEN) {
        return us * us;
    } else if constexpr (RING == RING_X) {
        return us;
    } else {
        // tanh^2(alpha us / 2)
        if constexpr (sizeof(R) == 4) {
            // tanh(h), h = |alpha us| / 2: below h = 1/2 its odd series to
            // h^13 (next term < 1e-7 relative), above (1 - e)/(1 + e) with
            // e = e^(-2h) <= 0.37 from the hardware exp2 (no cancellation)
            const float y = fabsf(alpha * us);
            const float h = 0.5f * y, h2 = h * h;
            float ser = fmaf(h2, 21844.0f / 6081075.0f, -1382.0f / 155925.0f);
            ser = fmaf(h2, ser, 62.0f / 2835.0f);
            ser = fmaf(h2, ser, -17.0f / 315.0f);
            ser = fmaf(h2, ser, 2.0f / 15.0f);
            ser = fmaf(h2, ser, -1.0f / 3.0f);
            ser = fmaf(h2 * h, ser, h);
            float e;
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.44269504f * y));
            const float t = h < 0.5f ? ser : __fdividef(1.0f - e, 1.0f + e);
            return t * t;
        } else {
            // tanh(y/2) = -em / (2 + em), em = expm1(-|y|), accurate also where tanh is small
            const R em = expm1(-fabs(alpha * us));
            const R t = -em / (2.0 + em);
            return t * t;
        }
    }
}

// V_j = V^(j)(x), j = 0..J, of a general potential from its families:
// polynomial table; Gaussians through the Hermite recurrence; sech^2 = tanh'
// through the Taylor coefficients a_k of tanh, (n+1) a_{n+1} = -sum_k a_k a_{n-k}
// from tanh' = 1 - tanh^2, which stay accurate where tanh is near +-1.
__device__ __forceinline__ void general_derivatives(double x, const GeneralDev *__restrict__ G,
                                                    double (&V)[kGenMaxSym]) {
    const int J = G->J;
    for (int j = 0; j <= J; ++j) {
        double v = 0.0;
        if (j <= 8)
            for (int i = 8; i >= j; --i) v = fma(v, x, G->poly_der[j][i]);
        V[j] = v;
    }
    for (int g = 0; g < G->ng; ++g) {
        const double u = x - G->gauss[g][2], sb = G->gauss[g][3];
        const double y = sb * u, e = G->gauss[g][0] * exp(-G->gauss[g][1] * u * u);
        double h0 = 1.0, h1 = 2.0 * y, f = 1.0;
        for (int n = 0; n <= J; ++n) {
            V[n] = fma(f * (n == 0 ? h0 : h1), e, V[n]);
            f *= -sb;
            if (n >= 1) {
                const double h2 = fma(2.0 * y, h1, -2.0 * n * h0);
                h0 = h1;
                h1 = h2;
            }
        }
    }
    for (int q = 0; q < G->ns; ++q) {
        const double w = G->sech[q][1] * (x - G->sech[q][2]);
        const double em = expm1(-2.0 * fabs(w)), e = exp(-2.0 * fabs(w));
        const double den = 2.0 + em;               // 1 + e^{-2|w|}
        double a[kGenMaxSym + 1];
        a[0] = copysign(-em / den, w);             // tanh w
        a[1] = 4.0 * e / (den * den);              // sech^2 w
        V[0] = fma(G->sech_scale[q][0], a[1], V[0]);
        for (int n = 1; n <= J; ++n) {
            double acc = 0.0;
            for (int k = 0; k < (n + 1) / 2; ++k) acc = fma(a[k], a[n - k], acc);
            acc += acc;
            if (!(n & 1)) acc = fma(a[n >> 1], a[n >> 1], acc);
            a[n + 1] = -acc * G->inv[n + 1];
            V[n] = fma(G->sech_scale[q][n], a[n + 1], V[n]);
        }
    }
    for (int q = 0; q < G->ne; ++q) {   // exponentials: (-kappa)^n E e^{-kappa (x - x0)}
        const double kap = G->expo[q][1];
        double e = G->expo[q][0] * exp(-kap * (x - G->expo[q][2]));
        for (int n = 0; n <= J; ++n) {
            V[n] += e;
            e *= -kap;
        }
    }
}

// -eps W_p of B = 1 or 2 slices (ql[b], qr[b]) for a general potential
// (double only).  The monomials of W_p in the V_j form a trie walked depth
// first: each node's monomial is its parent's (the top of a stack of depth
// <= 6 at p = 12) times one V_j, and its entries are the coefficients of
// vs^0, vs^2, .., vs^(2 count - 2), combined by Horner in vs^2 and added
// times the monomial.  Two slices share every node and coefficient load.
template <int B>
__device__ __noinline__ double2 slice_general(double ql0, double qr0, double ql1, double qr1,
                                              const double *__restrict__ coef,
                                              const GeneralDev *__restrict__ G) {
    const double ql[2] = {ql0, ql1}, qr[2] = {qr0, qr1};
    double V[B][kGenMaxSym], Y[B], stk[B][kGenMaxDepth + 1], w[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        general_derivatives(0.5 * (ql[b] + qr[b]), G, V[b]);
        const double vs = qr[b] - ql[b];
        Y[b] = vs * vs;
        stk[b][0] = 1.0;
        w[b] = 0.0;
    }
    const int nn = G->n_nodes;
    for (int t = 0; t < nn; ++t) {
        const GeneralNode nd = G->nodes[t];
        double mu[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            mu[b] = 1.0;
            if (t) {
                mu[b] = stk[b][nd.depth - 1] * V[b][nd.sym];
                stk[b][nd.depth] = mu[b];
            }
        }
        const int cnt = nd.count;
        if (cnt) {
            const double *c = coef + nd.first;
            double h[B];
            const double top = c[cnt - 1];
#pragma unroll
            for (int b = 0; b < B; ++b) h[b] = top;
#pragma unroll 4
            for (int e = cnt - 2; e >= 0; --e) {
                const double ce = c[e];
#pragma unroll
                for (int b = 0; b < B; ++b) h[b] = fma(h[b], Y[b], ce);
            }
#pragma unroll
            for (int b = 0; b < B; ++b) w[b] = fma(h[b], mu[b], w[b]);
        }
    }
    return make_double2(w[0], B > 1 ? w[B - 1] : 0.0);
}

// Entry i of a level table.  Tables hold scalars, or (the single-precision
// sampler) pairs {c, c} that feed the packed two-slice multiply-adds.
__device__ __forceinline__ float coef(const float *t, int i) { return t[i]; }
__device__ __forceinline__ double coef(const double *t, int i) { return t[i]; }
__device__ __forceinline__ float coef(const float2 *t, int i) { return t[i].x; }

// -eps W_p(x, xb; eps) of one slice, from the level's table in shared memory:
// sum_j (vs^2)^j sum_i T_ij Z^i, nested Horner (columns, then powers of vs^2).
template <typename R, int RING, typename TT, typename SP>
__device__ __forceinline__ R slice(R ql, R qr, const TT *__restrict__ tab, const SP &P, R alpha) {
    if constexpr (RING == RING_GENERAL) {
        static_assert(sizeof(R) == 8, "the general potential is evaluated in double");
        return slice_general<1>(ql, qr, ql, qr, tab, P.general).x;
    }
    const R us = ql + qr;
    const R vs = qr - ql;
    const R Y = vs * vs;
    const R Z = ring_var<R, RING>(us, alpha);
    int off = P.M;
    R acc = 0;
    for (int j = P.ncol - 1; j >= 0; --j) {
        const int L = P.len[j];
        off -= L;
        R h = coef(tab, off + L - 1);
#pragma unroll 4
        for (int i = L - 2; i >= 0; --i) h = fma(h, Z, coef(tab, off + i));
        acc = fma(acc, Y, h);
    }
    return acc;
}

// Sum of -eps W_p over NS slices of one level of a segment, the slices taken
// between the points q[k STR] and q[(k+1) STR].  Slices are evaluated in
// batches of B side by side: each table entry is loaded once per batch (a
// broadcast shared-memory read) and feeds B independent multiply-add chains.
//
// Double path (FP64-pipe bound): per slice T_00 + Z H(Z) + Y A(Y, Z), where H
// is column 0 without its constant and A the outer Horner over columns 1..;
// the two products go straight into two running sums and the NS constants
// are added once, one FP64 operation per slice fewer than summing whole
// slice values.  (The single path sums its slices two at a time in
// level_sum_pairs.)
template <typename R>
struct Batch {
    static constexpr int B = 8;
};

// The path code's view of the table shape when it is compiled in (shape K of
// fixed_shapes.h): M and ncol are constants, the column lengths a run-time
// copy for the few places that index them with a run-time column (the
// coarse levels' single slices).  ShapeOf<SP>::value is K, or -1 for the
// run-time shapes of SamplerParams and BatchView.
template <int K>
struct FixedView {
    static constexpr int M = fixed_M(K);
    static constexpr int ncol = fixed_ncol(K);
    int len[fixed_ncol(K)];
    double alpha, lwf, hcoef;
    int wf_on;
    const GeneralDev *general;
};

template <typename SP>
struct ShapeOf {
    static constexpr int value = -1;
};
template <int K>
struct ShapeOf<FixedView<K>> {
    static constexpr int value = K;
};

// Columns J, J-1, .., 0 of the packed nested Horner with shape K compiled
// in: acc <- acc Y + H_j(Z), H_j the column's Horner in Z, the chains
// started as in level_sum (fma(c_top, Z, c_next); a one-entry column goes
// straight into acc).
template <int K, int J, int BP>
__device__ __forceinline__ void fixed_columns(float2 (&acc)[BP], const float2 (&Y)[BP], const float2 (&Z)[BP],
                                              const float2 *__restrict__ tab) {
    if constexpr (J >= 0) {
        constexpr int L = fixed_len(K, J);
        constexpr int off = fixed_off(K, J);
        if constexpr (L == 1) {
            const float2 c = tab[off];
#pragma unroll
            for (int m = 0; m < BP; ++m) acc[m] = __ffma2_rn(acc[m], Y[m], c);
        } else {
            float2 h[BP];
            const float2 c = tab[off + L - 1], c0 = tab[off + L - 2];
#pragma unroll
            for (int m = 0; m < BP; ++m) h[m] = __ffma2_rn(c, Z[m], c0);
#pragma unroll
            for (int i = L - 3; i >= 0; --i) {
                const float2 ci = tab[off + i];
#pragma unroll
                for (int m = 0; m < BP; ++m) h[m] = __ffma2_rn(h[m], Z[m], ci);
            }
#pragma unroll
            for (int m = 0; m < BP; ++m) acc[m] = __ffma2_rn(acc[m], Y[m], h[m]);
        }
        fixed_columns<K, J - 1, BP>(acc, Y, Z, tab);
    }
}

// the whole table: the last column starts the outer Horner in xb^2
template <int K, int BP>
__device__ __forceinline__ void fixed_horner(float2 (&acc)[BP], const float2 (&Y)[BP], const float2 (&Z)[BP],
                                             const float2 *__restrict__ tab) {
    constexpr int J = fixed_ncol(K) - 1;
    constexpr int L = fixed_len(K, J);
    constexpr int off = fixed_off(K, J);
    const float2 c = tab[off + L - 1];
    if constexpr (L == 1) {
#pragma unroll
        for (int m = 0; m < BP; ++m) acc[m] = c;
    } else {
        const float2 c0 = tab[off + L - 2];
#pragma unroll
        for (int m = 0; m < BP; ++m) acc[m] = __ffma2_rn(c, Z[m], c0);
#pragma unroll
        for (int i = L - 3; i >= 0; --i) {
            const float2 ci = tab[off + i];
#pragma unroll
            for (int m = 0; m < BP; ++m) acc[m] = __ffma2_rn(acc[m], Z[m], ci);
        }
    }
    fixed_columns<K, J - 1, BP>(acc, Y, Z, tab);
}

template <typename R, int RING, int NS, int STR, int NQ, typename TT, typename SP>
__device__ __forceinline__ R level_sum(const R (&q)[NQ], const TT *__restrict__ tab, const SP &P, R alpha) {
    if constexpr (RING == RING_GENERAL) {
        R total = 0;
        if constexpr (NS == 1) {
            total = slice_general<1>(q[0], q[STR], q[0], q[STR], tab, P.general).x;
        } else {
#pragma unroll
            for (int k = 0; k < NS; k += 2) {   // unrolled: q stays in registers
                const double2 r = slice_general<2>(q[k * STR], q[(k + 1) * STR], q[(k + 1) * STR],
                                                   q[(k + 2) * STR], tab, P.general);
                total += r.x + r.y;
            }
        }
        return total;
    }
    constexpr int B = NS < Batch<R>::B ? NS : Batch<R>::B;
    constexpr bool kFold = sizeof(R) == 8;
    const int L0 = P.len[0];
    R ty = 0, tz = 0;
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
        const int jlast = kFold ? 1 : 0;          // last column of the outer Horner
        if (P.ncol - 1 >= jlast) {
            if constexpr (sizeof(R) == 4) {
                // single precision (issue bound): the first step of every Horner
                // chain peeled -- the chains start from fma(c_top, z, c_next), a
                // one-entry column goes straight into the outer chain -- so no
                // chain is seeded by register copies; the same operations in the
                // same order.  (In double the copies cost no FP64 issue and the
                // peeled form spills.)
                int off = P.M;
                {   // last column starts the outer Horner in x-bar^2
                    const int L = P.len[P.ncol - 1];
                    off -= L;
                    const R c = coef(tab, off + L - 1);
                    if (L == 1) {
#pragma unroll
                        for (int b = 0; b < B; ++b) acc[b] = c;
                    } else {
                        const R c0 = coef(tab, off + L - 2);
#pragma unroll
                        for (int b = 0; b < B; ++b) acc[b] = fma(c, Z[b], c0);
                    }
#pragma unroll 4
                    for (int i = L - 3; i >= 0; --i) {
                        const R ci = coef(tab, off + i);
#pragma unroll
                        for (int b = 0; b < B; ++b) acc[b] = fma(acc[b], Z[b], ci);
                    }
                }
                for (int j = P.ncol - 2; j >= jlast; --j) {
                    const int L = P.len[j];
                    off -= L;
                    const R c = coef(tab, off + L - 1);
                    if (L == 1) {
#pragma unroll
                        for (int b = 0; b < B; ++b) acc[b] = fma(acc[b], Y[b], c);
                        continue;
                    }
                    R h[B];
                    const R c0 = coef(tab, off + L - 2);
#pragma unroll
                    for (int b = 0; b < B; ++b) h[b] = fma(c, Z[b], c0);
#pragma unroll 4
                    for (int i = L - 3; i >= 0; --i) {
                        const R ci = coef(tab, off + i);
#pragma unroll
                        for (int b = 0; b < B; ++b) h[b] = fma(h[b], Z[b], ci);
                    }
#pragma unroll
                    for (int b = 0; b < B; ++b) acc[b] = fma(acc[b], Y[b], h[b]);
                }
            } else {
                int off = P.M;
                {   // last column starts the outer Horner in x-bar^2
                    const int L = P.len[P.ncol - 1];
                    off -= L;
                    const R c = coef(tab, off + L - 1);
#pragma unroll
                    for (int b = 0; b < B; ++b) acc[b] = c;
#pragma unroll 4
                    for (int i = L - 2; i >= 0; --i) {
                        const R ci = coef(tab, off + i);
#pragma unroll
                        for (int b = 0; b < B; ++b) acc[b] = fma(acc[b], Z[b], ci);
                    }
                }
                for (int j = P.ncol - 2; j >= jlast; --j) {
                    const int L = P.len[j];
                    off -= L;
                    R h[B];
                    const R c = coef(tab, off + L - 1);
#pragma unroll
                    for (int b = 0; b < B; ++b) h[b] = c;
#pragma unroll 4
                    for (int i = L - 2; i >= 0; --i) {
                        const R ci = coef(tab, off + i);
#pragma unroll
                        for (int b = 0; b < B; ++b) h[b] = fma(h[b], Z[b], ci);
                    }
#pragma unroll
                    for (int b = 0; b < B; ++b) acc[b] = fma(acc[b], Y[b], h[b]);
                }
            }
            if constexpr (kFold) {
#pragma unroll
                for (int b = 0; b < B; ++b) ty = fma(acc[b], Y[b], ty);
            } else {
#pragma unroll
                for (int b = 0; b < B; ++b) ty += acc[b];
            }
        }
        if constexpr (kFold) {
            if (L0 > 1) {
                R h[B];
                const R c = coef(tab, L0 - 1);
#pragma unroll
                for (int b = 0; b < B; ++b) h[b] = c;
#pragma unroll 4
                for (int i = L0 - 2; i >= 1; --i) {
                    const R ci = coef(tab, i);
#pragma unroll
                    for (int b = 0; b < B; ++b) h[b] = fma(h[b], Z[b], ci);
                }
#pragma unroll
                for (int b = 0; b < B; ++b) tz = fma(h[b], Z[b], tz);
            }
        }
    }
    if constexpr (kFold) return fma((R)NS, coef(tab, 0), ty + tz);
    return ty;
}

// The packed nested Horner of BP pairs of slices: acc = sum_j (xb^2)^j sum_i
// T_ij z^i for both slices of each pair (fma.rn.f32x2 on tables of pairs
// {c, c}), the chains started from fma(c_top, Z, c_next) and a one-entry
// column going straight into the outer chain; with the table shape compiled
// in (ShapeOf<SP>) every loop unrolled (fixed_horner), the same operations
// in the same order.
template <int BP, typename SP>
__device__ __forceinline__ void horner_packed(float2 (&acc)[BP], const float2 (&Y)[BP], const float2 (&Z)[BP],
                                              const float2 *__restrict__ tab, const SP &P) {
    if constexpr (ShapeOf<SP>::value >= 0) {
        fixed_horner<ShapeOf<SP>::value, BP>(acc, Y, Z, tab);
    } else {
        int off = P.M;
        {   // last column starts the outer Horner in x-bar^2
            const int L = P.len[P.ncol - 1];
            off -= L;
            const float2 c = tab[off + L - 1];
            if (L == 1) {
#pragma unroll
                for (int m = 0; m < BP; ++m) acc[m] = c;
            } else {
                const float2 c0 = tab[off + L - 2];
#pragma unroll
                for (int m = 0; m < BP; ++m) acc[m] = __ffma2_rn(c, Z[m], c0);
            }
#pragma unroll 4
            for (int i = L - 3; i >= 0; --i) {
                const float2 ci = tab[off + i];
#pragma unroll
                for (int m = 0; m < BP; ++m) acc[m] = __ffma2_rn(acc[m], Z[m], ci);
            }
        }
        for (int j = P.ncol - 2; j >= 0; --j) {
            const int L = P.len[j];
            off -= L;
            const float2 c = tab[off + L - 1];
            if (L == 1) {
#pragma unroll
                for (int m = 0; m < BP; ++m) acc[m] = __ffma2_rn(acc[m], Y[m], c);
                continue;
            }
            float2 h[BP];
            const float2 c0 = tab[off + L - 2];
#pragma unroll
            for (int m = 0; m < BP; ++m) h[m] = __ffma2_rn(c, Z[m], c0);
#pragma unroll 4
            for (int i = L - 3; i >= 0; --i) {
                const float2 ci = tab[off + i];
#pragma unroll
                for (int m = 0; m < BP; ++m) h[m] = __ffma2_rn(h[m], Z[m], ci);
            }
#pragma unroll
            for (int m = 0; m < BP; ++m) acc[m] = __ffma2_rn(acc[m], Y[m], h[m]);
        }
    }
}

// Single precision: a segment's points as pairs Pq[m] = (q_m, q_{m+H}),
// m = 0..H, H = 2^(F-1) (q_H in both Pq[0].y and Pq[H].x).  A level of NS >= 2
// slices of the segment (stride STR = 2^F / NS) pairs slice k with slice
// k + NS/2: both lie between Pq[k STR] and Pq[(k+1) STR], so the packed
// two-slice Horner takes them without moves.  The sum runs over the pairs in
// order, each pair's two slices in turn.  NS = 1: the one slice (q_0, q_2H).
template <int RING, int NS, int STR, int H, typename TT, typename SP>
__device__ __forceinline__ float level_sum_pairs(const float2 (&Pq)[H + 1], const TT *__restrict__ tab, const SP &P,
                                                 float alpha) {
    if constexpr (NS == 1) {
        return slice<float, RING>(Pq[0].x, Pq[H].y, tab, P, alpha);
    } else {
        constexpr int NP = NS / 2;                 // pairs of slices
        constexpr int BP = NP < 4 ? NP : 4;        // pairs per batch: each table entry feeds 2 BP slices
        const float2 m1 = make_float2(-1.0f, -1.0f);
        float ty = 0;
#pragma unroll
        for (int k0 = 0; k0 < NP; k0 += BP) {
            float2 Z[BP], Y[BP], acc[BP];
#pragma unroll
            for (int m = 0; m < BP; ++m) {
                const float2 ql = Pq[(k0 + m) * STR], qr = Pq[(k0 + m + 1) * STR];
                const float2 vs = __ffma2_rn(ql, m1, qr);     // qr - ql, exactly as a subtraction
                Y[m] = __fmul2_rn(vs, vs);
                const float2 us = __fadd2_rn(ql, qr);
                if constexpr (RING == RING_EVEN) {
                    Z[m] = __fmul2_rn(us, us);
                } else {
                    Z[m] = make_float2(ring_var<float, RING>(us.x, alpha), ring_var<float, RING>(us.y, alpha));
                }
            }
            horner_packed<BP>(acc, Y, Z, tab, P);
#pragma unroll
            for (int m = 0; m < BP; ++m) {
                ty += acc[m].x;
                ty += acc[m].y;
            }
        }
        return ty;
    }
}

// levels d = D..F of a single-precision segment held as pairs
template <int RING, int F, int D, typename TT, typename SP>
__device__ __forceinline__ void segment_levels_pairs(float (&acc)[F + 1], const float2 (&Pq)[(1 << (F - 1)) + 1],
                                                     const TT *__restrict__ tab, const SP &P, float alpha, int S) {
    if constexpr (D <= F) {
        if (D < S) {
            acc[D] += level_sum_pairs<RING, ((1 << F) >> D), (1 << D), (1 << (F - 1))>(Pq, tab + D * P.M, P, alpha);
            segment_levels_pairs<RING, F, D + 1>(acc, Pq, tab, P, alpha, S);
        }
    }
}

// levels d = D..F of a segment (level n = S - d uses every 2^d-th point)
template <typename R, int RING, int F, int D, typename TT, typename SP>
__device__ __forceinline__ void segment_levels(R (&acc)[F + 1], const R (&q)[(1 << F) + 1],
                                               const TT *__restrict__ tab, const SP &P, R alpha, int S) {
    if constexpr (D <= F) {
        if (D < S) {
            acc[D] += level_sum<R, RING, ((1 << F) >> D), (1 << D)>(q, tab + D * P.M, P, alpha);
            segment_levels<R, RING, F, D + 1>(acc, q, tab, P, alpha, S);
        }
    }
}

// (l + r)/2 for the bisection midpoint.  Double path: the halving on the
// exponent bits (an FP64 multiply costs as much as a multiply-add on this
// part); sums below 2^-1021 in magnitude become zero, infinities and NaNs
// pass through.
__device__ __forceinline__ double mid(double l, double r) {
    const long long u = __double_as_longlong(l + r);
    const int E = (int)((u >> 52) & 0x7FF);
    const long long h = E >= 2 ? (E == 0x7FF ? u : u - (1LL << 52)) : (u & (long long)0x8000000000000000ULL);
    return __longlong_as_double(h);
}
__device__ __forceinline__ float mid(float l, float r) { return 0.5f * (l + r); }

// --------------------------------------------------------------- a path
// Per-path configuration: endpoints, depth, sampled levels and the bisection
// widths sigma[n], n = 1..S, in the kernel's precision (shared memory).
template <typename R>
struct PathCfg {
    R a, b;
    int S;
    int levels;
    const R *sigma;
};

// The single path stages a segment's normals of levels 3..F in shared memory
// (Stream::zq) from one rolled loop before its bisection, in the order its
// paired bisection takes them: the same normals, but few copies of the Philox
// and Box-Muller code in the segment loop instead of one per quad, which keeps
// that loop inside the instruction cache.

// quads staged per thread for 2^F-slice segments: levels 3..F, or 4..F where
// level 3's one quad stays in registers (Z3REG: the batched kernel, for which
// the 2 KB per CTA decide its residency; in the sampler the registers are
// the tighter budget)
__host__ __device__ constexpr int staged_quads(int F, bool z3reg = false) {
    return z3reg ? (F >= 4 ? (1 << (F - 2)) - 2 : 0) : (F >= 3 ? (1 << (F - 2)) - 1 : 0);
}

// This thread's shared-memory columns (stride kThreads): qc holds the C+1
// segment endpoints, zz the per-level sums of z^2 (width-factor weight only).
// Writes the log-weight of sampled level d (level n = S - d) to wout[d * wstride].
template <typename R, int RING, int F, bool WF, bool Z3REG = false, typename TT, typename SP>
__device__ __forceinline__ void sample_path(const SP &P, const PathCfg<R> &pc,
                                            const TT *__restrict__ tab, R *__restrict__ qc,
                                            double *__restrict__ zz, const Stream<R> &st,
                                            R *__restrict__ wout, int wstride, float *qout = nullptr) {
    constexpr int NF = 1 << F;
    const int S = pc.S;
    const int C = 1 << (S - F);
    const bool hier = pc.levels > 1;
    const int M = P.M;
    const R alpha = (R)P.alpha;

    if constexpr (WF)
        for (int n = 0; n <= S; ++n) zz[n * kThreads] = 0.0;

    R cz[F + 1];
#pragma unroll
    for (int l = 0; l <= F; ++l) cz[l] = 0;

    // single path: the quads of levels 1 and 2, which span several segments
    // (or, with one segment, both levels)
    float Q1[4] = {0.f, 0.f, 0.f, 0.f}, Q2[4] = {0.f, 0.f, 0.f, 0.f};

    // ---- segment endpoints: bisection levels 1..S-F, heap order j = 0..C-2
    if (C > 1) {
        qc[0] = pc.a;
        qc[C * kThreads] = pc.b;
        R carry = 0;
        uint32_t j = 0;
        for (int n = 1; n <= S - F; ++n) {
            const int hc = C >> n;
            const R sg = pc.sigma[n];
            for (int i = 0; i < (1 << (n - 1)); ++i, ++j) {
                R z;
                if constexpr (sizeof(R) == 8) {
                    if ((j & 1u) == 0) {
                        R z0, z1;
                        st.pair(j >> 1, z0, z1);
                        z = z0;
                        carry = z1;
                    } else {
                        z = carry;
                    }
                } else {
                    const uint32_t jp = j + 1;
                    if (j == 0 || (jp & 3u) == 0) st.quad(jp >> 2, Q1);
                    z = pick4(Q1, jp);
                }
                if constexpr (WF) zz[n * kThreads] += (double)z * (double)z;
                const int idx = (2 * i + 1) * hc;
                qc[idx * kThreads] = fma(sg, z, mid(qc[(idx - hc) * kThreads], qc[(idx + hc) * kThreads]));
            }
        }
        cz[0] = carry;
    }

    // ---- segments: levels S-F+1..S in registers, all slices evaluated
    R acc[F + 1];
#pragma unroll
    for (int d = 0; d <= F; ++d) acc[d] = 0;

    for (int c = 0; c < C; ++c) {
        if constexpr (sizeof(R) == 4) {
            // ---- single precision: the segment as pairs Pq[m] = (q_m, q_{m+H})
            constexpr int H = NF / 2;
            float4 z3 = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (F >= 3) {
                // the normals of levels 3..F (level l: quads from
                // (2^(n-1) + c 2^(l-1)) / 4 on, normal il at slot il & 3 of quad
                // il / 4) in the order the paired bisection takes them: pair il
                // of level l is (z_il, z_{il + 2^(l-2)}); level 3's quad in
                // registers, levels 4..F staged, float4 slot 2^(l-3) - 2 + il / 2
                // holding pairs il (even) and il + 1 (2^(l-3) - 1 + il / 2 with
                // level 3 staged too)
                {   // level 3: one quad, pairs (z0, z2), (z1, z3)
                    const int n = S - F + 3;
                    float za[4];
                    st.quad(((1u << (n - 1)) + ((uint32_t)c << 2)) >> 2, za);
                    z3 = make_float4(za[0], za[2], za[1], za[3]);
                    if constexpr (!Z3REG) st.zq[0] = z3;
                }
#pragma unroll 1
                for (int l = 4; l <= F; ++l) {   // levels 4..F: quad k pairs with quad k + 2^(l-4)
                    const int n = S - F + l;
                    const uint32_t q0 = ((1u << (n - 1)) + ((uint32_t)c << (l - 1))) >> 2;
                    const int hq = 1 << (l - 4), base = (1 << (l - 3)) - (Z3REG ? 2 : 1);
#pragma unroll 1
                    for (int k = 0; k < hq; ++k) {
                        float za[4], zb[4];
                        st.quad(q0 + (uint32_t)k, za);
                        st.quad(q0 + (uint32_t)(k + hq), zb);
                        st.zq[(base + 2 * k) * kThreads] = make_float4(za[0], zb[0], za[1], zb[1]);
                        st.zq[(base + 2 * k + 1) * kThreads] = make_float4(za[2], zb[2], za[3], zb[3]);
                    }
                }
            }
            float2 Pq[H + 1];
            const R qa = C > 1 ? qc[c * kThreads] : pc.a;
            const R qb = C > 1 ? qc[(c + 1) * kThreads] : pc.b;
            {   // level 1: the midpoint q_H (normal j' = 2^(n-1) + c)
                const int n = S - F + 1;
                const uint32_t jp = (1u << (n - 1)) + (uint32_t)c;
                R z;
                if (C == 1) {
                    st.quad(0, Q1);
                    z = Q1[1];
                } else if (C == 2) {            // the endpoint levels' quad
                    z = c ? Q1[3] : Q1[2];
                } else {                        // a quad per four segments
                    if ((c & 3) == 0) st.quad(jp >> 2, Q1);
                    z = pick4(Q1, (uint32_t)c);
                }
                if constexpr (WF) zz[n * kThreads] += (double)z * (double)z;
                const R qm = fma(pc.sigma[n], z, mid(qa, qb));
                Pq[0] = make_float2(qa, qm);
                Pq[H] = make_float2(qm, qb);
            }
            // levels 2..F: midpoints idx and idx + H together, pair il < 2^(l-2)
#pragma unroll
            for (int l = 2; l <= F; ++l) {
                const int n = S - F + l;
                const R sg = pc.sigma[n];
                const float2 sg2 = make_float2(sg, sg), half2 = make_float2(0.5f, 0.5f);
                const int h = 1 << (F - l);
                float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int il = 0; il < (1 << (l - 2)); ++il) {
                    float2 zp;
                    if (l == 2) {                   // normals j' = 2^(n-1) + 2c + {0, 1}
                        if (C == 1) {               // j' = 2, 3: the quad of level 1
                            zp = make_float2(Q1[2], Q1[3]);
                        } else {                    // a quad per two segments
                            if ((c & 1) == 0) st.quad(((1u << (n - 1)) + 2u * (uint32_t)c) >> 2, Q2);
                            zp = (c & 1) ? make_float2(Q2[2], Q2[3]) : make_float2(Q2[0], Q2[1]);
                        }
                    } else {
                        if (Z3REG && l == 3)
                            v4 = z3;
                        else if ((il & 1) == 0)
                            v4 = st.zq[((1 << (l - 3)) - (Z3REG ? 2 : 1) + (il >> 1)) * kThreads];
                        zp = (il & 1) ? make_float2(v4.z, v4.w) : make_float2(v4.x, v4.y);
                    }
                    if constexpr (WF) {
                        zz[n * kThreads] += (double)zp.x * (double)zp.x;
                        zz[n * kThreads] += (double)zp.y * (double)zp.y;
                    }
                    const int idx = (2 * il + 1) * h;
                    // (0.5 (l + r), for both) then the widths: the scalar mid() and fma
                    Pq[idx] = __ffma2_rn(sg2, zp, __fmul2_rn(half2, __fadd2_rn(Pq[idx - h], Pq[idx + h])));
                }
            }
            if (qout) {   // path output (per-sample mode)
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    qout[c * NF + k] = Pq[k].x;
                    qout[c * NF + H + k] = Pq[k].y;
                }
                if (c == C - 1) qout[C * NF] = Pq[H].y;
            }
            // top level: every slice of the segment; then the coarser levels
            acc[0] += level_sum_pairs<RING, NF, 1, H>(Pq, tab, P, alpha);
            if (hier) segment_levels_pairs<RING, F, 1>(acc, Pq, tab, P, alpha, S);
        } else {
            // ---- double precision: the segment's points in registers
            R q[NF + 1];
            q[0] = C > 1 ? qc[c * kThreads] : pc.a;
            q[NF] = C > 1 ? qc[(c + 1) * kThreads] : pc.b;
#pragma unroll
            for (int l = 1; l <= F; ++l) {
                const int n = S - F + l;
                const uint32_t jbase = (1u << (n - 1)) - 1u + ((uint32_t)c << (l - 1));
                const R sg = pc.sigma[n];
                const int h = 1 << (F - l);
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
                    if constexpr (WF) zz[n * kThreads] += (double)z * (double)z;
                    const int idx = (2 * il + 1) * h;
                    q[idx] = fma(sg, z, mid(q[idx - h], q[idx + h]));
                }
            }
            // top level: every slice of the segment; then the coarser levels
            acc[0] += level_sum<R, RING, NF, 1>(q, tab, P, alpha);
            if (hier) segment_levels<R, RING, F, 1>(acc, q, tab, P, alpha, S);
        }
    }

    // ---- width-factor weight, cumulative over levels 1..n (stored in zz)
    if constexpr (WF) {
        double cum = 0;
        for (int n = 1; n <= S; ++n) {
            cum += (double)(1 << (n - 1)) * P.lwf + P.hcoef * zz[n * kThreads];
            zz[n * kThreads] = cum;
        }
    }
    auto out = [&](int d, R v) {
        if constexpr (WF)
            wout[d * wstride] = (R)((double)v + zz[(S - d) * kThreads]);
        else
            wout[d * wstride] = v;
    };

    // ---- outputs, level n = S - d
#pragma unroll
    for (int d = 0; d <= F; ++d)
        if (d == 0 || (hier && d < S)) out(d, acc[d]);
    if (hier) {
        for (int n = 1; n < S - F; ++n) {
            const int d = S - n;
            const int stp = C >> n;
            R sum = 0;
            for (int k = 0; k < (1 << n); ++k)
                sum += slice<R, RING>(qc[k * stp * kThreads], qc[(k + 1) * stp * kThreads], tab + d * M,
                                      P, alpha);
            out(d, sum);
        }
    }
}

// The width-factor weight is a template switch: as a run-time test inside
// the midpoint loop the compiler predicates it, and its double conversions
// and multiply-add then occupy the FP64 pipe on every midpoint.
template <typename R, int RING, bool WF, bool Z3REG = false, typename TT, typename SP>
__device__ __forceinline__ void sample_path_f(int F, const SP &P, const PathCfg<R> &pc,
                                              const TT *tab, R *qc, double *zz, const Stream<R> &st,
                                              R *wout, int wstride, float *qout) {
    switch (F) {
        case 1: sample_path<R, RING, 1, WF, Z3REG>(P, pc, tab, qc, zz, st, wout, wstride, qout); break;
        case 2: sample_path<R, RING, 2, WF, Z3REG>(P, pc, tab, qc, zz, st, wout, wstride, qout); break;
        case 3: sample_path<R, RING, 3, WF, Z3REG>(P, pc, tab, qc, zz, st, wout, wstride, qout); break;
        case 4: sample_path<R, RING, 4, WF, Z3REG>(P, pc, tab, qc, zz, st, wout, wstride, qout); break;
        default: sample_path<R, RING, 5, WF, Z3REG>(P, pc, tab, qc, zz, st, wout, wstride, qout); break;
    }
}

template <typename R, int RING, typename TT, typename SP>
__device__ __forceinline__ void sample_path_any(int F, const SP &P, const PathCfg<R> &pc,
                                                const TT *tab, R *qc, double *zz, const Stream<R> &st,
                                                R *wout, int wstride, float *qout = nullptr) {
    if (P.wf_on)
        sample_path_f<R, RING, true>(F, P, pc, tab, qc, zz, st, wout, wstride, qout);
    else
        sample_path_f<R, RING, false>(F, P, pc, tab, qc, zz, st, wout, wstride, qout);
}

// batched kernel: no width factor; the per-item view of the instance's
// table shape (BatchView, in shared memory) in place of SamplerParams; level
// 3's normals in registers
template <typename R, int RING, typename TT, typename SP>
__device__ __forceinline__ void sample_path_plain(int F, const SP &P, const PathCfg<R> &pc, const TT *tab, R *qc,
                                                  const Stream<R> &st, R *wout) {
    sample_path_f<R, RING, false, true>(F, P, pc, tab, qc, nullptr, st, wout, 1, nullptr);
}

// -------------------------------------------------------- warp helpers
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// e^x for x <= 0 in the reduction: double on the double path; on the single
// path the exponential is taken in float (its weights carry single-precision
// error already) and only the sums are kept in double
__device__ __forceinline__ double lse_exp(double x) { return exp(x); }
__device__ __forceinline__ double lse_exp(float x) { return (double)__expf(x); }

// running log-sum-exp tuple (M, S = sum e^{w-M}, Q = sum e^{2(w-M)}) of one
// thread: add the weight w
template <typename R>
__device__ __forceinline__ void lse_push(R &m, double &s, double &q, R w) {
    if (!(w > (R)-INFINITY)) return;          // zero weight
    if (w > m) {
        const double f = lse_exp((R)(m - w)); // 0 for the first weight
        s = fma(s, f, 1.0);
        q = fma(q, f * f, 1.0);
        m = w;
    } else {
        const double e = lse_exp((R)(w - m));
        s += e;
        q = fma(e, e, q);
    }
}

template <typename R>
struct Lse {
    R m = -INFINITY;
    double s = 0, q = 0;
    __device__ __forceinline__ void push(R w) { lse_push(m, s, q, w); }
};

// merge tuple b into tuple a (same convention) with the scale factor
// e^(m_a - m_b) in the kernel's precision (lse_exp): the sums stay in
// double; in single precision the
// factor carries float rounding like every per-sample term already does,
// and the batched kernel's CTA merges (a 32-lane butterfly per level and
// work item) stay off the FP64 pipe
template <typename R>
__device__ __forceinline__ void lse_merge_r(double &ma, double &sa, double &qa, double mb, double sb, double qb) {
    if (!(mb > -INFINITY)) return;
    if (mb > ma) {
        const double f = lse_exp((R)(ma - mb));   // 0 for ma = -inf
        sa = fma(sa, f, sb);
        qa = fma(qa, f * f, qb);
        ma = mb;
    } else {
        const double f = lse_exp((R)(mb - ma));
        sa = fma(sb, f, sa);
        qa = fma(qb, f * f, qa);
    }
}

// The log-sum-exp tuple (M, sum e^{w-M}, sum e^{2(w-M)}, n) of one item's
// cnt weights per level (sw[level][chunk]), one warp per level, written to
// partial[4 (item L + level)]; a fixed order, so a rerun gives the same bits.
template <typename R>
__device__ __forceinline__ void item_lse(const R *sw, int L, int chunk, int cnt, double *partial, int64_t item,
                                         int warp, int lane) {
    for (int d = warp; d < L; d += kThreads / 32) {
        const R *v = sw + (size_t)d * chunk;
        R m = (R)-INFINITY;
        for (int t = lane; t < cnt; t += 32) m = fmax(m, v[t]);
        m = warp_max(m);
        double s = 0, q = 0;
        if (m > (R)-INFINITY) {
            for (int t = lane; t < cnt; t += 32) {
                const double e = lse_exp((R)(v[t] - m));
                s += e;
                q = fma(e, e, q);
            }
        }
        s = warp_sum(s);
        q = warp_sum(q);
        if (lane == 0) {
            double *o = partial + 4 * (item * L + d);
            o[0] = (double)m;
            o[1] = s;
            o[2] = q;
            o[3] = (double)cnt;
        }
    }
}

// ----------------------------------------------------------- the kernel
// Shared memory: sw[levels][chunk] (R) | tables[levels][M] (R) | sigma[S+1] (R) |
//                qc[(C+1)][kThreads] (R) | zz[S+1][kThreads] (double, if wf_on) |
//                staged quads[2^(F-2) - 1][kThreads] (float4, single path) |
//                Box-Muller node tables (double path)
// CTAs per SM the register allocation is sized for: two for the double path
// (up to 255 registers: its segment, accumulators and Box-Muller state stay
// in registers; three CTAs at 168 registers spill and run slower), four for
// the single path (128 registers), three for single-path kernels with a
// compiled table shape of more than 30 entries (p >= 14), whose unrolled
// Horner spills at 128 registers (p = 18: 62.5 -> 57.6 ms at three)
template <typename R, int RING = RING_EVEN, int KS = -1>
struct MinCtas {
    static constexpr int value = sizeof(R) == 8 ? 2 : ((KS >= 0 && fixed_M(KS >= 0 ? KS : 0) > 30) ? 3 : 4);
};
// the general-potential evaluator keeps its derivatives and monomial stacks in
// local memory: more warps to hide their latency, shorter register segments
template <int KS>
struct MinCtas<double, RING_GENERAL, KS> {
    static constexpr int value = 4;
};

// KS >= 0: the single-precision sampler with table shape KS of
// fixed_shapes.h compiled in, for plans with 2^kMaxFine-slice segments and
// no width-factor weight (the host picks it only then).
template <typename R, int RING, bool GTAB = false, int KS = -1>
__global__ void __launch_bounds__(kThreads, MinCtas<R, RING, KS>::value) sampler_kernel(const __grid_constant__ SamplerParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int L = P.levels;
    const int chunk = kThreads * P.rounds;
    const bool per_sample = P.w_out != nullptr;
    const int C = 1 << (P.S - P.F);

    R *sw = reinterpret_cast<R *>(smem_raw);
    size_t off = per_sample ? 0 : sizeof(R) * (size_t)L * chunk;
    off = (off + 15) & ~(size_t)15;
    // the general program's level tables (thousands of entries per level),
    // and any tables too large to stage (levels p >~ 100), stay in global
    // memory: every lane reads the same entry, one broadcast load through L1
    constexpr bool kStage = RING != RING_GENERAL && !GTAB;
    // single precision stages every entry as a pair {c, c} for the packed
    // two-slice multiply-adds of level_sum
    using TT = typename std::conditional<sizeof(R) == 4, float2, R>::type;
    TT *tab_s = reinterpret_cast<TT *>(smem_raw + off);
    const TT *tab = kStage ? tab_s : reinterpret_cast<const TT *>(P.tables);
    off += kStage ? sizeof(TT) * (size_t)P.S * P.M : 0;
    R *sig = reinterpret_cast<R *>(smem_raw + off);
    off += sizeof(R) * (size_t)(SU_MAX_S + 1);
    off = (off + 15) & ~(size_t)15;
    R *qc = reinterpret_cast<R *>(smem_raw + off) + tid;
    off += sizeof(R) * (size_t)(C > 1 ? C + 1 : 0) * kThreads;
    off = (off + 15) & ~(size_t)15;
    double *zz = reinterpret_cast<double *>(smem_raw + off) + tid;
    off += P.wf_on ? sizeof(double) * (size_t)(P.S + 1) * kThreads : 0;
    off = (off + 15) & ~(size_t)15;
    float4 *zq = reinterpret_cast<float4 *>(smem_raw + off) + tid;           // single path only
    off += sizeof(R) == 4 ? sizeof(float4) * (size_t)staged_quads(P.F) * kThreads : 0;
    bm::Tables *bm_smem = reinterpret_cast<bm::Tables *>(smem_raw + off);   // double path only

    // stage the coefficient tables of every sampled level, the widths (and
    // the Box-Muller node tables of the double path)
    {
        const R *g = reinterpret_cast<const R *>(P.tables);
        const int n = kStage ? P.S * P.M : 0;
        for (int i = tid; i < n; i += kThreads) {
            if constexpr (sizeof(R) == 4)
                tab_s[i] = make_float2(g[i], g[i]);
            else
                tab_s[i] = g[i];
        }
        for (int i = tid; i <= SU_MAX_S; i += kThreads) sig[i] = (R)P.sigma[i];
        if constexpr (sizeof(R) == 8) bm::tables_init(bm_smem, tid, kThreads);
    }
    __syncthreads();
    const PathCfg<R> pc{(R)P.a, (R)P.b, P.S, L, sig};

    Stream<R> st;
    st.key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    st.inst = P.instance;
    st.bm = sizeof(R) == 8 ? bm_smem : nullptr;
    st.zq = zq;

    FixedView<(KS >= 0 ? KS : 0)> fv;
    if constexpr (KS >= 0) {
        static_assert(sizeof(R) == 4 && RING == RING_EVEN, "compiled shapes: single precision, even ring");
        for (int j = 0; j < fixed_ncol(KS); ++j) fv.len[j] = P.len[j];
        fv.alpha = P.alpha;
        fv.lwf = P.lwf;
        fv.hcoef = P.hcoef;
        fv.wf_on = 0;
        fv.general = nullptr;
    }

    const int warp = tid >> 5, lane = tid & 31;
    for (int64_t item = P.item0 + blockIdx.x; item < P.n_items; item += gridDim.x) {
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
            R wloc[SU_MAX_S];
            R *wout = per_sample ? wloc : sw + t;
            const int wstride = per_sample ? 1 : chunk;
            float *qout = (per_sample && P.q_out) ? P.q_out + (start + t) * (int64_t)((1 << P.S) + 1) : nullptr;
            if constexpr (KS >= 0)
                sample_path<R, RING, kMaxFine, false>(fv, pc, tab, qc, zz, st, wout, wstride, qout);
            else
                sample_path_any<R, RING>(P.F, P, pc, tab, qc, zz, st, wout, wstride, qout);
            bool bad = false;
            for (int d = 0; d < L; ++d) {
                const R w = wout[d * wstride];
                bad |= isnan(w) || (isinf(w) && w > 0);
            }
            if (bad) atomicOr(P.flags, 1);
            if (per_sample) {
                double *dst = P.w_out + (start + t) * (int64_t)P.S;
                for (int d = 0; d < L; ++d) dst[P.S - d - 1] = (double)wloc[d];
            }
        }
        if (per_sample) continue;

        // log-sum-exp tuple of this item, per level, in a fixed order
        __syncthreads();
        item_lse<R>(sw, L, chunk, cnt, P.partial, item, warp, lane);
        __syncthreads();
    }
}

// ---------------------------------------------------- the batched kernel
// Many instances (a_i, b_i, T_i, s_i, p_i, n_i) of one model in one
// persistent launch: CTAs take work items (instance, block, chunk) from an
// atomic queue ordered costliest first; each item's samples are reduced per
// thread (online log-sum-exp, one tuple per sampled level) and then across
// the CTA in a fixed order, so the tuples do not depend on which CTA took
// which item.  An instance samples its top level only, or (hierarchy) every
// level n = 1..s_i from the same paths.
// Shared memory: BatchView | tables[L_max * M_max] (R) | sigma[S_max+1] (R) |
//                qc[(C_max+1)][kThreads] (R) | level states m (R), s, q
//                (double) [L_max-1][kThreads] | staged quads[2^(kMaxFine-2) - 2]
//                [kThreads] (float4, single path) | Box-Muller node tables (double path)
// CTAs per SM for the register budget: the generic float form runs the
// amplitude matrix 2 % faster at 5 (96 registers) than at 4; with a table
// shape compiled in (KS >= 0) it spills more at 96 registers and runs the
// matrix 5 % faster at 4 (128 registers).
template <typename R, int RING, int KS>
struct BatchCtas {
    static constexpr int value = sizeof(R) == 8 ? 2 : (KS >= 0 ? 4 : 5);
};
// the general potential: as the sampler (local-memory stacks, more warps)
template <int KS>
struct BatchCtas<double, RING_GENERAL, KS> {
    static constexpr int value = 4;
};

// The table shape of the current item's instance (its level p), staged in
// shared memory; the path code reads it where the single-instance sampler
// reads SamplerParams.
struct BatchView {
    int ncol, M;
    double alpha, lwf, hcoef;
    int wf_on;
    const GeneralDev *general;
    int len[SU_MAX_P];
};

// KS >= 0: every item's instance has table shape KS of fixed_shapes.h
// (single precision, even ring; shapes[B.fixed_src]); items with
// 2^kMaxFine-slice segments run the path code with that shape compiled in.
template <typename R, int RING, int KS = -1>
__global__ void __launch_bounds__(kThreads, BatchCtas<R, RING, KS>::value) batch_kernel(const __grid_constant__ BatchParams B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ double s_red[kThreads / 32][SU_MAX_S][3];
    const SamplerParams &P = B.base;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    BatchView *view = reinterpret_cast<BatchView *>(smem_raw);
    size_t off = (sizeof(BatchView) + 15) & ~(size_t)15;
    // single precision stages the entries as pairs {c, c} (packed Horner);
    // the general potential's program entries stay in global memory
    using TT = typename std::conditional<sizeof(R) == 4, float2, R>::type;
    constexpr bool kStage = RING != RING_GENERAL;
    TT *tab_s = reinterpret_cast<TT *>(smem_raw + off);
    off += kStage ? sizeof(TT) * (size_t)B.tab_max : 0;
    R *sig = reinterpret_cast<R *>(smem_raw + off);
    off += sizeof(R) * (size_t)(SU_MAX_S + 1);
    off = (off + 15) & ~(size_t)15;
    R *qc = reinterpret_cast<R *>(smem_raw + off) + tid;
    off += sizeof(R) * (size_t)(B.C_max > 1 ? B.C_max + 1 : 0) * kThreads;
    off = (off + 15) & ~(size_t)15;
    double *ls = reinterpret_cast<double *>(smem_raw + off);          // [L_max-1][kThreads]
    off += sizeof(double) * (size_t)(B.L_max - 1) * kThreads;
    double *lq = reinterpret_cast<double *>(smem_raw + off);
    off += sizeof(double) * (size_t)(B.L_max - 1) * kThreads;
    R *lm = reinterpret_cast<R *>(smem_raw + off);
    off += sizeof(R) * (size_t)(B.L_max - 1) * kThreads;
    off = (off + 15) & ~(size_t)15;
    float4 *zq = reinterpret_cast<float4 *>(smem_raw + off) + tid;           // single path only
    off += sizeof(R) == 4 ? sizeof(float4) * (size_t)staged_quads(kMaxFine, true) * kThreads : 0;
    bm::Tables *bm_smem = reinterpret_cast<bm::Tables *>(smem_raw + off);
    if constexpr (sizeof(R) == 8) bm::tables_init(bm_smem, tid, kThreads);

    Stream<R> st;
    st.key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    st.bm = sizeof(R) == 8 ? bm_smem : nullptr;
    st.zq = zq;
    int cur_shape = -1;

    FixedView<(KS >= 0 ? KS : 0)> fv;
    if constexpr (KS >= 0) {
        static_assert(sizeof(R) == 4 && RING == RING_EVEN, "compiled shapes: single precision, even ring");
        for (int j = 0; j < fixed_ncol(KS); ++j) fv.len[j] = B.shapes[B.fixed_src].len[j];
        fv.alpha = P.alpha;
        fv.lwf = 0;
        fv.hcoef = 0;
        fv.wf_on = 0;
        fv.general = nullptr;
    }

    while (true) {
        __syncthreads();   // previous item's shared memory is free
        if (tid == 0) s_item = atomicAdd(B.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= B.n_items) break;
        const int2 it = B.items[item];
        const BatchInstance &in = B.inst[it.x];
        const int L = in.L;
        if (in.shape != cur_shape) {             // the same for every thread
            cur_shape = in.shape;
            const BatchShape &sh = B.shapes[cur_shape];
            if (tid == 0) {
                view->ncol = sh.ncol;
                view->M = sh.M;
                view->alpha = P.alpha;
                view->lwf = 0;
                view->hcoef = 0;
                view->wf_on = 0;
                view->general = sh.general;
            }
            for (int j = tid; j < sh.ncol; j += kThreads) view->len[j] = sh.len[j];
        }
        const TT *tab = tab_s;
        if constexpr (kStage) {
            const int n = L * B.shapes[in.shape].M;
            const R *g = reinterpret_cast<const R *>(P.tables) + in.tab;
            for (int i = tid; i < n; i += kThreads) {
                if constexpr (sizeof(R) == 4)
                    tab_s[i] = make_float2(g[i], g[i]);
                else
                    tab_s[i] = g[i];
            }
        } else {
            tab = reinterpret_cast<const TT *>(P.tables) + in.tab;
        }
        for (int i = tid; i <= SU_MAX_S; i += kThreads) sig[i] = (R)in.sigma[i];
        for (int d = 1; d < L; ++d) {
            lm[(d - 1) * kThreads + tid] = (R)-INFINITY;
            ls[(d - 1) * kThreads + tid] = 0.0;
            lq[(d - 1) * kThreads + tid] = 0.0;
        }
        __syncthreads();
        const PathCfg<R> pc{(R)in.a, (R)in.b, in.S, L, sig};
        st.inst = P.instance + (uint32_t)it.x;
        const int blk = it.y / in.chunks, chk = it.y - blk * in.chunks;
        const int64_t blo = (int64_t)blk * in.n_mc / in.n_blocks;
        const int64_t bhi = ((int64_t)blk + 1) * in.n_mc / in.n_blocks;
        const int64_t lo = blo + (bhi - blo) * chk / in.chunks;
        const int64_t hi = blo + (bhi - blo) * (chk + 1) / in.chunks;
        Lse<R> acc;
        bool bad = false;
        for (int64_t smp = lo + tid; smp < hi; smp += kThreads) {
            st.slo = (uint32_t)smp;
            st.shi = (uint32_t)((uint64_t)smp >> 32);
            R w[SU_MAX_S];
            if constexpr (KS >= 0) {
                if (in.F == kMaxFine)
                    sample_path<R, RING, kMaxFine, false, true>(fv, pc, tab, qc, nullptr, st, w, 1, nullptr);
                else
                    sample_path_plain<R, RING>(in.F, *view, pc, tab, qc, st, w);
            } else {
                sample_path_plain<R, RING>(in.F, *view, pc, tab, qc, st, w);
            }
            bad |= isnan(w[0]) || (isinf(w[0]) && w[0] > 0);
            acc.push(w[0]);
            for (int d = 1; d < L; ++d) {
                bad |= isnan(w[d]) || (isinf(w[d]) && w[d] > 0);
                const int k = (d - 1) * kThreads + tid;
                lse_push(lm[k], ls[k], lq[k], w[d]);
            }
        }
        if (bad) atomicOr(P.flags, 1);
        // CTA merge per level in a fixed order: lanes by butterfly, then warps in order
        for (int d = 0; d < L; ++d) {
            double m, s, q;
            if (d == 0) {
                m = (double)acc.m;
                s = acc.s;
                q = acc.q;
            } else {
                const int k = (d - 1) * kThreads + tid;
                m = (double)lm[k];
                s = ls[k];
                q = lq[k];
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const double mb = __shfl_xor_sync(0xffffffffu, m, o);
                const double sb = __shfl_xor_sync(0xffffffffu, s, o);
                const double qb = __shfl_xor_sync(0xffffffffu, q, o);
                lse_merge_r<R>(m, s, q, mb, sb, qb);
            }
            if (lane == 0) {
                s_red[warp][d][0] = m;
                s_red[warp][d][1] = s;
                s_red[warp][d][2] = q;
            }
        }
        __syncthreads();
        if (tid < L) {
            const int d = tid;
            double M0 = s_red[0][d][0], S0 = s_red[0][d][1], Q0 = s_red[0][d][2];
            for (int w2 = 1; w2 < kThreads / 32; ++w2)
                lse_merge_r<R>(M0, S0, Q0, s_red[w2][d][0], s_red[w2][d][1], s_red[w2][d][2]);
            double *o = B.tuples + 4 * (in.tup + (int64_t)it.y * L + d);
            o[0] = M0;
            o[1] = S0;
            o[2] = Q0;
            o[3] = (double)(hi - lo);
        }
    }
}

}  // namespace
}  // namespace su
