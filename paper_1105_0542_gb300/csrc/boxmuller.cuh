#pragma once
// Table-driven double-precision Box-Muller for the sampler (sm_103a).
//
// On this part the FP64 pipe runs at 1/60 of the FP32 rate, and the generic
// double log / sqrt / sincos cost about as much as W_p itself at low p.  The
// normal pair z0 = r cos(theta), z1 = r sin(theta), r = sqrt(-2 ln u1),
// theta = 2 pi u2 (Sec. 4.1, both branches) is therefore formed with table
// methods whose argument reduction is done on the integer bits:
//
//  * v = -2 ln u1: the table-driven logarithm (P. T. P. Tang, "Table-driven
//    implementation of the logarithm function in IEEE floating-point
//    arithmetic", ACM TOMS 16, 1990): u1 = 2^e m, m in [3/4, 3/2) taken from
//    the exponent and mantissa bits, nearest node c_j = 3/4 + j/128
//    (c_32 = 1 exactly), r = (m - c_j)/c_j with |r| <= 1/192, and
//    ln u1 = e ln 2 + ln c_j + ln(1 + r), ln(1 + r) by its Taylor series to
//    r^8 (truncation below 2^-60 relative).
//  * r = sqrt(v): two Newton steps for sqrt from the approximate reciprocal
//    square root (rsqrt.approx.f64).
//  * the exponent and mantissa of u1 come from the 53-bit integer itself and
//    the integer-to-double steps use bit patterns, so that the FP64 pipe only
//    runs the arithmetic (about 34 operations per pair).
//  * cos/sin(theta): the accurate-table method (Gal; Tang): theta =
//    a_i + delta with a_i = 2 pi (i + 1/2)/256 from the top 8 bits of the
//    53-bit integer behind u2, |delta| <= pi/256 from the remaining bits,
//    cos/sin(delta) by Taylor series (to delta^6 and delta^7), and the
//    addition formulas.
//
// The node values ln c_j, 1/c_j, cos a_i, sin a_i are computed once per CTA
// with the CUDA library functions and kept in shared memory.  Every result
// agrees with r cos(theta), r sin(theta) from the library functions to a few
// units in the last place (checked by the GPU tests through the oracle's
// normals).
#include <cstdint>

namespace su {
namespace {

constexpr int kLogNodes = 97;    // c_j = 3/4 + j/128, j = 0..96
constexpr int kTrigNodes = 256;  // a_i = 2 pi (i + 1/2) / 256
constexpr int kExpNodes = 56;    // -2 e ln 2, e = 0..-55

struct LogNode {
    double l2;                   // -2 ln c_j
    double inv;                  // 1 / c_j
    double c;                    // c_j
};

struct BMTables {
    LogNode lg[kLogNodes];
    double e2[kExpNodes];        // -2 ln 2 * e for e = -k, k = 0..55
    double2 tr[kTrigNodes];      // (cos a_i, sin a_i)
};

__device__ __forceinline__ void bm_tables_init(BMTables *t, int tid, int nthreads) {
    for (int j = tid; j < kLogNodes; j += nthreads) {
        const double c = 0.75 + j * (1.0 / 128.0);
        t->lg[j].l2 = -2.0 * log(c);
        t->lg[j].inv = 1.0 / c;
        t->lg[j].c = c;
    }
    for (int k = tid; k < kExpNodes; k += nthreads)
        t->e2[k] = 2.0 * k * 0.69314718055994530942;   // -2 ln 2 * (-k)
    for (int i = tid; i < kTrigNodes; i += nthreads) {
        double s, c;
        sincospi((i + 0.5) / 128.0, &s, &c);
        t->tr[i] = make_double2(c, s);
    }
}

// -2 ln(u1) for u1 = ((double)a + 1/2) 2^-53, a < 2^53, taking the binary
// exponent and mantissa of u1 from the integer a (the same rounding to
// nearest even as forming the double).
__device__ __forceinline__ double bm_minus2log(uint64_t a, const BMTables *__restrict__ t) {
    const uint64_t v = 2 * a + 1;               // u1 = v 2^-54, v odd
    int e;                                      // u1 = 2^e (1 + mant 2^-52)
    long long mant;
    if (v < (1ULL << 53)) {                     // exact
        const int pos = 63 - __clzll((long long)v);
        e = pos - 54;
        mant = (long long)((v << (52 - pos)) & ((1ULL << 52) - 1));
    } else {                                    // 54 bits: the last one is a tie
        uint64_t k = v >> 1;
        k += k & 1;                             // to even
        if (k >> 53) {
            e = 0;
            mant = 0;
        } else {
            e = -1;
            mant = (long long)(k - (1ULL << 52));
        }
    }
    long long mbits;
    int j;
    if (mant >= (1LL << 51)) {           // m in [1.5, 2): use m/2 in [0.75, 1)
        e += 1;
        mbits = mant | (1022LL << 52);
        j = (int)((mant - (1LL << 51) + (1LL << 45)) >> 46);
    } else {                             // m in [1, 1.5)
        mbits = mant | (1023LL << 52);
        j = 32 + (int)((mant + (1LL << 44)) >> 45);
    }
    const double m = __longlong_as_double(mbits);
    const LogNode node = t->lg[j];
    const double r = (m - node.c) * node.inv;   // m - c is exact
    // -2 ln(1 + r) = r * sum_{k>=0} (-2) (-r)^k / (k + 1), to r^8
    double p = 2.0 / 8.0;
    p = fma(p, r, -2.0 / 7.0);
    p = fma(p, r, 2.0 / 6.0);
    p = fma(p, r, -2.0 / 5.0);
    p = fma(p, r, 2.0 / 4.0);
    p = fma(p, r, -2.0 / 3.0);
    p = fma(p, r, 2.0 / 2.0);
    p = fma(p, r, -2.0);
    return fma(r, p, t->e2[-e] + node.l2);     // e in -54..0
}

// sqrt(v), v >= 0: Newton steps s <- s + (v - s^2) h from the hardware's
// approximate reciprocal square root (about 23 correct bits)
__device__ __forceinline__ double bm_sqrt(double v) {
    double y;
    asm("rsqrt.approx.f64 %0, %1;" : "=d"(y) : "d"(fmax(v, 1e-300)));
    const double h = 0.5 * y;
    double s = v * y;
    s = fma(fma(-s, s, v), h, s);
    s = fma(fma(-s, s, v), h, s);
    return s;
}

// z0 = r cos(2 pi u2), z1 = r sin(2 pi u2) with u2 = (b + 1/2) 2^-53, b < 2^53
__device__ __forceinline__ void bm_rotate(double r, uint64_t b, const BMTables *__restrict__ t,
                                          double &z0, double &z1) {
    const int i = (int)(b >> 45);
    // k = (b mod 2^45) - 2^44 as a double without a conversion: the bits of
    // 2^52 + 2^51 + k, minus that offset (exact for |k| < 2^51)
    const long long k = (long long)(b & ((1ULL << 45) - 1)) - (1LL << 44);
    const double kd = __longlong_as_double(0x4338000000000000LL + k) - 6755399441055744.0;
    const double C = 6.283185307179586477 * 0x1p-53;    // 2 pi / 2^53
    const double d = fma(kd, C, 0.5 * C);               // theta - a_i, |d| <= pi/256
    const double d2 = d * d;
    const double cm1 = d2 * fma(fma(d2, -1.0 / 720.0, 1.0 / 24.0), d2, -0.5);          // cos d - 1
    const double sd = fma(d * d2, fma(fma(d2, -1.0 / 5040.0, 1.0 / 120.0), d2, -1.0 / 6.0), d);  // sin d
    const double2 a = t->tr[i];
    const double rc = r * a.x, rs = r * a.y;
    z0 = fma(rc, cm1, fma(-rs, sd, rc));
    z1 = fma(rs, cm1, fma(rc, sd, rs));
}

}  // namespace
}  // namespace su
