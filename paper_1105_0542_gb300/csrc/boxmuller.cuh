#pragma once
// Table-driven double-precision Box-Muller for the sampler (sm_103a).
//
// The normal pair z0 = R cos(theta), z1 = R sin(theta), R = sqrt(-2 ln u1),
// theta = 2 pi u2 (Sec. 4.1, both branches) for the 53-bit uniforms
// u1 = (a + 1/2) 2^-53, u2 = (b + 1/2) 2^-53.
//
// On this part the FP64 pipe runs at 1/60 of the FP32 rate and every double
// conversion (integer or float to double and back) costs as much as a double
// multiply-add, while integer and single-precision work issues from other,
// nearly idle pipes.  The routines therefore do their argument reductions
// and conversions on the integer bits, evaluate the small high-order parts
// of each series in single precision, and keep in double only the terms
// that need 53 bits (19 FP64 operations per pair):
//
//  * -2 ln u1: the table-driven logarithm (P. T. P. Tang, "Table-driven
//    implementation of the logarithm function in IEEE floating-point
//    arithmetic", ACM TOMS 16, 1990).  The double nearest u1 is 2^e m with
//    m in [3/4, 3/2), both taken from the integer a; node c_j = 3/4 + j/512
//    (j = 0..384) is the nearest to m, r = m inv_j - 1 (inv_j the double
//    nearest 1/c_j, one fused multiply-add, |r| < 2^-9.5), and
//      -2 ln u1 = [(-e) 2 ln 2 + 2 ln inv_j] - 2 ln(1 + r).
//    The bracket is summed in 56-bit fixed point and rounded to double on
//    the integer bits; -2 ln(1 + r) = -2r + r^2 - 2r^3/3 + r^4 t(r) with
//    t = 1/2 - 2r/5 + r^2/3 in single precision (truncation below 2^-60).
//  * R = sqrt(v): a single-precision reciprocal-square-root seed and two
//    Newton steps s <- s + (v - s^2) / (2 y) in double.
//  * cos/sin(theta): octant reduction on the top three bits of b (theta =
//    o pi/4 + phi, odd octants reflected to pi/4 - phi), then the accurate
//    table method (Gal; Tang): phi = a_i + d, a_i = pi (i + 1/2)/2048 from
//    the next nine bits (512 nodes), d = pi k 2^-53 for the odd integer k of
//    the remaining bits, |d| <= pi/4096, and
//      cos d - 1 = d (-d/2) + d^4/24,   sin d = d + d (-d^2/6 + d^4/120)
//    with the d^4 and d^2 factors in single precision (next terms below
//    2^-58); then the addition formulas and the octant's swap and signs.
//
// The node values inv_j, 2 ln inv_j, cos a_i, sin a_i are computed once per
// CTA with the CUDA library functions and kept in shared memory.  Every
// result agrees with R cos(theta), R sin(theta) from the library functions
// to a few units in the last place (checked by the GPU tests through the
// oracle's normals).
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define SU_BM_FN __host__ __device__ __forceinline__
#else
#define SU_BM_FN inline
#endif

namespace su {
namespace bm {

constexpr int kLogNodes = 385;    // c_j = 3/4 + j/512, j = 0..384
constexpr int kTrigNodes = 512;   // a_i = pi (i + 1/2) / 2048, the first octant
// 2 ln 2 in 56-bit fixed point: round(2 ln 2 * 2^56)
constexpr long long kLn2x2Q56 = 99893036290645747LL;

struct LogNode {
    double inv;                   // inv_j, the double nearest 1/c_j
    long long l2q;                // 2 ln inv_j in 56-bit fixed point
};

struct TrigNode {
    double c, s;                  // cos a_i, sin a_i
};

struct Tables {
    LogNode lg[kLogNodes];
    TrigNode tr[kTrigNodes];
};

// ------------------------------------------------------------ bit helpers
SU_BM_FN uint64_t dbits(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}

SU_BM_FN double dfrom(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    std::memcpy(&x, &u, 8);
    return x;
#endif
}

SU_BM_FN uint32_t fbits(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
#endif
}

SU_BM_FN float ffrom(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    std::memcpy(&x, &u, 4);
    return x;
#endif
}

SU_BM_FN int clz64(uint64_t x) {   // x != 0
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

SU_BM_FN float rsqrt_seed(float x) {
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / std::sqrt(x);
#endif
}

// double -> float on the bits, rounded (half away from zero), for
// 2^-126 <= |x| < 2^127
SU_BM_FN float to_float(double x) {
    const uint64_t u = dbits(x);
    const uint32_t mag = (uint32_t)(((u & 0x7FFFFFFFFFFFFFFFULL) + (1ULL << 28)) >> 29) - (896u << 23);
    return ffrom(mag | ((uint32_t)(u >> 32) & 0x80000000u));
}

// float -> double on the bits: exact for normal x; zero and subnormal x give
// a value of magnitude below 2^-126
SU_BM_FN double to_double(float x) {
    const uint32_t u = fbits(x);
    const uint64_t mag = ((uint64_t)(u & 0x7FFFFFFFu) + (896ULL << 23)) << 29;
    return dfrom(mag | ((uint64_t)(u & 0x80000000u) << 32));
}

// n 2^scale as the nearest double (ties away from zero), 0 < n < 2^63
SU_BM_FN double scaled(uint64_t n, int scale) {
    const int lz = clz64(n);
    const uint64_t nn = n << lz;                       // leading one at bit 63
    const uint64_t t = (nn >> 11) + ((nn >> 10) & 1);  // 53 bits, 2^53 after a carry
    return dfrom(((uint64_t)(1086 + scale - lz) << 52) + t - (1ULL << 52));
}

// ------------------------------------------------------------ the tables
#ifdef __CUDACC__
__device__ __forceinline__ void tables_init(Tables *t, int tid, int nthreads) {
    for (int j = tid; j < kLogNodes; j += nthreads) {
        const double inv = 1.0 / (0.75 + j * (1.0 / 512.0));
        t->lg[j].inv = inv;
        t->lg[j].l2q = __double2ll_rn(ldexp(2.0 * log(inv), 56));
    }
    for (int i = tid; i < kTrigNodes; i += nthreads) {
        double s, c;
        sincospi((i + 0.5) / 2048.0, &s, &c);
        t->tr[i].c = c;
        t->tr[i].s = s;
    }
}
#endif

// ------------------------------------------------------------ -2 ln u1
// u1 = (a + 1/2) 2^-53, a < 2^53; the exponent and mantissa of the double
// nearest u1 (rounded to nearest even, as forming it in double would) come
// from the integer
SU_BM_FN double minus2log(uint64_t a, const Tables *__restrict__ t) {
    const uint64_t v = 2 * a + 1;               // u1 = v 2^-54, v odd
    int e;                                      // u1 = 2^e (1 + f 2^-52)
    long long f;
    if (v < (1ULL << 53)) {                     // exact
        const int pos = 63 - clz64(v);
        e = pos - 54;
        f = (long long)((v << (52 - pos)) & ((1ULL << 52) - 1));
    } else {                                    // 54 bits: the last one is a tie
        uint64_t k = v >> 1;
        k += k & 1;                             // to even
        if (k >> 53) {
            e = 0;
            f = 0;
        } else {
            e = -1;
            f = (long long)(k - (1ULL << 52));
        }
    }
    long long mb;
    int j;
    if (f >= (1LL << 51)) {             // 1 + f 2^-52 in [3/2, 2): m = half of it, in [3/4, 1)
        e += 1;
        mb = f | (1022LL << 52);
        j = (int)((f - (1LL << 51) + (1LL << 43)) >> 44);          // 0..128
    } else {                            // m in [1, 3/2)
        mb = f | (1023LL << 52);
        j = 128 + (int)((f + (1LL << 42)) >> 43);                   // 128..384
    }
    const double m = dfrom((uint64_t)mb);
    const LogNode nd = t->lg[j];
    const double r = fma(m, nd.inv, -1.0);
    // r^4 coefficient of -2 ln(1 + r), single precision from float copies
    const float rf = fmaf(to_float(m), to_float(nd.inv), -1.0f);
    const float tf = fmaf(fmaf(rf, 1.0f / 3.0f, -0.4f), rf, 0.5f);
    double p = fma(r, to_double(tf), -2.0 / 3.0);
    p = fma(r, p, 1.0);
    p = fma(r, p, -2.0);
    // (-e) 2 ln 2 + 2 ln inv_j >= 0 (zero only for u1 in [1 - 2^-10, 1))
    const long long bq = (long long)(-e) * kLn2x2Q56 + nd.l2q;
    const double base = bq > 0 ? scaled((uint64_t)bq, -56) : 0.0;
    return fma(r, p, base);
}

// ------------------------------------------------------------ sqrt
// v in [0, 2^7] (v = 0 for u1 rounded to 1)
SU_BM_FN double sqrt_pos(double v) {
    const uint64_t vb = dbits(v), lo = 0x39B4484BFEEBC2A0ULL;   // the double 1e-30
    const float y = rsqrt_seed(to_float(dfrom(vb > lo ? vb : lo)));
    const double yd = to_double(y), hd = to_double(0.5f * y);
    double s = v * yd;
    s = fma(fma(-s, s, v), hd, s);
    s = fma(fma(-s, s, v), hd, s);
    return s;
}

// ------------------------------------------------------------ rotation
// z0 = R cos(theta), z1 = R sin(theta), theta = 2 pi (b + 1/2) 2^-53, b < 2^53
SU_BM_FN void rotate(double R, uint64_t b, const Tables *__restrict__ t, double &z0, double &z1) {
    const uint32_t o = (uint32_t)(b >> 50);                         // octant
    uint64_t x = b & ((1ULL << 50) - 1);                            // phi = 2 pi (x + 1/2) 2^-53
    if (o & 1) x = ((1ULL << 50) - 1) - x;                          // pi/4 - phi
    const int i = (int)(x >> 41);
    // d = phi - a_i = pi k 2^-53, k = 2 (x mod 2^41) - 2^41 + 1 (odd, |k| < 2^41)
    const long long k = 2 * (long long)(x & ((1ULL << 41) - 1)) - (1LL << 41) + 1;
    const uint64_t dneg = k < 0 ? 0x8000000000000000ULL : 0;
    const double d = dfrom(dbits(scaled((uint64_t)(k < 0 ? -k : k), -53) * 3.14159265358979323846) | dneg);
    const float df = to_float(d);
    const float d2 = df * df;
    const double q4 = to_double(d2 * d2 * (1.0f / 24.0f));              // d^4/24
    const double m6 = to_double(d2 * fmaf(d2, 1.0f / 120.0f, -1.0f / 6.0f));   // -d^2/6 + d^4/120
    const double hd = dfrom((dbits(d) - (1ULL << 52)) ^ 0x8000000000000000ULL);  // -d/2
    const double cm1 = fma(d, hd, q4);                               // cos d - 1
    const double sd = fma(d, m6, d);                                 // sin d
    const TrigNode a = t->tr[i];
    const double cf = fma(a.c, cm1, fma(-a.s, sd, a.c));             // cos(reduced angle)
    const double sf = fma(a.s, cm1, fma(a.c, sd, a.s));              // sin(reduced angle)
    // theta = q pi/2 + psi, (cos psi, sin psi) = (cf, sf) for even octants and
    // (sf, cf) for odd ones; then the quadrant's quarter turns
    const uint32_t q = o >> 1;
    const bool swap = ((o ^ q) & 1) != 0;
    const uint64_t sx = (q == 1 || q == 2) ? 0x8000000000000000ULL : 0;
    const uint64_t sy = (q >= 2) ? 0x8000000000000000ULL : 0;
    const double P = dfrom(dbits(swap ? sf : cf) ^ sx);
    const double Q = dfrom(dbits(swap ? cf : sf) ^ sy);
    z0 = R * P;
    z1 = R * Q;
}

}  // namespace bm
}  // namespace su

// ---------------------------------------------------------------------------
// Single-precision Box-Muller (the single-precision sampler's normals) for the
// 24-bit uniforms u1 = fl(a + 1/2) 2^-24, u2 = fl(b + 1/2) 2^-24 (a, b the top
// 24 bits of two Philox words), in float, from the hardware approximations:
//  * -2 ln u1 = -2 ln 2 log2(u1) with lg2.approx.f32 (absolute error about
//    2^-22.6), except for u1 > 15/16, where that absolute error would be large
//    against ln u1 itself: there -ln(1 - t) = t (1 + t/2 + .. + t^6/7) with
//    t = 1 - u1 exact (truncation t^7/8 < 2^-31 relative);
//  * R = sqrt(v) by sqrt.approx.f32 (0 where u1 rounds to 1);
//  * cos/sin(2 pi u2) = -(cos, sin)(2 pi (u2 - 1/2)) by __sincosf on an
//    argument in (-pi, pi) (u2 - 1/2 is exact; absolute error about 2^-21).
// Largest error: about 5e-7 R from the sine and cosine, at most 3e-7 from
// the logarithm (at u1 = 15/16, where R = 0.36); the GPU tests hold the
// normals to 1e-6 (1 + R) of the oracle's double-precision Box-Muller on the
// same uniforms.  Earlier forms, table-driven like the double routines above
// (a 49-node logarithm, quadrant-reduced 33-node sin/cos), were a few units
// in the last place accurate but cost about 55 instructions per pair, the
// largest item of the issue-bound single-precision sampler after the W_p
// Horner; this one costs about 25.
namespace bm32 {

// z0 = R cos(2 pi u2), z1 = R sin(2 pi u2), R = sqrt(-2 ln u1)
__device__ __forceinline__ void pair(uint32_t a, uint32_t b, float &z0, float &z1) {
    // ((w >> 8) + 1/2) 2^-24 in one rounding: the scaling is exact
    const float u1 = fmaf((float)(a >> 8), 0x1p-24f, 0x1p-25f);
    const float u2 = fmaf((float)(b >> 8), 0x1p-24f, 0x1p-25f);

    // ---- v = -2 ln u1
    const float t = 1.0f - u1;
    float lg;
    asm("lg2.approx.f32 %0, %1;" : "=f"(lg) : "f"(u1));
    float ser = fmaf(t, 1.0f / 7.0f, 1.0f / 6.0f);
    ser = fmaf(t, ser, 0.2f);
    ser = fmaf(t, ser, 0.25f);
    ser = fmaf(t, ser, 0.333333343f);
    ser = fmaf(t, ser, 0.5f);
    ser = fmaf(t, ser, 1.0f);
    const float v = t < 0.0625f ? 2.0f * t * ser : -1.38629436f * lg;   // -2 ln 2 = -1.38629436

    // ---- R = sqrt(v), v in {0} u [2^-24, 35]
    float R;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(R) : "f"(v));

    // ---- cos, sin of 2 pi u2
    float sn, cs;
    __sincosf(6.28318530718f * (u2 - 0.5f), &sn, &cs);
    z0 = -R * cs;
    z1 = -R * sn;
}

}  // namespace bm32
