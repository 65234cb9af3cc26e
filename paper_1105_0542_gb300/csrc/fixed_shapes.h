// Table shapes compiled into specialised single-precision samplers.
//
// In the single-precision sampler the nested Horner of -eps W_p (Eq. SNp,
// collapsed in powers of xb^2 and z) is issue-bound, and with the shape read
// at run time a third of its instructions are loop control and table
// addressing.  The shapes below are those of the even ring (z = x^2) for the
// harmonic oscillator and for every quartic potential (anharmonic oscillator,
// double well) at p = 1..18; a plan whose level tables have one of them runs
// a sampler instantiated for it, with every Horner loop unrolled and every
// table offset a constant (the same operations in the same order, so the
// same bits), and so does a batch plan whose instances all have it.  Any
// other shape runs the generic kernels.
//
// Shape k is coded as nibbles: column j has (code >> 4 j) & 15 entries, the
// columns run up to the first empty nibble.
#pragma once

namespace su {

constexpr int kNumFixed = 20;
constexpr int kFixedGroups = 8;          // translation units the specialised kernels are spread over

__host__ __device__ constexpr unsigned fixed_code(int k) {
    return k == 0 ? 0x2u :               // harmonic oscillator, p = 1
           k == 1 ? 0x12u :              // harmonic oscillator, p >= 2
           k == 2 ? 0x3u :               // quartic, p = 1
           k == 3 ? 0x23u :              // p = 2
           k == 4 ? 0x124u :             // p = 3
           k == 5 ? 0x134u :             // p = 4
           k == 6 ? 0x235u :             // p = 5
           k == 7 ? 0x1245u :            // p = 6
           k == 8 ? 0x1346u :            // p = 7
           k == 9 ? 0x2356u :            // p = 8
           k == 10 ? 0x12457u :          // p = 9
           k == 11 ? 0x13467u :          // p = 10
           k == 12 ? 0x23568u :          // p = 11
           k == 13 ? 0x124578u :         // p = 12
           k == 14 ? 0x134679u :         // p = 13
           k == 15 ? 0x235689u :         // p = 14
           k == 16 ? 0x124578au :        // p = 15
           k == 17 ? 0x134679au :        // p = 16
           k == 18 ? 0x235689bu :        // p = 17
           0x124578abu;                  // p = 18
}

__host__ __device__ constexpr int fixed_len(int k, int j) { return (int)((fixed_code(k) >> (4 * j)) & 15u); }

__host__ __device__ constexpr int fixed_ncol(int k) {
    int n = 0;
    while (n < 8 && fixed_len(k, n)) ++n;
    return n;
}

// first entry of column j: the entries of columns 0..j-1
__host__ __device__ constexpr int fixed_off(int k, int j) {
    int o = 0;
    for (int i = 0; i < j; ++i) o += fixed_len(k, i);
    return o;
}

__host__ __device__ constexpr int fixed_M(int k) { return fixed_off(k, fixed_ncol(k)); }

// the compiled shape equal to (ncol, len[0..ncol-1]), or -1
inline int fixed_shape_index(int ncol, const int *len) {
    for (int k = 0; k < kNumFixed; ++k) {
        if (fixed_ncol(k) != ncol) continue;
        bool eq = true;
        for (int j = 0; j < ncol; ++j) eq = eq && fixed_len(k, j) == len[j];
        if (eq) return k;
    }
    return -1;
}

}  // namespace su
