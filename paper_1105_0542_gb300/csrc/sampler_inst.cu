// One instantiation of the sampler and batched kernels, selected at compile time:
//   SU_PREC = 64 or 32 (double / float path and W_p), SU_RING = 0, 1, 2
//   (z = x^2, x, sech^2(alpha x)) or 3 (a general potential through its
//   derivatives; double sampler only); SU_GTAB = 1 for the double sampler
//   that reads level tables too large for shared memory from global memory.
// The build compiles this file once per combination so the kernels compile
// in parallel.
#include "sampler_impl.cuh"

#ifdef SU_FIXED
// SU_FIXED = g: the single-precision even-ring samplers and batched kernels
// with the table shapes k = g, g + kFixedGroups, .. of fixed_shapes.h
// compiled in
namespace su {
namespace {
template <int K>
const void *fixed_entry(int k) {
    if constexpr (K >= kNumFixed) {
        return nullptr;
    } else {
        if (k == K) return (const void *)sampler_kernel<float, RING_EVEN, false, K>;
        return fixed_entry<K + kFixedGroups>(k);
    }
}
template <int K>
const void *fixed_batch_entry(int k) {
    if constexpr (K >= kNumFixed) {
        return nullptr;
    } else {
        if (k == K) return (const void *)batch_kernel<float, RING_EVEN, K>;
        return fixed_batch_entry<K + kFixedGroups>(k);
    }
}
}  // namespace

#define SU_FIXED_NAME2(a, g) a##_##g
#define SU_FIXED_NAME(a, g) SU_FIXED_NAME2(a, g)
const void *SU_FIXED_NAME(sampler_fixed_entry, SU_FIXED)(int k) { return fixed_entry<SU_FIXED>(k); }
const void *SU_FIXED_NAME(batch_fixed_entry, SU_FIXED)(int k) { return fixed_batch_entry<SU_FIXED>(k); }
}  // namespace su
#else

#ifndef SU_PREC
#error "SU_PREC must be 64 or 32"
#endif
#ifndef SU_RING
#error "SU_RING must be 0, 1, 2 or 3"
#endif
#ifndef SU_GTAB
#define SU_GTAB 0
#endif

#define SU_CAT2(a, b, c) a##b##_##c
#define SU_CAT(a, b, c) SU_CAT2(a, b, c)

namespace su {
#if SU_PREC == 64
using Real = double;
#else
using Real = float;
#endif

#if SU_GTAB
// the level tables read from global memory (too large to stage)
const void *SU_CAT(sampler_entry_gt_f, SU_PREC, SU_RING)() {
    return (const void *)sampler_kernel<Real, SU_RING, true>;
}
#else
const void *SU_CAT(sampler_entry_f, SU_PREC, SU_RING)() {
    return (const void *)sampler_kernel<Real, SU_RING>;
}
#endif

#if !SU_GTAB && (SU_RING != 3 || SU_PREC == 64)
const void *SU_CAT(batch_entry_f, SU_PREC, SU_RING)() {
    return (const void *)batch_kernel<Real, SU_RING>;
}
#endif
}  // namespace su
#endif  // SU_FIXED
