// Non-templated kernels of the amplitude estimator and the host launchers:
// the block combine, the raw Philox words, and the dispatch to the sampler
// instantiations (one translation unit per precision and ring, built from
// sampler_inst.cu).
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "sampler_impl.cuh"

namespace su {

// defined in the sampler_inst.cu instantiations
const void *sampler_entry_f64_0();
const void *sampler_entry_f64_1();
const void *sampler_entry_f64_2();
const void *sampler_entry_f32_0();
const void *sampler_entry_f32_1();
const void *sampler_entry_f32_2();
const void *sampler_entry_f64_3();
const void *sampler_entry_gt_f64_0();
const void *sampler_entry_gt_f64_1();
const void *sampler_entry_gt_f64_2();
const void *batch_entry_f64_0();
const void *batch_entry_f64_1();
const void *batch_entry_f64_2();
const void *batch_entry_f64_3();
const void *batch_entry_f32_0();
const void *batch_entry_f32_1();
const void *batch_entry_f32_2();
// the compiled-shape kernels of group g = k % kFixedGroups (sampler_inst.cu, SU_FIXED = g)
#define SU_FIXED_GROUP(g)                        \
    const void *sampler_fixed_entry_##g(int k); \
    const void *batch_fixed_entry_##g(int k);
SU_FIXED_GROUP(0)
SU_FIXED_GROUP(1)
SU_FIXED_GROUP(2)
SU_FIXED_GROUP(3)
SU_FIXED_GROUP(4)
SU_FIXED_GROUP(5)
SU_FIXED_GROUP(6)
SU_FIXED_GROUP(7)
#undef SU_FIXED_GROUP
static_assert(kFixedGroups == 8, "one entry pair per group");
using FixedEntry = const void *(*)(int);
static const FixedEntry kSamplerFixed[kFixedGroups] = {
    sampler_fixed_entry_0, sampler_fixed_entry_1, sampler_fixed_entry_2, sampler_fixed_entry_3,
    sampler_fixed_entry_4, sampler_fixed_entry_5, sampler_fixed_entry_6, sampler_fixed_entry_7};
static const FixedEntry kBatchFixed[kFixedGroups] = {
    batch_fixed_entry_0, batch_fixed_entry_1, batch_fixed_entry_2, batch_fixed_entry_3,
    batch_fixed_entry_4, batch_fixed_entry_5, batch_fixed_entry_6, batch_fixed_entry_7};

namespace {

// ----------------------------------------------------------- combine
__global__ void combine_kernel(const double *__restrict__ partial, double *__restrict__ tuples, int64_t b0,
                               int64_t n_blocks, int L, int64_t ipb) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_blocks * L) return;
    const int64_t b = b0 + id / L;
    const int d = (int)(id - (id / L) * L);
    double M = -INFINITY, S = 0, Q = 0, n = 0;
    for (int64_t r = 0; r < ipb; ++r) {
        const double *p = partial + 4 * ((b * ipb + r) * L + d);
        const double m2 = p[0];
        n += p[3];
        if (!(m2 > -INFINITY)) continue;
        if (m2 > M) {
            const double f = exp(M - m2);  // 0 when M = -inf
            S = S * f + p[1];
            Q = Q * f * f + p[2];
            M = m2;
        } else {
            const double f = exp(m2 - M);
            S += p[1] * f;
            Q += p[2] * f * f;
        }
    }
    double *o = tuples + 4 * (b * L + d);
    o[0] = M;
    o[1] = S;
    o[2] = Q;
    o[3] = n;
}

// ------------------------------------------------------- raw Philox words
__global__ void philox_words_kernel(uint64_t seed, uint32_t inst, int64_t sample0, int64_t ns,
                                    int ncalls, uint32_t *out) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= ns * ncalls) return;
    const int64_t i = id / ncalls;
    const uint32_t t = (uint32_t)(id - i * ncalls);
    const uint64_t s = (uint64_t)(sample0 + i);
    const uint4 w = philox4x32_10(make_uint4(t, inst, (uint32_t)s, (uint32_t)(s >> 32)),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    reinterpret_cast<uint4 *>(out)[id] = w;
}

// ------------------------------------------------ the sampler's normals
// out[i * n + j] = normal j of sample sample0 + i, as the sampler forms it:
// one thread per (sample, call); a call gives two normals on the double path
// (j = 2t, 2t + 1) and four on the single path (j + 1 = 4t .. 4t + 3)
__global__ void __launch_bounds__(128) normals_kernel_f64(uint64_t seed, uint32_t inst, int64_t sample0,
                                                          int64_t ns, int n, double *out) {
    __shared__ bm::Tables tabs;
    bm::tables_init(&tabs, threadIdx.x, blockDim.x);
    __syncthreads();
    const int calls = (n + 1) / 2;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= ns * calls) return;
    const int64_t i = id / calls;
    const uint32_t t = (uint32_t)(id - i * calls);
    Stream<double> st;
    const uint64_t smp = (uint64_t)(sample0 + i);
    st.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    st.inst = inst;
    st.slo = (uint32_t)smp;
    st.shi = (uint32_t)(smp >> 32);
    st.bm = &tabs;
    double z0, z1;
    st.pair(t, z0, z1);
    out[i * n + 2 * t] = z0;
    if (2 * (int)t + 1 < n) out[i * n + 2 * t + 1] = z1;
}

__global__ void __launch_bounds__(128) normals_kernel_f32(uint64_t seed, uint32_t inst, int64_t sample0,
                                                          int64_t ns, int n, double *out) {
    const int calls = n / 4 + 1;                 // j' = j + 1 runs over 1..n
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= ns * calls) return;
    const int64_t i = id / calls;
    const uint32_t t = (uint32_t)(id - i * calls);
    Stream<float> st;
    const uint64_t smp = (uint64_t)(sample0 + i);
    st.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    st.inst = inst;
    st.slo = (uint32_t)smp;
    st.shi = (uint32_t)(smp >> 32);
    st.bm = nullptr;
    float z[4];
    st.quad(t, z);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = 4 * (int)t + k - 1;
        if (j >= 0 && j < n) out[i * n + j] = (double)z[k];
    }
}

// the single-precision sampler with this plan's table shape compiled in, if
// there is one (fixed_shapes.h): even ring, 2^kMaxFine-slice segments, no
// width-factor weight
int fixed_index(const SamplerParams &P, int precision) {
    if (precision != SU_FP32 || P.generic || P.ring != RING_EVEN || P.tab_global || P.F != kMaxFine || P.wf_on)
        return -1;
    return fixed_shape_index(P.ncol, P.len);
}

const void *pick_fixed(const SamplerParams &P, int precision) {
    const int k = fixed_index(P, precision);
    return k < 0 ? nullptr : kSamplerFixed[k % kFixedGroups](k);
}

const void *pick(const SamplerParams &P, int precision) {
    if (const void *fn = pick_fixed(P, precision)) return fn;
    if (P.ring == RING_GENERAL) return precision == SU_FP64 ? sampler_entry_f64_3() : nullptr;
    if (P.tab_global) {
        if (precision != SU_FP64) return nullptr;
        return P.ring == RING_EVEN ? sampler_entry_gt_f64_0() : P.ring == RING_X ? sampler_entry_gt_f64_1()
                                                                                  : sampler_entry_gt_f64_2();
    }
    if (precision == SU_FP32)
        return P.ring == RING_EVEN ? sampler_entry_f32_0() : P.ring == RING_X ? sampler_entry_f32_1() : sampler_entry_f32_2();
    return P.ring == RING_EVEN ? sampler_entry_f64_0() : P.ring == RING_X ? sampler_entry_f64_1() : sampler_entry_f64_2();
}

}  // namespace

const void *batch_fn(const BatchParams &B, int precision) {
    const int ring = B.base.ring;
    if (precision == SU_FP32 && ring == RING_EVEN && B.fixed_shape >= 0 && B.fixed_shape < kNumFixed) {
        const int k = B.fixed_shape;
        return kBatchFixed[k % kFixedGroups](k);
    }
    if (ring == RING_GENERAL) return precision == SU_FP64 ? batch_entry_f64_3() : nullptr;
    if (precision == SU_FP32)
        return ring == RING_EVEN ? batch_entry_f32_0() : ring == RING_X ? batch_entry_f32_1() : batch_entry_f32_2();
    return ring == RING_EVEN ? batch_entry_f64_0() : ring == RING_X ? batch_entry_f64_1() : batch_entry_f64_2();
}

int sampler_fixed_shape(const SamplerParams &P, int precision) { return pick_fixed(P, precision) ? fixed_index(P, precision) : -1; }

size_t batch_smem_bytes(const BatchParams &B, int precision) {
    const size_t rs = precision == SU_FP32 ? sizeof(float) : sizeof(double);
    size_t off = (sizeof(BatchView) + 15) & ~(size_t)15;
    // staged tables (the general program's stay in global memory)
    const size_t staged = B.base.ring == RING_GENERAL ? 0 : (size_t)B.tab_max;
    off += (precision == SU_FP32 ? 8 : rs) * staged + rs * (size_t)(SU_MAX_S + 1);
    off = (off + 15) & ~(size_t)15;
    off += rs * (size_t)(B.C_max > 1 ? B.C_max + 1 : 0) * kThreads;
    off = (off + 15) & ~(size_t)15;
    off += (2 * sizeof(double) + rs) * (size_t)(B.L_max - 1) * kThreads;
    off = (off + 15) & ~(size_t)15;
    if (precision == SU_FP32) off += sizeof(float4) * (size_t)staged_quads(kMaxFine, true) * kThreads;
    if (precision == SU_FP64) off += sizeof(bm::Tables);
    return off;
}

size_t sampler_smem_bytes(const SamplerParams &P, int precision) {
    const size_t rs = precision == SU_FP32 ? sizeof(float) : sizeof(double);
    const int C = 1 << (P.S - P.F);
    size_t off = P.w_out ? 0 : rs * (size_t)P.levels * kThreads * P.rounds;
    off = (off + 15) & ~(size_t)15;
    // staged tables (single precision: pairs {c, c}); else read from global memory
    if (P.ring != RING_GENERAL && !P.tab_global) off += (precision == SU_FP32 ? 8 : rs) * (size_t)P.S * P.M;
    off += rs * (size_t)(SU_MAX_S + 1);
    off = (off + 15) & ~(size_t)15;
    off += rs * (size_t)(C > 1 ? C + 1 : 0) * kThreads;
    off = (off + 15) & ~(size_t)15;
    if (P.wf_on) off += sizeof(double) * (size_t)(P.S + 1) * kThreads;
    off = (off + 15) & ~(size_t)15;
    if (precision == SU_FP32) off += sizeof(float4) * (size_t)staged_quads(P.F) * kThreads;
    if (precision == SU_FP64) off += sizeof(bm::Tables);
    return off;
}

// Opt the kernel in to the device's full dynamic shared memory once, so that
// plans of different sizes can alternate without re-setting the attribute.
// (the opt-in limit covers static and dynamic shared memory together)
static cudaError_t allow_full_smem(const void *fn) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) cudaGetLastError();   // reported through the return value only
    return e;
}

int batch_occupancy(const BatchParams &B, int precision, size_t smem) {
    const void *fn = batch_fn(B, precision);
    if (allow_full_smem(fn) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

int sampler_occupancy(const SamplerParams &P, int precision, size_t smem) {
    const void *fn = pick(P, precision);
    if (allow_full_smem(fn) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_sampler(const SamplerParams &P, int precision, int grid, size_t smem,
                           cudaStream_t st) {
    void *args[] = {const_cast<SamplerParams *>(&P)};
    const void *fn = pick(P, precision);
    cudaGetLastError();
    if (smem > 48 * 1024) {
        cudaError_t e = allow_full_smem(fn);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, smem, st);
}

cudaError_t launch_combine(const double *partial, double *tuples, int64_t b0, int64_t n_blocks, int levels,
                           int64_t items_per_block, cudaStream_t st) {
    const int64_t n = n_blocks * levels;
    if (n == 0) return cudaSuccess;
    const int th = 128;
    cudaGetLastError();
    combine_kernel<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(partial, tuples, b0, n_blocks, levels,
                                                               items_per_block);
    return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint32_t instance, int64_t sample0, int64_t n_samples,
                           int n_normals, int precision, double *out, cudaStream_t st) {
    if (n_samples <= 0 || n_normals <= 0) return cudaSuccess;
    const int64_t calls = precision == SU_FP32 ? n_normals / 4 + 1 : (n_normals + 1) / 2;
    const int64_t n = n_samples * calls;
    const int th = 128;
    const unsigned grid = (unsigned)((n + th - 1) / th);
    cudaGetLastError();
    if (precision == SU_FP32)
        normals_kernel_f32<<<grid, th, 0, st>>>(seed, instance, sample0, n_samples, n_normals, out);
    else
        normals_kernel_f64<<<grid, th, 0, st>>>(seed, instance, sample0, n_samples, n_normals, out);
    return cudaGetLastError();
}

cudaError_t launch_philox_words(uint64_t seed, uint32_t instance, int64_t sample0, int64_t n_samples,
                                int n_calls, uint32_t *out, cudaStream_t st) {
    const int64_t n = n_samples * n_calls;
    if (n == 0) return cudaSuccess;
    const int th = 256;
    cudaGetLastError();
    philox_words_kernel<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(seed, instance, sample0, n_samples,
                                                                    n_calls, out);
    return cudaGetLastError();
}

}  // namespace su
