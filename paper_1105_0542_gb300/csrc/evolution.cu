// The space-discretized short-time evolution operator (Sec. 5, Fig. 3 of the
// paper: energy eigenvalues and eigenfunctions by diagonalising the matrix of
// transition amplitudes):
//
//   U_ij = Delta * A_1^(p)(x_i, x_j; t),  x_i = -L + i Delta,  Delta = 2L/(n-1),
//   A_1^(p)(a, b; t) = (2 pi t)^(-1/2) exp(-(b - a)^2 / (2t) - t W_p((a+b)/2, (b-a)/2; t)),
//
// the single-slice amplitude with the level-p effective potential (Eq.
// ansatz at eps = t).  U is symmetric; its eigenvalues approach e^(-t E_k).
// Elements with (x_j - x_i)^2/(2t) > 40 are zero: their free factor is below
// e^-40 (under double resolution relative to the diagonal) and there
// xb^2 >> t, outside the short-time ordering of the expansion, where the
// truncated W_p can outgrow the Gaussian (Poeschl-Teller: the xb-series has a
// finite radius).  One thread per element of the tiles on and above the
// diagonal (columns coalesced along x), the rest by symmetry; -t W_p from
// the sampler's per-slice table evaluation, the free factor in double.
#include <cmath>

#include "sampler_impl.cuh"

namespace su {
namespace {

constexpr double kBand = 40.0;   // largest (x_j - x_i)^2/(2t) of a nonzero element

template <typename R, int RING>
__global__ void __launch_bounds__(256) evolution_kernel(const __grid_constant__ SamplerParams P,
                                                        const R *__restrict__ gtab, double L, double delta,
                                                        int n, double t, double lognorm, double *__restrict__ U) {
    // U is symmetric (W_p is even in xb and the free factor symmetric, so
    // U_ij and U_ji are the same bits): 32 x 32 tiles on and above the
    // diagonal are computed, each stored as it is and, through shared
    // memory, transposed into its mirror tile (both writes coalesced)
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (ti > tj) return;
    extern __shared__ __align__(16) unsigned char esm[];
    __shared__ double tile[32][33];
    // the general potential's program table (thousands of entries) is read
    // from global memory, every lane the same entry; the others are staged
    constexpr bool kStage = RING != RING_GENERAL;
    R *tab_s = reinterpret_cast<R *>(esm);
    const R *tab = kStage ? tab_s : gtab;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (kStage)
        for (int k = tid; k < P.M; k += blockDim.x * blockDim.y) tab_s[k] = gtab[k];
    __syncthreads();
    const int j = tj * 32 + threadIdx.x;
    // grid points rounded as (k Delta) + (-L), the last one L itself
    const double xj = j == n - 1 ? L : __dadd_rn(__dmul_rn((double)j, delta), -L);
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = ti * 32 + r;
        double u = 0.0;
        if (i < n && j < n) {
            const double xi = i == n - 1 ? L : __dadd_rn(__dmul_rn((double)i, delta), -L);
            const double d = xj - xi;
            const double free = d * d / (2.0 * t);
            if (free <= kBand) {
                const R w = slice<R, RING>((R)xi, (R)xj, tab, P, (R)P.alpha);   // -t W_p
                u = exp(lognorm - free + (double)w);
            }
            U[(size_t)i * n + j] = u;
        }
        tile[r][threadIdx.x] = u;
    }
    if (ti == tj) return;
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int jj = tj * 32 + r, ii = ti * 32 + threadIdx.x;
        if (jj < n && ii < n) U[(size_t)jj * n + ii] = tile[threadIdx.x][r];
    }
}

// The upper band of U in diagonal-major storage: D[k * pitch + i] = U_{i,i+k},
// k = 0..w, i = 0..n-1 (zero where i + k >= n or outside the band of reading
// E-1).  One thread per i along a diagonal (coalesced writes), kKPerCta
// diagonals per CTA; the lower half is U's mirror image (U is symmetric bit
// for bit: x_i + x_j and (x_j - x_i)^2 do not depend on the order).
constexpr int kKPerCta = 16;

template <typename R, int RING>
__global__ void __launch_bounds__(256) band_kernel(const __grid_constant__ SamplerParams P,
                                                   const R *__restrict__ gtab, double L, double delta, int n,
                                                   double t, double lognorm, int w, int64_t pitch,
                                                   double *__restrict__ D) {
    extern __shared__ __align__(16) unsigned char esm[];
    constexpr bool kStage = RING != RING_GENERAL;   // as in evolution_kernel
    R *tab_s = reinterpret_cast<R *>(esm);
    const R *tab = kStage ? tab_s : gtab;
    if (kStage)
        for (int k = threadIdx.x; k < P.M; k += blockDim.x) tab_s[k] = gtab[k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xi = i == n - 1 ? L : __dadd_rn(__dmul_rn((double)i, delta), -L);
    const int k0 = blockIdx.y * kKPerCta;
    for (int k = k0; k < min(k0 + kKPerCta, w + 1); ++k) {
        const int j = i + k;
        double u = 0.0;
        if (j < n) {
            const double xj = j == n - 1 ? L : __dadd_rn(__dmul_rn((double)j, delta), -L);
            const double d = xj - xi;
            const double free = d * d / (2.0 * t);
            if (free <= kBand) {
                const R wv = slice<R, RING>((R)xi, (R)xj, tab, P, (R)P.alpha);   // -t W_p
                u = exp(lognorm - free + (double)wv);
            }
        }
        D[(int64_t)k * pitch + i] = u;
    }
}

// Y (+)= U X for a block of B vectors, X and Y laid out [row][column]: the
// diagonals [k0, k1) of split blockIdx.y, one thread per row (its B partial
// sums in registers), written to part[split][row][column] for an ordered
// reduction.  Per diagonal k a row takes D_k[i] X[i+k] (upper half) and
// D_k[i-k] X[i-k] (its mirror, k >= 1): 2B FP64 multiply-adds per stored
// element and row.
template <int B>
__global__ void __launch_bounds__(64) band_matvec_kernel(const double *__restrict__ D, int64_t pitch, int n, int w,
                                                         int klen, const double *__restrict__ X,
                                                         double *__restrict__ part) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k0 = blockIdx.y * klen, k1 = min(w + 1, k0 + klen);
    double acc[B];
#pragma unroll
    for (int c = 0; c < B; ++c) acc[c] = 0.0;
    // a row of X: B doubles, read as 16-byte pairs (B even; rows 16-byte aligned)
    auto axpy = [&](double d, const double *x) {
        if constexpr (B % 2 == 0) {
            const double2 *x2 = reinterpret_cast<const double2 *>(x);
#pragma unroll
            for (int c = 0; c < B / 2; ++c) {
                const double2 v = x2[c];
                acc[2 * c] = fma(d, v.x, acc[2 * c]);
                acc[2 * c + 1] = fma(d, v.y, acc[2 * c + 1]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < B; ++c) acc[c] = fma(d, x[c], acc[c]);
        }
    };
    for (int k = k0; k < k1; ++k) {
        const double *Dk = D + (int64_t)k * pitch;
        if (i + k < n) axpy(Dk[i], X + (int64_t)(i + k) * B);
        if (k > 0 && i - k >= 0) axpy(Dk[i - k], X + (int64_t)(i - k) * B);
    }
    double *o = part + ((int64_t)blockIdx.y * n + i) * B;
#pragma unroll
    for (int c = 0; c < B; ++c) o[c] = acc[c];
}

// Ynew = alpha * (sum over splits of part) + beta * Ycur + gamma * Yprev,
// elementwise over n * B (the splits summed in order: deterministic).  With
// alpha = 2/e, beta = -2c/e, gamma = -1 this is one step of the Chebyshev
// recurrence T_{m+1}(s) = 2 s T_m(s) - T_{m-1}(s), s = (U - c)/e.
__global__ void cheb_kernel(const double *__restrict__ part, int splits, int64_t nb, const double *__restrict__ Ycur,
                            const double *__restrict__ Yprev, double *__restrict__ Ynew, double alpha, double beta,
                            double gamma) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    double s = 0.0;
    for (int q = 0; q < splits; ++q) s += part[(int64_t)q * nb + e];
    double y = alpha * s;
    if (beta != 0.0) y = fma(beta, Ycur[e], y);
    if (gamma != 0.0) y = fma(gamma, Yprev[e], y);
    Ynew[e] = y;
}

// part[chunk][c1][c2] = sum over the chunk's rows of A[i][c1] * C[i][c2]
// (B x B threads, rows staged through shared memory).
template <int B>
__global__ void gram_kernel(const double *__restrict__ A, const double *__restrict__ C, int n, int rows,
                            double *__restrict__ part) {
    __shared__ double sa[32][B], sc[32][B];
    const int c1 = threadIdx.x / B, c2 = threadIdx.x % B;
    const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
    double acc = 0.0;
    for (int base = r0; base < r1; base += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * B; e += blockDim.x) {
            const int r = base + e / B;
            sa[e / B][e % B] = r < r1 ? A[(int64_t)r * B + e % B] : 0.0;
            sc[e / B][e % B] = r < r1 ? C[(int64_t)r * B + e % B] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) acc = fma(sa[r][c1], sc[r][c2], acc);
    }
    part[((int64_t)blockIdx.x * B + c1) * B + c2] = acc;
}

// X[i][c] = sum_j Y[i][j] Q[j][c] (Q: B x B, row-major, in shared memory)
template <int B>
__global__ void rotate_kernel(const double *__restrict__ Y, const double *__restrict__ Q, int n,
                              double *__restrict__ X) {
    __shared__ double sq[B * B];
    for (int e = threadIdx.x; e < B * B; e += blockDim.x) sq[e] = Q[e];
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * B) return;
    const int64_t i = e / B;
    const int c = (int)(e - i * B);
    const double *y = Y + i * B;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < B; ++j) s = fma(y[j], sq[j * B + c], s);
    X[e] = s;
}

// part[chunk][c] = sum over the chunk's rows of (UX[i][c] - theta[c] X[i][c])^2
template <int B>
__global__ void resid_kernel(const double *__restrict__ UX, const double *__restrict__ X,
                             const double *__restrict__ theta, int n, int rows, double *__restrict__ part) {
    const int c = threadIdx.x % B, lane_row = threadIdx.x / B, nr = blockDim.x / B;
    const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
    const double th = theta[c];
    double acc = 0.0;
    for (int r = r0 + lane_row; r < r1; r += nr) {
        const double d = UX[(int64_t)r * B + c] - th * X[(int64_t)r * B + c];
        acc = fma(d, d, acc);
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < B) {
        double s = 0.0;
        for (int q = 0; q < nr; ++q) s += red[q * B + threadIdx.x];
        part[(int64_t)blockIdx.x * B + threadIdx.x] = s;
    }
}

// vec[k * n + i] = X[i][k] for k < nev / sqrt(Delta) (eigenfunctions on the grid)
template <int B>
__global__ void vectors_kernel(const double *__restrict__ X, int n, int nev, double scale, double *__restrict__ vec) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nev) return;
    const int64_t k = e / n, i = e - k * n;
    vec[e] = X[i * B + k] * scale;
}

template <typename R>
const void *pick_evolution(int ring) {
    switch (ring) {
        case RING_EVEN: return (const void *)evolution_kernel<R, RING_EVEN>;
        case RING_X: return (const void *)evolution_kernel<R, RING_X>;
        case RING_GENERAL:
            if constexpr (sizeof(R) == 8) return (const void *)evolution_kernel<double, RING_GENERAL>;
            return nullptr;
        default: return (const void *)evolution_kernel<R, RING_TANH2>;
    }
}

template <typename R>
const void *pick_band(int ring) {
    switch (ring) {
        case RING_EVEN: return (const void *)band_kernel<R, RING_EVEN>;
        case RING_X: return (const void *)band_kernel<R, RING_X>;
        case RING_GENERAL:
            if constexpr (sizeof(R) == 8) return (const void *)band_kernel<double, RING_GENERAL>;
            return nullptr;
        default: return (const void *)band_kernel<R, RING_TANH2>;
    }
}

}  // namespace

cudaError_t launch_evolution(const SamplerParams &P, int precision, const void *tab, double L, double delta, int n,
                             double t, double lognorm, double *U, cudaStream_t st) {
    const void *fn = precision == SU_FP32 ? pick_evolution<float>(P.ring) : pick_evolution<double>(P.ring);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = P.ring == RING_GENERAL ? 0 : (size_t)P.M * (precision == SU_FP32 ? sizeof(float) : sizeof(double));
    const dim3 block(32, 8), grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    void *args[] = {(void *)&P, (void *)&tab, (void *)&L, (void *)&delta, (void *)&n, (void *)&t, (void *)&lognorm,
                    (void *)&U};
    cudaGetLastError();
    return cudaLaunchKernel(fn, grid, block, args, smem, st);
}

}  // namespace su

namespace su {

cudaError_t launch_band(const SamplerParams &P, int precision, const void *tab, double L, double delta, int n,
                        double t, double lognorm, int w, int64_t pitch, double *D, cudaStream_t st) {
    const void *fn = precision == SU_FP32 ? pick_band<float>(P.ring) : pick_band<double>(P.ring);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = P.ring == RING_GENERAL ? 0 : (size_t)P.M * (precision == SU_FP32 ? sizeof(float) : sizeof(double));
    const dim3 block(256), grid((unsigned)((n + 255) / 256), (unsigned)((w + kKPerCta) / kKPerCta));
    void *args[] = {(void *)&P, (void *)&tab, (void *)&L, (void *)&delta, (void *)&n, (void *)&t,
                    (void *)&lognorm, (void *)&w, (void *)&pitch, (void *)&D};
    cudaGetLastError();
    return cudaLaunchKernel(fn, grid, block, args, smem, st);
}

template <int B>
static cudaError_t matvec_b(const double *D, int64_t pitch, int n, int w, int splits, const double *X, double *part,
                            cudaStream_t st) {
    const int klen = (w + splits) / splits;   // ceil((w + 1) / splits)
    const dim3 grid((unsigned)((n + 63) / 64), (unsigned)splits);
    band_matvec_kernel<B><<<grid, 64, 0, st>>>(D, pitch, n, w, klen, X, part);
    return cudaGetLastError();
}

cudaError_t launch_band_matvec(int B, const double *D, int64_t pitch, int n, int w, int splits, const double *X,
                               double *part, cudaStream_t st) {
    cudaGetLastError();
    switch (B) {
        case 1: return matvec_b<1>(D, pitch, n, w, splits, X, part, st);
        case 8: return matvec_b<8>(D, pitch, n, w, splits, X, part, st);
        case 16: return matvec_b<16>(D, pitch, n, w, splits, X, part, st);
        case 32: return matvec_b<32>(D, pitch, n, w, splits, X, part, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cheb(const double *part, int splits, int64_t nb, const double *Ycur, const double *Yprev,
                        double *Ynew, double alpha, double beta, double gamma, cudaStream_t st) {
    cudaGetLastError();
    cheb_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(part, splits, nb, Ycur, Yprev, Ynew, alpha, beta,
                                                              gamma);
    return cudaGetLastError();
}

template <int B>
static cudaError_t block_ops_b(int op, const double *A, const double *C, const double *Q, int n, int chunks,
                               double *out, cudaStream_t st) {
    const int rows = (n + chunks - 1) / chunks;
    if (op == 0) {
        gram_kernel<B><<<chunks, B * B, 0, st>>>(A, C, n, rows, out);
    } else if (op == 1) {
        const int64_t e = (int64_t)n * B;
        rotate_kernel<B><<<(unsigned)((e + 255) / 256), 256, 0, st>>>(A, Q, n, out);
    } else {
        resid_kernel<B><<<chunks, 256, 0, st>>>(A, C, Q, n, rows, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_block_op(int op, int B, const double *A, const double *C, const double *Q, int n, int chunks,
                            double *out, cudaStream_t st) {
    cudaGetLastError();
    switch (B) {
        case 8: return block_ops_b<8>(op, A, C, Q, n, chunks, out, st);
        case 16: return block_ops_b<16>(op, A, C, Q, n, chunks, out, st);
        case 32: return block_ops_b<32>(op, A, C, Q, n, chunks, out, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_vectors(int B, const double *X, int n, int nev, double scale, double *vec, cudaStream_t st) {
    cudaGetLastError();
    const int64_t e = (int64_t)n * nev;
    const unsigned g = (unsigned)((e + 255) / 256);
    switch (B) {
        case 8: vectors_kernel<8><<<g, 256, 0, st>>>(X, n, nev, scale, vec); break;
        case 16: vectors_kernel<16><<<g, 256, 0, st>>>(X, n, nev, scale, vec); break;
        case 32: vectors_kernel<32><<<g, 256, 0, st>>>(X, n, nev, scale, vec); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace su
