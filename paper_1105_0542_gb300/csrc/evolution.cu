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
    R *tab = reinterpret_cast<R *>(esm);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < P.M; k += blockDim.x * blockDim.y) tab[k] = gtab[k];
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

template <typename R>
const void *pick_evolution(int ring) {
    switch (ring) {
        case RING_EVEN: return (const void *)evolution_kernel<R, RING_EVEN>;
        case RING_X: return (const void *)evolution_kernel<R, RING_X>;
        default: return (const void *)evolution_kernel<R, RING_TANH2>;
    }
}

}  // namespace

cudaError_t launch_evolution(const SamplerParams &P, int precision, const void *tab, double L, double delta, int n,
                             double t, double lognorm, double *U, cudaStream_t st) {
    const void *fn = precision == SU_FP32 ? pick_evolution<float>(P.ring) : pick_evolution<double>(P.ring);
    const size_t smem = (size_t)P.M * (precision == SU_FP32 ? sizeof(float) : sizeof(double));
    const dim3 block(32, 8), grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    void *args[] = {(void *)&P, (void *)&tab, (void *)&L, (void *)&delta, (void *)&n, (void *)&t, (void *)&lognorm,
                    (void *)&U};
    cudaGetLastError();
    return cudaLaunchKernel(fn, grid, block, args, smem, st);
}

}  // namespace su
