// Internal interface between the host API and the device kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/speedup.h"
#include "generator.h"

namespace su {

constexpr int kThreads = 128;   // threads per CTA of the sampler: one path per thread
constexpr int kMaxFine = 5;     // depth of the register-resident bisection subtree

// Everything the sampler needs, passed by value (it lives in the constant bank).
// General potential (RING_GENERAL): the device image of the monomial program
// and of the potential's families (built by the host from GeneralEffective
// and GeneralPotential, in device memory).
constexpr int kGenMaxSym = 2 * kGenMaxP - 1;   // V_0..V_{2p-2}
constexpr int kGenMaxDepth = 16;               // deepest monomial (6 at p = 12, 9 at p = 18; checked by the host)

struct GeneralNode {
    unsigned char depth, sym;                  // depth in the trie, symbol j of V_j
    unsigned short count;                      // entries of this monomial
    int first;                                 // its first entry
};

struct GeneralDev {
    int J, K, n_nodes, n_entries, ng, ns, ne;
    const GeneralNode *nodes;                  // depth-first; node 0 = the constant monomial;
                                               // a node's entries are vs^0, vs^2, .. in order
    double poly_der[kGenMaxSym][9];            // V^(j) polynomial part: sum_i poly_der[j][i] x^(i-j)
    double gauss[4][4];                        // A, beta, c, sqrt(beta)
    double sech[4][3];                         // B, alpha, d
    double sech_scale[4][kGenMaxSym];          // B alpha^n (n+1)!
    double expo[4][3];                         // E, kappa, x0
    double inv[kGenMaxSym + 1];                // 1 / n
};

struct SamplerParams {
    // path: q_0 = a, q_N = b, N = 2^S, bisection widths sigma[n] (n = 1..S)
    double a, b;
    double sigma[SU_MAX_S + 1];
    int S;
    int F;                    // fine subtree depth, min(S, kMaxFine)
    int levels;               // sampled levels: S with the hierarchy, else 1
    // width-factor reweighting (Sec. 4.1 literal width): w_n += n_mid(n) lwf + hcoef * sum z^2
    int wf_on;
    double lwf, hcoef;
    // effective potential tables: row d (level n = S - d), M entries each
    int ring, ncol, M;
    int len[SU_MAX_P];
    int tab_global;           // 1: the level tables are read from global memory (too large to stage)
    int generic;              // 1: never the compiled-shape sampler (su_options.kernel = 1)
    double alpha;
    const void *tables;       // device, levels * M elements of the kernel's precision
    // Philox stream
    uint64_t seed;
    uint32_t instance;
    // work decomposition: items = (block b, chunk r), chunk = kThreads * rounds samples
    int64_t n_mc, sample0;
    int64_t n_blocks;
    int64_t items_per_block;
    int64_t n_items;          // items [item0, n_items) are this launch's (block ranges)
    int64_t item0;
    int rounds;
    // outputs
    double *partial;          // device: per item and level, (M, S, Q, n)
    double *w_out;            // device: per-sample mode when non-null, [sample][S]
    float *q_out;             // device: per-sample mode, single precision only: path points [sample][N+1] (or null)
    int *flags;               // device: bit 0 = non-finite weight seen
    const GeneralDev *general;  // device: RING_GENERAL only
};

// One instance of a batch: its path (a, b, N = 2^S, widths), its table
// shape (one per distinct level p), its tables (L rows of M entries from
// element tab: row d for level n = S - d), its samples and error blocks,
// the chunks each block is split into (work items), and where its tuples go.
struct BatchInstance {
    double a, b;
    int S, F;
    int L;                    // sampled levels: 1 (top level only) or S (hierarchy)
    int shape;                // index into BatchParams::shapes
    int64_t tab;              // first table element of this instance
    int64_t n_mc;             // samples
    int n_blocks, chunks;     // error blocks; work items per block
    int64_t tup;              // first tuple: [block][chunk][level], 4 doubles each
    double sigma[SU_MAX_S + 1];
};

// The Horner shape of one level p's tables (columns in x-bar^2, entries per
// column), or for the general potential its program (M = the program's entries).
struct BatchShape {
    int ncol, M;
    int len[SU_MAX_P];
    const GeneralDev *general;   // the general potential: this level's program (device), else null
};

// The batched kernel's parameters: the model fields of base (ring, alpha,
// seed, stream id, tables, flags) are shared by all instances; the
// per-instance fields of base are unused.
struct BatchParams {
    SamplerParams base;
    const BatchInstance *inst;
    const BatchShape *shapes;
    const int2 *items;        // (instance, block * chunks + chunk), costliest first
    int n_items;
    int S_max;
    int C_max;                // largest 2^(S - F): segment endpoints per path
    int L_max;                // most sampled levels of an instance
    int64_t tab_max;          // largest L * M: table elements staged per item
    double *tuples;           // per instance from its tup offset
    int *counter;             // work-queue head, zeroed before every launch
    int fixed_shape;          // >= 0: every item's instance has this compiled table shape (fixed_shapes.h)
    int fixed_src;            // ... which is shapes[fixed_src]
};

// dynamic shared memory the sampler needs
size_t sampler_smem_bytes(const SamplerParams &P, int precision);
// the compiled table shape the sampler launch of P runs with, or -1 (generic)
int sampler_fixed_shape(const SamplerParams &P, int precision);
// max resident CTAs per SM for the sampler (after opting in to its smem)
int sampler_occupancy(const SamplerParams &P, int precision, size_t smem);

// U[i * n + j] = exp(lognorm - (x_j - x_i)^2 / (2t) - t W_p) on the grid
// x_i = -L + i delta (evolution.cu); tab: the device table for eps = t
cudaError_t launch_evolution(const SamplerParams &P, int precision, const void *tab, double L, double delta, int n,
                             double t, double lognorm, double *U, cudaStream_t st);

// The upper band of the evolution operator, diagonal-major:
// D[k * pitch + i] = U_{i,i+k}, k = 0..w (evolution.cu)
cudaError_t launch_band(const SamplerParams &P, int precision, const void *tab, double L, double delta, int n,
                        double t, double lognorm, int w, int64_t pitch, double *D, cudaStream_t st);
// part[split][i][c] = partial sums of (U X)[i][c] over the split's diagonals, B in {1, 8, 16, 32}
cudaError_t launch_band_matvec(int B, const double *D, int64_t pitch, int n, int w, int splits, const double *X,
                               double *part, cudaStream_t st);
// Ynew = alpha * sum_split part + beta * Ycur + gamma * Yprev (nb = n * B elements)
cudaError_t launch_cheb(const double *part, int splits, int64_t nb, const double *Ycur, const double *Yprev,
                        double *Ynew, double alpha, double beta, double gamma, cudaStream_t st);
// op 0: out[chunk][B][B] = A^T C over the chunk's rows; op 1: out = A Q (Q: B x B);
// op 2: out[chunk][B] = sum (A - Q[c] C)^2 over the chunk's rows (Q: B Ritz values)
cudaError_t launch_block_op(int op, int B, const double *A, const double *C, const double *Q, int n, int chunks,
                            double *out, cudaStream_t st);
// vec[k n + i] = scale X[i][k], k < nev
cudaError_t launch_vectors(int B, const double *X, int n, int nev, double scale, double *vec, cudaStream_t st);

// Systems of d = D x M coordinates (Sec. 2.2): one bisection path per
// thread, every coordinate an exact Brownian bridge (coordinate c of heap
// midpoint j takes normal j D + c of the sample's stream), built and weighed
// in segments of 2^kNdSeg slices (segment endpoints in a global scratch, one
// segment's points in local memory); W(x, xb; eps) per slice from the monomial program of
// NdEffective (nodes as GeneralNode; entries = powers of z_H), several
// slices at a time (two in double, eight in single precision); weights and
// per-item tuples as the one-dimensional sampler's.
constexpr int kNdSeg = 5;     // the several-coordinates path in segments of 2^5 slices
struct NdParams {
    SamplerParams base;       // S, levels, tables (per level, global), M, sigma, stream, items, outputs
    int D, H, G, n_nodes;     // Horner in z_H^G
    const GeneralNode *nodes; // device
    double a[kNdMaxDim], b[kNdMaxDim];
    void *paths;              // device (double or float): segment endpoint i, coordinate c of slot t
                              // at [(i D + c) pstride + t]
    int64_t pstride;          // slots = grid x kThreads
};
size_t nd_smem_bytes(const NdParams &Q, int precision);
int nd_occupancy(const NdParams &Q, int precision, size_t smem);
cudaError_t launch_nd(const NdParams &Q, int precision, int grid, size_t smem, cudaStream_t st);

cudaError_t launch_sampler(const SamplerParams &P, int precision, int grid, size_t smem,
                           cudaStream_t st);
size_t batch_smem_bytes(const BatchParams &B, int precision);
int batch_occupancy(const BatchParams &B, int precision, size_t smem);
const void *batch_fn(const BatchParams &B, int precision);
// tuples of blocks [b0, b0 + n_blocks) from their items' partial tuples
cudaError_t launch_combine(const double *partial, double *tuples, int64_t b0, int64_t n_blocks, int levels,
                           int64_t items_per_block, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, uint32_t instance, int64_t sample0, int64_t n_samples,
                           int n_normals, int precision, double *out, cudaStream_t st);
cudaError_t launch_philox_words(uint64_t seed, uint32_t instance, int64_t sample0,
                                int64_t n_samples, int n_calls, uint32_t *out, cudaStream_t st);

}  // namespace su
