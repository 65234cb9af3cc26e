// The lowest energies of the space-discretized evolution operator (Sec. 5,
// Fig. 3): the largest eigenvalues lambda_k = exp(-t E_k) of the symmetric
// band matrix U, from its upper band in diagonal-major storage
// (D[k * pitch + i] = U_{i,i+k}, k = 0..w), by Chebyshev-filtered block
// subspace iteration with Rayleigh-Ritz (Zhou and Saad, "A Chebyshev-Davidson
// algorithm"/"Self-consistent-field calculations using Chebyshev-filtered
// subspace iteration", 2006-2007), all in double precision:
//
//   bounds   a few Lanczos steps (Lanczos 1950) give the lower end lo of the
//            spectrum (smallest Ritz value minus the last off-diagonal);
//   filter   Y = T_m((U - c)/e) X with the interval [lo, cut] mapped onto
//            [-1, 1] (c = (cut + lo)/2, e = (cut - lo)/2), cut = the
//            smallest Ritz value of the block: components above cut grow
//            like T_m of their mapped value, the rest stay bounded;
//   basis    shifted Cholesky QR followed by two plain passes (Fukaya,
//            Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020) on the
//            column-scaled Gram matrix;
//   Ritz     H = Y^T U Y, its eigenpairs by cyclic Jacobi rotations (Golub
//            and Van Loan, Sec. 8.5), X = Y Q, residuals |U x_k - theta_k x_k|.
//
// The block width (8, 16 or 32 columns) holds nev wanted pairs plus at least
// six guard vectors, so nearly degenerate pairs (a tunnelling doublet) sit
// inside the block and are separated by the Rayleigh-Ritz step, not by the
// filter.  Device work: the band matrix-block product (FP64 FMA bound,
// 2B multiply-adds per stored element and row), the Chebyshev update, Gram
// products and rotations; host work: B x B Cholesky and Jacobi.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sampler.h"
#include "spectrum.h"

namespace su {
namespace {

// symmetric eigenpairs of the k x k matrix A (row-major) by cyclic Jacobi
// rotations; eigenvalues descending in ev, eigenvectors in the columns of V
void jacobi_eig(std::vector<double> A, int k, std::vector<double> &ev, std::vector<double> &V) {
    V.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) V[(size_t)i * k + i] = 1.0;
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * k + j]; };
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                tot += a(i, j) * a(i, j);
                if (i != j) off += a(i, j) * a(i, j);
            }
        if (off <= 1e-34 * tot || off == 0.0) break;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = a(p, q);
                if (apq == 0.0) continue;
                // rotation that annihilates a(p, q): tan(phi) = t, t the smaller root
                const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {   // A <- A J (columns p, q)
                    const double arp = a(r, p), arq = a(r, q);
                    a(r, p) = c * arp - s * arq;
                    a(r, q) = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {   // A <- J^T A (rows p, q)
                    const double apr = a(p, r), aqr = a(q, r);
                    a(p, r) = c * apr - s * aqr;
                    a(q, r) = s * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {   // V <- V J
                    const double vrp = V[(size_t)r * k + p], vrq = V[(size_t)r * k + q];
                    V[(size_t)r * k + p] = c * vrp - s * vrq;
                    V[(size_t)r * k + q] = s * vrp + c * vrq;
                }
            }
    }
    std::vector<int> ord((size_t)k);
    for (int i = 0; i < k; ++i) ord[(size_t)i] = i;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return a(x, x) > a(y, y); });
    ev.resize((size_t)k);
    std::vector<double> W((size_t)k * k);
    for (int c = 0; c < k; ++c) {
        ev[(size_t)c] = a(ord[(size_t)c], ord[(size_t)c]);
        for (int r = 0; r < k; ++r) W[(size_t)r * k + c] = V[(size_t)r * k + ord[(size_t)c]];
    }
    V.swap(W);
}

// lower Cholesky factor of the k x k matrix G (row-major); false if not
// positive definite
bool cholesky(const std::vector<double> &G, int k, std::vector<double> &Lf) {
    Lf.assign((size_t)k * k, 0.0);
    for (int j = 0; j < k; ++j) {
        double d = G[(size_t)j * k + j];
        for (int r = 0; r < j; ++r) d -= Lf[(size_t)j * k + r] * Lf[(size_t)j * k + r];
        if (!(d > 0.0)) return false;
        const double l = std::sqrt(d);
        Lf[(size_t)j * k + j] = l;
        for (int i = j + 1; i < k; ++i) {
            double s = G[(size_t)i * k + j];
            for (int r = 0; r < j; ++r) s -= Lf[(size_t)i * k + r] * Lf[(size_t)j * k + r];
            Lf[(size_t)i * k + j] = s / l;
        }
    }
    return true;
}

// (L^T)^{-1}: the inverse of the upper factor R = L^T, row-major
std::vector<double> inverse_upper(const std::vector<double> &Lf, int k) {
    std::vector<double> X((size_t)k * k, 0.0);   // X = R^{-1}, R[i][j] = L[j][i]
    for (int c = 0; c < k; ++c) {
        // solve R x = e_c by back substitution
        for (int i = k - 1; i >= 0; --i) {
            double s = i == c ? 1.0 : 0.0;
            for (int j = i + 1; j < k; ++j) s -= Lf[(size_t)j * k + i] * X[(size_t)j * k + c];
            X[(size_t)i * k + c] = s / Lf[(size_t)i * k + i];
        }
    }
    return X;
}

struct Work {
    double *D = nullptr;
    int64_t pitch = 0;
    int n = 0, w = 0, B = 0, splits = 1, chunks = 1;
    cudaStream_t st = nullptr;
    double *part = nullptr;      // splits x n x B
    double *gpart = nullptr;     // chunks x B x B
    double *dQ = nullptr;        // B x B (or B values)
    std::vector<double> hpart;
    int64_t matvecs = 0;         // vector products with U
    std::vector<cudaEvent_t> ev; // pairs around the block products (their device time)
    ~Work() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

#define SPC(call)                               \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

// part = the split partial sums of U X; block products (B = W.B) are
// bracketed by a pair of events for their device time
cudaError_t matvec(Work &W, int B, const double *X) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (B == W.B) {
        SPC(cudaEventCreate(&e0));
        W.ev.push_back(e0);
        SPC(cudaEventCreate(&e1));
        W.ev.push_back(e1);
        SPC(cudaEventRecord(e0, W.st));
    }
    SPC(launch_band_matvec(B, W.D, W.pitch, W.n, W.w, W.splits, X, W.part, W.st));
    if (e1) SPC(cudaEventRecord(e1, W.st));
    return cudaSuccess;
}

// Y = U X (block of W.B columns, or one column with B = 1)
cudaError_t apply(Work &W, int B, const double *X, double *Y) {
    SPC(matvec(W, B, X));
    SPC(launch_cheb(W.part, W.splits, (int64_t)W.n * B, nullptr, nullptr, Y, 1.0, 0.0, 0.0, W.st));
    W.matvecs += B;
    return cudaSuccess;
}

// G = A^T C (B x B, row-major), the chunks summed in order on the host
cudaError_t gram(Work &W, const double *A, const double *C, std::vector<double> &G) {
    const int B = W.B;
    SPC(launch_block_op(0, B, A, C, nullptr, W.n, W.chunks, W.gpart, W.st));
    W.hpart.resize((size_t)W.chunks * B * B);
    SPC(cudaMemcpyAsync(W.hpart.data(), W.gpart, W.hpart.size() * sizeof(double), cudaMemcpyDeviceToHost, W.st));
    SPC(cudaStreamSynchronize(W.st));
    G.assign((size_t)B * B, 0.0);
    for (int q = 0; q < W.chunks; ++q)
        for (int e = 0; e < B * B; ++e) G[(size_t)e] += W.hpart[(size_t)q * B * B + e];
    return cudaSuccess;
}

// out = A Q for a host B x B matrix Q
cudaError_t rotate(Work &W, const double *A, const std::vector<double> &Q, double *out) {
    SPC(cudaMemcpyAsync(W.dQ, Q.data(), Q.size() * sizeof(double), cudaMemcpyHostToDevice, W.st));
    SPC(launch_block_op(1, W.B, A, nullptr, W.dQ, W.n, W.chunks, out, W.st));
    // the host copy of Q must outlive the copy
    return cudaStreamSynchronize(W.st);
}

// orthonormal basis of the columns of Y into out: column scaling, one
// shifted Cholesky QR pass and two plain ones.  Returns false (in ok) when
// the block has lost rank.
cudaError_t orthonormalize(Work &W, const double *Y, double *tmp, double *out, bool &ok) {
    const int B = W.B;
    std::vector<double> G, Lf;
    SPC(gram(W, Y, Y, G));
    std::vector<double> dsc((size_t)B);
    for (int c = 0; c < B; ++c) dsc[(size_t)c] = G[(size_t)c * B + c] > 0 ? 1.0 / std::sqrt(G[(size_t)c * B + c]) : 0.0;
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) G[(size_t)i * B + j] *= dsc[(size_t)i] * dsc[(size_t)j];
    double tr = 0.0;
    for (int c = 0; c < B; ++c) tr += G[(size_t)c * B + c];
    const double shift = 11.0 * ((double)W.n * B + (double)B * (B + 1)) * 0x1p-53 * tr;
    for (int c = 0; c < B; ++c) G[(size_t)c * B + c] += shift;
    ok = cholesky(G, B, Lf);
    if (!ok) return cudaSuccess;
    std::vector<double> Q = inverse_upper(Lf, B);
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) Q[(size_t)i * B + j] *= dsc[(size_t)i];
    SPC(rotate(W, Y, Q, out));
    for (int pass = 0; pass < 2; ++pass) {
        SPC(gram(W, out, out, G));
        ok = cholesky(G, B, Lf);
        if (!ok) return cudaSuccess;
        Q = inverse_upper(Lf, B);
        SPC(rotate(W, out, Q, tmp));
        SPC(cudaMemcpyAsync(out, tmp, (size_t)W.n * B * sizeof(double), cudaMemcpyDeviceToDevice, W.st));
    }
    return cudaSuccess;
}

}  // namespace

int band_spectrum(const double *D, int64_t pitch, int n, int w, int nev, int degree, double tol, int max_iter,
                  uint64_t seed, double *d_vectors, double vec_scale, cudaStream_t st, SpectrumResult &res,
                  std::string &err) {
    res = SpectrumResult{};
    const int B = nev + 6 <= 8 ? 8 : nev + 6 <= 16 ? 16 : 32;
    if (nev < 1 || nev + 6 > 32 || nev > n / 2) {
        err = "nev must be in 1..26 and at most n/2";
        return SU_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    Work W;
    W.D = const_cast<double *>(D);
    W.pitch = pitch;
    W.n = n;
    W.w = w;
    W.B = B;
    W.st = st;
    const int rblocks = (n + 63) / 64;
    // split the diagonals so that about 32 CTAs of two warps per SM are
    // resident: the FP64 multiply-adds need the warps to hide load latency
    W.splits = std::max(1, std::min(w + 1, (32 * std::max(sms, 1) + rblocks - 1) / rblocks));
    W.chunks = std::max(1, std::min(std::max(sms, 1), (n + 31) / 32));
    struct Bufs {
        std::vector<void *> v;
        ~Bufs() {
            for (void *p : v) cudaFree(p);
        }
        cudaError_t get(double **p, size_t count) {
            void *q = nullptr;
            cudaError_t e = cudaMalloc(&q, count * sizeof(double));
            if (e == cudaSuccess) v.push_back(q);
            *p = static_cast<double *>(q);
            return e;
        }
    } bufs;
    const size_t nb = (size_t)n * B;
    double *X, *Y0, *Y1, *Y2, *Z, *UX, *T;
    cudaError_t e = cudaSuccess;
    for (double **p : {&X, &Y0, &Y1, &Y2, &Z, &UX, &T})
        if (e == cudaSuccess) e = bufs.get(p, nb);
    if (e == cudaSuccess) e = bufs.get(&W.part, (size_t)W.splits * nb);
    if (e == cudaSuccess) e = bufs.get(&W.gpart, (size_t)W.chunks * B * B);
    if (e == cudaSuccess) e = bufs.get(&W.dQ, (size_t)B * B);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = std::string("eigensolver buffers: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SU_ENOMEM : SU_ECUDA;
    }
    auto cuda_err = [&](cudaError_t c, const char *what) {
        err = std::string(what) + ": " + cudaGetErrorString(c);
        cudaGetLastError();
        return SU_ECUDA;
    };

    // ---- the lower end of the spectrum: Lanczos steps on one vector
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    {
        const int steps = std::min(40, n);
        std::vector<double> v((size_t)n), vp((size_t)n, 0.0), wv((size_t)n), al, be;
        double nrm = 0;
        for (double &x : v) {
            x = nd(rng);
            nrm += x * x;
        }
        nrm = std::sqrt(nrm);
        for (double &x : v) x /= nrm;
        double beta = 0.0;
        for (int j = 0; j < steps; ++j) {
            if ((e = cudaMemcpyAsync(X, v.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st)) ||
                (e = apply(W, 1, X, Y0)) ||
                (e = cudaMemcpyAsync(wv.data(), Y0, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st)))
                return cuda_err(e, "Lanczos bounds");
            double a = 0;
            for (int i = 0; i < n; ++i) a += v[(size_t)i] * wv[(size_t)i];
            double b2 = 0;
            for (int i = 0; i < n; ++i) {
                wv[(size_t)i] -= a * v[(size_t)i] + beta * vp[(size_t)i];
                b2 += wv[(size_t)i] * wv[(size_t)i];
            }
            al.push_back(a);
            beta = std::sqrt(b2);
            be.push_back(beta);
            if (!(beta > 0)) break;
            vp = v;
            for (int i = 0; i < n; ++i) v[(size_t)i] = wv[(size_t)i] / beta;
        }
        const int k = (int)al.size();
        std::vector<double> Tm((size_t)k * k, 0.0), ev, V;
        for (int i = 0; i < k; ++i) {
            Tm[(size_t)i * k + i] = al[(size_t)i];
            if (i + 1 < k) Tm[(size_t)i * k + i + 1] = Tm[(size_t)(i + 1) * k + i] = be[(size_t)i];
        }
        jacobi_eig(Tm, k, ev, V);
        res.upper = ev.front() + be.back();
        res.lower = ev.back() - be.back();
    }
    const double lo = res.lower;

    // ---- a random block, orthonormalized, and its Rayleigh-Ritz pairs
    std::vector<double> h(nb);
    for (double &x : h) x = nd(rng);
    if ((e = cudaMemcpyAsync(Y0, h.data(), nb * sizeof(double), cudaMemcpyHostToDevice, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_err(e, "initial block");
    std::vector<double> theta((size_t)B, 0.0), H, Q, r((size_t)B);
    const double *src = Y0;
    for (int it = 0; it <= max_iter; ++it) {
        bool ok = true;
        if ((e = orthonormalize(W, src, T, X, ok))) return cuda_err(e, "orthonormalization");
        if (!ok) {
            err = "the block lost rank (Cholesky QR failed)";
            return SU_ECUDA;
        }
        if ((e = apply(W, B, X, Z)) || (e = gram(W, X, Z, H))) return cuda_err(e, "Rayleigh-Ritz");
        for (int i = 0; i < B; ++i)   // symmetrize the projection's rounding
            for (int j = i + 1; j < B; ++j)
                H[(size_t)i * B + j] = H[(size_t)j * B + i] = 0.5 * (H[(size_t)i * B + j] + H[(size_t)j * B + i]);
        jacobi_eig(H, B, theta, Q);
        if ((e = rotate(W, X, Q, Y1)) || (e = rotate(W, Z, Q, UX))) return cuda_err(e, "Ritz vectors");
        std::swap(X, Y1);
        // residual norms of the Ritz pairs
        if ((e = cudaMemcpyAsync(W.dQ, theta.data(), (size_t)B * sizeof(double), cudaMemcpyHostToDevice, st)) ||
            (e = launch_block_op(2, B, UX, X, W.dQ, n, W.chunks, W.gpart, st)))
            return cuda_err(e, "residuals");
        std::vector<double> rp((size_t)W.chunks * B);
        if ((e = cudaMemcpyAsync(rp.data(), W.gpart, rp.size() * sizeof(double), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))
            return cuda_err(e, "residuals");
        double worst = 0.0;
        for (int c = 0; c < B; ++c) {
            double s = 0;
            for (int q = 0; q < W.chunks; ++q) s += rp[(size_t)q * B + c];
            r[(size_t)c] = std::sqrt(s);
            if (c < nev) worst = std::max(worst, r[(size_t)c]);
        }
        res.iterations = it;
        res.converged = worst <= tol * std::fabs(theta[0]) ? 1 : 0;
        if (res.converged || it == max_iter) break;
        // ---- filter: Y = T_m((U - c)/e) X on the interval [lo, cut]
        double cut = theta[(size_t)B - 1];
        cut = std::max(cut, lo + 1e-3 * (theta[0] - lo));
        const double c0 = 0.5 * (cut + lo), e0 = 0.5 * (cut - lo);
        const int m = it == 0 ? std::min(4, degree) : degree;
        double *ym1 = X, *y = Y0, *yp = Y1;
        if ((e = matvec(W, B, X)) ||
            (e = launch_cheb(W.part, W.splits, (int64_t)nb, X, nullptr, Y0, 1.0 / e0, -c0 / e0, 0.0, st)))
            return cuda_err(e, "filter");
        W.matvecs += B;
        for (int j = 1; j < m; ++j) {
            if ((e = matvec(W, B, y)) ||
                (e = launch_cheb(W.part, W.splits, (int64_t)nb, y, ym1, yp, 2.0 / e0, -2.0 * c0 / e0, -1.0, st)))
                return cuda_err(e, "filter");
            W.matvecs += B;
            // rotate the three buffers: the oldest becomes the next output
            double *old = ym1;
            ym1 = y;
            y = yp;
            yp = old == X ? Y2 : old;
        }
        src = y;
        if (src == X) {   // cannot happen for m >= 1; keep the orthonormalizer's output separate
            err = "internal: filter output aliases the basis";
            return SU_ECUDA;
        }
    }
    res.theta.assign(theta.begin(), theta.begin() + nev);
    res.resid.assign(r.begin(), r.begin() + nev);
    res.block = B;
    res.matvecs = W.matvecs;
    if ((e = cudaStreamSynchronize(st))) return cuda_err(e, "eigensolver");
    for (size_t q = 0; q + 1 < W.ev.size(); q += 2) {
        float ms = 0;
        if ((e = cudaEventElapsedTime(&ms, W.ev[q], W.ev[q + 1]))) return cuda_err(e, "event time");
        res.block_matvec_ms += ms;
        ++res.block_matvecs;
    }
    if (d_vectors) {
        if ((e = launch_vectors(B, X, n, nev, vec_scale, d_vectors, st)) || (e = cudaStreamSynchronize(st)))
            return cuda_err(e, "eigenvectors");
    }
    return SU_OK;
}

}  // namespace su
