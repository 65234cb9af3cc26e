// Host driver of the band eigensolver of the evolution operator (internal).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace su {

struct SpectrumResult {
    std::vector<double> theta;   // the nev largest Ritz values, descending
    std::vector<double> resid;   // |U x_k - theta_k x_k| of their unit Ritz vectors
    double lower = 0, upper = 0; // spectrum bounds from the Lanczos steps
    int iterations = 0;          // filter + Rayleigh-Ritz rounds after the first
    int block = 0;               // columns of the block
    int converged = 0;           // every residual <= tol * theta_0
    int64_t matvecs = 0;         // vector products with U
    int block_matvecs = 0;       // block products U X (B columns each)
    double block_matvec_ms = 0;  // their device time
};

// The nev largest eigenvalues of the symmetric band matrix whose upper band
// is D[k * pitch + i] = U_{i,i+k} (k = 0..w, device, double).  degree: the
// Chebyshev filter's degree; tol: residual tolerance relative to theta_0;
// max_iter: filter rounds; seed: the random start block; d_vectors (device,
// n * nev, may be null): scale * Ritz vector k at d_vectors[k * n + i].
// Returns SU_OK (res.converged says whether tol was met), SU_EINVAL,
// SU_ENOMEM or SU_ECUDA with a message in err.
int band_spectrum(const double *D, int64_t pitch, int n, int w, int nev, int degree, double tol, int max_iter,
                  uint64_t seed, double *d_vectors, double vec_scale, cudaStream_t st, SpectrumResult &res,
                  std::string &err);

}  // namespace su
