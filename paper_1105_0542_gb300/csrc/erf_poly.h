// erf(v/sqrt 2) ~ v Q(v^2) for |v| <= 3 sqrt 2 (v clamped beyond): the
// coefficients of Q, constant term first, from paper_1105_0542_gb300/erf_fit.py
// (least squares on Chebyshev points; largest error about 1e-4 with float
// Horner evaluation).
#pragma once

namespace su {
namespace mlp {
constexpr float kErfClamp = 4.2426407f;
constexpr int kErfTerms = 8;
// coefficient k of Q (a constant expression, usable in device code)
__host__ __device__ constexpr float erf_poly(int k) {
    return k == 0 ? 7.975821720e-01f :
           k == 1 ? -1.319999921e-01f :
           k == 2 ? 1.905591245e-02f :
           k == 3 ? -2.006924355e-03f :
           k == 4 ? 1.467288699e-04f :
           k == 5 ? -6.946592044e-06f :
           k == 6 ? 1.891344503e-07f :
           -2.230359241e-09f;
}
}  // namespace mlp
}  // namespace su
