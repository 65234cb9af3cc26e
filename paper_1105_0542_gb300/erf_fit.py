"""Writes csrc/erf_poly.h: the odd polynomial erf(v/sqrt 2) ~ v Q(v^2) on
|v| <= 3 sqrt 2 used by the proposal network's GELU epilogue (exact-erf GELU
v (1 + erf(v/sqrt 2))/2, evaluated with fused multiply-adds on pairs of
values).

Method: least squares on 6000 Chebyshev points of [0, 3 sqrt 2] (the
near-minimax Chebyshev fit; Cheney, "Introduction to Approximation Theory",
ch. 3), in the scaled variable y = v/(3 sqrt 2) (a well-conditioned basis),
then rescaled to powers of v.  Beyond |v| = 3 sqrt 2 the argument is
clamped: 1 - erf(3) = 2.2e-5.  The largest error, about 1e-4, is far below
the bfloat16 rounding (2^-9) of the activations the epilogue writes.  Run
from the repository root:
    python paper_1105_0542_gb300/erf_fit.py
"""
import math
import os

import numpy as np
from scipy.special import erf

VMAX, DEG = 3.0 * math.sqrt(2.0), 7      # v Q(v^2), Q of degree 7 in v^2: eight coefficients


def fit():
    v = np.cos(np.linspace(0.0, np.pi, 6000)) * VMAX / 2 + VMAX / 2
    y = v / VMAX
    A = np.stack([y ** (2 * k + 1) for k in range(DEG + 1)], axis=1)
    c, *_ = np.linalg.lstsq(A, erf(v / math.sqrt(2.0)), rcond=None)
    return [float(c[k] / VMAX ** (2 * k + 1)) for k in range(DEG + 1)]


def main():
    cx = fit()
    here = os.path.dirname(os.path.abspath(__file__))
    lines = ["// erf(v/sqrt 2) ~ v Q(v^2) for |v| <= 3 sqrt 2 (v clamped beyond): the",
             "// coefficients of Q, constant term first, from paper_1105_0542_gb300/erf_fit.py",
             "// (least squares on Chebyshev points; largest error about 1e-4 with float",
             "// Horner evaluation).",
             "#pragma once",
             "",
             "namespace su {",
             "namespace mlp {",
             f"constexpr float kErfClamp = {VMAX:.7f}f;",
             f"constexpr int kErfTerms = {DEG + 1};",
             "// coefficient k of Q (a constant expression, usable in device code)",
             "__host__ __device__ constexpr float erf_poly(int k) {",
             "    return " + " :\n           ".join(f"k == {k} ? {v:.9e}f" for k, v in enumerate(cx[:-1]))
             + f" :\n           {cx[-1]:.9e}f;",
             "}"]
    lines += ["}  // namespace mlp", "}  // namespace su", ""]
    with open(os.path.join(here, "csrc", "erf_poly.h"), "w") as f:
        f.write("\n".join(lines))
    print("\n".join(lines))


if __name__ == "__main__":
    main()
