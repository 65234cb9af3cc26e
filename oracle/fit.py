"""The continuum estimate of Sec. 4 (Eq. fit) from one run's levels (oracle
side).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

One run of the estimator gives A_N^(p) for N = 2^n, n = 0..s.  The paper
fits them with

    A_N^(p) = A^(p) + B^(p) / N^p + C^(p+1) / N^(p+1) + ...

and reads the constant as the continuum amplitude.  Reading C-9: the fit
uses the levels n_min..s, the first `n_terms` terms of the series (2: A and
B; 3: A, B and C), weights 1/err_n^2 (the levels' statistical errors), and
ordinary weighted least squares (the normal equations in exact rationals);
the error of A is the square root of its diagonal entry of (X^T W X)^-1 (levels from one run share samples, so this
treats them as independent), and chi^2 is the weighted residual sum.
"""
from __future__ import annotations

from fractions import Fraction
import math


def _solve(G, h):
    """Gauss-Jordan elimination in exact rationals: (G^-1 h, G^-1)."""
    k = len(G)
    M = [list(G[i]) + list(h[i:i + 1]) + [Fraction(int(i == j)) for j in range(k)] for i in range(k)]
    for c in range(k):
        piv = next(r for r in range(c, k) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        f = M[c][c]
        M[c] = [v / f for v in M[c]]
        for r in range(k):
            if r != c and M[r][c] != 0:
                g = M[r][c]
                M[r] = [a - g * b for a, b in zip(M[r], M[c])]
    return [M[i][k] for i in range(k)], [M[i][k + 1:] for i in range(k)]


def fit_continuum(amps, errs, p, n_min=1, n_terms=3):
    """(A, A_err, chi2) from amps[n], errs[n], n = 0..s: the normal equations
    X^T W X beta = X^T W y solved exactly (every double is a rational), so
    that the reference holds however ill-conditioned the columns N^-p are."""
    amps = [Fraction(float(v)) for v in amps]
    errs = [Fraction(float(v)) for v in errs]
    s = len(amps) - 1
    ns = list(range(n_min, s + 1))
    if len(ns) < n_terms:
        raise ValueError("fewer levels than fit terms")
    rows = []
    for n in ns:
        x = [Fraction(1), Fraction(1, 2 ** (p * n))]
        if n_terms == 3:
            x.append(Fraction(1, 2 ** ((p + 1) * n)))
        rows.append((x, 1 / errs[n] ** 2, amps[n]))
    G = [[sum(w * x[i] * x[j] for x, w, _ in rows) for j in range(n_terms)] for i in range(n_terms)]
    h = [sum(w * x[i] * y for x, w, y in rows) for i in range(n_terms)]
    beta, cov = _solve(G, h)
    chi2 = sum(w * (y - sum(b * xi for b, xi in zip(beta, x))) ** 2 for x, w, y in rows)
    return float(beta[0]), math.sqrt(float(cov[0][0])), float(chi2)
