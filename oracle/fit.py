"""The continuum estimate of Sec. 4 (Eq. fit) from one run's levels (oracle
side).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

One run of the estimator gives A_N^(p) for N = 2^n, n = 0..s.  The paper
fits them with

    A_N^(p) = A^(p) + B^(p) / N^p + C^(p+1) / N^(p+1) + ...

and reads the constant as the continuum amplitude.  Reading C-9: the fit
uses the levels n_min..s, the first `n_terms` terms of the series (2: A and
B; 3: A, B and C), weights 1/err_n^2 (the levels' statistical errors), and
ordinary weighted least squares; the error of A is the square root of its
diagonal entry of (X^T W X)^-1 (levels from one run share samples, so this
treats them as independent), and chi^2 is the weighted residual sum.
"""
from __future__ import annotations

import numpy as np


def fit_continuum(amps, errs, p, n_min=1, n_terms=3):
    """(A, A_err, chi2) from amps[n], errs[n], n = 0..s."""
    amps = np.asarray(amps, dtype=np.float64)
    errs = np.asarray(errs, dtype=np.float64)
    s = len(amps) - 1
    n = np.arange(n_min, s + 1)
    if len(n) < n_terms:
        raise ValueError("fewer levels than fit terms")
    N = 2.0 ** n
    cols = [np.ones_like(N), N ** (-float(p))]
    if n_terms == 3:
        cols.append(N ** (-float(p + 1)))
    X = np.stack(cols, axis=1)
    w = 1.0 / errs[n] ** 2
    XtW = X.T * w
    cov = np.linalg.inv(XtW @ X)
    beta = cov @ (XtW @ amps[n])
    r = amps[n] - X @ beta
    return float(beta[0]), float(np.sqrt(cov[0, 0])), float(np.sum(w * r * r))
