"""Pins of the oracle's continuum fit (Eq. fit, Sec. 4), CPU only:

* exact series data A + B/N^p + C/N^(p+1) are fitted exactly (any weights);
* the harmonic oscillator's exact discretized amplitudes (Gaussian
  integrals) extrapolate to the Mehler continuum value far more closely than
  the best level itself;
* the error of A is the least-squares standard error: for two terms and
  equal errors it matches the closed form of a straight-line fit in 1/N^p.
"""
import math

import numpy as np
import pytest

from oracle import exact
from oracle import fit


@pytest.mark.parametrize("p,n_terms", [(1, 2), (2, 3), (4, 3), (10, 2)])
def test_exact_series_are_recovered(p, n_terms):
    s = 10
    N = 2.0 ** np.arange(s + 1)
    A, B, C = 0.3, 0.7, -0.2 if n_terms == 3 else 0.0
    amps = A + B / N ** p + C / N ** (p + 1)
    errs = np.linspace(1e-4, 3e-4, s + 1)
    a, da, chi2 = fit.fit_continuum(amps, errs, p, n_min=1, n_terms=n_terms)
    assert a == pytest.approx(A, rel=1e-12, abs=1e-13)
    assert chi2 <= 1e-12


@pytest.mark.parametrize("p", [1, 2, 4])
def test_harmonic_oscillator_extrapolates_to_the_mehler_kernel(p):
    """Levels up to N = 32, not yet converged: the fit's constant lands two
    to three orders of magnitude closer to the continuum than the last level
    (the neglected N^-(p+2) terms remain)."""
    s = 5
    amps = np.array([exact.ho_discretized(p, 2 ** n, 0.0, 1.0, 1.0) for n in range(s + 1)])
    ref = exact.mehler(0.0, 1.0, 1.0)
    errs = np.full(s + 1, 1e-6)
    a, _, _ = fit.fit_continuum(amps, errs, p, n_min=2, n_terms=3)
    assert abs(a - ref) < 0.02 * abs(amps[s] - ref)


def test_standard_error_of_a_straight_line_fit():
    p, s = 2, 6
    n = np.arange(1, s + 1)
    x = 2.0 ** (-p * n)
    sig = 1e-3
    amps = np.concatenate([[0.0], 1.0 + 0.5 * x])
    errs = np.full(s + 1, sig)
    _, da, _ = fit.fit_continuum(amps, errs, p, n_min=1, n_terms=2)
    # intercept of y = a + b x with equal errors: sig^2 sum x^2 / (n sum x^2 - (sum x)^2)
    ref = sig * math.sqrt(np.sum(x * x) / (len(x) * np.sum(x * x) - np.sum(x) ** 2))
    assert da == pytest.approx(ref, rel=1e-12)
