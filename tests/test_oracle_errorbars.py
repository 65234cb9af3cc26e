"""Pins of the oracle's error bars (``mc.estimate``: ``err`` and ``err_naive``).

Every 3-sigma test, the GPU error parity and every time-to-1e-4 figure rest on
these two numbers, so they are checked against exact values, not against a
restatement of their formulas.

For the harmonic oscillator W_p is a quadratic form in (x, xb), so under the
bisection bridge (Sec. 4.1) every moment of the per-sample factor X = exp(w),
w = -eps sum_k W_p, is a Gaussian integral of the same kind as A_N^(p)
itself (Eq. SNp):

    E[X^k] = A_N^(p)[k W_p] / A_free,

computed in 40-digit arithmetic by ``exact.ho_discretized(w_scale=k)``.  That
gives the exact per-sample variance sigma^2 = E[X^2] - E[X]^2 and the fourth
central moment, hence the exact standard error of the mean, sigma / sqrt(n),
and the sampling spread of any estimate of it:

* ``err_naive`` (the <f^2> - <f>^2 error of Sec. 4.1) from one large run: its
  square times n is a variance estimate whose standard error follows from
  the fourth moment;
* ``err`` (standard deviation of block means / sqrt(n_blocks), reading C-5)
  over hundreds of independent runs: with two blocks its square is a chi^2_1
  variable of mean sigma^2 / n, so the mean of err^2 over R runs is known to
  within sqrt(2 / R) -- a ddof = 0 formula halves it, a missing
  1/sqrt(n_blocks) doubles it;
* the z-scores (amp - A_N) / err of many runs with ten blocks follow a
  Student t with nine degrees of freedom: E[z^2] = 9/7.

A_N itself is the exact discretized amplitude, so these runs also re-check
that the estimate is unbiased.
"""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import exact, mc

OMEGA, A, B, T, P, S = 2.0, 0.0, 1.0, 1.0, 4, 4


def _moments(N):
    """(m1, sigma^2, mu4): the mean, variance and fourth central moment of
    X = exp(w) at N = 2^n slices, exactly."""
    af = mp.exp(mp.mpf(mc.log_A_free(A, B, T)))
    m = [exact.ho_discretized(P, N, A, B, T, omega=OMEGA, as_mp=True, w_scale=k) / af for k in (1, 2, 3, 4)]
    var = m[1] - m[0] ** 2
    mu4 = m[3] - 4 * m[0] * m[2] + 6 * m[0] ** 2 * m[1] - 3 * m[0] ** 4
    return float(m[0]), float(var), float(mu4)


@pytest.fixture(scope="module")
def weights():
    o = mc.Oracle("ho", [OMEGA], P)
    w, _ = o.logweights(A, B, T, S, 20240, 400_000, threads=4)
    return o, w


def test_moments_are_consistent():
    """The moment integrals themselves: E[X] is the amplitude ratio the
    estimator targets, and the variance is positive and below E[X^2]."""
    for n in range(1, S + 1):
        m1, var, mu4 = _moments(2 ** n)
        ref = exact.ho_discretized(P, 2 ** n, A, B, T, omega=OMEGA) / math.exp(mc.log_A_free(A, B, T))
        assert m1 == pytest.approx(ref, rel=1e-13)
        assert 0 < var < m1 * m1 + var and mu4 > var * var


def test_err_naive_is_the_exact_standard_error(weights):
    o, w = weights
    n = w.shape[0]
    res = mc.estimate(w, o.level0(A, B, T), A, B, T, 64)
    scale = math.exp(mc.log_A_free(A, B, T))
    for lev in range(1, S + 1):
        m1, var, mu4 = _moments(2 ** lev)
        got = (res[lev]["err_naive"] / scale) ** 2 * n          # the run's variance estimate
        se = math.sqrt((mu4 - var * var) / n)                  # its sampling standard error
        assert abs(got - var) <= 5 * se, (lev, got, var, se)
        # a wrong power of n would be off by a factor n^(1/2) or more
        assert res[lev]["err_naive"] == pytest.approx(scale * math.sqrt(var / n), rel=0.05)


@pytest.mark.parametrize("nb,runs", [(2, 400), (10, 200)])
def test_blocked_err_has_the_exact_mean_square(weights, nb, runs):
    o, w = weights
    n = w.shape[0] // runs
    scale = math.exp(mc.log_A_free(A, B, T))
    w0 = o.level0(A, B, T)
    for lev in range(1, S + 1):
        _, var, _ = _moments(2 ** lev)
        e2 = [(mc.estimate(w[r * n:(r + 1) * n], w0, A, B, T, nb)[lev]["err"] / scale) ** 2 for r in range(runs)]
        ratio = float(np.mean(e2)) / (var / n)
        # err^2 (nb - 1) / (sigma^2 / n) is chi^2 with nb - 1 degrees of freedom
        # for Gaussian block means: the mean over R runs has relative spread sqrt(2 / (R (nb - 1)))
        tol = 5 * math.sqrt(2.0 / (runs * (nb - 1)))
        assert abs(ratio - 1) <= tol, (lev, nb, ratio, tol)


def test_z_scores_follow_student_t(weights):
    o, w = weights
    runs, nb = 200, 10
    n = w.shape[0] // runs
    w0 = o.level0(A, B, T)
    for lev in range(1, S + 1):
        ref = exact.ho_discretized(P, 2 ** lev, A, B, T, omega=OMEGA)
        z = np.array([(r["amp"] - ref) / r["err"] for r in
                      (mc.estimate(w[k * n:(k + 1) * n], w0, A, B, T, nb)[lev] for k in range(runs))])
        nu = nb - 1
        ez2 = nu / (nu - 2)                                    # E[z^2] of Student t_nu
        ez4 = 3 * nu * nu / ((nu - 2) * (nu - 4))
        sd = math.sqrt((ez4 - ez2 * ez2) / runs)
        assert abs(float(np.mean(z * z)) - ez2) <= 5 * sd, (lev, float(np.mean(z * z)))
        assert abs(float(np.mean(z))) <= 5 * math.sqrt(ez2 / runs), lev    # unbiased
