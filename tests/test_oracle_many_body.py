"""Pins of the oracle's d-dimensional effective potential (Sec. 2.2, Eq. EXP,
Eq. MBrec, Eq. DIA), CPU only:

* the defining equation Eq. eqWMB with sympy in two and three dimensions:
  zero residual through order eps^(p-1) (xb^2 counted as eps);
* d = 1 reproduces the one-dimensional coefficients c_{m,k}(x) of
  Eq. 1Drec exactly (W_{m,k} = xb^(2k) c_{m,k});
* a separable potential V_1(x_1) + V_2(x_2) gives W_1 + W_2 exactly;
* a coupled harmonic oscillator 1/2 x.K.x equals the sum of its normal
  modes' one-dimensional W (the recursion is rotation covariant), and a
  radial 2D anharmonic oscillator is rotation invariant;
* the Monte Carlo side: the coupled oscillator's estimate equals the exact
  discretized amplitude (the product of its normal modes' Gaussian
  integrals) within 3 sigma at every level;
* physics: the spectrum of Sec. 5's evolution operator built from the 2D
  radial anharmonic oscillator's W equals a two-dimensional sinc-DVR
  diagonalisation of its Hamiltonian (an independent method).
"""
from fractions import Fraction as F
import functools
import math

import numpy as np
import pytest

from oracle import effective_action as ea
from oracle import evolution as ev
from oracle import exact, mc
from oracle import many_body as mb

sp = pytest.importorskip("sympy")


def aho2(A=F(1), g=F(1)):
    """A/2 (x^2 + y^2) + g/24 (x^2 + y^2)^2 (Sec. 3.3, the 2D-AHO)."""
    return {(2, 0): A / 2, (0, 2): A / 2, (4, 0): g / 24, (0, 4): g / 24, (2, 2): g / 12}


GEN2 = {(2, 0): F(1, 2), (0, 2): F(3, 4), (1, 1): F(1, 5), (2, 1): F(1, 3), (0, 3): F(-1, 7), (4, 0): F(1, 10),
        (1, 3): F(1, 20), (0, 4): F(1, 12), (1, 0): F(-1, 3)}
GEN3 = {(2, 0, 0): F(1, 2), (0, 2, 0): F(1, 2), (0, 0, 2): F(1, 2), (1, 1, 0): F(1, 5), (0, 1, 1): F(1, 7),
        (2, 0, 2): F(1, 11), (4, 0, 0): F(1, 24), (0, 4, 0): F(1, 24), (0, 0, 4): F(1, 30), (1, 1, 1): F(1, 9)}


def _sym_poly(poly, xs, xbs):
    tot = sp.Integer(0)
    for mono, v in poly.items():
        term = sp.Rational(v.numerator, v.denominator)
        for var, e in zip(list(xs) + list(xbs), mono):
            term *= var ** e
        tot += term
    return tot


@pytest.mark.parametrize("V,d,p", [(GEN2, 2, 2), (GEN2, 2, 3), (GEN2, 2, 4), (aho2(), 2, 5), (GEN3, 3, 3)])
def test_residual_of_the_many_body_equation(V, d, p):
    xs = sp.symbols(f"x0:{d}")
    xbs = sp.symbols(f"xb0:{d}")
    eps, lam = sp.symbols("eps lam")
    W = sum(_sym_poly(poly, xs, xbs) * eps ** (m - k) for (m, k), poly in mb.coefficients(V, d, p).items())
    Vs = _sym_poly(mb.potential(V, d), xs, xbs)
    Vp = Vs.subs({x: x + xb for x, xb in zip(xs, xbs)}, simultaneous=True)
    Vm = Vs.subs({x: x - xb for x, xb in zip(xs, xbs)}, simultaneous=True)
    lap = sum(sp.diff(W, x, 2) for x in xs)
    lapb = sum(sp.diff(W, x, 2) for x in xbs)
    g2 = sum(sp.diff(W, x) ** 2 for x in xs)
    gb2 = sum(sp.diff(W, x) ** 2 for x in xbs)
    R = (W + sum(xb * sp.diff(W, xb) for xb in xbs) + eps * sp.diff(W, eps) - eps / 8 * lap - eps / 8 * lapb
         + eps ** 2 / 8 * g2 + eps ** 2 / 8 * gb2 - (Vp + Vm) / 2)
    # xb ~ lam, eps ~ lam^2: every order below lam^(2p) must vanish
    R = sp.expand(R.subs({**{xb: lam * xb for xb in xbs}, eps: lam ** 2 * eps}, simultaneous=True))
    P = sp.Poly(R, lam)
    for (e,), c in P.terms():
        if e < 2 * p:
            assert sp.expand(c) == 0, (e, c)


@pytest.mark.parametrize("name,params,p", [("aho", [1, 10], 6), ("dw", [5], 5), ("poly", [F(1, 5), F(-1, 2), F(3, 10), F(1, 4), F(1, 10)], 5)])
def test_one_dimension_reproduces_the_scalar_recursion(name, params, p):
    model = ea.make_model(name, [F(v) for v in params])
    c = ea.coefficients(model, p)
    V = {(i,): F(v) for i, v in enumerate(model.V) if v}
    W = mb.coefficients(V, 1, p)
    for (m, k), poly in W.items():
        ref = {(i, 2 * k): v for i, v in enumerate(c[(m, k)]) if v}
        assert poly == ref, (m, k)


def test_separable_potential_gives_the_sum_of_one_dimensional_actions():
    p = 6
    V1 = {(2,): F(1, 2), (4,): F(1, 6), (3,): F(-1, 5)}
    V2 = {(2,): F(3, 2), (1,): F(1, 4), (4,): F(1, 24)}
    V = {(e[0], 0): v for e, v in V1.items()}
    V.update({(0, e[0]): v for e, v in V2.items()})
    W = mb.coefficients(V, 2, p)
    W1, W2 = mb.coefficients(V1, 1, p), mb.coefficients(V2, 1, p)
    for (m, k), poly in W.items():
        ref = {(a, 0, b, 0): v for (a, b), v in W1[(m, k)].items()}
        for (a, b), v in W2[(m, k)].items():
            ref[(0, a, 0, b)] = ref.get((0, a, 0, b), F(0)) + v
        ref = {key: v for key, v in ref.items() if v}
        assert poly == ref, (m, k)


def _ho_wp_1d(omega, p, x, xb, eps):
    model = ea.make_model("ho", [omega])
    return np.array([ea.wp(model, p, float(a), float(b), eps) for a, b in zip(np.ravel(x), np.ravel(xb))])


def test_coupled_oscillator_equals_its_normal_modes():
    """V = 1/2 x.K.x with K = U diag(w^2) U^T: W(x, xb) = sum_i W_HO(w_i; (U^T x)_i, (U^T xb)_i)."""
    K = {(2, 0): F(1, 1), (0, 2): F(2, 1), (1, 1): F(3, 5)}   # 1/2 (2 x^2 + 4 y^2) + 3/5 x y -> K = [[2, .6], [.6, 4]]
    Km = np.array([[2.0, 0.6], [0.6, 4.0]])
    lam, U = np.linalg.eigh(Km)
    w = np.sqrt(lam)
    p = 8
    rng = np.random.default_rng(3)
    x = rng.uniform(-2, 2, (40, 2))
    xb = rng.uniform(-0.6, 0.6, (40, 2))
    for eps in (0.05, 0.2):
        got = mb.wp(K, 2, p, x, xb, eps)
        y, yb = x @ U, xb @ U
        ref = sum(_ho_wp_1d(w[i], p, y[:, i], yb[:, i], eps) for i in range(2))
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_radial_anharmonic_oscillator_is_rotation_invariant():
    p = 7
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.5, 1.5, (30, 2))
    xb = rng.uniform(-0.4, 0.4, (30, 2))
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    a = mb.wp(aho2(F(1), F(6)), 2, p, x, xb, 0.1)
    b = mb.wp(aho2(F(1), F(6)), 2, p, x @ R.T, xb @ R.T, 0.1)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_coupled_oscillator_monte_carlo_matches_the_exact_discretized_amplitude():
    Km = np.array([[2.0, 0.6], [0.6, 4.0]])
    K = {(2, 0): F(1), (0, 2): F(2), (1, 1): F(3, 5)}
    lam, U = np.linalg.eigh(Km)
    w = np.sqrt(lam)
    a, b, T, p, s, n = np.array([0.3, -0.2]), np.array([0.5, 0.4]), 1.0, 4, 3, 20000
    ws, _ = mb.logweights(K, 2, p, a, b, T, s, 11, n)
    w0 = mb.level0(K, 2, p, a, b, T)
    res = mc.estimate(ws, w0, 0.0, 0.0, T, 40)     # A_free of the d coordinates added below
    shift = mb.log_A_free(a, b, T) - mc.log_A_free(0.0, 0.0, T)
    ua, ub = a @ U, b @ U
    for r in res:
        N = 1 << r["n"]
        ref = math.prod(exact.ho_discretized(p, N, ua[i], ub[i], T, omega=w[i]) for i in range(2))
        amp = r["amp"] * math.exp(shift)
        err = r["err"] * math.exp(shift)
        if r["n"] == 0:
            assert amp == pytest.approx(ref, rel=1e-12)
        else:
            assert abs(amp - ref) <= 3 * err, (r["n"], amp, ref, err)


_RADIAL_AHO = {(2, 0): 0.5, (0, 2): 0.5, (4, 0): 1 / 24, (0, 4): 1 / 24, (2, 2): 1 / 12}


@functools.lru_cache(maxsize=1)
def _radial_aho_dvr():
    return exact.dvr_energies_2d(lambda x, y: 0.5 * (x * x + y * y) + (x * x + y * y) ** 2 / 24, 6.0, 0.1, 8)


@pytest.mark.parametrize("p", [8, 4])
def test_radial_anharmonic_spectrum_matches_two_dimensional_dvr(p):
    """Sec. 5's evolution operator built from the contracted W of the 2D
    radial anharmonic oscillator (a non-separable potential) on a 49 x 49
    grid, t = 0.1: its lowest eight energies (with the degenerate pairs of
    the rotation symmetry) equal a two-dimensional sinc-DVR diagonalisation
    of the Hamiltonian within 1e-9 at p = 8; at p = 4 the short-time error
    of the truncated action shows (> 1e-6)."""
    t = 0.1
    U = ev.evolution_matrix_nd(_RADIAL_AHO, 2, p, t, np.linspace(-6.0, 6.0, 49))
    E = ev.energies(U, t, 8)
    err = np.abs(E - _radial_aho_dvr()).max()
    if p == 8:
        assert err <= 1e-9, E - _radial_aho_dvr()
    else:
        assert err > 1e-6, err
