"""Pins of the oracle's general-potential effective action (derivative-symbol
form of W_p), CPU only:

* the defining PDE (Sec. 2.1, Eq. eqW) with a symbolic V(x) (sympy Function):
  zero residual through order eps^(p-1), xb^2 counted as eps;
* substituting the derivatives of a polynomial potential reproduces the
  model-specific c_{m,k}(x) exactly (exact rational polynomials);
* with sech^2 terms it reproduces the Poeschl-Teller model of the tanh ring
  (numerically, 1e-12);
* the derivative evaluators of the families against mpmath's numerical
  differentiation;
* term counts of the general form (1, 3, 15, 58, 193, 585 at p = 1, 2, 4, 6,
  8, 10: an independent sympy count).
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import effective_action as ea
from oracle import general_v as gv

sp = pytest.importorskip("sympy")
mp = pytest.importorskip("mpmath")


def _params(poly=(), gauss=(), sech=()):
    a = list(poly) + [0.0] * (gv.N_POLY - len(poly))
    g = [v for t in gauss for v in t] + [0.0] * (3 * (gv.N_GAUSS - len(gauss)))
    s = [v for t in sech for v in t] + [0.0] * (3 * (gv.N_SECH - len(sech)))
    return a + g + s


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_pde_residual_for_a_symbolic_potential(p):
    x, xb, eps = sp.symbols("x xb eps")
    V = sp.Function("V")
    c = gv.coefficients(p)
    J = 2 * p - 1
    syms = [V(x).diff(x, j) if j else V(x) for j in range(J + 1)]

    def to_sym(poly):
        tot = sp.Integer(0)
        for mono, v in poly.items():
            term = sp.Rational(v.numerator, v.denominator)
            for j, e in enumerate(mono):
                if e:
                    term *= syms[j] ** e
            tot += term
        return tot

    W = sp.expand(sum(to_sym(poly) * eps ** (m - k) * xb ** (2 * k) for (m, k), poly in c.items()))
    # (V(x + xb) + V(x - xb))/2 through xb^(2p-2)
    rhs = sum(V(x).diff(x, 2 * j) * xb ** (2 * j) / math.factorial(2 * j) if j else V(x) for j in range(p))
    R = (W + xb * sp.diff(W, xb) + eps * sp.diff(W, eps) - eps / 8 * sp.diff(W, x, 2)
         - eps / 8 * sp.diff(W, xb, 2) + eps ** 2 / 8 * sp.diff(W, x) ** 2 + eps ** 2 / 8 * sp.diff(W, xb) ** 2
         - rhs)
    R = sp.expand(R)
    P = sp.Poly(R, eps, xb)
    for (a, b), coeff in P.terms():
        if 2 * a + b <= 2 * (p - 1):
            assert sp.simplify(coeff) == 0, (a, b, coeff)


def _poly_derivs(V, J):
    out = [list(V)]
    for _ in range(J):
        prev = out[-1]
        out.append([i * prev[i] for i in range(1, len(prev))] or [Fraction(0)])
    return out


def _padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def _pmul(a, b):
    r = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, u in enumerate(a):
        for j, v in enumerate(b):
            r[i + j] += u * v
    return r


@pytest.mark.parametrize("name,params,p", [("aho", [1, 10], 8), ("dw", [5], 6),
                                           ("poly", [Fraction(1, 3), Fraction(-1, 5), Fraction(2, 7),
                                                     Fraction(1, 11), Fraction(-1, 13)], 6)])
def test_substituted_polynomial_reproduces_the_model_specific_coefficients(name, params, p):
    model = ea.make_model(name, [Fraction(v) for v in params])
    spec = ea.coefficients(model, p)
    gen = gv.coefficients(p)
    Vd = _poly_derivs(model.V, 2 * p - 1)
    for key, poly in gen.items():
        tot = [Fraction(0)]
        for mono, v in poly.items():
            term = [v]
            for j, e in enumerate(mono):
                for _ in range(e):
                    term = _pmul(term, Vd[j])
            tot = _padd(tot, term)
        while len(tot) > 1 and tot[-1] == 0:
            tot.pop()
        ref = list(spec.get(key, [])) or [Fraction(0)]
        assert tot == ref, key


def test_sech2_terms_reproduce_the_poeschl_teller_model():
    lam, alpha, p = 3.0, 0.8, 8
    params = _params(sech=[(-lam, alpha, 0.0)])
    model = ea.make_model("mpt", [lam, alpha])
    rng = np.random.default_rng(1)
    x = rng.uniform(-3, 3, 50)
    xb = rng.uniform(-0.5, 0.5, 50)
    for eps in (0.05, 0.3):
        got = gv.wp(params, p, x, xb, eps)
        ref = np.array([ea.wp(model, p, float(a), float(b), eps) for a, b in zip(x, xb)])
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_family_derivatives_against_numerical_differentiation():
    mp.mp.dps = 40
    params = _params(poly=[0.3, -0.1, 0.5, 0.0, 0.02], gauss=[(1.5, 0.7, 0.4), (-0.8, 2.0, -1.0)],
                     sech=[(-2.0, 1.3, 0.2)])

    def V(x):
        return (0.3 - 0.1 * x + 0.5 * x ** 2 + 0.02 * x ** 4 + 1.5 * mp.exp(-0.7 * (x - 0.4) ** 2)
                - 0.8 * mp.exp(-2.0 * (x + 1.0) ** 2) - 2.0 * mp.sech(1.3 * (x - 0.2)) ** 2)

    J = 9
    for x0 in (-1.3, 0.0, 0.77, 2.1):
        got = gv.derivatives(params, np.array([x0]), J)[:, 0]
        for j in range(J + 1):
            ref = float(mp.diff(V, mp.mpf(x0), j))
            assert got[j] == pytest.approx(ref, rel=1e-9, abs=1e-9 * max(1.0, abs(ref))), (x0, j)


def test_sech2_derivatives_to_the_highest_order_far_from_the_centre():
    """All orders the general mode uses (up to 2p - 2 = 22) where tanh is
    near +-1 and the derivatives are small against their polynomial
    coefficients (|u| up to 4): the cancellation-prone region."""
    mp.mp.dps = 60
    J = 22
    for B, alpha, d in ((-3.0, 1.0, 0.0), (0.4, 2.0, 0.5)):
        params = _params(sech=[(B, alpha, d)])
        for x0 in (-2.2, 0.3, 1.7, 3.0 / alpha + d, 4.0):
            got = gv.derivatives(params, np.array([x0]), J)[:, 0]
            f = lambda z: B * mp.sech(alpha * (z - d)) ** 2  # noqa: E731
            for j in range(J + 1):
                ref = float(mp.diff(f, mp.mpf(x0), j))
                assert got[j] == pytest.approx(ref, rel=1e-12, abs=1e-300), (B, x0, j)


def test_sech2_leibniz_rule_matches_the_tanh_polynomials():
    """The Leibniz recursion on tanh' = 1 - tanh^2 and the polynomials
    P_n(t) (P_0 = 1 - t^2, P_{n+1} = (1 - t^2) P_n') are the same
    derivatives: equal at rational t in exact arithmetic."""
    J = 12
    P = gv._sech2_polys(J)
    for t in (Fraction(0), Fraction(1, 3), Fraction(-5, 7), Fraction(9, 10)):
        T = [t]
        for n in range(J + 1):
            T.append((1 if n == 0 else 0) - sum(math.comb(n, k) * T[k] * T[n - k] for k in range(n + 1)))
        for n in range(J + 1):
            assert sum(c * t ** i for i, c in enumerate(P[n])) == T[n + 1], (t, n)


def test_term_counts():
    assert [gv.term_count(p) for p in (1, 2, 4, 6, 8, 10)] == [1, 3, 15, 58, 193, 585]


def test_exponential_terms_derivatives_to_the_highest_order():
    """A Morse potential D (1 - e^{-a (x - x0)})^2 = D - 2D e^{-a u} + D e^{-2a u}
    through the exponential family (45 parameters): every order up to 22
    against mpmath's numerical differentiation."""
    mp.mp.dps = 60
    D, a, x0 = 4.0, 1.0, 0.3
    params = _params(poly=[D]) + [-2 * D, a, x0, D, 2 * a, x0] + [0.0] * 6
    assert len(params) == gv.N_PARAMS_EXP
    J = 22
    f = lambda z: D * (1 - mp.exp(-a * (z - x0))) ** 2  # noqa: E731
    for xq in (-0.8, 0.3, 1.9):
        got = gv.derivatives(params, np.array([xq]), J)[:, 0]
        for j in range(J + 1):
            ref = float(mp.diff(f, mp.mpf(xq), j))
            assert got[j] == pytest.approx(ref, rel=1e-12, abs=1e-12 * max(1.0, abs(ref))), (xq, j)
    # 33 parameters are the same potential without exponential terms
    assert gv.split_params_all(_params(poly=[D]))[3] == []


def _read_golden_w3():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "w3_derivative_symbols.txt")
    out = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            m, k, coef, mono = line.split()
            e = [0] * 6
            for factor in mono.split("*"):
                sym, _, power = factor.partition("^")
                e[int(sym[1:])] += int(power) if power else 1
            out.setdefault((int(m), int(k)), {})[tuple(e)] = Fraction(coef)
    return out


def test_level_three_matches_the_hand_derivation():
    golden = _read_golden_w3()
    c = gv.coefficients(3)
    assert set(c) == set(golden)
    for key, poly in golden.items():
        assert c[key] == poly, key
