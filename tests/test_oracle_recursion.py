"""Pins of the oracle's effective-action coefficients (CPU only).

Each test checks the oracle's c_{m,k} against something the paper or
mathematics fixes, computed here by independent means (sympy / mpmath):

* the defining PDE for W (Sec. 2.1, Eq. eqW): W_p must satisfy it through
  order eps^(p-1), counting xb^2 as one power of eps (Eq. ansatz);
* the hand-derived W_3 (from Eq. 1Drec and Eq. diagonal by hand);
* the exact harmonic-oscillator W read off the Mehler kernel (Sec. 2.1);
* W_1 = V (the naive midpoint action, Sec. 2.1 and Eq. SNp at p = 1).
"""
from fractions import Fraction
import math
import random

import pytest

from oracle import effective_action as ea

sp = pytest.importorskip("sympy")
x, xb, eps, t = sp.symbols("x xb eps t")


def _to_sympy_poly(poly, var):
    return sp.Integer(0) + sum(sp.Rational(v.numerator, v.denominator) * var ** i
                               for i, v in enumerate(poly))


def _W_sympy(model, p, var):
    c = ea.coefficients(model, p)
    return sp.expand(sum(_to_sympy_poly(poly, var) * eps ** (m - k) * xb ** (2 * k)
                         for (m, k), poly in c.items()))


def _low_order_terms(expr, p):
    """Monomials eps^a xb^b (any power of the ring variable) with a + b/2 <= p-1."""
    P = sp.Poly(sp.expand(expr), eps, xb)
    bad = []
    for (a, b), coeff in P.terms():
        if 2 * a + b <= 2 * (p - 1) and sp.simplify(coeff) != 0:
            bad.append(((a, b), coeff))
    return bad


def _residual_x(model, p):
    V = _to_sympy_poly(model.V, x)
    W = _W_sympy(model, p, x)
    rhs = sp.Rational(1, 2) * (V.subs(x, x + xb) + V.subs(x, x - xb))
    R = (W + xb * sp.diff(W, xb) + eps * sp.diff(W, eps)
         - eps / 8 * sp.diff(W, x, 2) - eps / 8 * sp.diff(W, xb, 2)
         + eps ** 2 / 8 * sp.diff(W, x) ** 2 + eps ** 2 / 8 * sp.diff(W, xb) ** 2 - rhs)
    return R


@pytest.mark.parametrize("name,params,p", [
    ("aho", [1, 1], 6),
    ("aho", [Fraction(3, 2), 10], 5),
    ("dw", [5], 5),
    ("poly", [Fraction(1, 3), Fraction(-1, 5), Fraction(2, 7), Fraction(1, 11), Fraction(-1, 13)], 5),
    ("ho", [Fraction(7, 5)], 7),
])
def test_pde_residual_vanishes_through_order_p_minus_1(name, params, p):
    model = ea.make_model(name, params)
    R = _residual_x(model, p)
    assert _low_order_terms(R, p) == []
    # the truncation is really at p-1: some order-p term survives (not HO, whose
    # W is quadratic with every order present)
    P = sp.Poly(sp.expand(R), eps, xb)
    assert any(2 * a + b == 2 * p and sp.simplify(cf) != 0 for (a, b), cf in P.terms())


def test_pde_residual_mpt_in_tanh_ring():
    """Same check for -lambda/cosh^2(alpha x) with d/dx = alpha (1-t^2) d/dt."""
    lam, alpha, p = Fraction(3), Fraction(1, 2), 5
    model = ea.make_model("mpt", [lam, alpha])
    al = sp.Rational(alpha.numerator, alpha.denominator)
    D = lambda f: sp.expand(al * (1 - t ** 2) * sp.diff(f, t))
    V = -sp.Rational(lam.numerator) * (1 - t ** 2)
    W = _W_sympy(model, p, t)
    # (V(x+xb) + V(x-xb))/2 as its Taylor series in xb
    rhs, Dk = 0, V
    for k in range(0, p):
        rhs += Dk * xb ** (2 * k) / sp.factorial(2 * k)
        Dk = D(D(Dk))
    R = (W + xb * sp.diff(W, xb) + eps * sp.diff(W, eps)
         - eps / 8 * D(D(W)) - eps / 8 * sp.diff(W, xb, 2)
         + eps ** 2 / 8 * D(W) ** 2 + eps ** 2 / 8 * sp.diff(W, xb) ** 2 - rhs)
    assert _low_order_terms(R, p) == []


def test_hand_derived_W3_polynomial():
    rng = random.Random(7)
    coeffs = [Fraction(rng.randint(-9, 9), rng.randint(1, 9)) for _ in range(7)]
    model = ea.make_model("poly", coeffs)
    V = _to_sympy_poly(model.V, x)
    d = lambda n: sp.diff(V, x, n)
    hand = {
        (0, 0): V,
        (1, 0): d(2) / 12,
        (1, 1): d(2) / 6,
        (2, 0): d(4) / 240 - d(1) ** 2 / 24,
        (2, 1): d(4) / 120,
        (2, 2): d(4) / 120,
    }
    c = ea.coefficients(model, 3)
    assert set(c) == set(hand)
    for key, expr in hand.items():
        assert sp.expand(_to_sympy_poly(c[key], x) - expr) == 0, key


def test_hand_derived_W3_mpt_numeric():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    lam, alpha = 3.0, 0.7
    model = ea.make_model("mpt", [lam, alpha])
    c = ea.coefficients(model, 3)
    Vf = lambda y: -lam / mp.cosh(alpha * y) ** 2
    for xv in (-1.3, 0.0, 0.4, 2.2):
        d = lambda n: mp.diff(Vf, xv, n)
        hand = {(0, 0): d(0), (1, 0): d(2) / 12, (1, 1): d(2) / 6,
                (2, 0): d(4) / 240 - d(1) ** 2 / 24, (2, 1): d(4) / 120, (2, 2): d(4) / 120}
        z = math.tanh(alpha * xv)
        for key, ref in hand.items():
            got = ea.peval(c[key], z)
            assert abs(got - float(ref)) <= 1e-12 * max(1.0, abs(float(ref))), (xv, key)


def test_mpt_derivative_chain_matches_numeric_derivatives():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    lam, alpha = 2.5, 1.3
    model = ea.make_model("mpt", [lam, alpha])
    Vf = lambda y: -lam / mp.cosh(alpha * y) ** 2
    f = model.V
    for n in range(0, 11):
        for xv in (-0.9, 0.3, 1.7):
            ref = float(mp.diff(Vf, xv, n))
            got = ea.peval(f, math.tanh(alpha * xv))
            assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref)), (n, xv)
        f = model.D(f)


@pytest.mark.parametrize("omega", [Fraction(1), Fraction(3, 2)])
def test_harmonic_W_matches_mehler_series(omega):
    p = 8
    w = sp.Rational(omega.numerator, omega.denominator)
    sh, ch = sp.sinh(w * eps), sp.cosh(w * eps)
    f = w * (ch - 1) / sh / eps
    g = (w * (ch + 1) / sh - 2 / eps) / eps
    h = sp.log(sh / (w * eps)) / (2 * eps)
    fs = sp.series(f, eps, 0, p).removeO()
    gs = sp.series(g, eps, 0, p - 1).removeO()
    hs = sp.series(h, eps, 0, p).removeO()
    c = ea.coefficients(ea.make_model("ho", [omega]), p)
    al = sum(_to_sympy_poly(c[(m, 0)], x).coeff(x, 2) * eps ** m for m in range(p))
    ga = sum(_to_sympy_poly(c[(m, 0)], x).coeff(x, 0) * eps ** m for m in range(p))
    be = sum(_to_sympy_poly(c[(m, 1)], x).coeff(x, 0) * eps ** (m - 1) for m in range(1, p))
    assert sp.expand(al - fs) == 0
    assert sp.expand(be - gs) == 0
    assert sp.expand(ga - hs) == 0
    # nothing else: W_p is exactly alpha x^2 + beta xb^2 + gamma
    for (m, k), poly in c.items():
        for i, v in enumerate(poly):
            if v:
                assert (i, k) in ((2, 0), (0, 0), (0, 1))


def test_level_one_is_the_potential():
    for name, params in [("aho", [1, 10]), ("dw", [5]), ("mpt", [3, 1]), ("poly", [1, -2, 3])]:
        model = ea.make_model(name, params)
        c = ea.coefficients(model, 1)
        assert c == {(0, 0): model.V}


def test_diagonal_formula():
    model = ea.make_model("poly", [Fraction(1, 2), 3, Fraction(-1, 7), 0, 1, Fraction(2, 3), 0, 0, 1])
    V = _to_sympy_poly(model.V, x)
    c = ea.coefficients(model, 5)
    for m in range(5):
        ref = sp.diff(V, x, 2 * m) / sp.factorial(2 * m + 1)
        assert sp.expand(_to_sympy_poly(c[(m, m)], x) - ref) == 0
