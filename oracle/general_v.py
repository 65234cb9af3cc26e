"""The level-p effective potential for a general potential (oracle side):
W_p as a polynomial in the derivative symbols V_j = V^(j)(x).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

Sec. 2.1's recursion (Eq. 1Drec with the diagonal of Eq. diagonal, in the
order of Fig. 1) holds for any V; leaving V unspecified, every c_{m,k} is a
polynomial with rational coefficients in V_0, V_1, ..., V_{2p-2}, and the
x-derivative acts by the chain rule, d/dx V_j = V_{j+1} (the general 1D
effective action of Sec. 3.1, here derived with exact rational arithmetic).
A polynomial is a dict {exponent tuple (e_0..e_J): Fraction}.

The potentials of the general mode are sums of analytic families whose
derivatives of every order are evaluated here directly:

    V(x) = sum_{i<=8} a_i x^i + sum_g A_g exp(-beta_g (x - c_g)^2)
           + sum_s B_s sech^2(alpha_s (x - d_s)),

(and, optionally, four exponentials E e^{-kappa (x - x0)}, whose
derivatives are (-kappa)^n times themselves: Morse potentials are sums of
them), the Gaussian's through Hermite polynomials,
d^n/du^n e^{-beta u^2} = (-sqrt(beta))^n H_n(sqrt(beta) u) e^{-beta u^2},
and sech^2's as derivatives of tanh: sech^2 = tanh' and tanh' = 1 - tanh^2,
so by Leibniz's rule tanh^(n+1) = -sum_k C(n, k) tanh^(k) tanh^(n-k) for
n >= 1, started from tanh and sech^2 themselves.
(The same derivatives are polynomials P_n in t = tanh u -- kept below as a
pin -- but those polynomials summed in the monomial basis cancel badly for
|u| >~ 1: at order 22 and u = 3 they keep two correct digits.)
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
import math

import numpy as np

ZERO = Fraction(0)


def _add_into(acc, poly, scale=Fraction(1)):
    for mono, v in poly.items():
        w = acc.get(mono, ZERO) + scale * v
        if w:
            acc[mono] = w
        else:
            acc.pop(mono, None)
    return acc


def _mul(a, b):
    out = {}
    for ma, va in a.items():
        for mb, vb in b.items():
            mono = tuple(x + y for x, y in zip(ma, mb))
            w = out.get(mono, ZERO) + va * vb
            if w:
                out[mono] = w
            else:
                out.pop(mono, None)
    return out


def _D(poly, J):
    """d/dx with d/dx V_j = V_{j+1} (j < J)."""
    out = {}
    for mono, v in poly.items():
        for j, e in enumerate(mono):
            if e == 0:
                continue
            if j == J:
                raise ValueError("derivative order beyond the symbols")
            m = list(mono)
            m[j] -= 1
            m[j + 1] += 1
            m = tuple(m)
            w = out.get(m, ZERO) + v * e
            if w:
                out[m] = w
            else:
                out.pop(m, None)
    return out


@lru_cache(maxsize=16)
def coefficients(p):
    """dict (m, k) -> c_{m,k} as a polynomial in V_0..V_{2p-1} (the last
    symbol only in the never-used derivative of the last row), for
    0 <= k <= m <= p-1; c_{m,k} itself involves V_j with j <= 2m."""
    if p < 1:
        raise ValueError("p >= 1")
    J = 2 * p - 1
    nsym = J + 1

    def sym(j):
        e = [0] * nsym
        e[j] = 1
        return {tuple(e): Fraction(1)}

    c, dc = {}, {}
    for m in range(p):
        c[(m, m)] = {mono: v / math.factorial(2 * m + 1) for mono, v in sym(2 * m).items()}
        dc[(m, m)] = _D(c[(m, m)], J)
        for k in range(m - 1, -1, -1):
            acc = {}
            _add_into(acc, c[(m, k + 1)], Fraction((2 * k + 2) * (2 * k + 1)))
            _add_into(acc, _D(dc[(m - 1, k)], J))
            for l in range(0, m - 1):
                for r in range(max(0, k - m + l + 2), min(k, l) + 1):
                    _add_into(acc, _mul(dc[(l, r)], dc[(m - l - 2, k - r)]), Fraction(-1))
            for l in range(1, m - 1):
                for r in range(max(0, k - m + l + 2), min(k, l) + 1):
                    fac = 2 * r * (2 * k - 2 * r + 2)
                    if fac:
                        _add_into(acc, _mul(c[(l, r)], c[(m - l - 1, k - r + 1)]), Fraction(-fac))
            c[(m, k)] = {mono: v / (8 * (m + k + 1)) for mono, v in acc.items()}
            if m < p - 1:
                dc[(m, k)] = _D(c[(m, k)], J)
    return c


def term_count(p):
    return sum(len(poly) for poly in coefficients(p).values())


# ---------------------------------------------------------------------------
# potentials of the general mode and their derivatives
# ---------------------------------------------------------------------------

N_POLY, N_GAUSS, N_SECH, N_EXP = 9, 4, 4, 4
N_PARAMS = N_POLY + 3 * N_GAUSS + 3 * N_SECH     # 33
N_PARAMS_EXP = N_PARAMS + 3 * N_EXP               # 45: with the exponential terms


def split_params_all(params):
    """(a[9], gauss [(A, beta, c)], sech [(B, alpha, d)], exps [(E, kappa, x0)]),
    the terms with a nonzero amplitude; 33 parameters (no exponential terms)
    or 45."""
    if len(params) not in (N_PARAMS, N_PARAMS_EXP):
        raise ValueError(f"the general potential takes {N_PARAMS} or {N_PARAMS_EXP} parameters")
    a = [float(v) for v in params[:N_POLY]]
    g = [tuple(float(v) for v in params[N_POLY + 3 * i:N_POLY + 3 * i + 3]) for i in range(N_GAUSS)]
    o = N_POLY + 3 * N_GAUSS
    s = [tuple(float(v) for v in params[o + 3 * i:o + 3 * i + 3]) for i in range(N_SECH)]
    o = N_PARAMS
    e = [tuple(float(v) for v in params[o + 3 * i:o + 3 * i + 3]) for i in range(N_EXP)] \
        if len(params) == N_PARAMS_EXP else []
    return a, [t for t in g if t[0] != 0], [t for t in s if t[0] != 0], [t for t in e if t[0] != 0]


def split_params(params):
    """(a[9], gauss [(A, beta, c)] with A != 0, sech [(B, alpha, d)] with B != 0)."""
    a, g, s, _ = split_params_all(params)
    return a, g, s


@lru_cache(maxsize=64)
def _sech2_polys(J):
    """P_n(t), n = 0..J, with d^n/du^n sech^2(u) = P_n(tanh u) (alpha = 1)."""
    polys = [[Fraction(1), ZERO, Fraction(-1)]]          # 1 - t^2
    for _ in range(J):
        prev = polys[-1]
        der = [i * prev[i] for i in range(1, len(prev))]  # d/dt
        nxt = [ZERO] * (len(der) + 2)
        for i, v in enumerate(der):                     # (1 - t^2) * der
            nxt[i] += v
            nxt[i + 2] -= v
        polys.append(nxt)
    return tuple(tuple(p) for p in polys)


def derivatives(params, x, J):
    """V^(j)(x), j = 0..J, as an array (J+1, *x.shape) in float64."""
    x = np.asarray(x, dtype=np.float64)
    a, gs, ss, es = split_params_all(params)
    out = np.zeros((J + 1,) + x.shape)
    # polynomial
    for j in range(J + 1):
        coef = [a[i] * math.perm(i, j) for i in range(j, N_POLY)]
        v = np.zeros_like(x)
        for cf in reversed(coef):
            v = v * x + cf
        out[j] += v
    # Gaussians: (-sqrt(beta))^n H_n(sqrt(beta) u) e^{-beta u^2}
    for A, beta, c in gs:
        u = x - c
        sb = math.sqrt(beta)
        y = sb * u
        e = A * np.exp(-beta * u * u)
        h0, h1 = np.ones_like(y), 2 * y
        for n in range(J + 1):
            h = h0 if n == 0 else h1
            out[n] += (-sb) ** n * h * e
            if n >= 1:
                h0, h1 = h1, 2 * y * h1 - 2 * n * h0
    # sech^2: d^n/dx^n sech^2(alpha u) = alpha^n tanh^(n+1)(alpha u)
    for B, alpha, d in ss:
        w = alpha * (x - d)
        T = [np.tanh(w), 1.0 / np.cosh(w) ** 2]   # tanh' directly, not 1 - tanh^2
        for n in range(1, J + 1):
            acc = np.zeros_like(x)
            for k in range(n + 1):
                acc = acc - math.comb(n, k) * T[k] * T[n - k]
            T.append(acc)
        for n in range(J + 1):
            out[n] += B * alpha ** n * T[n + 1]
    # exponentials: d^n/dx^n E e^{-kappa (x - x0)} = (-kappa)^n E e^{-kappa (x - x0)}
    for E, kappa, x0 in es:
        e = E * np.exp(-kappa * (x - x0))
        for n in range(J + 1):
            out[n] += (-kappa) ** n * e
    return out


def wp(params, p, x, xb, eps):
    """W_p(x, xb; eps) of the general potential (float64, vectorised)."""
    c = coefficients(p)
    J = 2 * p - 1
    x = np.asarray(x, dtype=np.float64)
    Vd = derivatives(params, x, J)
    tot = np.zeros_like(x)
    for (m, k), poly in c.items():
        v = np.zeros_like(x)
        for mono, coef in poly.items():
            term = np.full_like(x, float(coef))
            for j, e in enumerate(mono):
                if e:
                    term = term * Vd[j] ** e
            v = v + term
        tot = tot + v * eps ** (m - k) * np.asarray(xb) ** (2 * k)
    return tot


def wp_abs(params, p, x, xb, eps):
    """sum over terms of |term|: the scale the terms of W_p are summed from."""
    c = coefficients(p)
    J = 2 * p - 1
    x = np.asarray(x, dtype=np.float64)
    Vd = derivatives(params, x, J)
    tot = np.zeros_like(x)
    for (m, k), poly in c.items():
        for mono, coef in poly.items():
            term = np.full_like(x, abs(float(coef)))
            for j, e in enumerate(mono):
                if e:
                    term = term * np.abs(Vd[j]) ** e
            tot = tot + term * eps ** (m - k) * np.abs(np.asarray(xb)) ** (2 * k)
    return tot
