"""Exact coefficients of the level-p effective potential W_p (oracle side).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

Sec. 2.1 writes the short-time amplitude through the effective potential W and
expands it as (Eq. ansatz)

    W(x, xb; eps) = sum_{m>=0} sum_{k=0..m} c_{m,k}(x) eps^(m-k) xb^(2k),

truncated at m <= p-1 for the level-p potential W_p.  The coefficients follow
from the Schroedinger equation for W (Eq. eqW) as the recursion Eq. 1Drec,

    8(m+k+1) c_{m,k} = (2k+2)(2k+1) c_{m,k+1} + c''_{m-1,k}
                       - sum_{l=0}^{m-2} sum_r c'_{l,r} c'_{m-l-2,k-r}
                       - sum_{l=1}^{m-2} sum_r 2r(2k-2r+2) c_{l,r} c_{m-l-1,k-r+1},
    r from max(0, k-m+l+2) to min(k, l),

with the diagonal (Eq. diagonal) c_{m,m} = V^(2m) / (2m+1)!, and for each m
the diagonal first, then k = m-1, ..., 0 (Fig. 1).

Everything here is exact rational arithmetic (``fractions.Fraction``) on
polynomials in one variable z, a list of coefficients, lowest power first.
The variable is z = x for polynomial potentials (the model-specific mode of
Sec. 3.3, where derivatives are taken explicitly) and z = t = tanh(alpha x)
for the modified Poeschl-Teller potential V = -lambda / cosh^2(alpha x)
(Eq. 1D-MPT), where V = -lambda (1 - t^2) and d/dx f(t) = alpha (1-t^2) f'(t)
keep every coefficient a polynomial in t (the content of Eq. 1D-MPTansatz).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
import math

ZERO = Fraction(0)


# ---------------------------------------------------------------------------
# polynomial arithmetic in z (lists of Fractions, lowest power first)
# ---------------------------------------------------------------------------

def _trim(a):
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return a


def padd(a, b):
    n = max(len(a), len(b))
    r = [ZERO] * n
    for i, v in enumerate(a):
        r[i] += v
    for i, v in enumerate(b):
        r[i] += v
    return _trim(r)


def pscale(a, s):
    return _trim([s * v for v in a])


def pmul(a, b):
    if not a or not b:
        return []
    r = [ZERO] * (len(a) + len(b) - 1)
    for i, u in enumerate(a):
        if u == 0:
            continue
        for j, v in enumerate(b):
            if v:
                r[i + j] += u * v
    return _trim(r)


def pder(a):
    """d/dz of a polynomial in z."""
    return _trim([i * a[i] for i in range(1, len(a))])


def peval(a, z):
    """sum_i a[i] z^i (Horner), in the arithmetic of z."""
    acc = 0 * z
    for v in reversed(a):
        acc = acc * z + (float(v) if isinstance(z, float) else v)
    return acc


# ---------------------------------------------------------------------------
# models: the ring variable, the x-derivative in that variable, and V
# ---------------------------------------------------------------------------

class Model:
    """A 1D potential in the ring of polynomials in z.

    kind 'x': z = x, D f = f'(z).
    kind 't': z = tanh(alpha x), D f = alpha (1 - z^2) f'(z).
    """

    def __init__(self, name, V, kind="x", alpha=Fraction(1)):
        self.name = name
        self.V = _trim([Fraction(v) for v in V])
        self.kind = kind
        self.alpha = Fraction(alpha)

    def D(self, f):
        """x-derivative of f(z(x)), again a polynomial in z."""
        if self.kind == "x":
            return pder(f)
        return pmul(pscale([Fraction(1), ZERO, Fraction(-1)], self.alpha), pder(f))

    def z_of_x(self, x):
        if self.kind == "x":
            return x
        return math.tanh(float(self.alpha) * float(x))

    def key(self):
        return (self.name, tuple(self.V), self.kind, self.alpha)


def make_model(name, params):
    """Models of the boundary: 'ho' (omega), 'aho' (A, g), 'dw' (h),
    'mpt' (lambda, alpha), 'poly' (v_0, v_1, ...).  Parameters are taken as
    exact rationals (every double is one)."""
    P = [Fraction(v) for v in params]
    if name == "ho":
        (w,) = P
        return Model(name, [0, 0, w * w / 2])                     # V = w^2 x^2 / 2
    if name == "aho":
        A, g = P
        return Model(name, [0, 0, A / 2, 0, g / 24])               # V = A x^2/2 + g x^4/24 (Sec. 3.3)
    if name == "dw":
        (h,) = P
        return Model(name, [h, 0, -2 * h, 0, h])                   # V = h (x^2 - 1)^2
    if name == "mpt":
        lam, alpha = P
        return Model(name, [-lam, 0, lam], kind="t", alpha=alpha)  # V = -lam (1 - t^2) = -lam / cosh^2(alpha x)
    if name == "poly":
        return Model(name, P)
    raise ValueError(f"unknown model {name!r}")


# ---------------------------------------------------------------------------
# the recursion
# ---------------------------------------------------------------------------

@lru_cache(maxsize=64)
def _coefficients(model_key, p):
    name, V, kind, alpha = model_key
    model = Model(name, V, kind, alpha)
    # x-derivatives of V up to order 2p-2, for the diagonal
    Vd = [model.V]
    for _ in range(2 * p):
        Vd.append(model.D(Vd[-1]))
    c = {}
    dc = {}                      # first x-derivatives c'_{m,k}
    for m in range(p):
        # diagonal first (Eq. diagonal)
        c[(m, m)] = pscale(Vd[2 * m], Fraction(1, math.factorial(2 * m + 1)))
        dc[(m, m)] = model.D(c[(m, m)])
        # then k = m-1 .. 0 (Fig. 1), each from Eq. 1Drec
        for k in range(m - 1, -1, -1):
            acc = pscale(c[(m, k + 1)], Fraction((2 * k + 2) * (2 * k + 1)))
            acc = padd(acc, model.D(dc[(m - 1, k)]))             # c''_{m-1,k}
            for l in range(0, m - 1):
                for r in range(max(0, k - m + l + 2), min(k, l) + 1):
                    acc = padd(acc, pscale(pmul(dc[(l, r)], dc[(m - l - 2, k - r)]), Fraction(-1)))
            for l in range(1, m - 1):
                for r in range(max(0, k - m + l + 2), min(k, l) + 1):
                    fac = 2 * r * (2 * k - 2 * r + 2)
                    if fac:
                        acc = padd(acc, pscale(pmul(c[(l, r)], c[(m - l - 1, k - r + 1)]), Fraction(-fac)))
            c[(m, k)] = pscale(acc, Fraction(1, 8 * (m + k + 1)))
            dc[(m, k)] = model.D(c[(m, k)])
    return c


def coefficients(model: Model, p: int):
    """dict (m, k) -> c_{m,k} as a polynomial in the model's ring variable,
    for 0 <= k <= m <= p-1."""
    if p < 1:
        raise ValueError("p >= 1")
    return _coefficients(model.key(), p)


def wp(model: Model, p: int, x, xb, eps):
    """W_p(x, xb; eps) = sum_{m<p} sum_{k<=m} c_{m,k}(x) eps^(m-k) xb^(2k).

    Exact when x, xb, eps are Fractions and the ring is 'x'; float otherwise."""
    c = coefficients(model, p)
    exact = all(isinstance(v, (Fraction, int)) for v in (x, xb, eps)) and model.kind == "x"
    if not exact:
        x, xb, eps = float(x), float(xb), float(eps)
    z = model.z_of_x(x)
    tot = 0 * eps
    for (m, k), poly in c.items():
        tot = tot + peval(poly, z) * eps ** (m - k) * xb ** (2 * k)
    return tot


def V_of_x(model: Model, x):
    return peval(model.V, model.z_of_x(x) if model.kind == "t" else x)


def flat_tables(model: Model, p: int):
    """c_{m,k} rounded to double, flattened for the C oracle:
    offsets[m*p + k] .. offsets[m*p + k] + lengths[m*p + k] index into coef."""
    c = coefficients(model, p)
    coef, offsets, lengths = [], [], []
    for m in range(p):
        for k in range(p):
            poly = c.get((m, k), []) if k <= m else []
            offsets.append(len(coef))
            lengths.append(len(poly))
            coef.extend(float(v) for v in poly)
    return coef, offsets, lengths
