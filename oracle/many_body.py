"""The level-p effective potential of a system in d = D x M dimensions
(oracle side): Sec. 2.2, the expansion Eq. EXP in fully contracted terms
W_{m,k}(x, xb), the recursion Eq. MBrec, the diagonal Eq. DIA, solved in
the order of Fig. 1.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

The potential is a polynomial V(x_1..x_d) given as {exponent tuple:
coefficient}.  Every W_{m,k} is then a polynomial in the 2d variables
(x_1..x_d, xb_1..xb_d), homogeneous of degree 2k in xb; a polynomial is a
dict {(e_1..e_d, f_1..f_d): Fraction}.  All arithmetic is exact.

    W(x, xb; eps) = sum_{m<p} sum_{k<=m} eps^(m-k) W_{m,k}(x, xb)

    8 (m+k+1) W_{m,k} = lap W_{m-1,k} + lapb W_{m,k+1}
        - sum_{l=0}^{m-2} sum_r grad W_{l,r} . grad W_{m-l-2,k-r}
        - sum_{l=1}^{m-2} sum_r gradb W_{l,r} . gradb W_{m-l-1,k-r+1}
    r from max(0, k-m+l+2) to min(k, l);  W_{m,m} = (xb . grad)^(2m) V / (2m+1)!

The Monte Carlo side (per-sample log-weights) builds each coordinate's
bisection path as the one-dimensional oracle does, with normal j*d + c of the
sample's stream for heap midpoint j and coordinate c, and sums
-eps_n W(x_k, xb_k; eps_n) over the slices of every level n.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
import math

import numpy as np

from . import mc

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


def _deriv(poly, i):
    """d/d(variable i); variables 0..d-1 are x, d..2d-1 are xb."""
    out = {}
    for mono, v in poly.items():
        e = mono[i]
        if e == 0:
            continue
        m = list(mono)
        m[i] -= 1
        m = tuple(m)
        w = out.get(m, ZERO) + v * e
        if w:
            out[m] = w
        else:
            out.pop(m, None)
    return out


def _lap(poly, d, bar):
    out = {}
    for i in range(d):
        _add_into(out, _deriv(_deriv(poly, d * bar + i), d * bar + i))
    return out


def _dot_grad(a, b, d, bar):
    out = {}
    for i in range(d):
        _add_into(out, _mul(_deriv(a, d * bar + i), _deriv(b, d * bar + i)))
    return out


def potential(V, d):
    """V as a polynomial of the 2d variables (no xb dependence)."""
    out = {}
    for e, c in V.items():
        if len(e) != d:
            raise ValueError("exponent tuple of the wrong length")
        if c:
            _add_into(out, {tuple(e) + (0,) * d: Fraction(c)})
    return out


def _xb_dot_grad(poly, d):
    """(xb . grad) poly."""
    out = {}
    for i in range(d):
        xi = tuple(1 if j == d + i else 0 for j in range(2 * d))
        _add_into(out, _mul({xi: Fraction(1)}, _deriv(poly, i)))
    return out


def _key(V):
    return tuple(sorted((tuple(e), Fraction(c)) for e, c in V.items() if c))


@lru_cache(maxsize=32)
def _coefficients(Vkey, d, p):
    V = potential(dict(Vkey), d)
    W = {}
    for m in range(p):
        # diagonal, Eq. DIA
        t = V
        for _ in range(2 * m):
            t = _xb_dot_grad(t, d)
        W[(m, m)] = {mono: v / math.factorial(2 * m + 1) for mono, v in t.items()}
        for k in range(m - 1, -1, -1):
            acc = {}
            if (m - 1, k) in W:
                _add_into(acc, _lap(W[(m - 1, k)], d, 0))
            _add_into(acc, _lap(W[(m, k + 1)], d, 1))
            for l in range(0, m - 1):
                for r in range(max(0, k - m + l + 2), min(k, l) + 1):
                    _add_into(acc, _dot_grad(W[(l, r)], W[(m - l - 2, k - r)], d, 0), Fraction(-1))
            for l in range(1, m - 1):
                for r in range(max(0, k - m + l + 2), min(k, l) + 1):
                    _add_into(acc, _dot_grad(W[(l, r)], W[(m - l - 1, k - r + 1)], d, 1), Fraction(-1))
            W[(m, k)] = {mono: v / (8 * (m + k + 1)) for mono, v in acc.items()}
    return W


def coefficients(V, d, p):
    """{(m, k): W_{m,k}} for m < p, k <= m."""
    return _coefficients(_key(V), int(d), int(p))


def collapsed(V, d, p, eps):
    """W(x, xb; eps) as one polynomial {monomial: value} (exact for rational eps)."""
    out = {}
    for (m, k), poly in coefficients(V, d, p).items():
        _add_into(out, poly, Fraction(eps) ** (m - k))
    return out


def term_count(V, d, p):
    return len(collapsed(V, d, p, Fraction(1, 7)))


def _eval(poly, x, xb, absolute=False):
    """poly at points x, xb of shape (..., d), float64."""
    x = np.asarray(x, dtype=np.float64)
    xb = np.asarray(xb, dtype=np.float64)
    d = x.shape[-1]
    z = np.concatenate([x, xb], axis=-1)
    tot = np.zeros(x.shape[:-1])
    for mono, v in poly.items():
        term = np.full(x.shape[:-1], abs(float(v)) if absolute else float(v))
        for i, e in enumerate(mono):
            if e:
                term = term * (np.abs(z[..., i]) if absolute else z[..., i]) ** e
        tot = tot + term
    assert len(next(iter(poly))) == 2 * d if poly else True
    return tot


def wp(V, d, p, x, xb, eps):
    """W_p(x, xb; eps), term by term in float64."""
    tot = 0.0
    for (m, k), poly in coefficients(V, d, p).items():
        if poly:
            tot = tot + _eval(poly, x, xb) * eps ** (m - k)
    return tot


def wp_abs(V, d, p, x, xb, eps):
    """sum over terms of |term|: the scale the terms of W_p are summed from."""
    tot = 0.0
    for (m, k), poly in coefficients(V, d, p).items():
        if poly:
            tot = tot + _eval(poly, x, xb, absolute=True) * eps ** (m - k)
    return tot


# ---------------------------------------------------------------------------
# Monte Carlo: per-sample log-weights of the d-dimensional bisection paths
# ---------------------------------------------------------------------------

def path(a, b, T, s, seed, sample, instance=0, bits=53):
    """Points q[0..2^s, 0..d-1] of one sample: coordinate c of heap midpoint j
    takes normal j*d + c of the sample's stream (Sec. 4.1, exact bridge)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = a.shape[0]
    N = 1 << s
    z = mc.normals(seed, instance, sample, max((N - 1) * d, 1), bits)
    q = np.empty((N + 1, d))
    q[0], q[N] = a, b
    for n in range(1, s + 1):
        sig = math.sqrt(T / float(1 << (n + 1)))
        h = 1 << (s - n)
        for i in range(1 << (n - 1)):
            j = (1 << (n - 1)) - 1 + i
            idx = (2 * i + 1) * h
            for c in range(d):
                q[idx, c] = 0.5 * (q[idx - h, c] + q[idx + h, c]) + sig * z[j * d + c]
    return q


def logweights(V, d, p, a, b, T, s, seed, n, sample0=0, instance=0, bits=53):
    """(n, s) array of w_n = -eps_n sum_k W_p on the level-n subpath, and the
    condition scales eps_n sum_k sum |terms|; bits = 53 or 24 selects the
    uniforms (and normal layout) of the double or single-precision stream."""
    q = np.stack([path(a, b, T, s, seed, sample0 + i, instance, bits) for i in range(n)])
    w = np.empty((n, s))
    wa = np.empty((n, s))
    for lev in range(1, s + 1):
        eps = T / 2 ** lev
        st = 1 << (s - lev)
        ql, qr = q[:, :-1:st, :], q[:, st::st, :]
        x, xb = 0.5 * (ql + qr), 0.5 * (qr - ql)
        w[:, lev - 1] = -eps * wp(V, d, p, x, xb, eps).sum(axis=1)
        wa[:, lev - 1] = eps * wp_abs(V, d, p, x, xb, eps).sum(axis=1)
    return w, wa


def log_A_free(a, b, T):
    """Free amplitude of d independent coordinates."""
    return float(sum(mc.log_A_free(float(u), float(v), T) for u, v in zip(a, b)))


def level0(V, d, p, a, b, T):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return -T * float(wp(V, d, p, 0.5 * (a + b), 0.5 * (b - a), T))
