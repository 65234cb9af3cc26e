"""The erf polynomial of the proposal network's GELU epilogue
(paper_1105_0542_gb300/csrc/erf_poly.h, written by erf_fit.py) against
scipy's erf, evaluated as the device evaluates it: erf(v/sqrt 2) = v Q(v^2)
with v clamped to [-3 sqrt 2, 3 sqrt 2], Horner in v^2 with single-precision
fused multiply-adds (each rounded once).  The largest error must stay far
below the bfloat16 rounding (2^-9) that the epilogue applies to every
activation."""
import os
import re

import numpy as np
from scipy.special import erf

HDR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_1105_0542_gb300", "csrc",
                   "erf_poly.h")


def _coefs():
    text = open(HDR).read()
    body = text[text.index("erf_poly(int k)"):]
    vals = [float(v.rstrip("f")) for v in re.findall(r"[-+]?\d\.\d+e[-+]\d+f", body)]
    clamp = float(re.search(r"kErfClamp = ([\d.]+)f", text).group(1))
    return np.array(vals, dtype=np.float32), np.float32(clamp)


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _erf_device(v):
    """erf(v / sqrt 2) as the device evaluates it"""
    c, clamp = _coefs()
    x = np.clip(v.astype(np.float32), -clamp, clamp)
    z = (x * x).astype(np.float32)
    p = np.full_like(z, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = _fma32(p, z, np.full_like(z, c[k]))
    return (x * p).astype(np.float32)


def test_erf_polynomial_error():
    v = np.linspace(-12, 12, 2_000_001).astype(np.float32)
    err = np.abs(_erf_device(v).astype(np.float64) - erf(v.astype(np.float64) / np.sqrt(2)))
    assert err.max() <= 1.2e-4, err.max()
    assert len(_coefs()[0]) == 8


def test_gelu_from_the_polynomial():
    v = np.linspace(-12, 12, 1_000_001).astype(np.float32)
    h = (v * np.float32(0.5)).astype(np.float32)
    g = _fma32(h, _erf_device(v), h)
    exact = 0.5 * v.astype(np.float64) * (1 + erf(v.astype(np.float64) / np.sqrt(2)))
    # relative to |v|: below a tenth of the bfloat16 rounding of the activation
    assert np.max(np.abs(g - exact) / (np.abs(v) + 1e-3)) <= 2.0 ** -9 / 10
