"""Python side of the CPU Monte Carlo oracle (builds and calls mc_oracle.c).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

The estimator (Sec. 4; the normalisation of Sec. 4.1 written out):
bisection samples the free Brownian bridge from a to b, whose density times
exp(-S_kin) (2 pi eps)^(-N/2) is the free amplitude
A_free = (2 pi T)^(-1/2) exp(-(b-a)^2 / (2T)) (Sec. 2.1 with W = 0), so

    A_N^(p)(a,b;T) = A_free * E[exp(w_n)],   w_n = -eps_n sum_k W_p(x_k, xb_k; eps_n).

The mean is taken over n_mc samples; the error is the standard deviation of
n_blocks contiguous block means divided by sqrt(n_blocks) (the paper's
<f^2> - <f>^2 error of Sec. 4.1 is reported beside it).  Level n = 0 is the
single analytic term A_free exp(-T W_p((a+b)/2, (b-a)/2; T)) with error 0.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from . import effective_action as ea

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile mc_oracle.c with gcc (plain C, OpenMP over samples)."""
    src = os.path.join(_HERE, "mc_oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fopenmp", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _WP(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("ring", ctypes.c_int), ("alpha", ctypes.c_double),
                ("coef", ctypes.POINTER(ctypes.c_double)),
                ("off", ctypes.POINTER(ctypes.c_int)),
                ("len", ctypes.POINTER(ctypes.c_int))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64, u32, i64, i32, d = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                     ctypes.c_int, ctypes.c_double)
            pd = ctypes.POINTER(ctypes.c_double)
            pu32 = ctypes.POINTER(ctypes.c_uint32)
            L.oracle_philox.argtypes = [pu32, pu32, pu32]
            L.oracle_philox_words.argtypes = [u64, u32, u64, u32, pu32]
            L.oracle_normals.argtypes = [u64, u32, u64, i64, i32, pd]
            L.oracle_Wp.argtypes = [ctypes.POINTER(_WP), d, d, d]
            L.oracle_Wp.restype = d
            L.oracle_path.argtypes = [u64, u32, u64, i32, d, d, d, i32, d, pd, pd]
            L.oracle_level0.argtypes = [ctypes.POINTER(_WP), d, d, d]
            L.oracle_level0.restype = d
            L.oracle_logweights.argtypes = [ctypes.POINTER(_WP), d, d, d, i32, u64, u32, i64, i64,
                                             i32, d, i32, pd]
            L.oracle_logweights.restype = i32
            L.oracle_logweights_abs.argtypes = [ctypes.POINTER(_WP), d, d, d, i32, u64, u32, i64, i64,
                                                i32, d, pd]
            L.oracle_logweights_abs.restype = None
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------

def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox(c, k, o)
    return [int(v) for v in o]


def philox_words(seed, instance, sample, call):
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox_words(seed, instance, sample, call, o)
    return [int(v) for v in o]


def normals(seed, instance, sample, n, bits=53):
    z = np.empty(n, dtype=np.float64)
    lib().oracle_normals(seed, instance, sample, n, bits, _dptr(z))
    return z


# ---------------------------------------------------------------------------
# the estimator
# ---------------------------------------------------------------------------

def log_A_free(a, b, T):
    return -0.5 * math.log(2.0 * math.pi * T) - (b - a) ** 2 / (2.0 * T)


class Oracle:
    """Level-p effective action of one model, ready for sampling."""

    def __init__(self, model_name, params, p):
        self.model = ea.make_model(model_name, params)
        self.p = int(p)
        coef, off, ln = ea.flat_tables(self.model, self.p)
        self._coef = np.asarray(coef if coef else [0.0], dtype=np.float64)
        self._off = np.asarray(off, dtype=np.int32)
        self._len = np.asarray(ln, dtype=np.int32)
        self._wp = _WP(self.p, 0 if self.model.kind == "x" else 1, float(self.model.alpha),
                       _dptr(self._coef),
                       self._off.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       self._len.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))

    def Wp(self, x, xb, eps):
        return lib().oracle_Wp(ctypes.byref(self._wp), float(x), float(xb), float(eps))

    def level0(self, a, b, T):
        return lib().oracle_level0(ctypes.byref(self._wp), a, b, T)

    def path(self, a, b, T, s, seed, sample, instance=0, bits=53, wf=1.0):
        q = np.empty((1 << s) + 1, dtype=np.float64)
        corr = np.empty(max(s, 1), dtype=np.float64)
        lib().oracle_path(seed, instance, sample, s, a, b, T, bits, wf, _dptr(q), _dptr(corr))
        return q, corr[:s]

    def logweights(self, a, b, T, s, seed, nsamples, sample0=0, instance=0, bits=53,
                   wf=1.0, threads=1):
        """(nsamples, s) array of w_n, n = 1..s; returns (w, threads used)."""
        w = np.empty((max(nsamples, 0), max(s, 0)), dtype=np.float64)
        used = 1
        if s >= 1 and nsamples > 0:
            used = lib().oracle_logweights(ctypes.byref(self._wp), a, b, T, s, seed, instance,
                                           sample0, nsamples, bits, wf, threads, _dptr(w))
        return w, used

    def logweights_abs(self, a, b, T, s, seed, nsamples, sample0=0, instance=0, bits=53, wf=1.0):
        """(nsamples, s) condition scales eps_n sum_k sum_terms |term| of the same
        samples: the size of the numbers each w_n is summed from."""
        out = np.empty((max(nsamples, 0), max(s, 0)), dtype=np.float64)
        if s >= 1 and nsamples > 0:
            lib().oracle_logweights_abs(ctypes.byref(self._wp), a, b, T, s, seed, instance, sample0,
                                        nsamples, bits, wf, _dptr(out))
        return out

    def amplitude(self, a, b, T, s, n_mc, seed, n_blocks=64, instance=0, bits=53, wf=1.0,
                  threads=1):
        w, _ = self.logweights(a, b, T, s, seed, n_mc, instance=instance, bits=bits, wf=wf,
                               threads=threads)
        return estimate(w, self.level0(a, b, T), a, b, T, n_blocks)


def block_bounds(n_mc, n_blocks):
    """Block b holds samples [b n_mc // n_blocks, (b+1) n_mc // n_blocks)."""
    return [(b * n_mc // n_blocks, (b + 1) * n_mc // n_blocks) for b in range(n_blocks)]


def _exp(x):
    """exp that returns inf instead of raising where the result overflows"""
    return math.exp(x) if x < 709.78 else float("inf")


def estimate(w, w0, a, b, T, n_blocks):
    """Per-level results from per-sample log-weights w (n_mc, s)."""
    n_mc, s = w.shape
    laf = log_A_free(a, b, T)
    out = [dict(n=0, amp=_exp(laf + w0), log_amp=laf + w0, err=0.0, rel_err=0.0,
                err_naive=0.0, ess=float(n_mc), max_share=1.0 / max(n_mc, 1))]
    nb = min(n_blocks, n_mc)
    for lev in range(1, s + 1):
        x = w[:, lev - 1]
        M = float(np.max(x))
        e = np.exp(x - M)
        S = float(np.sum(e))
        Q = float(np.sum(e * e))
        mean = S / n_mc
        mu = np.array([np.mean(e[lo:hi]) for lo, hi in block_bounds(n_mc, nb)])
        err_b = float(np.std(mu, ddof=1) / math.sqrt(nb)) if nb > 1 else float("nan")
        var = max(Q / n_mc - mean * mean, 0.0)
        err_n = math.sqrt(var / (n_mc - 1)) if n_mc > 1 else float("nan")
        scale = _exp(laf + M)
        out.append(dict(n=lev, amp=scale * mean, log_amp=laf + M + math.log(mean),
                        err=scale * err_b, rel_err=err_b / mean, err_naive=scale * err_n,
                        ess=S * S / Q, max_share=1.0 / S))
    return out
