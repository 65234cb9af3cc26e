"""Oracle of the learned bisection proposal (double precision, numpy).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

The proposal replaces the bridge density of each bisection midpoint (Sec. 4.1)
by a Gaussian whose shift and log-scale a small network predicts from the
instance and the midpoint's two parents; exact importance weights keep the
estimator of A_N^(p) unbiased.  Written out:

* network: x = (a, b, T, n/s, q_L, q_R) -> Linear(6,128) -> GELU ->
  Linear(128,128) -> GELU -> Linear(128,128) -> GELU -> Linear(128,2) =
  (shift, ls); GELU(v) = v (1 + erf(v / sqrt 2)) / 2 (the exact form);
  weights stored [out][in] with the bias after each matrix, in one flat float
  vector (W1, b1, W2, b2, W3, b3, W4, b4).
* proposal of a midpoint at level n with parents q_L, q_R: with
  mu = (q_L + q_R)/2 and the bridge width sigma_n (sigma_n^2 = T/2^(n+1)),
  q = mu + sigma_n (shift + e^ls z), z standard normal (the same normal j of
  the Philox stream the plain sampler would use).
* exact weight of that midpoint: log phi_bridge(q) - log phi_proposal(q)
  = z^2/2 - (shift + e^ls z)^2/2 + ls, added to w_n of every level n' >= n.
* training objective (weighted maximum likelihood on plain-sampler paths):
  L = sum_rows r_w [ls + (u - shift)^2 e^(-2 ls) / 2] / sum_rows r_w with
  u = (q - mu)/sigma_n the midpoint's standardized offset and r_w the
  self-normalised weight of its path.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from . import effective_action as ea
from . import mc

SIZES = [(128, 6), (128, 128), (128, 128), (2, 128)]


def n_params():
    return sum(o * i + o for o, i in SIZES)


def init(seed=0):
    """Uniform(+-1/sqrt(fan_in)) weights and biases, last layer zero (so the
    untrained proposal is the bridge itself)."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (o, i) in enumerate(SIZES):
        bound = 1.0 / math.sqrt(i)
        if li == len(SIZES) - 1:
            parts += [np.zeros(o * i), np.zeros(o)]
        else:
            parts += [rng.uniform(-bound, bound, o * i), rng.uniform(-bound, bound, o)]
    return np.concatenate(parts)


def unpack(theta):
    out, k = [], 0
    for o, i in SIZES:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def gelu(v):
    return 0.5 * v * (1.0 + erf(v / math.sqrt(2.0)))


def gelu_grad(v):
    return 0.5 * (1.0 + erf(v / math.sqrt(2.0))) + v * np.exp(-0.5 * v * v) / math.sqrt(2.0 * math.pi)


def forward(theta, X, bf16=False):
    """(n, 2) outputs (shift, ls) and the pre-activations.  With bf16=True the
    weights and every layer input are rounded to bfloat16 first (round to
    nearest even), as a bfloat16 tensor-core network sees them."""
    layers = unpack(theta)
    h = np.asarray(X, dtype=np.float64)
    pres = []
    for li, (W, b) in enumerate(layers):
        if bf16:
            h, W = round_bf16(h), round_bf16(W)
        pre = h @ W.T + b
        pres.append(pre)
        h = gelu(pre) if li < len(layers) - 1 else pre
    return h, pres


def loss_and_grad(theta, X, u, rw):
    """Weighted negative log-likelihood of standardized midpoints u and its
    gradient with respect to the flat parameter vector."""
    layers = unpack(theta)
    Y, pres = forward(theta, X)
    shift, ls = Y[:, 0], Y[:, 1]
    rw = np.asarray(rw, dtype=np.float64)
    norm = rw.sum()
    d = u - shift
    e2 = np.exp(-2.0 * ls)
    L = float(np.sum(rw * (ls + 0.5 * d * d * e2)) / norm)
    dY = np.stack([-(d * e2), 1.0 - d * d * e2], axis=1) * (rw / norm)[:, None]
    grads = [None] * len(layers)
    acts = [np.asarray(X, dtype=np.float64)] + [gelu(p) for p in pres[:-1]]
    g = dY
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (g.T @ acts[li], g.sum(axis=0))
        if li > 0:
            g = (g @ W) * gelu_grad(pres[li - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return L, flat


def round_bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# sampling with the proposal, one path at a time
# ---------------------------------------------------------------------------

def features(a, b, T, n, s, qL, qR):
    return np.array([a, b, T, n / s, qL, qR], dtype=np.float64)


def proposal_path(theta, a, b, T, s, seed, sample, instance=0, bits=24, bf16=True, outs=None):
    """Path q[0..2^s] and the cumulative log proposal weight per level
    (corr[n-1] = sum over midpoints of levels <= n).  If outs is given
    (sequence of (shift, ls) per heap index j), those network outputs are used
    instead of evaluating the network (to replay a device run exactly)."""
    N = 1 << s
    q = np.empty(N + 1)
    q[0], q[N] = a, b
    z = mc.normals(seed, instance, sample, N - 1, bits)
    corr = np.zeros(s)
    c = 0.0
    for n in range(1, s + 1):
        sig = math.sqrt(T / 2 ** (n + 1))
        h = 1 << (s - n)
        rows = []
        for i in range(1 << (n - 1)):
            k = (2 * i + 1) * h
            rows.append(features(a, b, T, n, s, q[k - h], q[k + h]))
        if outs is None:
            Y, _ = forward(theta, np.stack(rows), bf16=bf16)
        for i in range(1 << (n - 1)):
            j = (1 << (n - 1)) - 1 + i
            k = (2 * i + 1) * h
            sh, ls = (Y[i] if outs is None else outs[j])
            t = sh + math.exp(ls) * z[j]
            q[k] = 0.5 * (q[k - h] + q[k + h]) + sig * t
            c += 0.5 * z[j] * z[j] - 0.5 * t * t + ls
        corr[n - 1] = c
    return q, corr


def proposal_logweights(theta, model_name, params, p, a, b, T, s, seed, nsamples, sample0=0, instance=0,
                        bits=24, bf16=True):
    """(nsamples, s) log-weights w_n + proposal weight, n = 1..s."""
    model = ea.make_model(model_name, params)
    from .exact import _wp_vec
    out = np.empty((nsamples, s))
    for i in range(nsamples):
        q, corr = proposal_path(theta, a, b, T, s, seed, sample0 + i, instance, bits, bf16)
        for n in range(1, s + 1):
            qq = q[:: 1 << (s - n)]
            eps = T / 2 ** n
            W = _wp_vec(model, p, 0.5 * (qq[1:] + qq[:-1]), 0.5 * (qq[1:] - qq[:-1]), eps)
            out[i, n - 1] = -eps * float(np.sum(W)) + corr[n - 1]
    return out


def training_rows(q_paths, a, b, T, s):
    """Features X and standardized offsets u of every midpoint of every path
    (rows grouped by path, heap order within a path)."""
    X, U = [], []
    for q in q_paths:
        for n in range(1, s + 1):
            sig = math.sqrt(T / 2 ** (n + 1))
            h = 1 << (s - n)
            for i in range(1 << (n - 1)):
                k = (2 * i + 1) * h
                X.append(features(a, b, T, n, s, q[k - h], q[k + h]))
                U.append((q[k] - 0.5 * (q[k - h] + q[k + h])) / sig)
    return np.array(X), np.array(U)
