"""Pins of the oracle's learned-proposal network, reweighting and loss (CPU).

* the loss gradient against central finite differences;
* bfloat16 rounding against torch's float32 -> bfloat16 conversion;
* the zero-initialised output layer gives the bridge itself: proposal weights
  equal the plain weights sample by sample;
* exact reweighting keeps the estimator unbiased: with a non-trivial network
  the harmonic oscillator's exact discretized amplitude is recovered within
  3 sigma at every level.
"""
import math

import numpy as np
import pytest

from oracle import exact, mc
from oracle import proposal as pr


def _random_theta(seed, scale_last=0.3):
    th = pr.init(seed)
    rng = np.random.default_rng(seed + 1)
    k = pr.n_params() - (2 * 128 + 2)
    th[k:] = rng.normal(0, scale_last / math.sqrt(128), 2 * 128 + 2)
    return th


def test_gradient_matches_finite_differences():
    th = _random_theta(3)
    rng = np.random.default_rng(0)
    X = rng.normal(size=(20, 6))
    u = rng.normal(size=20)
    rw = rng.uniform(0.1, 2.0, size=20)
    L, g = pr.loss_and_grad(th, X, u, rw)
    idx = list(rng.choice(pr.n_params(), 60, replace=False)) + [pr.n_params() - 1, 0]
    for k in idx:
        h = 1e-6 * max(1.0, abs(th[k]))
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (pr.loss_and_grad(tp, X, u, rw)[0] - pr.loss_and_grad(tm, X, u, rw)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-8), k


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(size=5000) * 10 ** rng.uniform(-6, 6, 5000),
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -2.5, 0.0]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(pr.round_bf16(x), ref)


def test_zero_output_layer_is_the_bridge():
    th = pr.init(7)
    o = mc.Oracle("aho", [1.0, 1.0], 4)
    w_plain, _ = o.logweights(0.0, 1.0, 1.0, 4, 21, 30, bits=24)
    w_prop = pr.proposal_logweights(th, "aho", [1.0, 1.0], 4, 0.0, 1.0, 1.0, 4, 21, 30, bits=24)
    np.testing.assert_allclose(w_prop, w_plain, rtol=1e-12, atol=1e-13)


def test_reweighting_is_unbiased_for_the_harmonic_oscillator():
    th = _random_theta(11, scale_last=0.5)
    n = 6000
    w = pr.proposal_logweights(th, "ho", [1.0], 4, 0.0, 1.0, 1.0, 3, 99, n, bits=53, bf16=False)
    o = mc.Oracle("ho", [1.0], 4)
    res = mc.estimate(w, o.level0(0.0, 1.0, 1.0), 0.0, 1.0, 1.0, 20)
    for lev in range(1, 4):
        ref = exact.ho_discretized(4, 2 ** lev, 0.0, 1.0, 1.0)
        sig = max(res[lev]["err"], res[lev]["err_naive"])
        assert abs(res[lev]["amp"] - ref) <= 3 * sig, (lev, res[lev]["amp"], ref, sig)
    # the proposal really moved the paths: the weights are not the plain ones
    wp, _ = o.logweights(0.0, 1.0, 1.0, 3, 99, 50)
    assert np.abs(w[:50] - wp).max() > 1e-2


def test_training_rows_recover_the_normals():
    o = mc.Oracle("aho", [1.0, 1.0], 4)
    q, _ = o.path(0.0, 1.0, 1.0, 3, 5, 17)
    X, U = pr.training_rows([q], 0.0, 1.0, 1.0, 3)
    z = mc.normals(5, 0, 17, 7)
    assert X.shape == (7, 6)
    np.testing.assert_allclose(U, z, rtol=1e-12, atol=1e-12)
