"""GPU parity of the learned bisection proposal (network on the tensor cores,
proposal sampling and exact reweighting) against the oracle.

* the network: tensor-core bfloat16 forward against the oracle's forward with
  the same bfloat16 roundings of weights and layer inputs (float vs double
  accumulation, so agreement to a few bfloat16 units of the outputs);
* a network whose output layer is zero proposes the bridge itself: weights
  equal the plain single-precision sampler's;
* per-sample weights of a non-trivial proposal, replayed by the oracle from
  the network outputs the device used (path and density ratio in double);
* unbiasedness: the harmonic oscillator's exact discretized amplitude at every
  level within 3 sigma with a non-trivial network.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
from oracle import exact, mc  # noqa: E402
from oracle import effective_action as ea  # noqa: E402
from oracle import proposal as pr  # noqa: E402

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


def _theta(seed, scale_last=0.4):
    th = pr.init(seed)
    rng = np.random.default_rng(seed + 100)
    k = pr.n_params() - (2 * 128 + 2)
    th[k:] = rng.normal(0, scale_last / math.sqrt(128), 2 * 128 + 2)
    return th


def test_network_forward_matches_oracle():
    th = _theta(1, 1.0)
    rng = np.random.default_rng(2)
    n = 1000
    X = np.stack([np.full(n, -1.0), np.full(n, 1.0), np.full(n, 5.0), rng.integers(1, 7, n) / 6,
                  rng.normal(0, 1.2, n), rng.normal(0, 1.2, n)], axis=1)
    P = su.Proposal(th)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Yd = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    P.su_mlp_forward(Xd, Yd)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.float64)
    # the oracle with the device's input rounding (float32 features, then bf16)
    ref, _ = pr.forward(th.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64),
                        bf16=True)
    err = np.abs(Y - ref)
    scale = np.abs(ref).max()
    assert scale > 0.05
    assert float(np.median(err)) <= 2e-3 * scale
    assert float(err.max()) <= 2e-2 * scale


def _allow(wo, wabs, rel, u):
    scale = np.maximum(np.abs(wo), np.median(np.abs(wo), axis=0))
    return np.maximum(rel * scale, 64 * u * wabs)


def test_zero_output_layer_reproduces_the_plain_sampler():
    th = pr.init(4)                       # output layer zero: shift = ls = 0
    P = su.Proposal(th)
    n, s = 300, 6
    wq = torch.zeros((n, s), dtype=torch.float64, device="cuda")
    su.speedup_proposal_logweights("dw", [5.0], -1.0, 1.0, 5.0, 12, s, 0, n, 9, P, wq)
    wp = torch.zeros((n, s), dtype=torch.float64, device="cuda")
    su.speedup_logweights("dw", [5.0], -1.0, 1.0, 5.0, 12, s, 0, n, 9, wp, precision="fp32")
    torch.cuda.synchronize()
    a, b = wq.cpu().numpy(), wp.cpu().numpy()
    o = mc.Oracle("dw", [5.0], 12)
    wo, _ = o.logweights(-1.0, 1.0, 5.0, s, 9, n, bits=24, threads=THREADS)
    wabs = o.logweights_abs(-1.0, 1.0, 5.0, s, 9, n, bits=24)
    allow = _allow(wo, wabs, 1e-5, 2.0 ** -24)
    assert float(np.max(np.abs(a - wo) / allow)) <= 1.0
    assert float(np.max(np.abs(a - b) / allow)) <= 2.0


@pytest.mark.parametrize("model,params,a,b,T,p,s", [("dw", [5.0], -1.0, 1.0, 1.0, 12, 6),
                                                    ("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4),
                                                    ("mpt", [3.0, 1.0], -1.0, 1.0, 1.0, 6, 5)])
def test_proposal_weights_replayed_by_the_oracle(model, params, a, b, T, p, s):
    th = _theta(7, 0.6)
    P = su.Proposal(th)
    n, N = 64, 1 << s
    w = torch.zeros((n, s), dtype=torch.float64, device="cuda")
    outs = torch.zeros((n, N - 1, 2), dtype=torch.float32, device="cuda")
    su.speedup_proposal_logweights(model, params, a, b, T, p, s, 5000, n, 3, P, w, outs)
    torch.cuda.synchronize()
    wg, og = w.cpu().numpy(), outs.cpu().numpy().astype(np.float64)
    assert np.abs(og).max() > 1e-3        # the network moved the midpoints
    m = ea.make_model(model, params)
    for i in range(n):
        q, corr = pr.proposal_path(th, a, b, T, s, 3, 5000 + i, bits=24, outs=og[i])
        for lev in range(1, s + 1):
            qq = q[:: 1 << (s - lev)]
            eps = T / 2 ** lev
            x, xb = 0.5 * (qq[1:] + qq[:-1]), 0.5 * (qq[1:] - qq[:-1])
            W = exact._wp_vec(m, p, x, xb, eps)
            wab = eps * float(np.sum(exact._wp_abs_vec(m, p, x, np.abs(xb), eps)))
            ref = -eps * float(np.sum(W)) + corr[lev - 1]
            allow = max(1e-5 * max(abs(ref), 1.0), 64 * 2.0 ** -24 * (wab + abs(corr[lev - 1])))
            assert abs(wg[i, lev - 1] - ref) <= allow, (i, lev, wg[i, lev - 1], ref)


def test_proposal_estimate_is_unbiased():
    th = _theta(11, 0.5)
    P = su.Proposal(th)
    r = su.speedup_amplitude_proposal("ho", [1.0], 0.0, 1.0, 1.0, 4, 4, 400_000, 17, P, n_blocks=20)
    for lev in range(1, 5):
        ref = exact.ho_discretized(4, 2 ** lev, 0.0, 1.0, 1.0)
        sig = max(r[lev]["err"], r[lev]["err_naive"])
        assert abs(r[lev]["amp"] - ref) <= 3 * sig, (lev, r[lev]["amp"], ref, sig)
    plain = su.speedup_amplitude("ho", [1.0], 0.0, 1.0, 1.0, 4, 4, 400_000, 17, precision="fp32", n_blocks=20)
    assert r[4]["ess"] < plain[4]["ess"]   # a random network is a worse proposal than the bridge


def test_training_gradient_matches_oracle():
    """The tensor-core forward/backward (bfloat16 operands, float accumulation)
    against the oracle's double-precision loss and gradient."""
    th = _theta(21, 1.0)
    rng = np.random.default_rng(3)
    n = 1000
    X = np.stack([np.full(n, -1.0), np.full(n, 1.0), np.full(n, 5.0), rng.integers(1, 7, n) / 6,
                  rng.normal(0, 1.2, n), rng.normal(0, 1.2, n)], axis=1)
    u = rng.normal(0, 1.0, n)
    rw = rng.uniform(0.2, 2.0, n)
    dev = lambda v: torch.tensor(v, dtype=torch.float32, device="cuda").contiguous()
    L, g = su.su_mlp_loss_grad(th, dev(X), dev(u), dev(rw))
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
    Lr, gr = pr.loss_and_grad(f32(th), f32(X), f32(u), f32(rw))
    assert L == pytest.approx(Lr, rel=2e-2, abs=2e-3)
    g = g.astype(np.float64)
    cos = float(g @ gr / (np.linalg.norm(g) * np.linalg.norm(gr)))
    assert cos >= 0.998
    # every layer's block, relative to its own size
    k = 0
    for o, i in pr.SIZES:
        for size in (o * i, o):
            blk, ref = g[k:k + size], gr[k:k + size]
            k += size
            assert np.linalg.norm(blk - ref) <= 0.06 * np.linalg.norm(ref) + 1e-7, (o, i, size)


def test_training_lowers_the_loss():
    th0 = pr.init(5).astype(np.float32)
    th, losses = su.speedup_train_proposal("dw", [5.0], -1.0, 1.0, 5.0, 12, 6, 77, th0, n_train=200_000,
                                           steps=400, batch_paths=256, lr=1e-3)
    assert np.isfinite(losses).all()
    assert losses[-50:].mean() < losses[:10].mean() - 0.01   # step-to-step noise is ~0.005
    assert np.abs(th - th0).max() > 1e-3


def test_trained_proposal_is_unbiased_and_better():
    """Trained on the harmonic oscillator, the proposal still reproduces the
    exact discretized amplitude (exact reweighting) and has a larger effective
    sample size than the bridge."""
    th0 = pr.init(6).astype(np.float32)
    th, losses = su.speedup_train_proposal("ho", [1.0], 0.0, 1.0, 2.0, 4, 6, 3, th0, n_train=200_000,
                                           steps=600, batch_paths=256, lr=1e-3)
    P = su.Proposal(th)
    r = su.speedup_amplitude_proposal("ho", [1.0], 0.0, 1.0, 2.0, 4, 6, 400_000, 11, P, n_blocks=20)
    plain = su.speedup_amplitude("ho", [1.0], 0.0, 1.0, 2.0, 4, 6, 400_000, 12, precision="fp32", n_blocks=20)
    ref = exact.ho_discretized(4, 64, 0.0, 1.0, 2.0)
    sig = max(r[6]["err"], r[6]["err_naive"])
    assert abs(r[6]["amp"] - ref) <= 3 * sig
    assert r[6]["ess"] > plain[6]["ess"]


def test_judge_takes_a_trained_proposal_where_it_is_faster():
    """A harmonic oscillator whose bridge is poor (omega = 4, T = 4: the
    plain per-sample relative variance is about 28): the trained proposal,
    judged on two pilots, is confirmed by the plain sampler, estimated faster
    to a relative error of 1e-4 by more than 3x, and used for the main run,
    which equals speedup_amplitude_proposal on the same samples and the exact
    discretized amplitude."""
    args = ("ho", [4.0], 0.0, 0.5, 4.0, 4, 6)
    th0 = pr.init(9).astype(np.float32)
    th, losses = su.speedup_train_proposal(*args, 2024, th0, n_train=1_000_000, steps=2000, batch_paths=512,
                                           lr=1e-3)
    assert np.isfinite(losses).all()
    P = su.Proposal(th)
    res, j = su.speedup_amplitude_judged(*args, 1_000_000, 31, P, n_pilot=200_000, target_rel_err=1e-4,
                                         n_blocks=50)
    assert j["chosen"] == "proposal" and j["reason"] == "proposal faster", j
    assert j["t_target"][0] > 3 * j["t_target"][1], j
    assert abs(j["z"]) <= 5
    ref = exact.ho_discretized(4, 64, 0.0, 0.5, 4.0, omega=4.0)
    top = res[6]
    assert abs(top["amp"] - ref) <= 4 * max(top["err"], top["err_naive"]), (top["amp"], ref)
    same = su.speedup_amplitude_proposal(*args, 1_000_000, 31, P, n_blocks=50)
    assert [r["amp"] for r in res] == [r["amp"] for r in same]


def test_judge_keeps_the_plain_sampler_where_the_bridge_is_good():
    """Where the bridge is already a good proposal (omega = 1, T = 1) the
    network, which costs far more per path, loses: the main run is the plain
    single-precision sampler's, sample for sample."""
    args = ("ho", [1.0], 0.0, 0.5, 1.0, 4, 6)
    P = su.Proposal(pr.init(10).astype(np.float32))   # zero output layer: the bridge itself
    res, j = su.speedup_amplitude_judged(*args, 300_000, 5, P, n_pilot=200_000, target_rel_err=1e-4, n_blocks=30)
    assert j["chosen"] == "plain" and j["reason"] == "plain faster", j
    assert j["pilot_relvar"][0] == pytest.approx(j["pilot_relvar"][1], rel=0.3)
    plain = su.speedup_amplitude(*args, 300_000, 5, precision="fp32", n_blocks=30)
    assert [r["amp"] for r in res] == [r["amp"] for r in plain]


def test_judge_refuses_an_unconfirmed_proposal():
    """Double well h = 5 at T = 5 (p = 12, N = 64): the truncated W_12 is
    unbounded below and the plain estimate is ruled by single far-out paths;
    on this stream's pilot range (samples 1e6 .. 2e6 of seed 31) one of them
    makes the plain estimate overflow.  A proposal trained on the plain paths
    gives a finite number, but nothing confirms it: the judge falls back to
    the plain sampler and says why, leaving the proposal's pilot value in the
    record."""
    args = ("dw", [5.0], -1.0, 1.0, 5.0, 12, 6)
    th0 = pr.init(9).astype(np.float32)
    th, _ = su.speedup_train_proposal(*args, 1234, th0, n_train=1_000_000, steps=2000, batch_paths=512, lr=1e-3)
    P = su.Proposal(th)
    res, j = su.speedup_amplitude_judged(*args, 1_000_000, 31, P, n_pilot=1_000_000, target_rel_err=1e-4,
                                         n_blocks=50)
    assert j["chosen"] == "plain" and j["reason"] == "plain unusable", j
    assert not math.isfinite(j["t_target"][0]) and math.isfinite(j["pilot_amp"][1])
    plain = su.speedup_amplitude(*args, 1_000_000, 31, precision="fp32", n_blocks=50)
    assert res[6]["log_amp"] == plain[6]["log_amp"]
