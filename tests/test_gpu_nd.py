"""GPU parity of the estimator for systems of several coordinates (Sec. 2.2,
Eq. MBrec / Eq. DIA) against the oracle, through the C ABI.

* Per-sample log-weights w_n on identical Philox streams (coordinate c of
  midpoint j = normal j d + c) against the oracle's exact-rational W on the
  oracle's own paths: within 1e-12 relative, or the summation bound where the
  terms cancel; d = 1..4.
* d = 1 against the one-dimensional polynomial model on the same stream
  (two independent device paths: 1e-12).
* The estimator against the oracle's estimator on the same samples; the
  plan interface (execute / range / finalize) against the one-call entry.
* A coupled harmonic oscillator against the exact discretized amplitude
  (product of its normal modes' Gaussian integrals) within 3 sigma at every
  level; a separable 2D anharmonic oscillator against the product of the
  one-dimensional sinc-DVR continuum amplitudes within 4 sigma.
"""
from fractions import Fraction as F
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
from oracle import exact, mc  # noqa: E402
from oracle import many_body as mb  # noqa: E402

pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


def _gpu_w(V, a, b, T, p, s, n, seed, sample0=0, precision="fp64"):
    w = torch.full((n, s), float("nan"), dtype=torch.float64, device="cuda")
    su.speedup_logweights_nd(V, a, b, T, p, s, sample0, n, seed, w, precision=precision)
    torch.cuda.synchronize()
    return w.cpu().numpy()


def _excess(wg, wo, wabs, rel, u):
    scale = np.maximum(np.abs(wo), np.median(np.abs(wo), axis=0))
    allow = np.maximum(rel * scale, 64 * u * wabs)
    allow = np.maximum(allow, 1e-300)
    return float(np.max(np.abs(wg - wo) / allow))


def _frac(V):
    return {k: F(v) for k, v in V.items()}


AHO2 = {(2, 0): 0.5, (0, 2): 0.5, (4, 0): 1 / 24, (0, 4): 1 / 24, (2, 2): 1 / 12}
GEN2 = {(2, 0): 0.5, (0, 2): 0.75, (1, 1): 0.2, (2, 1): 1 / 3, (0, 3): -1 / 7, (4, 0): 0.1, (1, 3): 0.05,
        (0, 4): 1 / 12, (1, 0): -1 / 3}
GEN3 = {(2, 0, 0): 0.5, (0, 2, 0): 0.5, (0, 0, 2): 0.5, (1, 1, 0): 0.2, (0, 1, 1): 1 / 7, (2, 0, 2): 1 / 11,
        (4, 0, 0): 1 / 24, (0, 4, 0): 1 / 24, (0, 0, 4): 1 / 30, (1, 1, 1): 1 / 9}
TWO_2D = {(2, 0, 0, 0): 0.5, (0, 2, 0, 0): 0.5, (0, 0, 2, 0): 0.5, (0, 0, 0, 2): 0.5,
          (2, 0, 2, 0): 0.1, (1, 0, 1, 0): -0.2, (0, 1, 0, 1): -0.2, (0, 2, 0, 2): 0.1, (4, 0, 0, 0): 0.05}
SEXTIC2 = {(6, 0): 0.01, (0, 2): 0.5, (3, 3): 0.02, (2, 0): 0.5}

CASES = [
    # name, V, a, b, T, p, s, n, seed, sample0
    ("aho2-p10", AHO2, (0.0, 0.2), (1.0, -0.3), 1.0, 10, 6, 200, 1234, 0),
    ("gen2-p6", GEN2, (-0.5, 0.3), (0.7, 0.1), 1.0, 6, 5, 130, 7, 10_000),
    ("gen2-p12", GEN2, (0.1, 0.0), (0.4, 0.2), 0.5, 12, 4, 40, 9, 0),
    ("gen3-p6", GEN3, (0.0, 0.1, 0.2), (0.5, -0.5, 0.0), 1.0, 6, 4, 64, 3, (1 << 32) - 5),
    ("two-2d-p4", TWO_2D, (0.3, 0.0, -0.3, 0.1), (0.2, 0.4, -0.1, -0.2), 1.0, 4, 4, 50, 5, 0),
    ("sextic2-p6", SEXTIC2, (0.2, -0.1), (0.1, 0.6), 0.8, 6, 6, 60, 2, 0),
    ("d1-p8", {(2,): 0.5, (4,): 1 / 24, (3,): -0.1}, (0.0,), (1.0,), 1.0, 8, 7, 100, 1234, 0),
    ("s1", GEN2, (0.0, 0.0), (0.5, 0.5), 0.4, 8, 1, 33, 4, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_nd_logweights_match_oracle(case):
    _, V, a, b, T, p, s, n, seed, s0 = case
    d = len(a)
    wg = _gpu_w(V, a, b, T, p, s, n, seed, s0)
    wo, wabs = mb.logweights(_frac(V), d, p, np.array(a), np.array(b), T, s, seed, n, s0)
    assert np.isfinite(wg).all()
    assert _excess(wg, wo, wabs, 1e-12, U64) <= 1.0


@pytest.mark.parametrize("case", CASES[:6], ids=[c[0] for c in CASES[:6]])
def test_nd_logweights_fp32_match_oracle(case):
    """Single precision: path and W in float on the stream's float layout,
    against the oracle fed the same 24-bit uniforms (1e-5 relative, or the
    float summation bound where the terms cancel)."""
    _, V, a, b, T, p, s, n, seed, s0 = case
    d = len(a)
    wg = _gpu_w(V, a, b, T, p, s, n, seed, s0, precision="fp32")
    wo, wabs = mb.logweights(_frac(V), d, p, np.array(a), np.array(b), T, s, seed, n, s0, bits=24)
    assert np.isfinite(wg).all()
    assert _excess(wg, wo, wabs, 1e-5, U32) <= 1.0


def test_nd_fp32_and_fp64_amplitudes_agree():
    """Independent streams: the two precisions' amplitudes within 3 combined
    sigma at every level."""
    V, a, b, T, p, s = AHO2, (0.0, 0.2), (1.0, -0.3), 1.0, 10, 6
    r64 = su.speedup_amplitude_nd(V, a, b, T, p, s, 1_000_000, 5, n_blocks=64)
    r32 = su.speedup_amplitude_nd(V, a, b, T, p, s, 1_000_000, 5, n_blocks=64, precision="fp32")
    for lev in range(1, s + 1):
        sig = math.hypot(r64[lev]["err"], r32[lev]["err"])
        assert abs(r64[lev]["amp"] - r32[lev]["amp"]) <= 3 * sig, lev


def test_one_coordinate_equals_the_one_dimensional_model():
    """d = 1 draws midpoint j from normal j, as the one-dimensional sampler."""
    coeffs = [0.2, -0.5, 0.3, 0.25, 0.1]
    V = {(i,): v for i, v in enumerate(coeffs)}
    s, n = 8, 500
    wn = _gpu_w(V, (-0.5,), (0.7,), 0.8, 7, s, n, 8)
    w1 = torch.full((n, s), float("nan"), dtype=torch.float64, device="cuda")
    su.speedup_logweights("poly", coeffs, -0.5, 0.7, 0.8, 7, s, 0, n, 8, w1)
    torch.cuda.synchronize()
    w1 = w1.cpu().numpy()
    scale = np.maximum(np.abs(w1), np.median(np.abs(w1), axis=0))
    assert float(np.max(np.abs(wn - w1) / scale)) <= 1e-12


def test_nd_estimator_matches_oracle_estimator_and_the_plan_interface():
    V, a, b, T, p, s, n = GEN2, (-0.5, 0.3), (0.7, 0.1), 1.0, 6, 4, 3000
    r = su.speedup_amplitude_nd(V, a, b, T, p, s, n, 21, n_blocks=20)
    wo, _ = mb.logweights(_frac(V), 2, p, np.array(a), np.array(b), T, s, 21, n)
    w0 = mb.level0(_frac(V), 2, p, np.array(a), np.array(b), T)
    ref = mc.estimate(wo, w0, 0.0, 0.0, T, 20)
    shift = math.exp(mb.log_A_free(np.array(a), np.array(b), T) - mc.log_A_free(0.0, 0.0, T))
    for lev in range(s + 1):
        assert r[lev]["amp"] == pytest.approx(ref[lev]["amp"] * shift, rel=1e-10)
        if lev:
            assert r[lev]["err"] == pytest.approx(ref[lev]["err"] * shift, rel=1e-8)
    pl = su.PlanND(V, a, b, T, p, s, n, 21, n_blocks=20)
    t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
    sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
    assert pl.su_plan_execute(t, sc) == 2
    torch.cuda.synchronize()
    rp = pl.su_plan_finalize(t.cpu().numpy(), sc)
    t2 = torch.zeros_like(t)
    pl.su_plan_execute_range(0, 7, t2, sc)
    pl.su_plan_execute_range(7, 20, t2, sc)
    torch.cuda.synchronize()
    rr = pl.su_plan_finalize(t2.cpu().numpy(), sc)
    for lev in range(s + 1):
        assert rp[lev]["amp"] == r[lev]["amp"] and rr[lev]["amp"] == r[lev]["amp"]


def test_coupled_oscillator_matches_the_exact_discretized_amplitude():
    V = {(2, 0): 1.0, (0, 2): 2.0, (1, 1): 0.6}          # K = [[2, .6], [.6, 4]]
    lam, U = np.linalg.eigh(np.array([[2.0, 0.6], [0.6, 4.0]]))
    w = np.sqrt(lam)
    a, b, T, p, s = np.array([0.3, -0.2]), np.array([0.5, 0.4]), 1.0, 4, 4
    r = su.speedup_amplitude_nd(V, a, b, T, p, s, 2_000_000, 99, n_blocks=64)
    ua, ub = a @ U, b @ U
    for lev in r:
        N = 1 << lev["level"]
        ref = math.prod(exact.ho_discretized(p, N, ua[i], ub[i], T, omega=w[i]) for i in range(2))
        if lev["level"] == 0:
            assert lev["amp"] == pytest.approx(ref, rel=1e-12)
        else:
            assert abs(lev["amp"] - ref) <= 3 * lev["err"], (lev["level"], lev["amp"], ref, lev["err"])


def test_separable_anharmonic_oscillator_matches_the_product_of_dvr_amplitudes():
    """V = (x^2 + y^2)/2 + g (x^4 + 2 y^4)/24: A = A_x A_y; p = 10, N = 32 is
    converged far below the statistical error."""
    g = 6.0
    V = {(2, 0): 0.5, (0, 2): 0.5, (4, 0): g / 24, (0, 4): 2 * g / 24}
    a, b, T = (0.0, -0.4), (0.6, 0.2), 1.0
    r = su.speedup_amplitude_nd(V, a, b, T, 10, 5, 2_000_000, 1234, n_blocks=64)
    Ax, _ = exact.dvr_amplitude(lambda x: 0.5 * x * x + g * x ** 4 / 24, a[0], b[0], T, L=8.0, dx=0.02)
    Ay, _ = exact.dvr_amplitude(lambda x: 0.5 * x * x + 2 * g * x ** 4 / 24, a[1], b[1], T, L=8.0, dx=0.02)
    top = r[5]
    sig = max(top["err"], top["err_naive"])
    assert sig < 0.01 * Ax * Ay
    assert abs(top["amp"] - Ax * Ay) <= 4 * sig, (top["amp"], Ax * Ay, sig)


def test_nd_edge_cases():
    """s = 0 is the analytic level 0; a single sample; the hierarchy off
    gives the same top level as the hierarchy on (same stream)."""
    V, a, b, T, p = GEN2, (0.2, -0.1), (0.4, 0.3), 0.7, 6
    r0 = su.speedup_amplitude_nd(V, a, b, T, p, 0, 10, 1)
    w0 = mb.level0(_frac(V), 2, p, np.array(a), np.array(b), T)
    laf = mb.log_A_free(np.array(a), np.array(b), T)
    assert r0[0]["log_amp"] == pytest.approx(laf + w0, rel=1e-13)
    r1 = su.speedup_amplitude_nd(V, a, b, T, p, 3, 1, 5)
    assert r1[3]["n"] == 1 and np.isfinite(r1[3]["amp"])
    on = su.speedup_amplitude_nd(V, a, b, T, p, 7, 5000, 9, n_blocks=10)
    off = su.speedup_amplitude_nd(V, a, b, T, p, 7, 5000, 9, n_blocks=10, hierarchy=False)
    assert off[7]["amp"] == on[7]["amp"] and off[7]["err"] == on[7]["err"]
