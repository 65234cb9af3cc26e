"""GPU parity of the general-potential mode (W_p in the derivatives of V,
Eq. 1Drec with V's derivatives as symbols) against the oracle, through the C ABI.

* Per-sample log-weights w_n on identical Philox streams against the oracle's
  general W_p (exact-rational coefficients, numpy evaluation) on the oracle's
  own paths: within 1e-12 relative, or the summation bound where the level's
  terms cancel.
* A polynomial potential given through the general mode reproduces the
  model-specific (collapsed-table) weights of the same potential, and a sech^2
  term the Poeschl-Teller model's: two independent device evaluations.
* The amplitude of a mixed potential (polynomial + Gaussian + sech^2) against
  the sinc-DVR continuum value, within 4 sigma.
* The batched launch with per-instance levels p against the oracle's
  estimator on the same samples.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
from oracle import exact, mc  # noqa: E402
from oracle import general_v as gv  # noqa: E402

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


def _gpu_w(model, params, a, b, T, p, s, n, seed, sample0=0, **kw):
    w = torch.full((n, s), float("nan"), dtype=torch.float64, device="cuda")
    su.speedup_logweights(model, params, a, b, T, p, s, sample0, n, seed, w, **kw)
    torch.cuda.synchronize()
    return w.cpu().numpy()


def _oracle_w(params, a, b, T, p, s, n, seed, sample0=0, instance=0):
    """w_n = -eps_n sum_k W_p over the level-n subpath of the oracle's path
    (Sec. 4.1), with W_p the oracle's general form; and eps_n sum_k sum|terms|."""
    paths = mc.Oracle("ho", [1.0], 1)   # the path does not depend on the potential
    q = np.stack([paths.path(a, b, T, s, seed, sample0 + i, instance=instance)[0] for i in range(n)])
    w = np.empty((n, s))
    wabs = np.empty((n, s))
    for lev in range(1, s + 1):
        eps = T / 2 ** lev
        st = 1 << (s - lev)
        ql, qr = q[:, :-1:st], q[:, st::st]
        x, xb = 0.5 * (ql + qr), 0.5 * (qr - ql)
        w[:, lev - 1] = -eps * gv.wp(params, p, x, xb, eps).sum(axis=1)
        wabs[:, lev - 1] = eps * gv.wp_abs(params, p, x, xb, eps).sum(axis=1)
    return w, wabs


def _excess(wg, wo, wabs, rel, u):
    scale = np.maximum(np.abs(wo), np.median(np.abs(wo), axis=0))
    allow = np.maximum(rel * scale, 64 * u * wabs)
    allow = np.maximum(allow, 1e-300)
    return float(np.max(np.abs(wg - wo) / allow))


P_AHO10 = su.general_params((0.0, 0.0, 0.5, 0.0, 10.0 / 24.0))
P_MIXED = su.general_params((0.1, -0.2, 0.5, 0.05, 0.04), [(1.5, 2.0, 0.3), (-0.7, 0.5, -1.0)],
                            [(-3.0, 1.0, 0.0), (0.4, 2.0, 0.5)])
P_MPT = su.general_params((), (), [(-3.0, 1.0, 0.0)])
P_BARRIER = su.general_params((0.0, 0.0, 0.5), [(2.0, 1.0, 0.0)])
P_SEXTIC = su.general_params((0.0, 0.3, -1.0, 0.0, 0.2, 0.0, 0.01))
# Morse D (1 - e^{-a (x - x0)})^2, D = 4, a = 1, x0 = 0.3, plus a Gaussian bump
P_MORSE = su.general_params((4.0,), [(0.5, 3.0, -0.2)], (), [(-8.0, 1.0, 0.3), (4.0, 2.0, 0.3)])

CASES = [
    # name, params, a, b, T, p, s, n, seed, sample0
    ("aho10", P_AHO10, 0.0, 1.0, 1.0, 10, 6, 200, 1234, 0),
    ("mixed", P_MIXED, -0.5, 0.7, 1.0, 6, 5, 150, 7, 0),
    ("mixed-p12", P_MIXED, -0.5, 0.7, 1.0, 12, 4, 64, 11, 10_000),
    ("p1", P_MIXED, -0.5, 0.7, 1.0, 1, 8, 40, 3, 0),
    ("mpt", P_MPT, -1.0, 1.0, 1.0, 12, 6, 100, 1234, 0),
    ("barrier", P_BARRIER, -1.5, 1.5, 2.0, 8, 6, 100, 5, (1 << 32) - 7),
    ("sextic", P_SEXTIC, 0.2, -0.4, 0.5, 9, 7, 60, 9, 0),
    ("s0-edge", P_MIXED, 0.0, 0.0, 0.3, 12, 1, 33, 2, 0),
    ("morse", P_MORSE, -0.2, 0.9, 1.0, 10, 6, 100, 31, 0),
    ("mixed-p16", P_MIXED, -0.5, 0.7, 1.0, 16, 3, 24, 13, 0),
    ("aho10-p18", P_AHO10, 0.0, 1.0, 1.0, 18, 4, 24, 1234, 500),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_general_logweights_match_oracle(case):
    _, params, a, b, T, p, s, n, seed, s0 = case
    wg = _gpu_w("general", params, a, b, T, p, s, n, seed, s0)
    wo, wabs = _oracle_w(params, a, b, T, p, s, n, seed, s0)
    assert np.isfinite(wg).all()
    assert _excess(wg, wo, wabs, 1e-12, U64) <= 1.0


@pytest.mark.parametrize("model,mparams,gparams,p", [
    ("aho", [1.0, 10.0], P_AHO10, 10),
    ("aho", [1.0, 10.0], P_AHO10, 12),
    ("aho", [1.0, 10.0], P_AHO10, 18),
    ("dw", [5.0], su.general_params((5.0, 0.0, -10.0, 0.0, 5.0)), 12),
    ("poly", [0.2, -0.5, 0.3, 0.25, 0.1], su.general_params((0.2, -0.5, 0.3, 0.25, 0.1)), 7),
    ("mpt", [3.0, 1.0], P_MPT, 12),
])
def test_general_mode_reproduces_the_model_tables(model, mparams, gparams, p):
    """Two device evaluations of the same W_p: the collapsed per-model table
    and the derivative-symbol program."""
    a, b, T, s, n = -1.0, 1.0, 1.0, 6, 500
    wm = _gpu_w(model, mparams, a, b, T, p, s, n, 77)
    wg = _gpu_w("general", gparams, a, b, T, p, s, n, 77)
    scale = np.maximum(np.abs(wm), np.median(np.abs(wm), axis=0))
    assert float(np.max(np.abs(wg - wm) / scale)) <= 1e-11


def test_general_amplitude_estimator_matches_oracle_estimator():
    """Amplitudes and block errors of the device estimator against the
    oracle's estimator applied to the oracle's weights of the same samples."""
    params, a, b, T, p, s, n = P_MIXED, -0.5, 0.7, 1.0, 8, 4, 4000
    r = su.speedup_amplitude("general", params, a, b, T, p, s, n, 21, n_blocks=20)
    wo, _ = _oracle_w(params, a, b, T, p, s, n, 21)
    w0 = -T * float(gv.wp(params, p, 0.5 * (a + b), 0.5 * (b - a), T))
    ref = mc.estimate(wo, w0, a, b, T, 20)
    for lev in range(s + 1):
        assert r[lev]["amp"] == pytest.approx(ref[lev]["amp"], rel=1e-11)
        if lev:
            assert r[lev]["err"] == pytest.approx(ref[lev]["err"], rel=1e-8)


def test_general_batch_equals_oracle_per_instance():
    """The batched launch with the general potential: instances of levels
    p = 4, 10, 18 (one program each), depths 3..7, the top level alone or
    every level, against the oracle's estimator applied to the oracle's
    weights of the same samples (instance id = the batch's first id + i)."""
    inst = [(-0.5, 0.7, 1.0, 5, 4, 900, 1), (0.2, -0.3, 0.5, 7, 10, 700, 0), (1.0, 0.0, 2.0, 3, 18, 500, 1),
            (0.0, 0.4, 1.0, 6, 10, 800, 1)]
    nb, seed = 5, 31
    res = su.speedup_amplitude_batch("general", P_MIXED, 10, inst, 1000, seed, n_blocks=nb, instance=7)
    for i, (a, b, T, s, p, n, hier) in enumerate(inst):
        wo, _ = _oracle_w(P_MIXED, a, b, T, p, s, n, seed, instance=7 + i)
        w0 = -T * float(gv.wp(P_MIXED, p, 0.5 * (a + b), 0.5 * (b - a), T))
        ref = mc.estimate(wo, w0, a, b, T, nb)
        got = res[i] if hier else [None] * s + [res[i]]
        assert len(got) == s + 1
        for lev in (range(s + 1) if hier else [s]):
            g, r = got[lev], ref[lev]
            assert g["n"] == n and g["level"] == lev
            # (coarse levels at p = 18 sit far outside the expansion's radius:
            # log-amplitudes of order 1e12, equal to 1e-10 relative)
            assert abs(g["log_amp"] - r["log_amp"]) <= 1e-10 * max(1.0, abs(r["log_amp"])), (i, p, s, lev)
            if lev:
                assert g["err"] == pytest.approx(r["err"], rel=1e-7), (i, p, s, lev)


def test_general_amplitude_matches_dvr():
    """A(a, b; T) of V = x^2/2 + 1.5 e^{-2 (x - 0.3)^2} - sech^2(2 x), p = 12,
    N = 32 (converged: eps^12 is far below the statistical error) against the
    sinc-DVR continuum value."""
    params = su.general_params((0.0, 0.0, 0.5), [(1.5, 2.0, 0.3)], [(-1.0, 2.0, 0.0)])
    a, b, T = -0.5, 0.7, 1.0
    r = su.speedup_amplitude("general", params, a, b, T, 12, 5, 4_000_000, 1234, n_blocks=64)
    V = lambda x: 0.5 * x * x + 1.5 * np.exp(-2.0 * (x - 0.3) ** 2) - 1.0 / np.cosh(2.0 * x) ** 2  # noqa: E731
    ref, _ = exact.dvr_amplitude(V, a, b, T, L=10.0, dx=0.02)
    top = r[5]
    sig = max(top["err"], top["err_naive"])
    assert sig < 0.01 * ref
    assert abs(top["amp"] - ref) <= 4 * sig, (top["amp"], ref, sig)


def test_general_edge_cases():
    """s = 0 is the analytic level 0; the hierarchy off gives the same top
    level as the hierarchy on (same stream)."""
    a, b, T, p = -0.5, 0.7, 1.0, 8
    r0 = su.speedup_amplitude("general", P_MIXED, a, b, T, p, 0, 10, 1)
    w0 = -T * float(gv.wp(P_MIXED, p, 0.5 * (a + b), 0.5 * (b - a), T))
    assert r0[0]["log_amp"] == pytest.approx(mc.log_A_free(a, b, T) + w0, rel=1e-13)
    on = su.speedup_amplitude("general", P_MIXED, a, b, T, p, 6, 5000, 9, n_blocks=10)
    off = su.speedup_amplitude("general", P_MIXED, a, b, T, p, 6, 5000, 9, n_blocks=10, hierarchy=False)
    assert off[6]["amp"] == on[6]["amp"] and off[6]["err"] == on[6]["err"]


def test_morse_amplitude_matches_dvr():
    """A(a, b; T) of the Morse potential 4 (1 - e^{-(x - 0.3)})^2 through the
    exponential family, p = 12, N = 32, against sinc-DVR."""
    params = su.general_params((4.0,), (), (), [(-8.0, 1.0, 0.3), (4.0, 2.0, 0.3)])
    a, b, T = 0.0, 0.6, 1.0
    r = su.speedup_amplitude("general", params, a, b, T, 12, 5, 4_000_000, 77, n_blocks=64)
    V = lambda x: 4.0 * (1.0 - np.exp(-(x - 0.3))) ** 2  # noqa: E731
    ref, _ = exact.dvr_amplitude(V, a, b, T, L=12.0, dx=0.02)
    top = r[5]
    sig = max(top["err"], top["err_naive"])
    assert sig < 0.01 * ref
    assert abs(top["amp"] - ref) <= 4 * sig, (top["amp"], ref, sig)
