"""GPU parity of the CUDA path against the oracle, through the C ABI.

* Philox4x32-10 words: bit-exact.
* Per-sample log-weights w_n (Sec. 4.1 normalisation, Eq. SNp) on identical
  Philox streams: within 1e-12 (double) and 1e-5 (single precision, against
  the oracle fed the same 24-bit uniforms), relative to max(|w|, the median
  |w| of that level) so that weights near zero are not judged by their own
  vanishing size.
* Amplitudes and block errors from the same samples: the same numbers as the
  oracle's estimator up to reduction order.
* Against closed forms: the harmonic oscillator's exact discretized value,
  quadrature for N = 2, 4, the exact-diagonalisation continuum value at the
  full convergence-sweep size, within 3 sigma (plus the discretization bound
  where the level is not converged).
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
from oracle import exact, mc  # noqa: E402

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


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


def _rel_err(wg, wo):
    scale = np.maximum(np.abs(wo), np.median(np.abs(wo), axis=0))
    scale = np.maximum(scale, 1e-300)
    return float(np.max(np.abs(wg - wo) / scale))


U64, U32 = 2.0 ** -53, 2.0 ** -24


def _excess(wg, wo, wabs, rel, u):
    """Largest |wg - wo| over its allowance: rel * max(|w|, median |w| of the
    level), or, where the level's terms cancel (large eps, outside the
    expansion's convergence radius), 64 u times the sum of the absolute terms
    (Horner's rounding bound, gamma_2n sum |a_i x^i| with degrees <= 32)."""
    scale = np.maximum(np.abs(wo), np.median(np.abs(wo), axis=0))
    allow = np.maximum(rel * scale, 64 * u * wabs)
    allow = np.maximum(allow, 1e-300)
    return float(np.max(np.abs(wg - wo) / allow))


@pytest.mark.parametrize("seed,inst,sample0", [(1234, 0, 0), (0xFEDCBA9876543210, 7, (1 << 32) - 3),
                                               (1, 0xFFFFFFFF, 10_000_000 - 50)])
def test_philox_words_bit_exact(seed, inst, sample0):
    ns, nc = 100, 37
    out = torch.zeros((ns, nc, 4), dtype=torch.int32, device="cuda")
    su.speedup_philox_words(seed, inst, sample0, ns, nc, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    for i in (0, 1, 17, ns - 1):
        for t in (0, 1, 5, nc - 1):
            assert list(got[i, t]) == mc.philox_words(seed, inst, sample0 + i, t), (i, t)


@pytest.mark.parametrize("prec,bits,tol", [("fp64", 53, 1e-15), ("fp32", 24, 1e-6)])
def test_normals_match_oracle_box_muller(prec, bits, tol):
    """The sampler's table-driven (double) and float Box-Muller against the
    oracle's libm Box-Muller on the same Philox words: |dz| <= tol (1 + r)
    with r the pair's radius (the oracle's own rounding of 2 pi u2 is
    ~1e-16 |theta|, which moves both normals by up to r times that)."""
    ns, nn = 4000, 64
    out = torch.zeros((ns, nn), dtype=torch.float64, device="cuda")
    su.speedup_normals(77, 3, 123456789, ns, nn, out, precision=prec)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = np.stack([mc.normals(77, 3, 123456789 + i, nn, bits) for i in range(ns)])
    # both normals of a pair carry the error of its radius r = |(z0, z1)|
    r = np.repeat(np.hypot(ref[:, 0::2], ref[:, 1::2]), 2, axis=1)
    assert float(np.max(np.abs(got - ref) / (1 + r))) <= tol
    assert np.isfinite(got).all()


CASES = [
    # model, params, a, b, T, p, s, n, seed, sample0
    ("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 1000, 1234, 0),
    ("ho", [1.0], 0.0, 1.0, 1.0, 4, 4, 300, 1234, 0),
    ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 1, 10, 129, 1234, 0),
    ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 10, 10, 200, 1234, 9_999_800),
    ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 18, 10, 131, 99, 0),
    ("aho", [1.0, 1.0], -4.9, 3.2, 0.25, 10, 2, 333, 5, 0),
    ("aho", [1.0, 1.0], 5.0, -5.0, 2.0, 10, 8, 257, 5, 77),
    ("dw", [5.0], -1.0, 1.0, 5.0, 12, 6, 300, 1234, 0),
    ("dw", [1.0], -1.0, 1.0, 1.0, 12, 6, 200, 1234, 12345),
    ("dw", [5.0], -1.0, 1.0, 5.0, 12, 6, 5, 8, 350412),      # a rare path with w_6 = 3350
    ("mpt", [3.0, 1.0], -1.0, 1.0, 1.0, 12, 6, 200, 1234, 0),
    ("mpt", [3.0, 1.0], -1.0, 1.0, 5.0, 6, 7, 150, 3, 0),
    ("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 21, 10, 96, 1234, 0),     # levels above the convergence sweep
    ("aho", [1.0, 48.0], 0.0, 0.5, 0.5, 32, 8, 64, 7, 5000),
    ("aho", [1.0, 48.0], 0.0, 0.5, 0.5, 48, 6, 64, 3, 0),         # p = 48: exact oracle in ~10 s
    ("poly", [0.2, -0.5, 0.3, 0.25, 0.1], -0.5, 0.7, 0.8, 5, 5, 140, 8, 0),
    ("poly", [0.0, 1.0, 0.5], 0.3, -0.2, 1.5, 3, 9, 64, 8, 0),
    ("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 6, 1, 65, 2, 0),
    ("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 6, 3, 1, 2, 0),
    ("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 6, 5, 33, 2, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-p{c[5]}-s{c[6]}-n{c[7]}" for c in CASES])
def test_logweights_fp64_match_oracle(case):
    model, params, a, b, T, p, s, n, seed, s0 = case
    wg = _gpu_w(model, params, a, b, T, p, s, n, seed, s0, precision="fp64")
    o = mc.Oracle(model, params, p)
    wo, _ = o.logweights(a, b, T, s, seed, n, sample0=s0, bits=53, threads=THREADS)
    wabs = o.logweights_abs(a, b, T, s, seed, n, sample0=s0, bits=53)
    assert not np.isnan(wg).any()
    assert _excess(wg, wo, wabs, 1e-12, U64) <= 1.0


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-p{c[5]}-s{c[6]}-n{c[7]}" for c in CASES])
def test_logweights_fp32_match_oracle(case):
    model, params, a, b, T, p, s, n, seed, s0 = case
    wg = _gpu_w(model, params, a, b, T, p, s, n, seed, s0, precision="fp32")
    o = mc.Oracle(model, params, p)
    wo, _ = o.logweights(a, b, T, s, seed, n, sample0=s0, bits=24, threads=THREADS)
    wabs = o.logweights_abs(a, b, T, s, seed, n, sample0=s0, bits=24)
    assert _excess(wg, wo, wabs, 1e-5, U32) <= 1.0


def _allowance_counts(wg, wo, wabs, rel, u):
    """Per level: how many samples meet the plain relative tolerance
    |dw| <= rel |w|, how many pass only through the median floor
    rel * median |w|, and how many only through Horner's bound 64 u A."""
    d = np.abs(wg - wo)
    plain = d <= rel * np.abs(wo)
    med = ~plain & (d <= rel * np.median(np.abs(wo), axis=0))
    horner = ~plain & ~med & (d <= 64 * u * wabs)
    return plain.sum(axis=0), med.sum(axis=0), horner.sum(axis=0)


@pytest.mark.parametrize("prec,bits,tol,u", [("fp64", 53, 1e-12, U64), ("fp32", 24, 1e-5, U32)])
def test_converged_levels_meet_the_plain_tolerance(prec, bits, tol, u):
    """Which allowance decides, case by case and level by level (printed with
    -s), and the plain relative tolerance of the benchmark spec (1e-12 in double,
    1e-5 in single precision, no floor) on every sample whose sum is well
    conditioned, A / |w| <= tol / (64 u) (A = eps sum |terms|): the floor and
    Horner's bound decide only where the terms of W_p cancel -- in these
    cases the double well h = 5 at T = 5 on levels eps >= 0.16 and
    Poeschl-Teller at T = 5 on eps >= 1.25, outside the expansion's
    convergence radius, and single samples whose weight is near zero
    (A / |w| of several hundred, e.g. the odd polynomial)."""
    rows, fails = [], []
    kmax = tol / (64 * u)
    for case in CASES:
        model, params, a, b, T, p, s, n, seed, s0 = case
        wg = _gpu_w(model, params, a, b, T, p, s, n, seed, s0, precision=prec)
        o = mc.Oracle(model, params, p)
        wo, _ = o.logweights(a, b, T, s, seed, n, sample0=s0, bits=bits, threads=THREADS)
        wabs = o.logweights_abs(a, b, T, s, seed, n, sample0=s0, bits=bits)
        plain, med, horner = _allowance_counts(wg, wo, wabs, tol, u)
        rows.append((f"{model}-p{p}-s{s}-n{n}", plain.tolist(), med.tolist(), horner.tolist()))
        miss = np.abs(wg - wo) > tol * np.abs(wo)
        for lev in range(1, s + 1):
            eps = T / 2 ** lev
            m = miss[:, lev - 1]
            kappa = wabs[:, lev - 1] / np.maximum(np.abs(wo[:, lev - 1]), 1e-300)
            if (m & (kappa <= kmax)).any():
                fails.append((f"{model}-p{p}-s{s}-n{n}", lev, eps, int(m.sum()), float(kappa[m].min())))
    print(f"\n{prec}: samples per level n = 1..s meeting rel {tol:g} | only via the median floor | "
          f"only via Horner's bound")
    for name, pl, md, hr in rows:
        print(f"  {name:28s} {pl} | {md} | {hr}")
    assert not fails, fails


@pytest.mark.parametrize("prec,bits,tol", [("fp64", 53, 1e-12), ("fp32", 24, 1e-5)])
def test_width_factor_weights_match_oracle(prec, bits, tol):
    wf = math.sqrt(2.0)
    for s in (3, 7):
        wg = _gpu_w("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, s, 200, 42, 0, precision=prec, width_factor=wf)
        wo, _ = mc.Oracle("aho", [1.0, 1.0], 4).logweights(0.0, 1.0, 1.0, s, 42, 200, bits=bits, wf=wf,
                                                          threads=THREADS)
        assert _rel_err(wg, wo) <= tol


def test_instance_selects_an_independent_stream():
    w0 = _gpu_w("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 64, 9, 0, instance=0)
    w5 = _gpu_w("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 64, 9, 0, instance=5)
    wo, _ = mc.Oracle("aho", [1.0, 1.0], 4).logweights(0.0, 1.0, 1.0, 4, 9, 64, instance=5)
    assert _rel_err(w5, wo) <= 1e-12
    assert np.abs(w0 - w5).max() > 1e-3


@pytest.mark.parametrize("prec,bits", [("fp64", 53), ("fp32", 24)])
@pytest.mark.parametrize("n_mc,n_blocks", [(1, 4), (5, 2), (33, 10), (1000, 10), (4099, 64)])
def test_amplitude_equals_oracle_estimator_on_the_same_samples(prec, bits, n_mc, n_blocks):
    model, params, a, b, T, p, s, seed = "aho", [1.0, 10.0], 0.0, 1.0, 1.0, 10, 6, 77
    res = su.speedup_amplitude(model, params, a, b, T, p, s, n_mc, seed, precision=prec, n_blocks=n_blocks)
    o = mc.Oracle(model, params, p)
    wo, _ = o.logweights(a, b, T, s, seed, n_mc, bits=bits, threads=THREADS)
    ref = mc.estimate(wo, o.level0(a, b, T), a, b, T, n_blocks)
    tol = 1e-10 if prec == "fp64" else 1e-4
    for lev in range(s + 1):
        r, g = ref[lev], res[lev]
        assert g["n"] == n_mc
        assert abs(g["amp"] - r["amp"]) <= tol * r["amp"], lev
        assert abs(g["log_amp"] - r["log_amp"]) <= tol
        if lev and n_mc > 1 and min(n_blocks, n_mc) > 1:
            assert abs(g["err"] - r["err"]) <= 100 * tol * r["err"] + 1e-300, lev
            assert abs(g["err_naive"] - r["err_naive"]) <= 100 * tol * r["err_naive"] + 1e-300
            assert abs(g["ess"] - r["ess"]) <= 100 * tol * r["ess"]


def test_hierarchy_off_gives_the_top_level_only():
    full = su.speedup_amplitude("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 6, 7, 5000, 3, n_blocks=8)
    top = su.speedup_amplitude("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 6, 7, 5000, 3, n_blocks=8, hierarchy=False)
    assert top[7]["amp"] == pytest.approx(full[7]["amp"], rel=1e-13)
    assert top[0]["amp"] == full[0]["amp"]


def test_sample_ranges_compose():
    """Disjoint sample ranges (one per device in a sharded run) are one run."""
    kw = dict(n_blocks=1)
    parts = [su.Plan("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 5, 3000, 11, sample0=s0, **kw) for s0 in (0, 3000)]
    whole = su.speedup_amplitude("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 5, 6000, 11, n_blocks=2)
    tuples = []
    for pl in parts:
        t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
        sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
        pl.su_plan_execute(t, sc)
        torch.cuda.synchronize()
        tuples.append(t.cpu().numpy().reshape(-1, pl.levels, 4))
    merged = np.concatenate(tuples, axis=0)
    pl2 = su.Plan("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 5, 6000, 11, n_blocks=2)
    res = pl2.su_plan_finalize(merged.reshape(-1))
    for lev in range(6):
        assert res[lev]["amp"] == pytest.approx(whole[lev]["amp"], rel=1e-13)
        assert res[lev]["err"] == pytest.approx(whole[lev]["err"], rel=1e-9, abs=1e-300)


def _within(res, ref, extra=0.0, nsig=3.0):
    sig = max(res["err"], res["err_naive"])
    return abs(res["amp"] - ref) <= nsig * sig + extra


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_harmonic_against_exact_discretized(prec):
    r = su.speedup_amplitude("ho", [1.0], 0.0, 1.0, 1.0, 4, 4, 100_000, 1234, precision=prec, n_blocks=10)
    for lev in r:
        ref = exact.ho_discretized(4, 2 ** lev["level"], 0.0, 1.0, 1.0)
        if lev["level"] == 0:
            assert lev["amp"] == pytest.approx(ref, rel=1e-13)
        else:
            assert _within(lev, ref), (lev["level"], lev["amp"], ref)
    assert r[4]["amp"] == pytest.approx(exact.mehler(0.0, 1.0, 1.0), abs=5 * r[4]["err"] + 2e-8)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_anharmonic_against_quadrature(prec):
    r = su.speedup_amplitude("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 100_000, 1234, precision=prec, n_blocks=10)
    for n, N in ((0, 1), (1, 2), (2, 4)):
        ref, edge = exact.quadrature("aho", [1.0, 1.0], 4, N, 0.0, 1.0, 1.0)
        assert edge < 1e-12
        if n == 0:
            assert r[0]["amp"] == pytest.approx(ref, rel=1e-12)
        else:
            assert _within(r[n], ref)


@pytest.mark.parametrize("name,params,a,b,T,p", [("dw", [1.0], -1.0, 1.0, 1.0, 4),
                                                  ("mpt", [3.0, 1.0], -1.0, 1.0, 1.0, 4),
                                                  ("poly", [0.2, -0.5, 0.3, 0.25, 0.1], -0.5, 0.7, 0.8, 3)])
def test_tiny_N_models_against_quadrature(name, params, a, b, T, p):
    r = su.speedup_amplitude(name, params, a, b, T, p, 2, 400_000, 4321, n_blocks=20)
    for n, N in ((1, 2), (2, 4)):
        ref, edge = exact.quadrature(name, params, p, N, a, b, T)
        assert edge < 1e-12
        assert _within(r[n], ref), (N, r[n]["amp"], ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_convergence_sweep_full_size_against_diagonalisation(prec):
    """AHO g = 10, T = 1, a = 0, b = 1, p = 10, s = 10, 1e7 samples in 100
    blocks: the plan the benchmark times.  Converged levels agree with the
    exact-diagonalisation amplitude within 3 sigma plus the discretization
    bound |A_n - A_{n+1}| 2^p / (2^p - 1)."""
    pl = su.Plan("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 10, 10, 10_000_000, 1234, precision=prec, n_blocks=100)
    t = torch.empty(pl.tuple_bytes // 8, dtype=torch.float64, device="cuda")
    sc = torch.empty(pl.scratch_bytes, dtype=torch.uint8, device="cuda")
    pl.su_plan_execute(t, sc)
    torch.cuda.synchronize()
    res = pl.su_plan_finalize(t.cpu().numpy(), sc)
    ref = exact.ed_amplitude([0, 0, 0.5, 0, 10 / 24], 0.0, 1.0, 1.0, 200)[0]
    for n in range(5, 10):
        bound = abs(res[n]["amp"] - res[n + 1]["amp"]) * 2 ** 10 / (2 ** 10 - 1)
        assert _within(res[n], ref, extra=bound), (n, res[n]["amp"], ref, res[n]["err"])
    assert res[10]["rel_err"] < 3e-4
    # sampled outputs of the same run, one by one against the oracle
    idx0 = 9_999_900
    wg = _gpu_w("aho", [1.0, 10.0], 0.0, 1.0, 1.0, 10, 10, 100, 1234, idx0, precision=prec)
    wo, _ = mc.Oracle("aho", [1.0, 10.0], 10).logweights(0.0, 1.0, 1.0, 10, 1234, 100, sample0=idx0,
                                                        bits=53 if prec == "fp64" else 24, threads=THREADS)
    assert _rel_err(wg, wo) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("name,params,T,levels", [
    ("dw", [5.0], 1.0, (3, 4, 5, 6)),
    ("dw", [1.0], 1.0, (1, 2, 3, 4, 5, 6)),
    ("mpt", [3.0, 1.0], 5.0, (5, 6)),     # eps >= 5/8: rare weights near e^1000 in 2e5
])
def test_fp32_and_fp64_means_agree(name, params, T, levels):
    """Single- and double-precision W_p give the same amplitude within the
    combined statistical error (independent seeds) on the double-well and
    Poeschl-Teller workloads (p = 12, N = 64).  Levels with eps beyond the
    expansion's radius of convergence are excluded: there the truncated W_p is
    unbounded below and single rare paths carry astronomically large weights.
    (The double well h = 5 at T = 5 is heavy-tailed even at N = 64: sample
    350414 of seed 8 has w_6 = 3350; its weight is checked per sample in
    test_logweights_*, where both precisions agree with the oracle.)"""
    r64 = su.speedup_amplitude(name, params, -1.0, 1.0, T, 12, 6, 1_000_000, 7, precision="fp64")
    r32 = su.speedup_amplitude(name, params, -1.0, 1.0, T, 12, 6, 1_000_000, 8, precision="fp32")
    for lev in levels:
        s = math.hypot(r64[lev]["err"], r32[lev]["err"])
        assert math.isfinite(r64[lev]["amp"]) and math.isfinite(s)
        assert abs(r64[lev]["amp"] - r32[lev]["amp"]) <= 4 * s, lev


def test_highest_levels_read_their_tables_from_global_memory():
    """p = 144 at s = 10 does not fit its tables in shared memory and reads
    them from global memory; its converged levels (eps <= T/64) equal the
    staged p = 96 ones sample by sample."""
    wg = _gpu_w("aho", [1.0, 48.0], 0.0, 0.5, 1.0, 144, 10, 64, 5, precision="fp64")
    ws = _gpu_w("aho", [1.0, 48.0], 0.0, 0.5, 1.0, 96, 10, 64, 5, precision="fp64")
    top = slice(5, 10)
    scale = np.maximum(np.abs(ws[:, top]), np.median(np.abs(ws[:, top]), axis=0))
    assert float(np.max(np.abs(wg[:, top] - ws[:, top]) / scale)) <= 1e-12


@pytest.mark.parametrize("p", [1, 2, 10])
def test_continuum_fit_of_one_run_matches_dvr(p):
    """Fig. 2's case (modified Poeschl-Teller, lambda = alpha = 1,
    A(-0.5, 0.5; 1), s = 10, 1e6 samples): the constant of Eq. fit over the
    levels N = 8..1024 equals the sinc-DVR continuum amplitude within 4 of
    its standard errors (the levels share samples, so the error is taken as
    the larger of the fit's and the top level's)."""
    r = su.speedup_amplitude("mpt", [1.0, 1.0], -0.5, 0.5, 1.0, p, 10, 1_000_000, 2011, n_blocks=100)
    A, dA, _ = su.su_fit_continuum(r, p, n_min=3, n_terms=3)
    ref, _ = exact.dvr_amplitude(lambda y: -1.0 / np.cosh(y) ** 2, -0.5, 0.5, 1.0, L=25.0, dx=0.02)
    sig = max(dA, r[10]["err"])
    assert abs(A - ref) <= 4 * sig, (A, ref, dA, r[10]["err"])


def test_cli_prints_the_library_levels():
    """The command-line front end (T a b s Nmc seed par..., Sec. 4's argument
    order) prints exactly speedup_amplitude's levels, negative endpoints and
    the continuum fit included."""
    import subprocess
    from paper_1105_0542_gb300 import build as _b
    out = subprocess.run([_b.CLI, "-m", "dw", "-p", "6", "-B", "20", "-t", "1.5", "-1.0", "0.5", "6", "20000",
                          "77", "2.0"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if not l.startswith("#")]
    r = su.speedup_amplitude("dw", [2.0], -1.0, 0.5, 1.5, 6, 6, 20000, 77, n_blocks=20)
    assert len(lines) == 7
    for n, l in enumerate(lines):
        k, N, amp, err = l.split()
        assert int(k) == n and int(N) == 2 ** n
        assert float(amp) == r[n]["amp"]
        assert float(err) == pytest.approx(r[n]["err"], rel=1e-5)
    assert any(l.startswith("# continuum fit") for l in out.stdout.splitlines())
