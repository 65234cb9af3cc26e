"""Host-side checks of the C-ABI library (no GPU needed).

* the library builds, loads, and exports every entry point include/speedup.h
  declares;
* the host generator of W_p (double-double recursion + collapse) agrees with
  the oracle's exact-rational c_{m,k} collapsed by hand (Eq. ansatz at fixed
  eps), coefficient by coefficient, for every model family and p up to 18;
* argument validation fails loudly with SU_EINVAL, and without a CUDA device
  the compute entry points fail with SU_ECUDA instead of falling back;
* the host evaluators of W (speedup_wp, speedup_wp_nd: the collapsed tables,
  the general mode's derivative-symbol program and the several-coordinates
  program the kernels run) against the oracle's term-by-term W at random
  points, within 1e-12 of the terms' absolute sum.
"""
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import paper_1105_0542_gb300 as su
from oracle import effective_action as ea

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "speedup.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:su|speedup)_\w+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    lib = su.load()
    declared = _declared_functions()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(su.EXPORTS)


def test_version_string():
    v = su.su_version()
    assert "sm_103a" in v


def _exact_collapse(name, params, p, eps):
    """P_ij from the oracle's exact c_{m,k}: W_p = sum_j xb^2j sum_i P_ij z^i."""
    model = ea.make_model(name, [Fraction(v) for v in params])
    c = ea.coefficients(model, p)
    eps = Fraction(eps)
    cols = {}
    for (m, k), poly in c.items():
        acc = cols.setdefault(k, [])
        for i, v in enumerate(poly):
            while len(acc) <= i:
                acc.append(Fraction(0))
            acc[i] += v * eps ** (m - k)
    if model.kind == "t":
        # the library's ring variable is t^2 = tanh^2(alpha x): keep even powers
        return {k: poly[0::2] for k, poly in cols.items()}, 2
    even = all(v == 0 for poly in cols.values() for v in poly[1::2])
    if even:
        return {k: poly[0::2] for k, poly in cols.items()}, 0
    return cols, 1


@pytest.mark.parametrize("name,params,p,eps", [
    ("aho", [1.0, 10.0], 18, 0.5),
    ("aho", [1.0, 10.0], 18, 1.0 / 1024),
    ("aho", [1.0, 1.0], 10, 0.25),
    ("aho", [1.0, 10.0], 4, 1.0 / 16),
    ("ho", [1.0], 12, 0.125),
    ("dw", [5.0], 12, 5.0 / 64),
    ("mpt", [3.0, 1.0], 12, 1.0 / 64),
    ("mpt", [2.0, 0.7], 6, 0.3),
    ("poly", [0.2, -0.5, 0.3, 0.25, 0.1], 8, 0.1),
    ("aho", [1.0, 10.0], 1, 1.0),
    ("aho", [1.0, 48.0], 21, 0.02),          # the level of the evolution-operator spectra (Fig. 3)
    ("aho", [-10.0, 12.0], 21, 0.1),
    ("aho", [1.0, 10.0], 32, 1.0 / 64),
    ("dw", [1.0], 24, 0.25),
    ("aho", [1.0, 48.0], 48, 0.02),          # levels beyond the convergence sweep
    ("mpt", [3.0, 1.0], 24, 1.0 / 64),
])
def test_generator_matches_oracle_exact_collapse(name, params, p, eps):
    P, ncol, ring, lens = su.speedup_generate_coeffs(name, params, p, eps)
    cols, ring_ref = _exact_collapse(name, params, p, eps)
    assert ring == ring_ref
    off = 0
    for j in range(ncol):
        ref = cols.get(j, [])
        got = P[off:off + lens[j]]
        off += lens[j]
        # exact zeros come out as double-double residue far below the column's scale
        floor = 1e-28 * max([abs(float(v)) for v in ref] + [1e-300])
        for i in range(max(len(ref), len(got))):
            r = float(ref[i]) if i < len(ref) else 0.0
            g = float(got[i]) if i < len(got) else 0.0
            assert abs(g - r) <= 2.3e-16 * abs(r) + floor, (j, i, g, r)
    assert off == len(P)
    # no coefficient of the exact collapse is missing from the shape
    for j, ref in cols.items():
        if any(ref):
            assert j < ncol


def _eval_table(P, ncol, ring, lens, x, xb, alpha=1.0):
    import mpmath as mp
    z = {0: mp.mpf(x) ** 2, 1: mp.mpf(x), 2: mp.tanh(alpha * mp.mpf(x)) ** 2}[ring]
    tot, tabs, off = mp.mpf(0), mp.mpf(0), 0
    for j in range(ncol):
        for i in range(lens[j]):
            t = mp.mpf(P[off + i]) * z ** i * mp.mpf(xb) ** (2 * j)
            tot += t
            tabs += abs(t)
        off += lens[j]
    return tot, tabs


def test_generator_at_the_paper_s_highest_levels():
    """p = 144 (the anharmonic oscillator's highest level of Sec. 3.3): the
    harmonic oscillator's collapsed table equals its closed-form W (the
    Mehler kernel, 50 digits) to the table's rounding; the anharmonic
    oscillator's p = 144 table equals its p = 96 one where both have
    converged; the Poeschl-Teller p = 41 table is finite."""
    import mpmath as mp
    mp.mp.dps = 50
    w, eps = 1.3, 0.25
    P, ncol, ring, lens = su.speedup_generate_coeffs("ho", [w], 144, eps)
    for x, xb in ((0.3, 0.1), (-1.2, 0.4), (2.0, -0.05)):
        got, scale = _eval_table(P, ncol, ring, lens, x, xb)
        we = mp.mpf(w) * eps
        sh, ch = mp.sinh(we), mp.cosh(we)
        ref = ((w / sh) * (x * x * (ch - 1) + xb * xb * (ch + 1)) - 2 * mp.mpf(xb) ** 2 / eps) / eps \
            + mp.log(sh / we) / (2 * eps)
        assert abs(got - ref) <= 1e-14 * scale, (x, xb, got, ref)
    a = su.speedup_generate_coeffs("aho", [1.0, 48.0], 144, 0.02)
    b = su.speedup_generate_coeffs("aho", [1.0, 48.0], 96, 0.02)
    for x, xb in ((0.4, 0.05), (-0.9, 0.1)):
        ga, sa = _eval_table(*a, x, xb)
        gb, sb = _eval_table(*b, x, xb)
        assert abs(ga - gb) <= 1e-13 * max(sa, sb)
    m = su.speedup_generate_coeffs("mpt", [3.0, 1.0], 41, 1.0 / 64)
    assert np.isfinite(m[0]).all() and len(m[0]) > 1000


def test_generator_term_counts_of_the_anharmonic_oscillator():
    counts = [len(su.speedup_generate_coeffs("aho", [1.0, 10.0], p, 0.1)[0]) for p in (4, 10, 12, 18)]
    assert counts == [8, 21, 27, 48]


def test_compiled_shapes_cover_the_quartic_and_harmonic_tables():
    """Every even-ring table of the harmonic oscillator and of the quartic
    potentials at p = 1..18 has a compiled shape (the single-precision plans
    of the convergence sweep all run specialised samplers); the shape is the
    generator's, so the quartic shapes are distinct per p and shared by the
    anharmonic oscillator and the double well; other rings and the polynomial
    model keep the generic sampler."""
    aho = [su.su_fixed_shape("aho", [1.0, 10.0], p) for p in range(1, 19)]
    assert min(aho) >= 0 and len(set(aho)) == 18
    assert aho == [su.su_fixed_shape("dw", [5.0], p) for p in range(1, 19)]
    assert aho == [su.su_fixed_shape("aho", [0.0, 1.0], p) for p in range(1, 19)]
    ho = {su.su_fixed_shape("ho", [1.0], p) for p in range(2, 19)}
    assert len(ho) == 1 and min(ho) >= 0 and su.su_fixed_shape("ho", [1.0], 1) >= 0
    assert su.su_fixed_shape("mpt", [3.0, 1.0], 10) == -1
    assert su.su_fixed_shape("poly", [0.0, 1.0, 0.5], 4) == -1
    with pytest.raises(su.SpeedupError) as e:
        su.su_fixed_shape("general", su.general_params(poly=(0, 0, 1)), 4)
    assert e.value.code == -6


@pytest.mark.parametrize("args,kw", [
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 0, 4, 100, 1), {}),        # p = 0
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 145, 4, 100, 1), {}),      # p = 145
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 11, 100, 1), {}),       # s = 11
    (("aho", [1.0, 1.0], 0.0, 1.0, 0.0, 4, 4, 100, 1), {}),        # T = 0
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 0, 1), {}),          # n_mc = 0
    (("aho", [1.0, 1.0], float("nan"), 1.0, 1.0, 4, 4, 10, 1), {}),
    (("aho", [1.0], 0.0, 1.0, 1.0, 4, 4, 10, 1), {}),              # wrong n_params
    (("mpt", [3.0, 0.0], 0.0, 1.0, 1.0, 4, 4, 10, 1), {}),         # alpha = 0
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 10, 1), {"n_blocks": 0}),
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 10, 1), {"width_factor": -1.0}),
    ((9, [1.0], 0.0, 1.0, 1.0, 4, 4, 10, 1), {}),                  # unknown model
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 10, 1), {"seg_log2": 6}),   # launch shape out of range
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 10, 1), {"rounds": 9}),
    (("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 10, 1), {"kernel": 2}),
])
def test_invalid_arguments_are_rejected(args, kw):
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude(*args, **kw)
    assert e.value.code == -1


def test_no_device_means_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 1000, 1234)
    assert e.value.code == -3


def test_level_zero_needs_no_sampling_but_still_a_plan():
    # s = 0 is analytic; the plan still checks for a device, so without one it fails
    import torch
    if torch.cuda.is_available():
        r = su.speedup_amplitude("ho", [1.0], 0.0, 1.0, 1.0, 4, 0, 10, 1)
        assert r[0]["err"] == 0.0
    else:
        with pytest.raises(su.SpeedupError):
            su.speedup_amplitude("ho", [1.0], 0.0, 1.0, 1.0, 4, 0, 10, 1)


@pytest.mark.parametrize("kw", [{"t": 0.0}, {"L": -1.0}, {"n": 1}, {"n": 70000}, {"p": 145}])
def test_evolution_matrix_rejects_bad_arguments(kw):
    args = {"model": "aho", "params": [1.0, 1.0], "p": 4, "t": 0.1, "L": 5.0, "n": 100}
    args.update(kw)
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_evolution_matrix(args["model"], args["params"], args["p"], args["t"], args["L"], args["n"], 1 << 20)
    assert e.value.code == -1


def test_fault_hooks_validate_and_the_nan_table_fails_before_any_device_work():
    with pytest.raises(su.SpeedupError) as e:
        su.su_fault_inject(9)
    assert e.value.code == -1
    with pytest.raises(su.SpeedupError) as e:
        su.su_fault_inject("alloc", 0)
    assert e.value.code == -1
    # the tables are built and checked before the device is touched
    su.su_fault_inject("table_nan")
    try:
        with pytest.raises(su.SpeedupError) as e:
            su.speedup_amplitude("aho", [1.0, 1.0], 0.0, 1.0, 1.0, 4, 4, 100, 1)
        assert e.value.code == -5
    finally:
        su.su_fault_inject("clear")



# ---- the general-potential mode: argument checks come before any device work
P_GEN = su.general_params((0.0, 0.0, 0.5), [(1.5, 2.0, 0.3)], [(-1.0, 2.0, 0.0)])


def test_general_params_layout():
    p = su.general_params((1.0, 2.0), [(3.0, 4.0, 5.0)], [(6.0, 7.0, 8.0), (9.0, 10.0, 11.0)])
    assert len(p) == 33
    assert p[:3] == (1.0, 2.0, 0.0) and p[9:12] == (3.0, 4.0, 5.0) and p[12:21] == (0.0,) * 9
    assert p[21:27] == (6.0, 7.0, 8.0, 9.0, 10.0, 11.0) and p[27:] == (0.0,) * 6
    with pytest.raises(ValueError):
        su.general_params(tuple(range(10)))
    q = su.general_params((1.0,), (), (), [(2.0, 0.5, 0.1)])
    assert len(q) == 45 and q[33:36] == (2.0, 0.5, 0.1) and q[36:] == (0.0,) * 9


@pytest.mark.parametrize("params,kw,code", [
    (P_GEN, {"p": 19}, -6),                                  # above the general program's p <= 18
    (P_GEN, {"precision": "fp32"}, -6),                      # double only
    (P_GEN[:32], {}, -1),                                    # 32 parameters
    (P_GEN[:9] + (1.0, 0.0, 0.0) + P_GEN[12:], {}, -1),      # a Gaussian with beta = 0
    (P_GEN[:21] + (1.0, 0.0, 0.0) + P_GEN[24:], {}, -1),     # a sech^2 term with alpha = 0
    (P_GEN[:4] + (float("nan"),) + P_GEN[5:], {}, -1),       # a non-finite parameter
    (P_GEN + (1.0, 1.0, 0.0) * 3 + (1.0, 1.0), {}, -1),       # 44 parameters
    (P_GEN + (1.0, float("inf"), 0.0) + (0.0,) * 9, {}, -1),  # a non-finite exponential parameter
])
def test_general_mode_rejects_bad_requests(params, kw, code):
    args = {"p": 6, "precision": "fp64"}
    args.update(kw)
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude("general", params, 0.0, 1.0, 1.0, args["p"], 4, 1000, 1, precision=args["precision"])
    assert e.value.code == code


def test_general_mode_is_refused_where_a_collapsed_table_is_needed():
    # the evolution operator and the batched launch take the general potential
    # in double precision only (its derivatives up to V^(2p-2) carry factors
    # like (2p-1)!, beyond the single-precision range at p = 18)
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_evolution_matrix("general", P_GEN, 4, 0.1, 5.0, 100, 1 << 20, precision="fp32")
    assert e.value.code == -6
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude_batch("general", P_GEN, 4, [(0.0, 1.0, 1.0, 4)], 1000, 1, precision="fp32")
    assert e.value.code == -6
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude_noalloc("general", P_GEN, 0.0, 1.0, 1.0, 4, 4, 1000, 1)
    assert e.value.code == -6


# ---- systems of several coordinates: the host generator against the oracle
from fractions import Fraction as _F  # noqa: E402

ND_GEN2 = {(2, 0): 0.5, (0, 2): 0.75, (1, 1): 0.2, (2, 1): 1 / 3, (0, 3): -1 / 7, (4, 0): 0.1, (1, 3): 0.05,
           (0, 4): 1 / 12, (1, 0): -1 / 3}
ND_GEN3 = {(2, 0, 0): 0.5, (0, 2, 0): 0.5, (0, 0, 2): 0.5, (1, 1, 0): 0.2, (0, 1, 1): 1 / 7, (2, 0, 2): 1 / 11,
           (4, 0, 0): 1 / 24, (0, 4, 0): 1 / 24, (0, 0, 4): 1 / 30, (1, 1, 1): 1 / 9}
ND_TWO_2D = {(2, 0, 0, 0): 0.5, (0, 2, 0, 0): 0.5, (0, 0, 2, 0): 0.5, (0, 0, 0, 2): 0.5,   # two particles in 2D
             (2, 0, 2, 0): 0.1, (1, 0, 1, 0): -0.2, (0, 1, 0, 1): -0.2, (0, 2, 0, 2): 0.1, (4, 0, 0, 0): 0.05}


@pytest.mark.parametrize("V,d,p", [(ND_GEN2, 2, 1), (ND_GEN2, 2, 5), (ND_GEN2, 2, 9), (ND_GEN3, 3, 6),
                                   (ND_TWO_2D, 4, 4), ({(2,): 0.5, (4,): 1 / 24, (3,): -0.1}, 1, 10),
                                   ({(6, 0): 0.01, (0, 2): 0.5, (3, 3): 0.02}, 2, 6)])
def test_nd_generator_matches_the_oracle(V, d, p):
    from oracle import many_body as mb
    Vf = {k: _F(v) for k, v in V.items()}
    for eps in (0.05, 0.4):
        got = su.speedup_generate_nd(V, p, eps)
        ref = mb.collapsed(Vf, d, p, _F(eps))
        assert set(got) == set(ref)
        for k, v in ref.items():
            assert got[k] == pytest.approx(float(v), rel=1e-14, abs=1e-300), k


@pytest.mark.parametrize("V,kw,code", [
    ({(2, 0, 0, 0, 0): 1.0}, {}, -1),                 # d = 5
    ({(7, 0): 1.0}, {}, -1),                          # degree 7
    ({(4, 3): 1.0}, {}, -1),                          # total degree 7
    ({(-1, 2): 1.0}, {}, -1),                         # negative exponent
    ({(2, 0): float("inf")}, {}, -1),                 # non-finite coefficient
    ({(2, 0): 1.0}, {"p": 13}, -6),
    ({(2, 0): 1.0}, {"width_factor": 1.4}, -6),
    ({(2, 0): 1.0}, {"a": (float("nan"), 0.0)}, -1),
])
def test_nd_rejects_bad_requests(V, kw, code):
    d = len(next(iter(V)))
    args = {"p": 4, "a": (0.0,) * d, "b": (1.0,) * d}
    args.update({k: v for k, v in kw.items() if k in ("p", "a")})
    opts = {k: v for k, v in kw.items() if k not in ("p", "a")}
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_amplitude_nd(V, args["a"], args["b"], 1.0, args["p"], 3, 1000, 1, **opts)
    assert e.value.code == code


def test_nd_generator_term_limit():
    big = {(i, j): 1.0 for i in range(7) for j in range(7) if i + j <= 6}   # 28 terms: fine
    assert len(su.speedup_generate_nd(big, 2, 0.1)) > 0
    with pytest.raises(su.SpeedupError) as e:
        su.speedup_generate_nd({(2,): 1.0}, 0, 0.1)
    assert e.value.code == -1


def test_nd_table_fault_fails_before_any_device_work():
    su.su_fault_inject("table_nan")
    try:
        with pytest.raises(su.SpeedupError) as e:
            su.speedup_amplitude_nd({(2, 0): 0.5, (0, 2): 0.5}, (0.0, 0.0), (1.0, 1.0), 1.0, 4, 3, 100, 1)
        assert e.value.code == -5
    finally:
        su.su_fault_inject("clear")
    with pytest.raises(ValueError):
        su.speedup_amplitude_nd({(2, 0): 0.5}, (0.0,), (1.0, 1.0), 1.0, 4, 3, 100, 1)


# ---- the continuum fit (Eq. fit): host only, against the oracle's
def _levels(amps, errs):
    return [{"amp": float(a), "err": float(e), "n": 1} for a, e in zip(amps, errs)]


@pytest.mark.parametrize("p,n_min,n_terms", [(1, 1, 2), (2, 1, 3), (10, 2, 3), (4, 3, 2), (18, 1, 3)])
def test_fit_continuum_matches_the_oracle(p, n_min, n_terms):
    from oracle import fit
    rng = np.random.default_rng(p)
    s = 10
    N = 2.0 ** np.arange(s + 1)
    errs = rng.uniform(1e-5, 1e-4, s + 1)
    amps = 0.2 + 0.3 / N ** min(p, 30) + errs * rng.normal(size=s + 1)
    a, da, c2 = su.su_fit_continuum(_levels(amps, errs), p, n_min, n_terms)
    ra, rda, rc2 = fit.fit_continuum(amps, errs, p, n_min, n_terms)
    assert a == pytest.approx(ra, rel=1e-9, abs=1e-14)
    assert da == pytest.approx(rda, rel=1e-6)
    assert c2 == pytest.approx(rc2, rel=1e-6, abs=1e-12)


def test_fit_continuum_recovers_exact_series_and_rejects_bad_input():
    s, p = 8, 3
    N = 2.0 ** np.arange(s + 1)
    amps = 0.4 - 0.6 / N ** p + 0.25 / N ** (p + 1)
    a, _, c2 = su.su_fit_continuum(_levels(amps, np.full(s + 1, 1e-3)), p, 1, 3)
    assert a == pytest.approx(0.4, rel=1e-13) and c2 <= 1e-20
    for kw in ({"n_min": 0}, {"n_terms": 4}, {"n_min": 7}):
        args = {"n_min": 1, "n_terms": 3}
        args.update(kw)
        with pytest.raises(su.SpeedupError) as e:
            su.su_fit_continuum(_levels(amps, np.full(s + 1, 1e-3)), p, args["n_min"], args["n_terms"])
        assert e.value.code == -1
    bad = np.full(s + 1, 1e-3)
    bad[4] = 0.0
    with pytest.raises(su.SpeedupError):
        su.su_fit_continuum(_levels(amps, bad), p, 1, 3)


# ---- the command-line front end (the paper's argument order)
def _cli(*args):
    import subprocess
    from paper_1105_0542_gb300 import build as _b
    return subprocess.run([_b.CLI, *map(str, args)], capture_output=True, text=True, timeout=120)


def test_cli_usage_and_argument_errors():
    r = _cli()
    assert r.returncode == 0 and r.stdout.startswith("usage: speedup")
    assert _cli("-m", "nope", 1, 0, 1, 4, 100, 1).returncode == 2
    assert _cli(1, 0, 1).returncode == 2                      # fewer than six positional arguments
    assert _cli(1, 0, "x", 4, 100, 1).returncode == 2         # not a number
    assert _cli("-f", "fp16", 1, 0, 1, 4, 100, 1).returncode == 2
    r = _cli("-m", "aho", 1, 0, 1, 4, 100, 1, 1.0)             # wrong parameter count: the library's check
    assert r.returncode == 1 and "speedup:" in r.stderr


# ---- the host evaluators of W (speedup_wp, speedup_wp_nd)

def _wp_points(rng, n, d=None, x_scale=1.5, xb_scale=0.4):
    shape = (n,) if d is None else (n, d)
    return rng.uniform(-x_scale, x_scale, shape), rng.uniform(-xb_scale, xb_scale, shape)


@pytest.mark.parametrize("model,params,p", [("ho", [1.3], 6), ("aho", [1.0, 10.0], 10), ("dw", [5.0], 12),
                                            ("mpt", [3.0, 1.0], 8), ("poly", [0.0, -0.3, 0.5, 0.2, 1 / 24], 7),
                                            ("aho", [1.0, 48.0], 21)])
def test_host_wp_matches_the_oracle(model, params, p):
    from oracle import exact
    rng = np.random.default_rng(11)
    x, xb = _wp_points(rng, 64)
    for eps in (0.02, 0.25):
        got = su.speedup_wp(model, params, p, eps, x, xb)
        mdl = ea.make_model(model, [_F(v) for v in params] if model != "mpt" else params)
        ref = exact._wp_vec(mdl, p, x, xb, eps)
        scale = exact._wp_abs_vec(mdl, p, x, np.abs(xb), eps)
        assert np.all(np.abs(got - ref) <= 1e-13 * scale + 1e-300), (model, eps)


def test_host_wp_of_the_general_mode_matches_the_oracle_and_the_model_tables():
    from oracle import general_v as gv
    rng = np.random.default_rng(12)
    x, xb = _wp_points(rng, 48)
    gp = su.general_params((0.1, -0.2, 0.5, 0.0, 0.05), [(1.5, 2.0, 0.3)], [(-1.0, 2.0, 0.0)], [(0.4, 1.2, 0.5)])
    for p, eps in ((6, 0.1), (12, 0.02)):
        got = su.speedup_wp("general", gp, p, eps, x, xb)
        ref = gv.wp(gp, p, x, xb, eps)
        scale = gv.wp_abs(gp, p, x, xb, eps)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), p
    # the same anharmonic oscillator through the derivative-symbol program and
    # through the collapsed tables
    aho = su.general_params((0.0, 0.0, 0.5, 0.0, 10.0 / 24.0))
    for p in (4, 10):
        a = su.speedup_wp("general", aho, p, 0.05, x, xb)
        b = su.speedup_wp("aho", [1.0, 10.0], p, 0.05, x, xb)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14), p


@pytest.mark.parametrize("V,d,p", [(ND_GEN2, 2, 9), (ND_GEN3, 3, 6), (ND_TWO_2D, 4, 4),
                                   ({(2,): 0.5, (4,): 1 / 24, (3,): -0.1}, 1, 10),
                                   ({(2, 0): 0.5, (0, 2): 0.5, (4, 0): 1 / 24, (0, 4): 1 / 24, (2, 2): 1 / 12}, 2, 10)])
def test_host_wp_nd_program_matches_the_oracle(V, d, p):
    from oracle import many_body as mb
    rng = np.random.default_rng(13)
    x, xb = _wp_points(rng, 40, d)
    Vf = {k: _F(v) for k, v in V.items()}
    for eps in (0.05, 0.3):
        got = su.speedup_wp_nd(V, p, eps, x, xb)
        ref = mb.wp(Vf, d, p, x, xb, eps)
        scale = mb.wp_abs(Vf, d, p, x, xb, eps)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), eps


def test_host_wp_rejects_bad_requests():
    x = np.zeros(3)
    for call, code in [(lambda: su.speedup_wp("aho", [1.0, 1.0], 4, 0.0, x, x), -1),
                       (lambda: su.speedup_wp("aho", [1.0, 1.0], 4, float("nan"), x, x), -1),
                       (lambda: su.speedup_wp("aho", [1.0], 4, 0.1, x, x), -1),
                       (lambda: su.speedup_wp("aho", [1.0, 1.0], 145, 0.1, x, x), -1),
                       (lambda: su.speedup_wp("general", su.general_params((0, 0, 0.5)), 19, 0.1, x, x), -6),
                       (lambda: su.speedup_wp_nd({(2, 0): 1.0}, 4, -1.0, np.zeros((3, 2)), np.zeros((3, 2))), -1),
                       (lambda: su.speedup_wp_nd({(2, 0): 1.0}, 13, 0.1, np.zeros((3, 2)), np.zeros((3, 2))), -1)]:
        with pytest.raises(su.SpeedupError) as e:
            call()
        assert e.value.code == code
    with pytest.raises(ValueError):
        su.speedup_wp_nd({(2, 0): 1.0}, 4, 0.1, np.zeros((3, 3)), np.zeros((3, 3)))
    # no points: nothing to do
    assert su.speedup_wp("ho", [1.0], 3, 0.1, np.zeros(0), np.zeros(0)).shape == (0,)


def test_host_wp_nd_program_on_random_polynomials():
    """Random sparse polynomials (d = 1..3, degree <= 6, with and without a
    parity, so that the Horner variable, its step G and the groups' offsets
    j0 vary): the program's W equals the oracle's at random points."""
    from oracle import many_body as mb
    rng = np.random.default_rng(2024)
    for trial in range(20):
        d = int(rng.integers(1, 4))
        p = int(rng.integers(2, 7 if d < 3 else 5))
        V = {}
        for _ in range(int(rng.integers(3, 8))):
            e = [0] * d
            for _ in range(int(rng.integers(1, 7 if d < 3 else 5))):
                e[int(rng.integers(0, d))] += 1
            if trial % 3 == 0:                       # even in every coordinate
                e = [2 * (k // 2) for k in e]
            V[tuple(e)] = V.get(tuple(e), 0.0) + float(rng.integers(-8, 9)) / 8.0
        V = {k: v for k, v in V.items() if v and sum(k) > 0}
        if not V:
            continue
        x, xb = _wp_points(rng, 24, d, 1.0, 0.3)
        Vf = {k: _F(v) for k, v in V.items()}
        got = su.speedup_wp_nd(V, p, 0.1, x, xb)
        ref = mb.wp(Vf, d, p, x, xb, 0.1)
        scale = mb.wp_abs(Vf, d, p, x, xb, 0.1)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300), (V, d, p)


def test_host_wp_general_program_at_high_levels():
    """p = 14, 16, 18 (the paper's compiled W_p reaches 18; 24 196
    monomial-power entries at p = 18): the library's derivative-symbol
    program equals the oracle's exact-rational W_p on a polynomial + Gaussian
    + sech^2 potential at random points."""
    from oracle import general_v as gv
    rng = np.random.default_rng(78)
    gp = su.general_params((0.1, -0.2, 0.5, 0.05, 0.04), [(1.5, 2.0, 0.3)], [(-1.0, 1.0, 0.1)])
    for p in (14, 16, 18):
        x, xb = _wp_points(rng, 16, None, 1.0, 0.2)
        eps = 0.05
        got = su.speedup_wp("general", gp, p, eps, x, xb)
        ref = gv.wp(gp, p, x, xb, eps)
        scale = gv.wp_abs(gp, p, x, xb, eps)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300), (p, np.max(np.abs(got - ref) / scale))
    assert gv.term_count(18) == 24196


def test_host_wp_general_program_on_random_potentials():
    """Random general potentials (a polynomial and up to two terms of each
    family, p = 1..12): the library's derivative-symbol program equals the
    oracle's W_p at random points."""
    from oracle import general_v as gv
    rng = np.random.default_rng(77)
    for trial in range(10):
        p = int(rng.integers(1, 13))
        poly = [float(v) for v in rng.integers(-4, 5, size=int(rng.integers(1, 6))) / 4.0]
        gauss = [(float(rng.uniform(-2, 2)), float(rng.uniform(0.3, 3)), float(rng.uniform(-1, 1)))
                 for _ in range(int(rng.integers(0, 3)))]
        sech = [(float(rng.uniform(-2, 2)), float(rng.uniform(0.3, 2)), float(rng.uniform(-1, 1)))
                for _ in range(int(rng.integers(0, 3)))]
        expo = [(float(rng.uniform(-1, 1)), float(rng.uniform(0.2, 1.5)), float(rng.uniform(-1, 1)))
                for _ in range(int(rng.integers(0, 3)))]
        gp = su.general_params(poly, gauss, sech, expo)
        x, xb = _wp_points(rng, 24, None, 1.2, 0.3)
        eps = float(rng.uniform(0.01, 0.2))
        got = su.speedup_wp("general", gp, p, eps, x, xb)
        ref = gv.wp(gp, p, x, xb, eps)
        scale = gv.wp_abs(gp, p, x, xb, eps)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300), (trial, p)
