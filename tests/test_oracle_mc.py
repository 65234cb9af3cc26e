"""Pins of the oracle's Monte Carlo estimate of A_N^(p)(a,b;T) (CPU only).

* free particle (V = 0): every weight is exactly 1, the estimate is the free
  amplitude with zero error (the bridge normalisation of Sec. 4.1);
* harmonic oscillator: the exact Gaussian value of A_N^(p) (Eq. SNp with a
  quadratic W_p) within 3 sigma, at every level of the hierarchy (Sec. 4.1);
* anharmonic, double-well, Poeschl-Teller and odd polynomial potentials:
  tensor-grid quadrature over the N-1 intermediate points (N = 2, 4);
* p = 1 is the naive midpoint action -eps sum V(x_k) (Sec. 2.1, Eq. SNp);
* the level-n weight is -eps_n sum W_p over the level-n subpath (Sec. 4.1),
  checked with an independent numpy evaluation of W_p;
* the literal bisection width sqrt(T/2^n) (Sec. 4.1) with its Gaussian
  reweighting gives the same amplitude;
* the convergence law A_N - A ~ 1/N^p (Sec. 2.1, Eq. fit) against exact
  diagonalisation, and the Mehler limit.
"""
import math

import numpy as np
import pytest

from oracle import exact, mc
from oracle import effective_action as ea

A, B, T = 0.0, 1.0, 1.0


def _within(res, ref, nsig=3.0):
    sig = max(res["err"], res["err_naive"])
    return abs(res["amp"] - ref) <= nsig * sig, (res["amp"], ref, sig)


def test_free_particle_has_zero_variance():
    o = mc.Oracle("poly", [0.0], 4)
    r = o.amplitude(A, B, T, 5, 2000, 7, n_blocks=10)
    free = math.exp(mc.log_A_free(A, B, T))
    for lev in r:
        assert lev["amp"] == pytest.approx(free, rel=1e-15)
        assert lev["err"] == 0.0 and lev["err_naive"] == 0.0


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_harmonic_matches_exact_discretized(p):
    o = mc.Oracle("ho", [1.0], p)
    r = o.amplitude(A, B, T, 4, 100000, 1234, n_blocks=10, threads=4)
    for lev in r:
        ref = exact.ho_discretized(p, 2 ** lev["n"], A, B, T)
        if lev["n"] == 0:
            assert lev["amp"] == pytest.approx(ref, rel=1e-13)
        else:
            ok, info = _within(lev, ref)
            assert ok, (lev["n"], info)


@pytest.mark.parametrize("name,params,p,a,b,Tq", [
    ("aho", [1.0, 1.0], 4, 0.0, 1.0, 1.0),
    ("aho", [1.0, 10.0], 3, 0.0, 1.0, 1.0),
    ("dw", [1.0], 4, -1.0, 1.0, 1.0),
    ("mpt", [3.0, 1.0], 4, -1.0, 1.0, 1.0),
    ("poly", [0.2, -0.5, 0.3, 0.25, 0.1], 3, -0.5, 0.7, 0.8),
])
def test_tiny_N_matches_quadrature(name, params, p, a, b, Tq):
    o = mc.Oracle(name, params, p)
    r = o.amplitude(a, b, Tq, 2, 100000, 4321, n_blocks=10, threads=4)
    q1, _ = exact.quadrature(name, params, p, 1, a, b, Tq)
    assert r[0]["amp"] == pytest.approx(q1, rel=1e-12)
    for n, N in ((1, 2), (2, 4)):
        ref, edge = exact.quadrature(name, params, p, N, a, b, Tq)
        assert edge < 1e-12
        ok, info = _within(r[n], ref)
        assert ok, (N, info)


def test_p1_is_the_naive_midpoint_action():
    o = mc.Oracle("aho", [1.0, 10.0], 1)
    s, seed = 5, 11
    w, _ = o.logweights(A, B, T, s, seed, 20)
    V = lambda y: 0.5 * y * y + 10.0 / 24.0 * y ** 4
    for i in range(20):
        q, _ = o.path(A, B, T, s, seed, i)
        for n in range(1, s + 1):
            qq = q[:: 2 ** (s - n)]
            eps = T / 2 ** n
            ref = -eps * np.sum(V(0.5 * (qq[1:] + qq[:-1])))
            assert w[i, n - 1] == pytest.approx(ref, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("name,params,p", [("aho", [1.0, 10.0], 10), ("mpt", [3.0, 1.0], 6),
                                           ("poly", [0.1, 0.2, -0.3, 0.05], 5)])
def test_level_weights_are_subpath_sums(name, params, p):
    o = mc.Oracle(name, params, p)
    model = ea.make_model(name, params)
    s, seed = 6, 5
    w, _ = o.logweights(-0.3, 0.8, 1.5, s, seed, 8, sample0=1000, instance=2)
    for i in range(8):
        q, _ = o.path(-0.3, 0.8, 1.5, s, seed, 1000 + i, instance=2)
        for n in range(1, s + 1):
            qq = q[:: 2 ** (s - n)]
            eps = 1.5 / 2 ** n
            W = exact._wp_vec(model, p, 0.5 * (qq[1:] + qq[:-1]), 0.5 * (qq[1:] - qq[:-1]), eps)
            ref = -eps * float(np.sum(W))
            assert w[i, n - 1] == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_bisection_points_are_bridge_midpoints():
    o = mc.Oracle("ho", [1.0], 2)
    s, seed, samp = 4, 3, 17
    q, _ = o.path(A, B, T, s, seed, samp)
    z = mc.normals(seed, 0, samp, 2 ** s - 1)
    assert q[0] == A and q[-1] == B
    for n in range(1, s + 1):
        h = 2 ** (s - n)
        sig = math.sqrt(T / 2 ** (n + 1))
        for i in range(2 ** (n - 1)):
            j = 2 ** (n - 1) - 1 + i
            k = (2 * i + 1) * h
            assert q[k] == pytest.approx(0.5 * (q[k - h] + q[k + h]) + sig * z[j], rel=1e-15, abs=1e-15)


def test_literal_width_with_reweighting_is_unbiased():
    o = mc.Oracle("aho", [1.0, 1.0], 4)
    r1 = o.amplitude(A, B, T, 4, 100000, 99, n_blocks=10, threads=4)
    r2 = o.amplitude(A, B, T, 4, 100000, 98, n_blocks=10, threads=4, wf=math.sqrt(2.0))
    for a_, b_ in zip(r1[1:], r2[1:]):
        sig = math.hypot(max(a_["err"], a_["err_naive"]), max(b_["err"], b_["err_naive"]))
        assert abs(a_["amp"] - b_["amp"]) <= 3 * sig


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_convergence_law_against_exact_diagonalisation(p):
    a, b, Tq = 0.0, 0.5, 0.3
    ref = exact.ed_amplitude([0, 0, 0.5, 0, 1 / 24], a, b, Tq, 200)[0]
    e2 = exact.quadrature("aho", [1.0, 1.0], p, 2, a, b, Tq)[0] - ref
    e4 = exact.quadrature("aho", [1.0, 1.0], p, 4, a, b, Tq, npts=120)[0] - ref
    assert 0.6 * 2 ** p < e2 / e4 < 1.6 * 2 ** p


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
def test_harmonic_convergence_slope_and_mehler_limit(p):
    m = exact.mehler_mp(A, B, T, dps=80)
    e = [exact.ho_discretized(p, N, A, B, T, dps=80, as_mp=True) - m for N in (16, 32, 64, 4096)]
    slope = math.log2(float(abs(e[1] / e[2])))
    assert abs(slope - p) < 0.15
    # and the error keeps shrinking as 1/N^p all the way to N = 4096
    assert abs(e[3]) < 2 * abs(e[2]) * (64.0 / 4096.0) ** p


def test_exact_references_agree():
    m = exact.mehler(0.0, 1.0, 1.0)
    assert m == pytest.approx(0.19086749087772256, rel=1e-15)
    assert exact.ed_amplitude([0, 0, 0.5], 0.0, 1.0, 1.0)[0] == pytest.approx(m, rel=1e-12)
    assert exact.dvr_amplitude(lambda y: 0.5 * y * y, 0.0, 1.0, 1.0)[0] == pytest.approx(m, rel=1e-9)
    # Poeschl-Teller with l(l-1)/2 = 3: bound states at -alpha^2 (l-1-n)^2 / 2 = -2, -1/2
    E = exact.dvr_amplitude(lambda y: -3.0 / np.cosh(y) ** 2, -1.0, 1.0, 1.0, L=25.0, dx=0.02)[1]
    assert E[0] == pytest.approx(-2.0, abs=1e-8) and E[1] == pytest.approx(-0.5, abs=1e-8)
    # anharmonic oscillator: two independent methods
    aho = exact.ed_amplitude([0, 0, 0.5, 0, 10 / 24], 0.0, 1.0, 1.0, 200)[0]
    assert aho == pytest.approx(exact.ed_amplitude([0, 0, 0.5, 0, 10 / 24], 0.0, 1.0, 1.0, 300)[0], rel=1e-12)
    assert aho == pytest.approx(exact.dvr_amplitude(lambda y: 0.5 * y * y + 10 / 24 * y ** 4,
                                                    0.0, 1.0, 1.0, L=10.0, dx=0.02)[0], rel=1e-9)
