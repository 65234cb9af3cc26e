"""Pins of the oracle's space-discretized evolution operator (Sec. 5, Fig. 3)
and its spectrum, CPU only.

* harmonic oscillator: U equals Delta times the Mehler kernel (the exact
  short-time amplitude) and its eigenvalues give E_k = k + 1/2;
* the two potentials of Fig. 3 at the figure's level p = 21 and times t
  (anharmonic A = 1, g = 48, t = 0.02, L = 8; double well A = -10, g = 12,
  t = 0.1, L = 10): the lowest eight energies equal the sinc-DVR
  diagonalisation of the Hamiltonian (an independent method) within 1e-9;
* the effective action's convergence: at p = 4 the short-time error is
  visible (> 1e-7), at p = 8 it is below 1e-9;
* the Poeschl-Teller model (tanh^2 ring): the three bound states of
  -6/cosh^2 x equal the closed form -(3 - n)^2/2 within 1e-10 at p = 8.
"""
import math

import numpy as np

from oracle import evolution as ev
from oracle import exact


def test_harmonic_oscillator_matrix_is_the_mehler_kernel():
    L, n, t = 8.0, 401, 0.1
    U = ev.evolution_matrix("ho", [1.0], 12, t, L, n)
    x = ev.grid(L, n)
    delta = 2 * L / (n - 1)
    Um = np.array([[exact.mehler(a, b, t) for b in x] for a in x]) * delta
    assert np.abs(U - Um).max() <= 1e-12 * Um.max()
    E = ev.energies(U, t, 10)
    np.testing.assert_allclose(E, np.arange(10) + 0.5, rtol=0, atol=1e-11)


def _dvr_energies(V, L, k):
    _, E = exact.dvr_amplitude(V, 0.0, 0.0, 1.0, L=L, dx=0.01)
    return E[:k]


def test_figure3_anharmonic_spectrum_matches_dvr():
    U = ev.evolution_matrix("aho", [1.0, 48.0], 21, 0.02, 8.0, 401)
    E = ev.energies(U, 0.02, 8)
    Ed = _dvr_energies(lambda x: 0.5 * x * x + 2.0 * x ** 4, 8.0, 8)
    assert np.abs(E - Ed).max() <= 1e-9, E - Ed


def test_figure3_double_well_spectrum_matches_dvr():
    U = ev.evolution_matrix("aho", [-10.0, 12.0], 21, 0.1, 10.0, 401)
    E = ev.energies(U, 0.1, 8)
    Ed = _dvr_energies(lambda x: -5.0 * x * x + 0.5 * x ** 4, 10.0, 8)
    assert np.abs(E - Ed).max() <= 1e-9, E - Ed
    # the ground-state tunnelling doublet
    assert 0 < E[1] - E[0] < 1e-3


def test_spectrum_converges_with_the_level_p():
    Ed = _dvr_energies(lambda x: 0.5 * x * x + 2.0 * x ** 4, 8.0, 6)
    err = {}
    for p in (4, 8):
        U = ev.evolution_matrix("aho", [1.0, 48.0], p, 0.02, 8.0, 401)
        err[p] = np.abs(ev.energies(U, 0.02, 6) - Ed).max()
    assert err[4] > 1e-7 and err[8] < 1e-9, err


def test_poeschl_teller_model_spectrum_is_the_closed_form():
    """The model-specific Poeschl-Teller action (the tanh^2 ring) in the
    evolution operator: V = -6/cosh^2 x = -l(l+1)/2 sech^2 x with l = 3 has
    the bound states E_n = -(l - n)^2/2 = -4.5, -2, -0.5; p = 8 gives them
    within 1e-10, p = 4 misses them by > 1e-8."""
    exact_E = np.array([-4.5, -2.0, -0.5])
    err = {}
    for p in (8, 4):
        U = ev.evolution_matrix("mpt", [6.0, 1.0], p, 0.02, 14.0, 1401)
        err[p] = np.abs(ev.energies(U, 0.02, 3) - exact_E).max()
    assert err[8] <= 1e-10 and err[4] > 1e-8, err
