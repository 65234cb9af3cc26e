"""Pins of the general-potential oracle (W_p in the derivative symbols,
Sec. 3.1, with the families' derivatives of every order) through the
spectrum of its evolution operator (Sec. 5), CPU only.

Each family is pinned against an energy spectrum that owes nothing to the
effective action:

* exponentials: the Morse potential D (1 - e^{-a x})^2 = D - 2D e^{-a x} +
  D e^{-2a x}, whose bound states are E_n = w (n + 1/2) - w^2 (n + 1/2)^2/(4D)
  with w = a sqrt(2D) (hbar = m = 1);
* sech^2: the Poeschl-Teller well -l(l+1)/2 sech^2(x), E_n = -(l - n)^2/2;
* Gaussians: a harmonic trap with a displaced Gaussian dip, against the
  sinc-DVR diagonalisation of the Hamiltonian.

At level p = 8..10 and t = 0.02 the lowest levels agree to ~1e-12; at p = 4
the short-time error of the truncated action is visible, so the pins see the
higher derivative terms, not only V itself.
"""
import math

import numpy as np
import pytest

from oracle import evolution as ev
from oracle import exact
from oracle import general_v as gv


def _energies(params, p, t, lo, hi, n, k):
    U = ev.evolution_matrix_general(params, p, t, np.linspace(lo, hi, n))
    return ev.energies(U, t, k)


def _morse(D, a):
    params = [0.0] * gv.N_PARAMS_EXP
    params[0] = D
    o = gv.N_PARAMS
    params[o:o + 3] = [-2.0 * D, a, 0.0]
    params[o + 3:o + 6] = [D, 2.0 * a, 0.0]
    return params


def _poeschl_teller(l):
    params = [0.0] * gv.N_PARAMS
    o = gv.N_POLY + 3 * gv.N_GAUSS
    params[o:o + 3] = [-l * (l + 1) / 2.0, 1.0, 0.0]
    return params


@pytest.mark.parametrize("p, tol", [(10, 1e-10), (4, None)])
def test_morse_spectrum_is_the_closed_form(p, tol):
    D, a = 12.5, 1.0
    w = a * math.sqrt(2.0 * D)
    exact_E = np.array([w * (n + 0.5) - w * w * (n + 0.5) ** 2 / (4.0 * D) for n in range(4)])
    E = _energies(_morse(D, a), p, 0.02, -1.8, 12.0, 691, 4)
    err = np.abs(E - exact_E).max()
    if tol is None:
        assert err > 1e-7, err           # the level-4 action's short-time error
    else:
        assert err <= tol, E - exact_E


@pytest.mark.parametrize("p, tol", [(8, 1e-10), (4, None)])
def test_poeschl_teller_spectrum_is_the_closed_form(p, tol):
    l = 3.0
    exact_E = np.array([-(l - n) ** 2 / 2.0 for n in range(3)])
    E = _energies(_poeschl_teller(l), p, 0.02, -20.0, 20.0, 2001, 3)
    err = np.abs(E - exact_E).max()
    if tol is None:
        assert err > 1e-8, err
    else:
        assert err <= tol, E - exact_E


@pytest.mark.parametrize("p, tol", [(8, 1e-10), (4, None)])
def test_gaussian_dip_spectrum_matches_dvr(p, tol):
    params = [0.0] * gv.N_PARAMS
    params[2] = 0.5
    params[gv.N_POLY:gv.N_POLY + 3] = [-4.0, 1.5, 0.4]
    _, Ed = exact.dvr_amplitude(lambda x: 0.5 * x * x - 4.0 * np.exp(-1.5 * (x - 0.4) ** 2),
                                0.0, 0.0, 1.0, L=8.0, dx=0.01)
    E = _energies(params, p, 0.02, -8.0, 8.0, 801, 6)
    err = np.abs(E - Ed[:6]).max()
    if tol is None:
        assert err > 1e-8, err
    else:
        assert err <= tol, E - Ed[:6]
