"""The stored reference values under tests/golden/ against the oracle that
wrote them and against an independent method.

* ed_aho_g10.json -- the continuum amplitude A(0, 1; 1) of the anharmonic
  oscillator g = 10 (the convergence sweep's exact-diagonalisation reference,
  200 harmonic-oscillator states): equal to what oracle/exact.ed_amplitude
  gives now, to its 300-state value, and to a sinc-DVR diagonalisation of the
  same Hamiltonian on a grid (a different basis and discretisation).
"""
import json
import os

import pytest

from oracle import exact

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_ed_reference_of_the_convergence_sweep():
    with open(os.path.join(HERE, "ed_aho_g10.json")) as f:
        ref = json.load(f)
    g = ref["g"]
    V = [0.0, 0.0, 0.5, 0.0, g / 24.0]
    A, _ = exact.ed_amplitude(V, ref["a"], ref["b"], ref["T"], nbasis=200)
    assert A == pytest.approx(ref["A"], rel=1e-13)
    assert ref["A_300_states"] == pytest.approx(ref["A"], rel=1e-10)
    dvr, _ = exact.dvr_amplitude(lambda x: 0.5 * x * x + g / 24.0 * x ** 4, ref["a"], ref["b"], ref["T"],
                                 L=8.0, dx=0.02)
    assert dvr == pytest.approx(ref["A"], rel=1e-8)
