"""Writes ed_aho_g10.json: the continuum amplitude A(0, 1; 1) of the
anharmonic oscillator V = q^2/2 + g q^4/24, g = 10 (Sec. 3.3), by exact
diagonalisation in the first 200 harmonic-oscillator states (the reference
the convergence sweep's errors are stated against), checked against 300
states.  Calls only the oracle (oracle/exact.py); run from the repository
root:  python tests/golden/make_ed_reference.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402


def main():
    g, a, b, T = 10.0, 0.0, 1.0, 1.0
    V = [0.0, 0.0, 0.5, 0.0, g / 24.0]
    A200, E200 = exact.ed_amplitude(V, a, b, T, nbasis=200)
    A300, E300 = exact.ed_amplitude(V, a, b, T, nbasis=300)
    out = {"potential": "q^2/2 + g q^4/24", "g": g, "a": a, "b": b, "T": T,
           "A": A200, "A_300_states": A300, "E0": float(E200[0]), "E1": float(E200[1]),
           "method": "exact diagonalisation, harmonic-oscillator basis (omega = 1) of 200 states; "
                     "A = sum_n psi_n(a) psi_n(b) exp(-E_n T) (Sec. 5 / Sec. 4 continuum limit)",
           "written_by": "tests/golden/make_ed_reference.py (oracle/exact.ed_amplitude)"}
    with open(os.path.join(HERE, "ed_aho_g10.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
