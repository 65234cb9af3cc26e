"""Oracle for the SPEEDUP effective-action path-integral Monte Carlo.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may.

The oracle is a plain, slow, obviously correct CPU restatement of what the
method computes, written from the paper (Balaz et al., "SPEEDUP Code for
Calculation of Transition Amplitudes via the Effective Action Approach"):

* ``effective_action`` -- exact-rational coefficients c_{m,k}(x) of the level-p
  effective potential (Sec. 2.1, Eq. ansatz, Eq. 1Drec, Eq. diagonal, Fig. 1
  order) over a polynomial ring in x (polynomial potentials) or in
  t = tanh(alpha x) (modified Poeschl-Teller, Sec. 3.3), and W_p itself.
* ``mc_oracle.c`` / ``mc`` -- the Monte Carlo estimate of the discretized
  amplitude A_N^(p)(a,b;T) (Sec. 4, Eq. SNp) by bisection paths (Sec. 4.1)
  fed by its own Philox4x32-10 and Box-Muller, one sample at a time.
* ``exact`` -- closed forms and brute force that pin the oracle: the Mehler
  kernel, the exact Gaussian value of A_N^(p) for the harmonic oscillator,
  tensor-grid quadrature over the N-1 intermediate points for tiny N, and
  exact-diagonalisation references (harmonic basis, sinc-DVR in one and two
  dimensions) for continuum amplitudes and spectra.
* ``evolution`` -- the evolution-operator matrix of Sec. 5 and its spectrum
  (the model potentials, the general potentials and systems of several
  coordinates on a tensor grid).
* ``proposal`` -- the learned proposal's network, loss and paths in numpy.
* ``general_v`` -- W_p of a general potential in the derivative symbols
  V_j (Sec. 3.1) and the derivatives of its families.
* ``many_body`` -- the contracted W_{m,k} of a system of d = D x M
  coordinates (Sec. 2.2, Eq. MBrec, Eq. DIA) and its Monte Carlo weights.

It shares no code with the CUDA path; only ``workloads`` (seeded input
definitions, none of the method's arithmetic) serves both.
"""
