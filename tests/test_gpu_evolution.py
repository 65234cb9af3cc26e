"""GPU parity of the space-discretized evolution operator (Sec. 5, Fig. 3).

* elements against the oracle's matrix (same grid, W_p from the exact
  coefficients), compared in the exponent: |d log U| <= max(tol, 64 u A),
  A = t sum_terms |term| of W_p (the rounding scale of -t W_p), tol = 1e-12
  (double) or 1e-5 (single-precision W_p);
* the matrix is exactly symmetric;
* spectra: the eigenvalues of the device matrix (torch's symmetric
  eigensolver) give the oracle's energies on the same grid (1e-10) and the
  sinc-DVR energies of both Fig. 3 potentials at the figure's level p = 21
  (1e-9);
* the paper's grid of Fig. 3 (anharmonic, L = 8, Delta = 9.77e-4, n = 16385):
  finite, positive, symmetric, and its diagonal matches the oracle at sampled
  points;
* the band storage: every diagonal equal, bit for bit, to the dense matrix's,
  nothing outside the band, on a ragged grid for six potentials;
* the band eigensolver (Chebyshev-filtered subspace iteration, no library
  eigensolver): the lowest eight energies equal the oracle's numpy
  diagonalisation of its own matrix (1e-10), and on both of Fig. 3's
  16 385-point grids the lowest ten equal sinc-DVR (1e-9), the tunnelling
  doublet of the double well included; the returned eigenfunctions are
  orthonormal on the grid and the ground state has no node.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1105_0542_gb300 as su  # noqa: E402
from oracle import effective_action as ea  # noqa: E402
from oracle import evolution as ev  # noqa: E402
from oracle import exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    torch.cuda.set_device(0)


def _device_matrix(model, params, p, t, L, n, precision="fp64"):
    U = torch.empty((n, n), dtype=torch.float64, device="cuda")
    su.speedup_evolution_matrix(model, params, p, t, L, n, U, precision=precision)
    torch.cuda.synchronize()
    return U


CASES = [("ho", [1.0], 12, 0.1, 8.0), ("aho", [1.0, 48.0], 21, 0.02, 8.0), ("aho", [-10.0, 12.0], 21, 0.1, 10.0),
         ("dw", [5.0], 12, 0.05, 3.0), ("mpt", [3.0, 1.0], 12, 0.05, 6.0), ("aho", [1.0, 10.0], 32, 0.01, 4.0)]


@pytest.mark.parametrize("prec,tol,u", [("fp64", 1e-12, 2.0 ** -53), ("fp32", 1e-5, 2.0 ** -24)])
@pytest.mark.parametrize("model,params,p,t,L", CASES)
def test_elements_match_oracle(model, params, p, t, L, prec, tol, u):
    n = 203                              # ragged against the 32 x 8 thread blocks
    got = _device_matrix(model, params, p, t, L, n, prec).cpu().numpy()
    ref = ev.evolution_matrix(model, params, p, t, L, n)
    A = ev.evolution_matrix_abs(model, params, p, t, L, n)
    live = ref > 0
    assert live.sum() > 3 * n            # a band around the diagonal
    x = ev.grid(L, n)
    free = (x[None, :] - x[:, None]) ** 2 / (2 * t)
    # the same band (reading E-1); a difference only on its edge
    assert np.all(np.abs(free[(got > 0) != live] - ev.BAND) < 1e-9)
    live &= got > 0
    d = np.abs(np.log(got[live]) - np.log(ref[live]))
    allow = np.maximum(tol, 64 * u * A[live])
    assert float(np.max(d / allow)) <= 1.0


def test_matrix_is_exactly_symmetric():
    U = _device_matrix("aho", [1.0, 48.0], 21, 0.02, 8.0, 1001)
    assert torch.equal(U, U.T)


@pytest.mark.parametrize("params,t,L,V", [([1.0, 48.0], 0.02, 8.0, lambda x: 0.5 * x * x + 2.0 * x ** 4),
                                          ([-10.0, 12.0], 0.1, 10.0, lambda x: -5.0 * x * x + 0.5 * x ** 4)])
def test_figure3_spectra(params, t, L, V):
    n = 401
    U = _device_matrix("aho", params, 21, t, L, n)
    lam = torch.linalg.eigvalsh(U).cpu().numpy()[::-1][:8]
    E = -np.log(lam) / t
    Eo = ev.energies(ev.evolution_matrix("aho", params, 21, t, L, n), t, 8)
    assert np.abs(E - Eo).max() <= 1e-10, E - Eo
    _, Ed = exact.dvr_amplitude(V, 0.0, 0.0, 1.0, L=L, dx=0.01)
    assert np.abs(E - Ed[:8]).max() <= 1e-9, E - Ed[:8]


def test_paper_grid_of_figure3():
    n, L, t, p = 16385, 8.0, 0.02, 21
    U = _device_matrix("aho", [1.0, 48.0], p, t, L, n)
    assert bool(torch.isfinite(U).all()) and bool((U >= 0).all())
    idx = torch.arange(0, n, 997, device="cuda")
    assert torch.equal(U[idx][:, idx], U[idx][:, idx].T)
    # sampled elements near the diagonal against the oracle's formula
    x = np.linspace(-L, L, n)
    delta = 2 * L / (n - 1)
    model = ea.make_model("aho", [1.0, 48.0])
    Uh = U[idx].cpu().numpy()
    for r, i in enumerate(idx.cpu().numpy()):
        for j in (i, min(i + 3, n - 1), max(i - 50, 0)):
            xm, xb = 0.5 * (x[i] + x[j]), 0.5 * (x[j] - x[i])
            w = exact._wp_vec(model, p, np.array([xm]), np.array([xb]), t)[0]
            ref = math.exp(math.log(delta) - 0.5 * math.log(2 * math.pi * t) - (x[j] - x[i]) ** 2 / (2 * t) - t * w)
            assert Uh[r, j] == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("model,params,p,t,L", CASES)
def test_band_equals_the_dense_matrix(model, params, p, t, L):
    n = 203
    U = _device_matrix(model, params, p, t, L, n).cpu().numpy()
    w, pitch = su.su_evolution_band_size(t, L, n)
    D = torch.full(((w + 1) * pitch,), float("nan"), dtype=torch.float64, device="cuda")
    su.speedup_evolution_band(model, params, p, t, L, n, D)
    torch.cuda.synchronize()
    Dh = D.cpu().numpy().reshape(w + 1, pitch)
    for k in range(w + 1):
        assert np.array_equal(Dh[k, :n - k], np.diagonal(U, k)), k
        assert not Dh[k, n - k:n].any(), k
    assert not np.triu(U, w + 1).any()


SPECTRUM_CASES = [("ho", [1.0], 12, 0.1, 8.0), ("aho", [1.0, 48.0], 21, 0.02, 8.0), ("aho", [-10.0, 12.0], 21, 0.1, 10.0),
                  ("dw", [5.0], 12, 0.05, 3.0), ("mpt", [3.0, 1.0], 12, 0.05, 6.0)]


@pytest.mark.parametrize("model,params,p,t,L", SPECTRUM_CASES)
def test_band_spectrum_matches_the_oracle(model, params, p, t, L):
    n = 401
    E, R, info = su.speedup_evolution_spectrum(model, params, p, t, L, n, 8)
    Eo = ev.energies(ev.evolution_matrix(model, params, p, t, L, n), t, 8)
    assert info["converged"] == 1 and info["block"] == 16
    assert np.all(np.abs(np.array(E) - Eo) <= 1e-10 * np.maximum(1.0, np.abs(Eo))), np.array(E) - Eo
    assert max(R) <= 1e-11 * math.exp(-t * Eo[0])


@pytest.mark.parametrize("params,t,L,V", [([1.0, 48.0], 0.02, 8.0, lambda x: 0.5 * x * x + 2.0 * x ** 4),
                                          ([-10.0, 12.0], 0.1, 10.0, lambda x: -5.0 * x * x + 0.5 * x ** 4)])
def test_figure3_spectra_on_the_paper_grid(params, t, L, V):
    n, nev = 16385, 10
    vec = torch.empty((nev, n), dtype=torch.float64, device="cuda")
    E, R, info = su.speedup_evolution_spectrum("aho", params, 21, t, L, n, nev, vectors=vec)
    _, Ed = exact.dvr_amplitude(V, 0.0, 0.0, 1.0, L=L, dx=0.01)
    assert info["converged"] == 1
    assert np.abs(np.array(E) - Ed[:nev]).max() <= 1e-9, np.array(E) - Ed[:nev]
    assert info["band_bytes"] < 0.4e9                   # the band, not the 2.1 GB dense matrix
    delta = 2 * L / (n - 1)
    G = (vec @ vec.T).cpu().numpy() * delta
    assert np.abs(G - np.eye(nev)).max() <= 1e-10
    g = vec[0].cpu().numpy()
    assert (g * np.sign(g[n // 2]) > -1e-12).all()      # the ground state has no node


def _morse_params(D, a, x0):
    """D (1 - e^{-a (x - x0)})^2 = D - 2D e^{-a (x - x0)} + D e^{-2a (x - x0)}"""
    return list(su.general_params((D,), (), (), [(-2.0 * D, a, x0), (D, 2.0 * a, x0)]))


def test_general_potential_band_equals_dense_and_oracle():
    """The evolution operator of a general potential (W_p from the
    derivative-symbol program): band storage equal to the dense matrix bit
    for bit, and the dense matrix equal to the oracle's (general_v W_p) in
    the exponent."""
    gp = list(su.general_params((0.0, 0.0, 0.5), [(-4.0, 1.5, 0.4)], [(-1.0, 2.0, -0.3)]))
    p, t, L, n = 8, 0.05, 5.0, 151
    U = _device_matrix("general", gp, p, t, L, n).cpu().numpy()
    w, pitch = su.su_evolution_band_size(t, L, n)
    D = torch.full(((w + 1) * pitch,), float("nan"), dtype=torch.float64, device="cuda")
    su.speedup_evolution_band("general", gp, p, t, L, n, D)
    torch.cuda.synchronize()
    Dh = D.cpu().numpy().reshape(w + 1, pitch)
    for k in range(w + 1):
        assert np.array_equal(Dh[k, :n - k], np.diagonal(U, k)), k
    x = ev.grid(L, n)
    ref = ev.evolution_matrix_general(gp, p, t, x)
    live = (ref > 0) & (U > 0)
    assert live.sum() > 3 * n
    assert np.abs(np.log(U[live]) - np.log(ref[live])).max() <= 1e-11


@pytest.mark.parametrize("name,params,p,t,L,n,ref", [
    ("morse", _morse_params(12.5, 1.0, -5.1), 10, 0.02, 7.0, 701,
     [5.0 * (k + 0.5) - 25.0 * (k + 0.5) ** 2 / 50.0 for k in range(4)]),
    ("poeschl-teller", list(su.general_params((), (), [(-6.0, 1.0, 0.0)])), 8, 0.02, 20.0, 2001,
     [-(3.0 - k) ** 2 / 2.0 for k in range(3)]),
])
def test_general_potential_spectrum_is_the_closed_form(name, params, p, t, L, n, ref):
    """Sec. 5 with a general potential through the band eigensolver: the
    Morse levels w (n + 1/2) - w^2 (n + 1/2)^2 / (4D) (w = a sqrt(2D)) and the
    Poeschl-Teller levels -(l - n)^2 / 2 (l = 3), within 1e-9."""
    E, R, info = su.speedup_evolution_spectrum("general", params, p, t, L, n, len(ref))
    assert info["converged"] == 1
    assert np.abs(np.array(E) - np.array(ref)).max() <= 1e-9, np.array(E) - np.array(ref)
