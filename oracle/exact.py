"""Closed forms and brute force that pin the oracle (no Monte Carlo here).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

* ``mehler`` -- the exact harmonic-oscillator amplitude (Mehler kernel), the
  continuum limit the discretized amplitudes converge to (Sec. 4, Eq. fit).
* ``ho_W_exact`` -- the exact effective potential of the harmonic oscillator,
  read off from the Mehler kernel through the definition of Sec. 2.1
  (A = (2 pi eps)^(-1/2) exp(-2 xb^2/eps - eps W)).
* ``ho_discretized`` -- the exact value of A_N^(p) (Eq. SNp) for the harmonic
  oscillator, whose W_p is a quadratic form in (x, xb): a Gaussian integral
  over q_1..q_{N-1} with a tridiagonal matrix, done in 40-digit arithmetic.
* ``quadrature`` -- A_N^(p) for N = 1, 2, 4 by tensor-grid Gauss-Legendre
  quadrature over the N-1 intermediate points (Eq. SNp written out) on a
  finite box.
* ``ed_amplitude`` / ``dvr_amplitude`` -- the continuum amplitude
  A(a,b;T) = sum_n psi_n(a) psi_n(b) exp(-E_n T) from exact diagonalisation
  in a harmonic-oscillator basis (polynomial potentials) or on a sinc-DVR
  grid (any potential).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import effective_action as ea


def mehler(a, b, T, omega=1.0):
    sh, ch = math.sinh(omega * T), math.cosh(omega * T)
    return math.sqrt(omega / (2 * math.pi * sh)) * math.exp(
        -omega * ((a * a + b * b) * ch - 2 * a * b) / (2 * sh))


def ho_W_exact(x, xb, eps, omega=1.0):
    """W of the harmonic oscillator from the Mehler kernel (any eps > 0)."""
    we = omega * eps
    sh, ch = math.sinh(we), math.cosh(we)
    return ((omega / sh) * (x * x * (ch - 1) + xb * xb * (ch + 1)) - 2 * xb * xb / eps) / eps \
        + math.log(sh / we) / (2 * eps)


def ho_quadratic_form(p, eps, omega=1.0):
    """W_p = alpha x^2 + beta xb^2 + gamma for the harmonic oscillator, from
    the oracle's c_{m,k}; raises if any other monomial appears."""
    c = ea.coefficients(ea.make_model("ho", [omega]), p)
    eps = Fraction(eps)
    al = be = ga = Fraction(0)
    for (m, k), poly in c.items():
        for i, v in enumerate(poly):
            if v == 0:
                continue
            term = v * eps ** (m - k)
            if (i, k) == (2, 0):
                al += term
            elif (i, k) == (0, 1):
                be += term
            elif (i, k) == (0, 0):
                ga += term
            else:
                raise AssertionError(f"unexpected monomial x^{i} xb^{2*k} in harmonic W_{p}")
    return al, be, ga


def mehler_mp(a, b, T, omega=1, dps=60):
    """The Mehler kernel in dps-digit arithmetic (an mpmath number)."""
    import mpmath as mp
    with mp.workdps(dps):
        w, T = mp.mpf(omega), mp.mpf(T)
        a, b = mp.mpf(a), mp.mpf(b)
        sh, ch = mp.sinh(w * T), mp.cosh(w * T)
        return +(mp.sqrt(w / (2 * mp.pi * sh)) * mp.exp(-w * ((a * a + b * b) * ch - 2 * a * b) / (2 * sh)))


def ho_discretized(p, N, a, b, T, omega=1.0, dps=40, as_mp=False, w_scale=1):
    """Exact A_N^(p)(a,b;T) of the harmonic oscillator (Gaussian integral).

    w_scale = k replaces W_p by k W_p (Eq. SNp otherwise unchanged): then
    A_N[k W_p] / A_free = E[exp(k w)] under the bisection bridge, the k-th
    moment of the estimator's per-sample factor exp(w) (Sec. 4.1), which
    pins the error bars of the Monte Carlo estimate."""
    import mpmath as mp
    with mp.workdps(dps):
        eps = mp.mpf(T) / N
        al, be, ga = ho_quadratic_form(p, Fraction(T) / N, omega)
        al, be, ga = (mp.mpf(v.numerator) / v.denominator * w_scale for v in (al, be, ga))
        # per slice: (q'-q)^2/(2 eps) + eps (al x^2 + be xb^2 + ga)
        #          = Ac (q'-q)^2 + Bc (q'+q)^2 + eps ga
        Ac = 1 / (2 * eps) + eps * be / 4
        Bc = eps * al / 4
        a_, b_ = mp.mpf(a), mp.mpf(b)
        if N == 1:
            S = Ac * (b_ - a_) ** 2 + Bc * (b_ + a_) ** 2 + eps * ga
            val = (2 * mp.pi * eps) ** (-0.5) * mp.exp(-S)
            return +val if as_mp else float(val)
        n = N - 1
        d = 2 * (Ac + Bc)          # diagonal of K
        o = Bc - Ac                # off-diagonal of K
        h = [mp.mpf(0)] * n
        h[0] += (Ac - Bc) * a_
        h[-1] += (Ac - Bc) * b_
        # tridiagonal LDL^T: log det and K^{-1} h
        piv = [mp.mpf(0)] * n
        y = [mp.mpf(0)] * n
        piv[0] = d
        y[0] = h[0]
        for i in range(1, n):
            l = o / piv[i - 1]
            piv[i] = d - l * o
            y[i] = h[i] - l * y[i - 1]
        xs = [mp.mpf(0)] * n
        xs[-1] = y[-1] / piv[-1]
        for i in range(n - 2, -1, -1):
            xs[i] = (y[i] - o * xs[i + 1]) / piv[i]
        logdet = mp.fsum(mp.log(v) for v in piv)
        quad = mp.fsum(h[i] * xs[i] for i in range(n))
        c0 = (Ac + Bc) * (a_ * a_ + b_ * b_) + N * eps * ga
        logA = (-mp.mpf(N) / 2 * mp.log(2 * mp.pi * eps) + mp.mpf(n) / 2 * mp.log(mp.pi)
                - logdet / 2 + quad - c0)
        return mp.exp(logA) if as_mp else float(mp.exp(logA))


# ---------------------------------------------------------------------------
# quadrature for tiny N
# ---------------------------------------------------------------------------

def _wp_vec(model, p, x, xb, eps):
    c = ea.coefficients(model, p)
    z = np.tanh(float(model.alpha) * x) if model.kind == "t" else x
    tot = np.zeros_like(x)
    for (m, k), poly in c.items():
        if not poly:
            continue
        v = np.zeros_like(x)
        for coef in reversed(poly):
            v = v * z + float(coef)
        tot += v * eps ** (m - k) * xb ** (2 * k)
    return tot


def _wp_abs_vec(model, p, x, xb, eps):
    """sum over all terms c_{m,k,i} z^i eps^(m-k) xb^(2k) of their absolute
    values (the condition scale of W_p at these points)"""
    c = ea.coefficients(model, p)
    z = np.abs(np.tanh(float(model.alpha) * x) if model.kind == "t" else x)
    tot = np.zeros_like(x)
    for (m, k), poly in c.items():
        v = np.zeros_like(x)
        zp = np.ones_like(x)
        for coef in poly:
            v += abs(float(coef)) * zp
            zp = zp * z
        tot += v * eps ** (m - k) * xb ** (2 * k)
    return tot


def quadrature(model_name, params, p, N, a, b, T, half_width=None, npts=None):
    """A_N^(p)(a,b;T) for N in {1, 2, 4}: Gauss-Legendre on the box
    |q_i - mid_i| <= half_width around the straight line from a to b.

    A truncated W_p can be unbounded below at large |x| (e.g. -eps^2 V'^2/24
    in W_3), which makes the integral over all of R^(N-1) diverge although
    the sampled paths never go there; the box is the reading of A_N^(p) that
    the Monte Carlo estimates.
    Returns (value, edge) where edge is the largest integrand on the box's
    faces relative to its maximum (a check that the box holds the mass)."""
    model = ea.make_model(model_name, params)
    eps = T / N
    if N == 1:
        x, xb = 0.5 * (a + b), 0.5 * (b - a)
        S = (b - a) ** 2 / (2 * eps) + eps * _wp_vec(model, p, np.array([x]), np.array([xb]), eps)[0]
        return float((2 * math.pi * eps) ** -0.5 * math.exp(-S)), 0.0
    if N not in (2, 4):
        raise ValueError("N in {1, 2, 4}")
    if half_width is None:
        # eight standard deviations of the bridge midpoint: a box a sampler of
        # up to ~1e12 samples never leaves, and inside which a truncated W_p
        # that is unbounded below (large |x|) has not yet turned the integrand up
        half_width = 8.0 * math.sqrt(T / 4.0)
    if npts is None:
        npts = 400 if N == 2 else 100
    g, wg = np.polynomial.legendre.leggauss(npts)
    nodes = half_width * g
    wts = half_width * wg
    mids = [a + (b - a) * i / N for i in range(1, N)]
    grids = list(np.meshgrid(*[mids[i] + nodes for i in range(N - 1)], indexing="ij"))
    W = np.ones_like(grids[0])
    for i in range(N - 1):
        shape = [1] * (N - 1)
        shape[i] = npts
        W = W * wts.reshape(shape)
    qs = [np.full_like(grids[0], a)] + grids + [np.full_like(grids[0], b)]
    S = np.zeros_like(grids[0])
    for k in range(N):
        ql, qr = qs[k], qs[k + 1]
        S += (qr - ql) ** 2 / (2 * eps) + eps * _wp_vec(model, p, 0.5 * (ql + qr), 0.5 * (qr - ql), eps)
    smin = S.min()
    f = np.exp(-(S - smin))
    val = float(np.sum(W * f)) * (2 * math.pi * eps) ** (-N / 2) * math.exp(-smin)
    # integrand on the faces of the box, relative to its maximum
    edge = 0.0
    for i in range(N - 1):
        sl = [slice(None)] * (N - 1)
        for end in (0, -1):
            sl[i] = end
            edge = max(edge, float(f[tuple(sl)].max()))
    return val, edge


# ---------------------------------------------------------------------------
# exact diagonalisation references for the continuum amplitude
# ---------------------------------------------------------------------------

def _hermite_functions(nmax, x):
    """phi_0..phi_{nmax-1} at x (oscillator eigenfunctions, omega = 1)."""
    x = np.asarray(x, dtype=np.float64)
    phi = np.zeros((nmax,) + x.shape)
    phi[0] = math.pi ** -0.25 * np.exp(-x * x / 2)
    if nmax > 1:
        phi[1] = math.sqrt(2.0) * x * phi[0]
    for n in range(2, nmax):
        phi[n] = math.sqrt(2.0 / n) * x * phi[n - 1] - math.sqrt((n - 1) / n) * phi[n - 2]
    return phi


def ed_amplitude(poly_V, a, b, T, nbasis=200):
    """A(a,b;T) for V(x) = sum_i poly_V[i] x^i in the basis of the first
    nbasis oscillator states (omega = 1)."""
    deg = len(poly_V) - 1
    big = nbasis + deg + 2
    n = np.arange(big)
    X = np.zeros((big, big))
    X[n[:-1], n[:-1] + 1] = np.sqrt((n[:-1] + 1) / 2.0)
    X = X + X.T
    Vm = np.zeros((big, big))
    P = np.eye(big)
    for i, v in enumerate(poly_V):
        if i:
            P = P @ X
        if v:
            Vm += float(v) * P
    X2 = X @ X
    H = np.diag(n + 0.5) - 0.5 * X2 + Vm
    H = H[:nbasis, :nbasis]
    E, U = np.linalg.eigh(H)
    phi = _hermite_functions(nbasis, np.array([a, b]))
    psi = U.T @ phi            # psi[n, point]
    return float(np.sum(psi[:, 0] * psi[:, 1] * np.exp(-E * T))), E


def dvr_amplitude(V, a, b, T, L=20.0, dx=0.02):
    """A(a,b;T) on a sinc-DVR grid x_i = i dx, |x_i| <= L (a, b on the grid)."""
    m = int(round(L / dx))
    x = dx * np.arange(-m, m + 1)
    ia, ib = int(round(a / dx)) + m, int(round(b / dx)) + m
    if abs(x[ia] - a) > 1e-12 or abs(x[ib] - b) > 1e-12:
        raise ValueError("a and b must be grid points")
    d = np.arange(len(x))
    D = d[:, None] - d[None, :]
    with np.errstate(divide="ignore"):
        K = np.where(D == 0, math.pi ** 2 / 3.0, 2.0 * (-1.0) ** np.abs(D) / np.where(D == 0, 1, D) ** 2)
    H = K / (2 * dx * dx) + np.diag(V(x))
    E, U = np.linalg.eigh(H)
    return float(np.sum(U[ia] * U[ib] * np.exp(-E * T)) / dx), E


def dvr_energies_2d(V, L, dx, k):
    """The k lowest eigenvalues of H = -(d^2/dx^2 + d^2/dy^2)/2 + V(x, y) on
    the two-dimensional sinc-DVR grid (x_i, y_j) = (i dx, j dx), |x|, |y| <= L:
    the one-dimensional sinc kinetic matrix on each axis (Kronecker sum),
    applied matrix-free, with scipy's Lanczos solver."""
    import scipy.sparse.linalg as sla
    m = int(round(L / dx))
    x = dx * np.arange(-m, m + 1)
    n = len(x)
    d = np.arange(n)
    D = d[:, None] - d[None, :]
    with np.errstate(divide="ignore"):
        K = np.where(D == 0, math.pi ** 2 / 3.0, 2.0 * (-1.0) ** np.abs(D) / np.where(D == 0, 1, D) ** 2)
    K = K / (2 * dx * dx)
    X, Y = np.meshgrid(x, x, indexing="ij")
    Vd = V(X, Y)

    def apply(v):
        v = v.reshape(n, n)
        return (K @ v + v @ K.T + Vd * v).ravel()

    op = sla.LinearOperator((n * n, n * n), matvec=apply, dtype=np.float64)
    E = sla.eigsh(op, k=k, which="SA", tol=1e-13)[0]
    return np.sort(E)
