"""Space-discretized evolution operator and its spectrum (oracle side).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__``.

Sec. 5 (Fig. 3) obtains energy eigenvalues and eigenfunctions by
diagonalising the matrix of short-time transition amplitudes on a grid: with
x_i = -L + i Delta, i = 0..n-1, Delta = 2L/(n-1),

    U_ij = Delta (2 pi t)^(-1/2) exp(-(x_j - x_i)^2/(2t) - t W_p(x, xb; t)),
    x = (x_i + x_j)/2,  xb = (x_j - x_i)/2,

the single-slice amplitude with the level-p effective potential (Eq.
ansatz at eps = t), a quadrature of the integral kernel of e^(-tH).  Its
eigenvalues approach e^(-t E_k), so E_k = -ln(lambda_k)/t.

Elements whose free-particle factor is below e^-40, (x_j - x_i)^2/(2t) > 40,
are zero (reading E-1): they are below double resolution relative to the
diagonal, and there xb^2 >> t, outside the short-time ordering of the
expansion, where the truncated W_p can grow faster than the Gaussian decays
(for the Poeschl-Teller potential the xb-series has a finite radius).

Written out plainly: W_p from the exact coefficients (``exact._wp_vec``) on
every pair of grid points, numpy's symmetric eigensolver for the spectrum.
"""
from __future__ import annotations

import math

import numpy as np

from . import effective_action as ea
from . import exact
from . import general_v
from . import many_body


BAND = 40.0   # largest (x_j - x_i)^2/(2t) of a nonzero element (reading E-1)


def grid(L, n):
    return np.linspace(-L, L, n)


def evolution_matrix(model_name, params, p, t, L, n):
    """U (n x n, float64) of the docstring."""
    model = ea.make_model(model_name, params)
    x = grid(L, n)
    delta = 2.0 * L / (n - 1)
    xi, xj = np.meshgrid(x, x, indexing="ij")
    xm, xb = 0.5 * (xi + xj), 0.5 * (xj - xi)
    W = exact._wp_vec(model, p, xm, xb, t)
    free = (xj - xi) ** 2 / (2.0 * t)
    band = free <= BAND
    expo = math.log(delta) - 0.5 * math.log(2.0 * math.pi * t) - free - t * np.where(band, W, 0.0)
    return np.where(band, np.exp(expo), 0.0)


def evolution_matrix_general(params, p, t, x):
    """U of the docstring for a general potential (``general_v`` parameters,
    W_p from the derivative symbols) on the equally spaced grid x, which
    need not be symmetric about 0."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    delta = (x[-1] - x[0]) / (n - 1)
    xi, xj = np.meshgrid(x, x, indexing="ij")
    free = (xj - xi) ** 2 / (2.0 * t)
    band = free <= BAND
    W = np.zeros((n, n))
    W[band] = general_v.wp(params, p, 0.5 * (xi[band] + xj[band]), 0.5 * (xj[band] - xi[band]), t)
    expo = math.log(delta) - 0.5 * math.log(2.0 * math.pi * t) - free - t * W
    return np.where(band, np.exp(expo), 0.0)


def evolution_matrix_nd(V, d, p, t, x1):
    """U of the docstring for a system of d coordinates (``many_body``
    polynomial V) on the tensor grid x1^d, points in C order: the element of
    grid points q and q' is Delta^d (2 pi t)^(-d/2) exp(-|q' - q|^2/(2t) - t
    W_p(x, xb; t)), zero where |q' - q|^2/(2t) > 40."""
    x1 = np.asarray(x1, dtype=np.float64)
    delta = (x1[-1] - x1[0]) / (x1.shape[0] - 1)
    P = np.stack([g.ravel() for g in np.meshgrid(*([x1] * d), indexing="ij")], axis=1)
    n = P.shape[0]
    free = ((P[None, :, :] - P[:, None, :]) ** 2).sum(axis=-1) / (2.0 * t)
    I, J = np.nonzero(free <= BAND)
    W = many_body.wp(V, d, p, 0.5 * (P[I] + P[J]), 0.5 * (P[J] - P[I]), t)
    U = np.zeros((n, n))
    U[I, J] = np.exp(d * math.log(delta) - 0.5 * d * math.log(2.0 * math.pi * t) - free[I, J] - t * W)
    return U


def evolution_matrix_abs(model_name, params, p, t, L, n):
    """t sum_terms |term| of W_p at every element: the size of the numbers
    -t W_p is summed from (for rounding allowances)."""
    model = ea.make_model(model_name, params)
    x = grid(L, n)
    xi, xj = np.meshgrid(x, x, indexing="ij")
    return t * exact._wp_abs_vec(model, p, 0.5 * (xi + xj), np.abs(0.5 * (xj - xi)), t)


def energies(U, t, k):
    """The k lowest E = -ln(lambda)/t from the k largest eigenvalues of U."""
    lam = np.linalg.eigvalsh(0.5 * (U + U.T))
    lam = np.sort(lam)[::-1][:k]
    return -np.log(lam) / t
