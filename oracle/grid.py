"""Oracle: tau / omega grids and the tau -> i omega weights (Sec. 2, cosine transform).

Test infrastructure only (see the package docstring).

The paper takes non-uniform tau_j, omega_k grids from GreenX and fits the
cosine-transform coefficients gamma_jk by an L2 minimisation.  GreenX's
tables are not available here, so the grid is built as follows (the same
construction the library states for its own host code):

* omega_k, W_k: an N-point Gauss-Legendre rule on t in (-1, 1) mapped to
  (0, inf) by omega = omega0 (1 + t) / (1 - t), omega0 = sqrt(dmin * dmax),
  W_k = omega0 * 2 w_k / (1 - t_k)^2;
* tau_j: the same rule mapped with tau0 = 1 / sqrt(dmin * dmax);
* Gamma_kj (= gamma_jk cos(omega_k tau_j)): for every k, the least-squares
  fit of the exact transform 2 D / (D^2 + omega_k^2) by sum_j Gamma_kj
  exp(-D tau_j) in relative error, on M log-spaced D in [dmin, dmax],
  solved by SVD with singular values below ``rcond`` * s_max dropped.

The fitted function sum_j Gamma_kj exp(-D tau_j) is unique; the
coefficients are unique only when no singular value is dropped.
"""
from __future__ import annotations

import math

import numpy as np

M_SAMPLES = 1000
RCOND = 1e-12


def gauss_legendre(n):
    """Nodes and weights of the n-point Gauss-Legendre rule on (-1, 1)."""
    return np.polynomial.legendre.leggauss(n)


def make_grid(n, dmin, dmax, m=M_SAMPLES, rcond=RCOND):
    """Returns dict(tau[n], omega[n], w_omega[n], gamma[n][n]) in Ha units."""
    if not (0 < dmin <= dmax):
        raise ValueError("need 0 < dmin <= dmax")
    t, w = gauss_legendre(n)
    omega0 = math.sqrt(dmin * dmax)
    omega = omega0 * (1 + t) / (1 - t)
    w_omega = omega0 * 2 * w / (1 - t) ** 2
    tau0 = 1.0 / omega0
    tau = tau0 * (1 + t) / (1 - t)
    return dict(tau=tau, omega=omega, w_omega=w_omega, gamma=fit_gamma(tau, omega, dmin, dmax, m, rcond))


def fit_gamma(tau, omega, dmin, dmax, m=M_SAMPLES, rcond=RCOND):
    """Gamma_kj: for every k, the least-squares fit of 2 D / (D^2 + omega_k^2) by sum_j Gamma_kj
    exp(-D tau_j) in relative error on m log-spaced D in [dmin, dmax] (SVD, singular values below
    rcond * s_max dropped)."""
    n = len(tau)
    d = dmin * np.exp(np.linspace(0.0, math.log(dmax / dmin), m)) if dmax > dmin else np.full(m, dmin)
    E = np.exp(-np.outer(d, tau))
    gamma = np.empty((len(omega), n))
    for k in range(len(omega)):
        f = 2 * d / (d * d + omega[k] ** 2)
        A = E / f[:, None]
        U, s, Vt = np.linalg.svd(A, full_matrices=False)
        keep = s > rcond * s[0]
        gamma[k] = Vt[keep].T @ ((U[:, keep].T @ np.ones(m)) / s[keep])
    return gamma


def transform_error(grid, dmin, dmax, m=4000):
    """eps_k = max over D in [dmin, dmax] of |sum_j Gamma_kj e^{-D tau_j} - 2D/(D^2+omega_k^2)|."""
    d = dmin * np.exp(np.linspace(0.0, math.log(dmax / dmin), m)) if dmax > dmin else np.full(m, dmin)
    E = np.exp(-np.outer(d, grid["tau"]))
    fit = E @ grid["gamma"].T                                  # [m][k]
    exact = 2 * d[:, None] / (d[:, None] ** 2 + grid["omega"][None] ** 2)
    return np.abs(fit - exact).max(axis=0)


def quadrature_error(grid, dmin, dmax, m=4000):
    """max over D of |sum_k W_k 4D^2/(D^2+omega_k^2)^2 - pi/D| * D / pi (relative)."""
    d = dmin * np.exp(np.linspace(0.0, math.log(dmax / dmin), m)) if dmax > dmin else np.full(m, dmin)
    q = (grid["w_omega"][None] * 4 * d[:, None] ** 2
         / (d[:, None] ** 2 + grid["omega"][None] ** 2) ** 2).sum(axis=1)
    return float(np.abs(q * d / math.pi - 1.0).max())
