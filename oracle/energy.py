"""Oracle: RPA correlation energy (Sec. 2, Eq. for E_c^RPA with Pi = chi0 V).

Test infrastructure only (see the package docstring).

E_c = (1/2 pi) (1/N_q) sum_q int_0^inf d omega { ln det[1 - Pi(q, i omega)] + Tr Pi(q, i omega) }

with the frequency integral replaced by the quadrature sum_k W_k f(omega_k).
ln det(1 - Pi) comes from an LU factorisation of 1 - chi0 V (the paper
uses ScaLAPACK LU for this step); ``integrand_eig`` gives the same number
from the eigenvalues lambda of Pi as sum ln(1 - lambda) + lambda.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg


def integrand_lu(chi_q, vq):
    """ln det(1 - chi V) + Tr(chi V) for one (q, omega), by LU; also returns
    the phase of det (should be ~0 for Hermitian chi <= 0, V > 0)."""
    pi_ = chi_q @ vq
    n = pi_.shape[0]
    lu, piv = scipy.linalg.lu_factor(np.eye(n) - pi_)
    d = np.diag(lu)
    # each row swap flips the sign of det
    nswap = int(np.sum(piv != np.arange(n)))
    logabs = float(np.sum(np.log(np.abs(d))))
    phase = float(np.angle(np.prod(d / np.abs(d)) * (-1.0) ** nswap))
    return logabs + float(np.trace(pi_).real), phase, float(np.trace(pi_).imag)


def integrand_eig(chi_q, vq):
    """sum over eigenvalues lambda of Pi = chi V of ln(1 - lambda) + lambda."""
    lam = np.linalg.eigvals(chi_q @ vq)
    return float(np.sum(np.log(1.0 - lam) + lam).real)


def correlation_energy(chi_qw, vq, w_omega, wq=None, method="lu"):
    """E_c in Ha per cell from chi_qw [nq][nomega][N][N] and V [nq][N][N].

    Returns (E_c, per-q [nq], per-omega [nomega], integrand [nq][nomega]).
    """
    nq, nw = chi_qw.shape[:2]
    if wq is None:
        wq = np.full(nq, 1.0 / nq)
    f = np.zeros((nq, nw))
    for iq in range(nq):
        for k in range(nw):
            if method == "lu":
                f[iq, k] = integrand_lu(chi_qw[iq, k], vq[iq])[0]
            else:
                f[iq, k] = integrand_eig(chi_qw[iq, k], vq[iq])
    contrib = f * np.asarray(w_omega)[None, :] * np.asarray(wq)[:, None] / (2.0 * math.pi)
    return float(contrib.sum()), contrib.sum(axis=1), contrib.sum(axis=0), f
