"""Oracle: tau -> i omega cosine transform and R -> q Fourier transform (Sec. 2).

Test infrastructure only (see the package docstring).

* chi0(R, i omega_k) = sum_j Gamma_kj chi0(R, tau_j), with the real
  Gamma_kj = gamma_jk cos(omega_k tau_j) (the paper's -i factors absorbed,
  see the package docstring);
* chi0(q, i omega) = sum_{R in BvK} e^{+i q.R} chi0(R, i omega).
"""
from __future__ import annotations

import numpy as np

from .green import bvk_vectors


def tau_to_omega(chi_tau, gamma):
    """chi_tau [ntau][...] -> [nomega][...] with Gamma [nomega][ntau]."""
    chi_tau = np.asarray(chi_tau)
    flat = chi_tau.reshape(chi_tau.shape[0], -1)
    return (np.asarray(gamma) @ flat).reshape((gamma.shape[0],) + chi_tau.shape[1:])


def r_to_q(chi_r, kmesh, qfrac, iqs=None):
    """chi_r [nR][N][N] (real) -> [len(iqs)][N][N] complex."""
    Rv = bvk_vectors(kmesh)
    qfrac = np.asarray(qfrac)
    if iqs is None:
        iqs = range(len(qfrac))
    out = []
    for iq in iqs:
        ph = np.exp(2j * np.pi * (Rv @ qfrac[iq]))
        out.append(np.tensordot(ph, chi_r, axes=(0, 0)))
    return np.array(out)
