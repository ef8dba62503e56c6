"""Oracle: chi0_{mu nu}(q) by a sum over KS states (an independent route).

Test infrastructure only (see the package docstring).

Insert Eq. green_mat into the definition of ``chi0_definition`` and sum
the phases over the BvK cells.  With the pair densities

    rho^mu(k, n; k', m) = sum_{i(R1), kap(R3)} Chat^{mu(0)}_{i(R1), kap(R3)}
                          c_im(k') e^{+i k'.R1} c*_kap n(k) e^{-i k.R3}

the R -> q transform of Sec. 2 (chi0(q) = sum_R e^{iq.R} chi0(R)) picks
k' = k + q and gives

    chi0_{mu nu}(q, tau) = -(s/N_k) sum_k sum_{n,m} f_nk (1 - f_m,k+q)
                            e^{-Delta tau} rho^mu rho^nu*,   Delta = e_m,k+q - e_nk.

This is exact in tau.  Replacing e^{-Delta tau} by its cosine transform
2 Delta / (Delta^2 + omega^2) (the continuous form of the tau -> i omega
step) gives the exact chi0(q, i omega) that a finite minimax grid
approximates.
"""
from __future__ import annotations

import numpy as np

from .chi0_definition import Neighbourhood


def _kplusq(kmesh, ik, iq):
    n1, n2, n3 = kmesh

    def split(i):
        return i // (n2 * n3), (i // n3) % n2, i % n3
    a, b, c = split(ik)
    d, e, f = split(iq)
    return (((a + d) % n1) * n2 + (b + e) % n2) * n3 + (c + f) % n3


def pair_densities(nb: Neighbourhood, kfrac, wfc, ik, ikq, chat):
    """rho^mu(k, n; k', m) as [mu][n][m] for k = ik, k' = ikq."""
    # Phi(k)[a, n] = c_{i(a) n}(k) e^{+2 pi i k.R(a)}
    ph_k = np.exp(2j * np.pi * (nb.row_cell @ kfrac[ik]))
    ph_kq = np.exp(2j * np.pi * (nb.row_cell @ kfrac[ikq]))
    phi_k = wfc[ik].T[nb.row_ao] * ph_k[:, None]       # [dim][nb]
    phi_kq = wfc[ikq].T[nb.row_ao] * ph_kq[:, None]
    # rho[mu, n, m] = sum_ab Chat_ab Phi(k')_am conj(Phi(k))_bn
    t = np.einsum('uab,bn->uan', chat, phi_k.conj(), optimize=True)
    return np.einsum('uan,am->unm', t, phi_kq, optimize=True)


def chi0_sos(st, lri, kfrac, eig, occ, wfc, iq, tau=None, omega=None, spin=2.0):
    """chi0(q) for one q index: returns [len(tau)][N][N] (tau form, kernel
    e^{-Delta tau}) or [len(omega)][N][N] (frequency form, kernel
    2 Delta/(Delta^2 + omega^2)).  Complex Hermitian."""
    nb = Neighbourhood(st, lri)
    chat = nb.chat()
    naux = chat.shape[0]
    kmesh = st.kmesh
    nk = st.nk
    if (tau is None) == (omega is None):
        raise ValueError("give exactly one of tau, omega")
    pts = np.asarray(tau if tau is not None else omega, dtype=np.float64)
    out = np.zeros((len(pts), naux, naux), dtype=np.complex128)
    for ik in range(nk):
        ikq = _kplusq(kmesh, ik, iq)
        rho = pair_densities(nb, kfrac, wfc, ik, ikq, chat)      # [mu][n][m]
        w = occ[ik][:, None] * (1.0 - occ[ikq][None, :])         # [n][m]
        delta = eig[ikq][None, :] - eig[ik][:, None]
        mask = w > 0
        r = rho[:, mask]                                         # [mu][pairs]
        d = delta[mask]
        ww = w[mask]
        for p, x in enumerate(pts):
            if tau is not None:
                ker = np.exp(-d * x)
            else:
                ker = 2.0 * d / (d * d + x * x)
            out[p] += (r * (ww * ker)) @ r.conj().T
    out *= -spin / nk
    return out
