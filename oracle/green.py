"""Oracle: real-space imaginary-time Green's functions (Eq. green_mat).

Test infrastructure only (see the package docstring).

G^occ_{ij}(R, tau) = (1/N_k) sum_{k,n} f_nk c_in(k) c*_jn(k) e^{-i k.R} e^{-(mu - e_nk) tau}
G^vir_{ij}(R, tau) = (1/N_k) sum_{k,n} (1 - f_nk) c_in(k) c*_jn(k) e^{-i k.R} e^{-(e_nk - mu) tau}

These are the paper's two branches with the prefactors -i and +i taken out
(tau >= 0 in both; the occupied branch is the paper's tau <= 0 branch
evaluated at -tau).  For time-reversal-symmetric inputs (real H(R), a
k-mesh closed under k -> -k) both are real; ``green`` returns the real
part and, on request, the largest imaginary part as a check.
"""
from __future__ import annotations

import numpy as np


def bvk_index(R, kmesh) -> int:
    """Flat BvK index of an integer lattice vector (folded into the mesh)."""
    n1, n2, n3 = kmesh
    return ((int(R[0]) % n1) * n2 + int(R[1]) % n2) * n3 + int(R[2]) % n3


def bvk_vectors(kmesh) -> np.ndarray:
    n1, n2, n3 = kmesh
    return np.array([(a, b, c) for a in range(n1) for b in range(n2) for c in range(n3)],
                    dtype=np.float64)


def green(kmesh, kfrac, eig, occ, wfc, efermi, tau, return_imag=False):
    """G^occ, G^vir as arrays [ntau][nR][nao][nao] (FP64).

    ``wfc[k, n, i]`` = c_in(k); ``occ`` in [0, 1] per spin-orbital.
    """
    kfrac = np.asarray(kfrac, dtype=np.float64)
    nk, nb, nao = wfc.shape
    Rv = bvk_vectors(kmesh)
    nR = len(Rv)
    tau = np.asarray(tau, dtype=np.float64)
    go = np.zeros((len(tau), nR, nao, nao), dtype=np.complex128)
    gv = np.zeros_like(go)
    # phase[k, R] = exp(-2 pi i k.R)
    phase = np.exp(-2j * np.pi * (kfrac @ Rv.T))
    for ik in range(nk):
        c = wfc[ik].T                      # c[i, n]
        e = eig[ik]
        f = occ[ik]
        for it, t in enumerate(tau):
            wo = f * np.exp(-(efermi - e) * t)
            wv = (1.0 - f) * np.exp(-(e - efermi) * t)
            po = (c * wo) @ c.conj().T     # sum_n c_in w_n c*_jn
            pv = (c * wv) @ c.conj().T
            for iR in range(nR):
                go[it, iR] += phase[ik, iR] * po
                gv[it, iR] += phase[ik, iR] * pv
    go /= nk
    gv /= nk
    if return_imag:
        imag = max(np.abs(go.imag).max(), np.abs(gv.imag).max())
        return go.real.copy(), gv.real.copy(), float(imag)
    return go.real.copy(), gv.real.copy()
