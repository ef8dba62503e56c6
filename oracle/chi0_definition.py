"""Oracle: chi0_{mu nu}(R, tau) as the plain definition (Eqs. LRI, chi0_NAOs, chi0_ABFs).

Test infrastructure only (see the package docstring).

Eq. LRI expands the product of NAO i (atom I, cell R1) and NAO k (atom K,
cell R3) over ABFs on *both* atoms.  Written as one pair coefficient of the
ABF mu in cell R_mu:

    Chat^{mu(R_mu)}_{i(R1), k(R3)} = [mu on I, R_mu = R1] C[I, K, R3 - R1]_{mu i k}
                                    + [mu on K, R_mu = R3] C[K, I, R1 - R3]_{mu k i}

(the second term uses the product's symmetry phi_i phi_k = phi_k phi_i to
store every coefficient with mu on its first atom).  For an on-site pair
(I = K, R1 = R3) both terms are taken, as Eq. LRI writes them.

Inserting Eq. green_func into chi0 = -i G(i tau) G(-i tau) gives Eq.
chi0_NAOs; expanding both NAO products with Eq. LRI and reading off the
coefficient of P_mu(0) P_nu(R) (Eq. chi0_ABFs) gives, in the real
convention of the package docstring,

    chi0_{mu nu}(R, tau) = -s sum Chat^{mu(0)}_{a b} G^vir_{a c} Chat^{nu(R)}_{c d} G^occ_{d b}

with a = i(R1), b = k(R3), c = j(R2), d = l(R4), G^vir_{a c} =
G^vir_{ij}(R2 - R1, tau) and G^occ_{d b} = G^occ_{lk}(R3 - R4, tau).

This module evaluates that sum with dense matrices over the finite set of
(atom, cell) sites on which some Chat^{mu(0)} is non-zero.  It needs
memory ~ N_aux * (sites * NAO)^2 and is meant for small cells.
"""
from __future__ import annotations

import numpy as np

from .green import bvk_index


class Neighbourhood:
    """Sites (atom, cell) touched by the pair coefficients of home-cell ABFs."""

    def __init__(self, st, lri):
        self.st = st
        nat = st.natoms
        self.aux_off = np.concatenate([[0], np.cumsum(st.n_aux)]).astype(int)
        sites = {(U, (0, 0, 0)) for U in range(nat)}
        for I, K, R, _ in lri:
            sites.add((K, tuple(R)))
            sites.add((I, (0, 0, 0)))
        self.sites = sorted(sites, key=lambda s: (s[1], s[0]))
        self.site_off = {}
        off = 0
        for s in self.sites:
            self.site_off[s] = off
            off += int(st.n_ao[s[0]])
        self.dim = off
        # flat description of every row: (atom, cell, orbital)
        self.row_atom = np.empty(self.dim, dtype=int)
        self.row_cell = np.empty((self.dim, 3), dtype=int)
        self.row_orb = np.empty(self.dim, dtype=int)
        ao_off = np.concatenate([[0], np.cumsum(st.n_ao)]).astype(int)
        self.row_ao = np.empty(self.dim, dtype=int)   # global NAO index in the cell
        for s in self.sites:
            o = self.site_off[s]
            n = int(st.n_ao[s[0]])
            self.row_atom[o:o + n] = s[0]
            self.row_cell[o:o + n] = s[1]
            self.row_orb[o:o + n] = np.arange(n)
            self.row_ao[o:o + n] = ao_off[s[0]] + np.arange(n)
        self.lri = lri

    def chat(self, mus=None):
        """Dense pair coefficients Chat^{mu(0)} [len(mus)][dim][dim] (Eq. LRI)."""
        st = self.st
        if mus is None:
            mus = range(int(self.aux_off[-1]))
        mus = list(mus)
        index = {m: t for t, m in enumerate(mus)}
        out = np.zeros((len(mus), self.dim, self.dim))
        home = (0, 0, 0)
        for I, K, R, C in self.lri:
            a0 = int(self.aux_off[I])
            ri = self.site_off[(I, home)]
            ck = self.site_off[(K, tuple(R))]
            ni, nk = int(st.n_ao[I]), int(st.n_ao[K])
            # mu on I: rows i(0) on the home site of I, columns k(R) on site (K, R)
            # mu on I as the *second* atom of the pair (K, R) -- (I, 0):
            #   Chat^{mu(0)}_{k(R), i(0)} = C[I, K, R]_{mu i k}
            for m in range(C.shape[0]):
                t = index.get(a0 + m)
                if t is None:
                    continue
                out[t, ri:ri + ni, ck:ck + nk] += C[m]
                out[t, ck:ck + nk, ri:ri + ni] += C[m].T
        return out

    def green_block(self, G, R, kmesh, left_shift, right_shift):
        """Dense [dim][dim] matrix G_{a c} = G_{ij}(cell_c + right_shift - cell_a - left_shift)."""
        ca = self.row_cell + np.asarray(left_shift)
        cc = self.row_cell + np.asarray(right_shift)
        out = np.empty((self.dim, self.dim))
        # group by (site_a, site_c) to index the BvK arrays blockwise
        for sa in self.sites:
            oa = self.site_off[sa]
            na = int(self.st.n_ao[sa[0]])
            ia = self.row_ao[oa:oa + na]
            for sc in self.sites:
                oc = self.site_off[sc]
                nc = int(self.st.n_ao[sc[0]])
                ic = self.row_ao[oc:oc + nc]
                d = np.asarray(sc[1]) + np.asarray(right_shift) - np.asarray(sa[1]) - np.asarray(left_shift)
                iR = bvk_index(d, kmesh)
                out[oa:oa + na, oc:oc + nc] = G[iR][np.ix_(ia, ic)]
        return out


def chi0_definition(st, lri, go, gv, points, spin=2.0, mu_chunk=64):
    """chi0(R, tau) [len(points)][N_aux][N_aux] for the (iR, itau) pairs given.

    ``go``/``gv``: [ntau][nR][nao][nao] from ``oracle.green``.
    """
    nb = Neighbourhood(st, lri)
    naux = int(nb.aux_off[-1])
    kmesh = st.kmesh
    n1, n2, n3 = kmesh
    out = np.zeros((len(points), naux, naux))
    for p, (iR, it) in enumerate(points):
        R = np.array([iR // (n2 * n3), (iR // n3) % n2, iR % n3])
        # G^vir_{a c}: a = i(R1) in the home neighbourhood, c = j(R + R2'') in the one around R
        gva = nb.green_block(gv[it], R, kmesh, left_shift=(0, 0, 0), right_shift=R)
        # G^occ_{d b}: d = l(R + R4''), b = k(R3)
        goa = nb.green_block(go[it], R, kmesh, left_shift=R, right_shift=(0, 0, 0))
        for m0 in range(0, naux, mu_chunk):
            cm = nb.chat(range(m0, min(naux, m0 + mu_chunk)))
            for n0 in range(0, naux, mu_chunk):
                cn = cm if n0 == m0 else nb.chat(range(n0, min(naux, n0 + mu_chunk)))
                # F^nu = G^vir Chat^nu G^occ, chi_{mu nu} = -s sum_ab Chat^mu_ab F^nu_ab
                F = np.matmul(np.matmul(gva[None], cn), goa[None])
                out[p, m0:m0 + cm.shape[0], n0:n0 + cn.shape[0]] = -spin * np.einsum(
                    'mab,nab->mn', cm, F, optimize=True)
    return out
