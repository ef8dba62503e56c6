"""Oracle: the whole path for one request, step by step (Sec. 2).

Test infrastructure only (see the package docstring).

G (Eq. green_mat) -> chi0(R, tau) (the four-term matrix form, or the plain definition)
-> chi0(R, i omega) (cosine transform) -> chi0(q, i omega) (Fourier
transform) -> E_c (ln det by LU, quadrature over omega, mean over q).  With a screening
threshold the Green's functions pass through ``screen.screen_blocks`` first
(Sec. 5, Green's-function screening).
"""
from __future__ import annotations

import numpy as np

from . import energy, freq, green, screen as _screen
from .chi0_matrix import chi0_matrix_form
from .chi0_definition import chi0_definition


def spin_factor(nspins: int) -> float:
    """Spin factor s of chi0 per channel: 2 for a spin-unpolarised calculation (one channel
    standing for both spins), 1 per channel for a spin-polarised one (chi0 = sum over spins)."""
    if nspins == 1:
        return 2.0
    if nspins == 2:
        return 1.0
    raise ValueError("nspins must be 1 or 2")


def greens(inp, grid, screen=0.0):
    """[(G^occ, G^vir)] per spin channel; blocks below the threshold ``screen`` dropped
    when it is > 0."""
    st = inp.st
    gs = [green.green(st.kmesh, inp.kfrac, e, o, w, inp.efermi, grid["tau"]) for e, o, w in inp.channels()]
    if screen > 0:
        gs = [(_screen.screen_blocks(go, st.n_ao, screen)[0], _screen.screen_blocks(gv, st.n_ao, screen)[0])
              for go, gv in gs]
    return gs


def chi0_tau(inp, grid, route="matrix", go=None, gv=None):
    """chi0(R, tau) as [ntau][nR][N][N]: the contraction of each spin channel with its own
    Green's functions, summed.  go / gv: one channel's arrays, or [nspins] of them."""
    st = inp.st
    if go is None:
        gs = greens(inp, grid)
    else:
        gs = [(go, gv)] if st.nspins == 1 else list(zip(go, gv))
    ntau = len(grid["tau"])
    pts = [(iR, it) for it in range(ntau) for iR in range(st.nk)]
    s = spin_factor(st.nspins)
    c = 0.0
    for g_o, g_v in gs:
        if route == "matrix":
            c = c + chi0_matrix_form(st, inp.lri, g_o, g_v, pts, spin=s)
        elif route == "definition":
            c = c + chi0_definition(st, inp.lri, g_o, g_v, pts, spin=s)
        else:
            raise ValueError(route)
    return c.reshape(ntau, st.nk, st.naux, st.naux)


def chi0_q_omega(inp, grid, chi_tau):
    """chi0(q, i omega) as [nq][nomega][N][N] complex."""
    st = inp.st
    chi_w = freq.tau_to_omega(chi_tau, grid["gamma"])            # [nw][nR][N][N]
    out = np.empty((st.nk, chi_w.shape[0], st.naux, st.naux), dtype=np.complex128)
    for k in range(chi_w.shape[0]):
        out[:, k] = freq.r_to_q(chi_w[k], st.kmesh, inp.kfrac)
    return out


def rpa_energy(inp, grid, route="matrix", vq=None, screen=0.0):
    """Dict with G ([nspins] leading axis when nspins = 2; screened when ``screen`` > 0),
    chi0 in every representation and E_c (Ha per cell)."""
    st = inp.st
    gs = greens(inp, grid, screen)
    if st.nspins == 1:
        go, gv = gs[0]
    else:
        go, gv = np.stack([g[0] for g in gs]), np.stack([g[1] for g in gs])
    ct = chi0_tau(inp, grid, route=route, go=go, gv=gv)
    cq = chi0_q_omega(inp, grid, ct)
    v = inp.vq if vq is None else vq
    ec, ec_q, ec_w, f = energy.correlation_energy(cq, v, grid["w_omega"])
    return dict(go=go, gv=gv, chi_tau=ct, chi_qw=cq, ec=ec, ec_q=ec_q, ec_w=ec_w, integrand=f)
