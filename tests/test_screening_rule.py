"""The point-selection rule of the screened contraction, checked against the oracle (no GPU).

The library leaves out the (R, tau) points where one of G^occ, G^vir has no kept block among
the blocks the contraction reads there (N-step: (L, K) at R1 - R - R2 for (L, R2) in N[V] and
(K, R1) in the union of the neighbour lists; X-step: (I, L) at R + R2; O assembly: (U, V) at R
and (V, K) at R1 - R), because every term of chi0 pairs a G^occ with a G^vir factor.  Here the
same rule, restated in Python, must only leave out points where the oracle's chi0 (matrix form) on the
screened G gives exactly zero, and must leave some out.  With the on-site block C[V, V, 0] in
N[V] the O-assembly sets are inside the X- and N-step sets; the rule keeps them for neighbour
lists without it.  Dropping the X- or the N-step set from the rule fails the single-block test.
"""
import numpy as np
import pytest

from oracle import grid as ogrid, pipeline, screen
from oracle.chi0_matrix import chi0_matrix_form
from paper_2407_19930_gb300 import synthetic as syn


def _needed_any(mask, nb, uni, kmesh, R):
    """Whether any block the contraction reads at lattice vector R is kept (mask [nR][I][J])."""
    n1, n2, n3 = kmesh

    def idx(v):
        return ((v[0] % n1) * n2 + v[1] % n2) * n3 + v[2] % n3

    if mask[idx(R)].any():                                   # (U, V) at R
        return True
    for K, R1 in uni:                                        # (V, K) at R1 - R, any V
        if mask[idx((R1[0] - R[0], R1[1] - R[1], R1[2] - R[2]))][:, K].any():
            return True
    for V in range(len(nb)):
        for L, R2 in nb[V]:
            if mask[idx((R[0] + R2[0], R[1] + R2[1], R[2] + R2[2]))][:, L].any():   # (I, L) at R + R2
                return True
            for K, R1 in uni:                                # (L, K) at R1 - R - R2
                if mask[idx((R1[0] - R[0] - R2[0], R1[1] - R[1] - R2[1], R1[2] - R[2] - R2[2]))][L, K]:
                    return True
    return False


@pytest.mark.parametrize("name,theta", [("cubic", 1e-2), ("cubic_3x3x1", 1e-2), ("mixed", 3e-3)])
def test_left_out_points_have_zero_chi0(name, theta):
    inp = {"cubic": syn.config_cubic, "mixed": syn.config_mixed,
           "cubic_3x3x1": lambda: syn.make_inputs(syn.cubic_two_atom(nao=4, naux=16, nlow=2, kmesh=(3, 3, 1)),
                                                  41, vscale=2e-3)}[name]()
    st = inp.st
    grid = ogrid.make_grid(8 if name != "mixed" else 10, *inp.delta_range)
    go, gv = pipeline.greens(inp, grid, screen=theta)[0]
    ko = screen.block_max(go, st.n_ao) > 0.0       # kept blocks (dropped ones are exactly zero)
    kv = screen.block_max(gv, st.n_ao) > 0.0
    nb = [[] for _ in range(st.natoms)]
    for I, K, R, C in inp.lri:
        nb[I].append((K, tuple(int(x) for x in R)))
    uni = sorted({e for lst in nb for e in lst})
    n1, n2, n3 = st.kmesh
    cells = [(a, b, c) for a in range(n1) for b in range(n2) for c in range(n3)]
    ntau = len(grid["tau"])
    pts = [(iR, it) for it in range(ntau) for iR in range(st.nk)]
    chi = chi0_matrix_form(st, inp.lri, go, gv, pts).reshape(ntau, st.nk, st.naux, st.naux)
    left_out = 0
    for it in range(ntau):
        for iR, R in enumerate(cells):
            active = _needed_any(ko[it], nb, uni, st.kmesh, R) and _needed_any(kv[it], nb, uni, st.kmesh, R)
            if not active:
                left_out += 1
                assert np.all(chi[it, iR] == 0.0), (it, iR)
    assert left_out > 0


@pytest.mark.parametrize("g_single", ["occ", "vir"])
def test_every_block_that_reaches_chi0_is_read(g_single):
    """Completeness of the rule, one block at a time: with a single atom-pair block of one Green's
    function kept (the other Green's function whole), every point where the oracle's chi0 gives a
    non-zero chi0 must be one the rule keeps.  Run over every block of a 2-atom cell on a 9x1x1
    mesh, long enough that the N-step blocks (near -R) and the X-step blocks (near +R) are the
    only route for some block and point."""
    inp = syn.make_inputs(syn.cubic_two_atom(nao=3, naux=8, nlow=1, kmesh=(9, 1, 1)), 43, vscale=2e-3)
    st = inp.st
    grid = ogrid.make_grid(4, *inp.delta_range)
    go, gv = pipeline.greens(inp, grid)[0]
    go, gv = go[:1], gv[:1]                          # one tau
    ao = np.concatenate([[0], np.cumsum(st.n_ao)])
    nb = [[] for _ in range(st.natoms)]
    for I, K, R, C in inp.lri:
        nb[I].append((K, tuple(int(x) for x in R)))
    uni = sorted({e for lst in nb for e in lst})
    n1, n2, n3 = st.kmesh
    cells = [(a, b, c) for a in range(n1) for b in range(n2) for c in range(n3)]
    pts = [(iR, 0) for iR in range(st.nk)]
    full = np.ones((st.nk, st.natoms, st.natoms), dtype=bool)
    reached = 0
    for iRb in range(st.nk):
        for I in range(st.natoms):
            for J in range(st.natoms):
                single = np.zeros_like(go)
                src = go if g_single == "occ" else gv
                single[0, iRb, ao[I]:ao[I + 1], ao[J]:ao[J + 1]] = src[0, iRb, ao[I]:ao[I + 1], ao[J]:ao[J + 1]]
                mask = np.zeros((st.nk, st.natoms, st.natoms), dtype=bool)
                mask[iRb, I, J] = True
                g_o, g_v = (single, gv) if g_single == "occ" else (go, single)
                chi = chi0_matrix_form(st, inp.lri, g_o, g_v, pts).reshape(st.nk, st.naux, st.naux)
                for iR, R in enumerate(cells):
                    if np.any(chi[iR] != 0.0):
                        reached += 1
                        assert _needed_any(mask, nb, uni, st.kmesh, R), (iRb, I, J, iR)
                        assert _needed_any(full, nb, uni, st.kmesh, R)
    assert reached > 0
