"""Oracle: Green's-function block screening (Sec. 5 runs its production
calculations with "Green's function-based screening" at a threshold of 1e-3;
Sec. 2 ties the O(N) limit to the spatial decay of G).  Test infrastructure
only (see the package docstring).

The paper states the threshold but no formula.  Reading taken here: for every
tau, every lattice vector R of the BvK cell and every atom pair (I, J), the NAO
block G^occ_{IJ}(R, tau) is dropped (replaced by zeros) when the largest
absolute value of its elements is below the threshold theta, and kept
unchanged otherwise; G^vir is screened the same way on its own blocks.  The
threshold is absolute (G is dimensionless).  theta = 0 keeps every block.
chi0 then runs on the screened Green's functions unchanged: a term whose
G block was dropped contributes nothing, so the cost follows the number of
kept blocks, and lattice vectors R whose G blocks are all dropped drop out of
chi0 altogether (the R range limited by the decay of G).
"""
from __future__ import annotations

import numpy as np


def block_max(G, n_ao):
    """Largest |element| of every atom-pair block: [ntau][nR][nat][nat] from
    G [ntau][nR][nao][nao]."""
    off = np.concatenate([[0], np.cumsum(n_ao)]).astype(int)
    nat = len(n_ao)
    out = np.zeros(G.shape[:2] + (nat, nat))
    for I in range(nat):
        for J in range(nat):
            blk = G[:, :, off[I]:off[I + 1], off[J]:off[J + 1]]
            out[:, :, I, J] = np.abs(blk).max(axis=(2, 3))
    return out


def screen_blocks(G, n_ao, theta):
    """(screened copy of G, keep mask [ntau][nR][nat][nat] of bool).

    A block is kept when its largest |element| is >= theta."""
    if theta < 0:
        raise ValueError("theta must be >= 0")
    off = np.concatenate([[0], np.cumsum(n_ao)]).astype(int)
    keep = block_max(G, n_ao) >= theta
    out = np.array(G, dtype=np.float64, copy=True)
    nat = len(n_ao)
    for I in range(nat):
        for J in range(nat):
            drop = ~keep[:, :, I, J]
            out[drop, off[I]:off[I + 1], off[J]:off[J + 1]] = 0.0
    return out, keep
