"""Writes ``oracle_energies.json``: E_c (Ha per cell) with its per-q and per-omega parts, computed
by the CPU oracle alone (``oracle.pipeline.rpa_energy``, matrix-form route of chi0) on seeded synthetic
requests, without and with Green's-function screening.  Run from the repository root:

    python tests/golden/make_golden.py

The stored values pin the oracle against later changes of its arithmetic: a change that moves
one of them must say in its commit message which passage of the paper, or which reading of it,
justifies the new value.
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import grid as ogrid, pipeline  # noqa: E402
from paper_2407_19930_gb300 import synthetic as syn  # noqa: E402


def molecule():
    ang = math.radians(104.5) / 2
    o = np.array([20.0, 20.0, 20.0])
    pos = np.array([o, o + 1.81 * np.array([math.sin(ang), 0.0, -math.cos(ang)]),
                    o + 1.81 * np.array([-math.sin(ang), 0.0, -math.cos(ang)])])
    st = syn.Structure(lat=np.eye(3) * 40.0, pos=pos, n_ao=np.array([5, 5, 5]), n_aux=np.array([30, 30, 30]),
                       n_low=np.array([2, 1, 1]), kmesh=(1, 1, 1))
    return syn.make_inputs(st, 17, vscale=2e-3)


CASES = {
    "tiny": (syn.config_tiny, 8, 0.0),
    "cubic": (syn.config_cubic, 8, 0.0),
    "cubic_screened_1e-2": (syn.config_cubic, 8, 1e-2),
    "cubic_spin": (syn.config_spin, 8, 0.0),
    "molecule": (molecule, 16, 0.0),
}


def compute(name):
    make, ntau, theta = CASES[name]
    inp = make()
    grid = ogrid.make_grid(ntau, *inp.delta_range)
    out = pipeline.rpa_energy(inp, grid, screen=theta)
    return {"ntau": ntau, "screen": theta, "ec": float(out["ec"]), "ec_q": [float(x) for x in out["ec_q"]],
            "ec_w": [float(x) for x in out["ec_w"]]}


def main():
    res = {"generator": "tests/golden/make_golden.py (oracle only)", "cases": {n: compute(n) for n in CASES}}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_energies.json"), "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
