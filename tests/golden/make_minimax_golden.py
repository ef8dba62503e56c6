"""Writes ``minimax_grids.json``: minimax tau / omega grids computed by the CPU oracle alone
(``oracle.minimax.make_minimax_grid``, Remez exchange in mpmath) for a few (n, dmin, dmax),
from one term up to the 16 points of the benchmark workload, ranges at and above the floor
R_floor(n).  Run from the repository root (a few minutes):

    python tests/golden/make_minimax_golden.py

The stored grids pin the oracle against later changes of its arithmetic and are what the
library's grids are compared with; a change that moves one of them must say in its commit
message which property of the minimax grids (Sec. 2, the non-uniform grids the paper takes
from GreenX) justifies the new values.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import minimax  # noqa: E402

CASES = [(1, 0.1, 1.0), (4, 0.2, 6.0), (8, 0.1, 4.0), (10, 0.3, 12.0), (12, 0.05, 500.0), (16, 0.1, 30.0),
         (16, 0.7, 1.3)]


def main():
    out = []
    for n, dmin, dmax in CASES:
        g = minimax.make_minimax_grid(n, dmin, dmax)
        out.append(dict(n=n, dmin=dmin, dmax=dmax, r_eff=g["r_eff"], tau=[float(v) for v in g["tau"]],
                        omega=[float(v) for v in g["omega"]], w_omega=[float(v) for v in g["w_omega"]],
                        a_tau=[float(v) for v in g["a_tau"]],
                        err_tau=g["err_tau"], err_omega=g["err_omega"]))
        print(n, dmin, dmax, "R_b %.4g" % g["r_eff"], "errors %.3e %.3e" % (g["err_tau"], g["err_omega"]), flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "minimax_grids.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
