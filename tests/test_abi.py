"""Host-side checks of the C-ABI library (no GPU needed).

* the library builds and exports every entry point include/librpa_gpu.h declares;
* the host grid construction (librpa_gpu_build_grid) agrees with the oracle's;
* argument checking of the host-only entry points.
"""
import os
import re

import numpy as np
import pytest

from paper_2407_19930_gb300 import librpa_gpu as L
from oracle import grid as ogrid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "librpa_gpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(librpa_gpu_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = L.load()
    names = declared_symbols()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps each of them under the same name
    for n in names:
        assert n in L._SIGS, n


def test_header_compiles_as_c():
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write('#include "librpa_gpu.h"\nint main(void){librpa_gpu_opts o; '
                           'librpa_gpu_default_opts(&o); return o.n_tau == 16 ? 0 : 1;}\n')
        r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", "-I", os.path.join(ROOT, "include"),
                            c, "-o", os.path.join(d, "t.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("n,dmin,dmax", [(1, 1.0, 1.0), (8, 0.7, 1.3), (16, 0.727, 1.302), (16, 0.5, 5.0),
                                         (24, 0.2, 3.0), (32, 0.1, 10.0)])
def test_grid_matches_oracle(n, dmin, dmax):
    """Nodes and weights are closed-form (Gauss-Legendre) and agree to rounding;
    the least-squares transform is compared through the fitted function, which is
    unique even where truncated singular directions make the coefficients differ."""
    a = L.librpa_gpu_build_grid(n, dmin, dmax)
    b = ogrid.make_grid(n, dmin, dmax)
    # elementwise relative: the (1 - t)^-2 of the mapping amplifies node rounding near t = 1
    for key in ("tau", "omega", "w_omega"):
        assert np.all(np.abs(a[key] - b[key]) <= 1e-12 * np.abs(b[key])), key
    d = np.exp(np.linspace(np.log(dmin), np.log(dmax), 777)) if dmax > dmin else np.array([dmin])
    fa = np.exp(-np.outer(d, a["tau"])) @ a["gamma"].T
    fb = np.exp(-np.outer(d, b["tau"])) @ b["gamma"].T
    assert np.abs(fa - fb).max() <= 1e-9 * np.abs(fb).max()
    # and the library's fit meets the oracle's error bound for the exact transform
    exact = 2 * d[:, None] / (d[:, None] ** 2 + a["omega"][None] ** 2)
    eps_b = ogrid.transform_error(b, dmin, dmax) if dmax > dmin else np.abs(fb - exact).max(axis=0)
    assert np.all(np.abs(fa - exact).max(axis=0) <= eps_b * 1.01 + 1e-12 * np.abs(exact).max())


def test_build_grid_rejects_bad_arguments():
    for n, dmin, dmax in [(0, 1.0, 2.0), (65, 1.0, 2.0), (8, 0.0, 1.0), (8, 2.0, 1.0), (8, -1.0, 1.0)]:
        with pytest.raises(L.LibrpaError) as e:
            L.librpa_gpu_build_grid(n, dmin, dmax)
        assert e.value.code == L.LIBRPA_E_ARG
