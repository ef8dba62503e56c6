"""Minimax tau / omega grids (Sec. 2: the non-uniform tau_j, omega_k grids the paper takes from
GreenX, built here from their defining property; oracle/minimax.py, csrc/minimax.cpp).

* The oracle's grids (tests/golden/minimax_grids.json, written by make_minimax_golden.py from
  oracle/ alone) equioscillate: 2n + 1 alternating extrema of equal modulus, checked on a dense
  sample in numpy, independently of the Remez solver that produced them.
* One term: a brute-force minimisation of the largest error finds the oracle's optimum.
* At equal n the minimax grids integrate the squared Lorentzians of every transition in the range
  better than the Gauss-Legendre rule.
* The library's host construction equals the oracle's (nodes and weights to 1e-12, the fitted
  transform to 1e-9), serves repeated ranges from its cache, and checks its arguments.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import grid as ogrid

omm = pytest.importorskip("oracle.minimax")   # needs mpmath

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "minimax_grids.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)


def _curves(g, x):
    """Error curves of the two fits in scaled units on x (numpy)."""
    d = g["dmin"]
    t, a = np.array(g["tau"]) * d, np.array(g["a_tau"]) * d
    o, w = np.array(g["omega"]) / d, np.array(g["w_omega"]) / d
    r_tau = 1 / x - np.exp(-np.outer(x, t)) @ a
    r_om = 1 / x - (4 * x[:, None] ** 2 / (x[:, None] ** 2 + o[None] ** 2) ** 2) @ w / math.pi
    return r_tau, r_om


def _alternation(r):
    """Alternating extrema of a sampled curve: per run of equal sign, the largest |r|."""
    out = []
    for v in r:
        if out and np.sign(v) == np.sign(out[-1]):
            if abs(v) > abs(out[-1]):
                out[-1] = v
        else:
            out.append(v)
    return np.array(out)


@pytest.mark.parametrize("case", range(7))
def test_oracle_grid_equioscillates(case):
    g = _cases()[case]
    n, R = g["n"], g["r_eff"]
    assert R == omm.range_ratio(n, g["dmin"], g["dmax"]) and R >= g["dmax"] / g["dmin"]
    u = np.linspace(0.0, 1.0, 40001)
    x = R ** (u * u)
    for r, err in zip(_curves(g, x), (g["err_tau"], g["err_omega"])):
        alt = _alternation(r)
        E = np.abs(r).max()
        assert abs(E / err - 1) < 1e-4, (E, err)
        level = alt[np.abs(alt) > (1 - 1e-4) * E]
        # at least 2n + 1 alternating extrema at the largest modulus
        assert len(level) >= 2 * n + 1, (len(level), 2 * n + 1)
        assert np.all(np.sign(level[1:]) != np.sign(level[:-1]))


def test_one_term_brute_force():
    """n = 1: minimise max |r| over (log a, log t) by Nelder-Mead on a dense sample."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    g = _cases()[0]
    assert g["n"] == 1
    R, d = g["r_eff"], g["dmin"]
    x = R ** (np.linspace(0.0, 1.0, 20001) ** 2)

    def f_tau(p):
        return np.abs(1 / x - math.exp(p[0]) * np.exp(-math.exp(p[1]) * x)).max()

    def f_om(p):
        return np.abs(1 / x - math.exp(p[0]) * 4 * x ** 2 / (x ** 2 + math.exp(2 * p[1])) ** 2 / math.pi).max()

    for f, (a_or, t_or, err) in ((f_tau, (g["a_tau"][0] * d, g["tau"][0] * d, g["err_tau"])),
                                 (f_om, (g["w_omega"][0] / d, g["omega"][0] / d, g["err_omega"]))):
        best = None
        for start in ([0.0, 0.0], [0.5, -1.0], [1.0, 1.0]):
            r = scipy_opt.minimize(f, start, method="Nelder-Mead",
                                   options=dict(xatol=1e-10, fatol=1e-14, maxiter=20000, maxfev=40000))
            if best is None or r.fun < best.fun:
                best = r
        assert abs(best.fun / err - 1) < 1e-5, (best.fun, err)
        assert abs(math.exp(best.x[0]) / a_or - 1) < 1e-3
        assert abs(math.exp(best.x[1]) / t_or - 1) < 1e-3


@pytest.mark.parametrize("case", [1, 2, 3, 4, 5])
def test_minimax_beats_gauss_legendre(case):
    """The squared-Lorentzian integral over the transition range, in the maximum norm (scaled units):
    the minimax weights do better than the Gauss-Legendre rule with the same number of points."""
    g = _cases()[case]
    n, dmin, dmax = g["n"], g["dmin"], g["dmax"]
    gl = ogrid.make_grid(n, dmin, dmax)
    D = dmin * np.exp(np.linspace(0.0, math.log(dmax / dmin), 20001))

    def qerr(om, w):
        q = (w[None] * 4 * D[:, None] ** 2 / (D[:, None] ** 2 + om[None] ** 2) ** 2).sum(axis=1)
        return np.abs(q / math.pi - 1 / D).max() * dmin

    e_mm = qerr(np.array(g["omega"]), np.array(g["w_omega"]))
    e_gl = qerr(gl["omega"], gl["w_omega"])
    assert e_mm <= g["err_omega"] * (1 + 1e-6)
    assert e_mm < e_gl, (e_mm, e_gl)


@pytest.mark.parametrize("case", range(7))
def test_library_grid_equals_oracle(case):
    from paper_2407_19930_gb300 import librpa_gpu as L
    g = _cases()[case]
    n, dmin, dmax = g["n"], g["dmin"], g["dmax"]
    a = L.librpa_gpu_build_grid_minimax(n, dmin, dmax)
    assert a["r_eff"] == g["r_eff"]
    for key in ("tau", "omega", "w_omega"):
        ref = np.array(g[key])
        assert np.all(np.abs(a[key] - ref) <= 1e-12 * np.abs(ref)), key
    assert abs(a["err_tau"] / g["err_tau"] - 1) < 1e-6
    assert abs(a["err_omega"] / g["err_omega"] - 1) < 1e-6
    # the transform fitted on [dmin, R_b dmin], compared through the fitted function
    hi = g["r_eff"] * dmin
    gam = ogrid.fit_gamma(np.array(g["tau"]), np.array(g["omega"]), dmin, hi)
    D = dmin * np.exp(np.linspace(0.0, math.log(hi / dmin), 777))
    fa = np.exp(-np.outer(D, a["tau"])) @ a["gamma"].T
    fb = np.exp(-np.outer(D, np.array(g["tau"]))) @ gam.T
    assert np.abs(fa - fb).max() <= 1e-9 * np.abs(fb).max()


def test_library_grid_cache_and_arguments():
    import time
    from paper_2407_19930_gb300 import librpa_gpu as L
    g = _cases()[3]
    a = L.librpa_gpu_build_grid_minimax(g["n"], g["dmin"], g["dmax"])
    t0 = time.time()
    # the same 1/8-octave range, other dmin and dmax: scaled copy from the cache
    b = L.librpa_gpu_build_grid_minimax(g["n"], 2 * g["dmin"], 2 * g["dmax"] * 0.999)
    assert time.time() - t0 < 0.05
    assert np.array_equal(b["tau"] * 2, a["tau"]) and np.array_equal(b["omega"], 2 * a["omega"])
    for n, dmin, dmax in [(0, 1.0, 2.0), (21, 1.0, 2.0), (8, 0.0, 1.0), (8, 2.0, 1.0), (8, -1.0, 1.0),
                          (8, 1.0, float("inf"))]:
        with pytest.raises(L.LibrpaError) as e:
            L.librpa_gpu_build_grid_minimax(n, dmin, dmax)
        assert e.value.code == L.LIBRPA_E_ARG
