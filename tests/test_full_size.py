"""The benchmark's workload shape at its full auxiliary size, end to end against the oracle.

The graphene slab (35 atoms: 32 C + a water-shaped molecule; n_ao 431, N_aux 2010) with the
k-mesh cut to 1x1x1 and 2x2x1 and 8 tau/omega points, so that the oracle (the matrix form of chi0 in
plain C, LU of 1 - chi0 V) finishes in about a minute.  Every chi0(q, i omega) element, E_c and its
per-q and per-omega parts are compared: the N_aux = 2010 matrices run the ln det stage's 32-panel
tile loops, its workspace chunking and the chi0 contraction's full atom-pair tables, which the
small parity cases do not reach.

Tolerances: FP64 as everywhere (chi0 1e-10 normwise per matrix, E_c 1e-8 Ha); the FP64-accurate
tensor-core mode with chi0(q, i omega) against the bound propagated through the transform
(N_R 1e-10 sum_j |Gamma_kj| max|chi0(tau_j)|), E_c 1e-8 Ha; the mixed mode (3 digit planes)
within 0.1 meV/atom.
"""
import numpy as np
import pytest

from paper_2407_19930_gb300 import librpa_gpu as L
from paper_2407_19930_gb300 import synthetic as syn
from oracle import grid as ogrid, pipeline

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_CHI = 1e-10
TOL_EC = 1e-8
MEV = 27211.386245988
NTAU = 8


def _run(inp, grid, precision):
    o = L.librpa_gpu_default_opts()
    o.precision = precision
    h = L.librpa_gpu_create(o)
    st = inp.st
    nw = len(grid["omega"])
    try:
        L.set_inputs(h, inp, grid)
        chi = L.librpa_gpu_chi0(h, out=(st.nk, nw, st.naux))
        ec, ecq, ecw = L.librpa_gpu_ec(h, st.nk, nw)
        ct = np.array([[L.librpa_gpu_get_chi0_tau(h, it, iR, st.naux) for iR in range(st.nk)]
                       for it in range(len(grid["tau"]))])
    finally:
        L.librpa_gpu_destroy(h)
    return dict(chi_qw=chi, chi_tau=ct, ec=ec, ec_q=ecq, ec_w=ecw)


@pytest.fixture(scope="module", params=[(1, 1, 1), (2, 2, 1)], ids=["gamma", "2x2x1"])
def full(request):
    inp = syn.config_graphene(kmesh=request.param)
    grid = ogrid.make_grid(NTAU, *inp.delta_range)
    ref = pipeline.rpa_energy(inp, grid)
    return inp, grid, ref


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_fp64_full_aux(full):
    inp, grid, ref = full
    st = inp.st
    assert st.naux == 2010 and st.natoms == 35
    gpu = _run(inp, grid, L.LIBRPA_FP64)
    for it in range(NTAU):
        for iR in range(st.nk):
            assert _rel(gpu["chi_tau"][it, iR], ref["chi_tau"][it, iR]) < TOL_CHI, (it, iR)
    for iq in range(st.nk):
        for k in range(NTAU):
            assert _rel(gpu["chi_qw"][iq, k], ref["chi_qw"][iq, k]) < TOL_CHI, (iq, k)
    assert abs(gpu["ec"] - ref["ec"]) < TOL_EC, (gpu["ec"], ref["ec"])
    assert np.abs(gpu["ec_q"] - ref["ec_q"]).max() < TOL_EC
    assert np.abs(gpu["ec_w"] - ref["ec_w"]).max() < TOL_EC


def test_fp64_tc_full_aux(full):
    inp, grid, ref = full
    st = inp.st
    gpu = _run(inp, grid, L.LIBRPA_FP64_TC)
    assert _rel(gpu["chi_tau"], ref["chi_tau"]) < TOL_CHI
    mx = np.abs(ref["chi_tau"]).reshape(NTAU, -1).max(axis=1)
    for k in range(NTAU):
        bound = st.nk * TOL_CHI * np.sum(np.abs(grid["gamma"][k]) * mx)
        for iq in range(st.nk):
            assert np.abs(gpu["chi_qw"][iq, k] - ref["chi_qw"][iq, k]).max() <= bound, (iq, k)
    assert abs(gpu["ec"] - ref["ec"]) < TOL_EC, (gpu["ec"], ref["ec"])
    assert np.abs(gpu["ec_q"] - ref["ec_q"]).max() < TOL_EC
    assert np.abs(gpu["ec_w"] - ref["ec_w"]).max() < TOL_EC


@pytest.mark.parametrize("precision", [L.LIBRPA_SPLIT, L.LIBRPA_SPLIT_FAST])
def test_split_full_aux(full, precision):
    inp, grid, ref = full
    gpu = _run(inp, grid, precision)
    err = abs(gpu["ec"] - ref["ec"]) * MEV / inp.st.natoms
    print("mixed mode %d at N_aux 2010 (%s k): E_c error %.2e meV/atom" % (
        precision, "x".join(map(str, inp.st.kmesh)), err))
    assert err < 0.1, err
