"""Green's-function block screening (Sec. 5's threshold; the block rule is the one stated with
librpa_gpu_set_screening): the GPU path against the oracle run on the screened G.

The screened G, chi0(R, tau), chi0(q, i omega) and E_c must match the oracle at the FP64
tolerances of the unscreened parity tests.  The keep/drop decision compares FP64 block maxima
with the threshold on both sides; G differs between them in the last bits, so each case first
checks on the oracle's G that no block maximum lies within 1e-9 (relative) of the threshold.
"""
import numpy as np
import pytest

from paper_2407_19930_gb300 import librpa_gpu as L
from oracle import grid as ogrid, pipeline, screen

from test_gpu_parity import CONFIGS, MEV, TOL_CHI, TOL_EC, TOL_G, TOL_MIXED_MEV_PER_ATOM, _opts, _rel, _run

pytestmark = pytest.mark.gpu

CASES = [("cubic", 1e-2), ("cubic", 1e-3), ("mixed", 3e-3), ("cubic_3x1x2", 3e-3), ("cubic_3x3x1", 1e-2),
         ("cubic_spin", 1e-3), ("molecule", 1e-2)]


def _grid(name, inp):
    return ogrid.make_grid(8 if name != "mixed" else 10, *inp.delta_range)


def _canonical_points(inp, ntau):
    """(R, tau) points the library contracts per spin channel: R with flat index <= that of -R."""
    n1, n2, n3 = inp.st.kmesh
    nr = 0
    for a in range(n1):
        for b in range(n2):
            for c in range(n3):
                i = (a * n2 + b) * n3 + c
                j = (((n1 - a) % n1) * n2 + (n2 - b) % n2) * n3 + (n3 - c) % n3
                nr += i <= j
    return nr * ntau


def _block_margin(inp, grid, theta):
    bm = np.concatenate([screen.block_max(g, inp.st.n_ao).ravel() for pr in pipeline.greens(inp, grid) for g in pr])
    return np.abs(bm - theta).min() / theta, int((bm >= theta).sum()), bm.size


@pytest.fixture(scope="module", params=CASES, ids=[f"{n}-{t:g}" for n, t in CASES])
def scase(request):
    name, theta = request.param
    inp = CONFIGS[name]()
    grid = _grid(name, inp)
    margin, kept, total = _block_margin(inp, grid, theta)
    assert margin > 1e-9, "threshold too close to a block maximum for a two-sided decision"
    ref = pipeline.rpa_energy(inp, grid, screen=theta)
    gpu = _run(inp, grid, screening=theta)
    return name, theta, inp, grid, ref, gpu, kept, total


def test_screened_green(scase):
    name, theta, inp, grid, ref, gpu, kept, total = scase
    go, gv = (ref["go"], ref["gv"]) if inp.st.nspins == 1 else (ref["go"][0], ref["gv"][0])
    assert _rel(gpu["go"], go) < TOL_G and _rel(gpu["gv"], gv) < TOL_G
    # the same blocks dropped: exact zeros in the same places
    assert np.array_equal(gpu["go"] == 0.0, go == 0.0) and np.array_equal(gpu["gv"] == 0.0, gv == 0.0)
    s = gpu["stats"]
    assert s["n_blocks_total"] == total and s["n_blocks_kept"] == kept


def test_screened_chi0_and_energy(scase):
    name, theta, inp, grid, ref, gpu, kept, total = scase
    assert _rel(gpu["chi_tau"], ref["chi_tau"]) < TOL_CHI
    assert _rel(gpu["chi_qw"], ref["chi_qw"]) < TOL_CHI
    assert abs(gpu["ec"] - ref["ec"]) < TOL_EC
    assert np.abs(gpu["ec_w"] - ref["ec_w"]).max() < TOL_EC
    s = gpu["stats"]
    ntau = len(grid["tau"])
    assert s["n_points_chi0"] + s["n_points_skipped"] == inp.st.nspins * _canonical_points(inp, ntau)


def test_skipped_points_are_the_zero_ones():
    """At 1e-2 the cubic cell's largest tau has no kept block: its points are not contracted,
    chi0 there is exactly zero, and the algorithmic flop count drops by their share."""
    inp = CONFIGS["cubic"]()
    grid = _grid("cubic", inp)
    full = _run(inp, grid)
    scr = _run(inp, grid, screening=1e-2)
    assert scr["stats"]["n_points_skipped"] > 0 and full["stats"]["n_points_skipped"] == 0
    assert np.all(scr["chi_tau"][-1] == 0.0)
    per_point = full["stats"]["flop_chi0"] / full["stats"]["n_points_chi0"]
    assert scr["stats"]["flop_chi0"] <= per_point * scr["stats"]["n_points_chi0"] * (1 + 1e-12)


def test_everything_dropped_gives_zero_energy():
    """A threshold above every block maximum: no point is contracted, chi0 = 0, E_c = 0."""
    inp = CONFIGS["cubic"]()
    grid = _grid("cubic", inp)
    gpu = _run(inp, grid, screening=10.0)
    assert gpu["stats"]["n_points_chi0"] == 0 and gpu["stats"]["n_blocks_kept"] == 0
    assert np.all(gpu["chi_tau"] == 0.0) and gpu["ec"] == 0.0


@pytest.mark.parametrize("precision", [L.LIBRPA_FP64_TC, L.LIBRPA_SPLIT])
def test_screening_in_tensor_core_modes(precision):
    """The tensor-core routes contract the same selected points; FP64_TC keeps the FP64 bar,
    SPLIT its 0.1 meV/atom bar, against the screened oracle."""
    inp = CONFIGS["cubic_3x3x1"]()
    grid = _grid("cubic_3x3x1", inp)
    ref = pipeline.rpa_energy(inp, grid, screen=1e-2)
    gpu = _run(inp, grid, opts=_opts(precision), screening=1e-2)
    assert gpu["stats"]["n_points_skipped"] > 0
    if precision == L.LIBRPA_FP64_TC:
        assert abs(gpu["ec"] - ref["ec"]) < TOL_EC
    else:
        assert abs(gpu["ec"] - ref["ec"]) * MEV / inp.st.natoms < TOL_MIXED_MEV_PER_ATOM


def test_screened_handle_in_a_batch():
    """A screened handle takes its own path in a batched pass and gives the energy it gives
    alone; the unscreened handles of the pass are unaffected."""
    names = ["cubic", "cubic", "tiny"]
    thetas = [1e-2, 0.0, 0.0]
    hs, b = [], None
    try:
        for n, t in zip(names, thetas):
            inp = CONFIGS[n]()
            h = L.librpa_gpu_create(_opts())
            L.set_inputs(h, inp, _grid(n, inp))
            L.librpa_gpu_set_screening(h, t)
            hs.append(h)
        b = L.librpa_gpu_batch_create(hs)
        ec = L.librpa_gpu_batch_run(b)
    finally:
        L.librpa_gpu_batch_destroy(b)
        for h in hs:
            L.librpa_gpu_destroy(h)
    for (n, t), e in zip(zip(names, thetas), ec):
        inp = CONFIGS[n]()
        alone = _run(inp, _grid(n, inp), screening=t)["ec"]
        assert abs(e - alone) <= 1e-12 * abs(alone), (n, t, e, alone)
    assert abs(ec[0] - ec[1]) > 1e-4


def test_set_screening_arguments():
    h = L.librpa_gpu_create(_opts())
    try:
        for bad in (-1e-3, float("nan"), float("inf")):
            with pytest.raises(L.LibrpaError) as e:
                L.librpa_gpu_set_screening(h, bad)
            assert e.value.code == L.LIBRPA_E_ARG
        L.librpa_gpu_set_screening(h, 0.0)
    finally:
        L.librpa_gpu_destroy(h)


@pytest.mark.parametrize("precision", [L.LIBRPA_FP64, L.LIBRPA_FP64_TC])
def test_block_sparse_work_follows_the_kept_blocks(precision):
    """Inside a contracted point the GEMM tiles sum only the K chunks that meet kept G blocks and the
    O blocks without a kept contribution are zeros: the algorithmic work falls below that of the
    contracted points done densely, while the result stays the oracle's on the screened G."""
    inp = CONFIGS["cubic_3x3x1"]()
    grid = _grid("cubic_3x3x1", inp)
    theta = 1e-2   # about a quarter of the G blocks kept
    ref = pipeline.rpa_energy(inp, grid, screen=theta)
    full = _run(inp, grid, opts=_opts(precision))
    scr = _run(inp, grid, opts=_opts(precision), screening=theta)
    per_point = full["stats"]["flop_chi0"] / full["stats"]["n_points_chi0"]
    dense_on_points = per_point * scr["stats"]["n_points_chi0"]
    frac = scr["stats"]["flop_chi0"] / dense_on_points
    print("block-sparse chi0 work: %.3f of the contracted points done densely (%s)" % (frac, precision))
    assert frac < 0.9
    assert _rel(scr["chi_tau"], ref["chi_tau"]) < TOL_CHI
    assert abs(scr["ec"] - ref["ec"]) < TOL_EC
