"""Per-q weights of the E_c sum (librpa_gpu_set_q_weights; Appendix B passes irreducible k
points with weights): the library against the oracle's weighted energy, q of zero weight left
out, and the weights moved onto q <= -q reproducing the 1/N_q result."""
import numpy as np
import pytest

from paper_2407_19930_gb300 import librpa_gpu as L
from paper_2407_19930_gb300 import synthetic as syn
from oracle import energy, grid as ogrid, pipeline

from test_gpu_parity import CONFIGS, TOL_EC, _opts

pytestmark = pytest.mark.gpu


def _energy(inp, grid, w=None, precision=L.LIBRPA_FP64):
    h = L.librpa_gpu_create(_opts(precision))
    try:
        L.set_inputs(h, inp, grid)
        if w is not None:
            L.librpa_gpu_set_q_weights(h, w)
        L.librpa_gpu_chi0(h)
        ec, ecq, ecw = L.librpa_gpu_ec(h, inp.st.nk, len(grid["omega"]))
        return ec, ecq, L.librpa_gpu_get_stats(h)
    finally:
        L.librpa_gpu_destroy(h)


@pytest.mark.parametrize("name", ["cubic", "cubic_3x3x1", "cubic_3x1x2"])
def test_weighted_energy_matches_oracle(name):
    inp = CONFIGS[name]()
    st = inp.st
    grid = ogrid.make_grid(8, *inp.delta_range)
    ref = pipeline.rpa_energy(inp, grid)
    rng = np.random.default_rng(5)
    w = rng.uniform(0.2, 1.0, st.nk)
    w[rng.permutation(st.nk)[: st.nk // 3]] = 0.0     # some q left out
    w /= w.sum()
    want, want_q, _, _ = energy.correlation_energy(ref["chi_qw"], inp.vq, grid["w_omega"], wq=w)
    for prec in (L.LIBRPA_FP64, L.LIBRPA_FP64_TC):
        ec, ecq, _ = _energy(inp, grid, w, prec)
        assert abs(ec - want) < TOL_EC
        assert np.abs(ecq - want_q).max() < TOL_EC
        assert np.all(ecq[w == 0.0] == 0.0)


def test_folded_weights_compute_fewer_q():
    """Each pair's weight on q <= -q and 0 on its partner: the same E_c as 1/N_q, with the q of
    zero weight not computed when V(-q) = conj V(q) does not already pair them (here it does,
    so the ln det work is the same), and uniform weights given explicitly change nothing."""
    inp = CONFIGS["cubic_3x3x1"]()
    st = inp.st
    grid = ogrid.make_grid(8, *inp.delta_range)
    base, _, s0 = _energy(inp, grid)
    mi = syn.minus_index(st.kmesh)
    w = np.zeros(st.nk)
    for q in range(st.nk):
        w[min(q, mi[q])] += 1.0 / st.nk
    folded, fq, s1 = _energy(inp, grid, w)
    assert abs(folded - base) < 1e-12 * abs(base)
    assert np.all(fq[w == 0.0] == 0.0)
    uni, _, _ = _energy(inp, grid, np.full(st.nk, 1.0 / st.nk))
    assert abs(uni - base) < 1e-13 * abs(base)
    # one q only: the ln det stage factorises only that q (and its V)
    w1 = np.zeros(st.nk)
    w1[0] = 1.0
    one, oq, s2 = _energy(inp, grid, w1)
    assert s2["flop_ec"] < s0["flop_ec"] and oq[0] == one and np.all(oq[1:] == 0.0)


def test_set_q_weights_arguments():
    inp = CONFIGS["cubic"]()
    h = L.librpa_gpu_create(_opts())
    try:
        with pytest.raises(L.LibrpaError) as e:
            L.librpa_gpu_set_q_weights(h, np.ones(inp.st.nk))
        assert e.value.code == L.LIBRPA_E_STATE
        L.set_inputs(h, inp)
        for bad in (np.zeros(inp.st.nk), np.full(inp.st.nk, -0.1), np.full(inp.st.nk, np.nan)):
            with pytest.raises(L.LibrpaError) as e:
                L.librpa_gpu_set_q_weights(h, bad)
            assert e.value.code == L.LIBRPA_E_ARG
        L.librpa_gpu_set_q_weights(h, None)
    finally:
        L.librpa_gpu_destroy(h)
