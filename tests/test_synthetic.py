"""The input recipe (seeded synthetic requests) has the properties the path and its readings
rely on (no GPU): real H(R) with H(-R) = H(R)^T and a gap; orthonormal KS vectors per k;
LRI blocks only within r_cut, on-site blocks symmetric in (i, k); V(q) Hermitian positive
definite with V(-q) = conj V(q) and real at q = -q (the ln det stage's pairing of q with -q
and its real route at q = -q depend on these two when the inputs have them)."""
import numpy as np
import pytest

from paper_2407_19930_gb300 import synthetic as syn

CASES = {
    "cubic": syn.config_cubic,
    "mixed": syn.config_mixed,
    "cubic_3x3x1": lambda: syn.make_inputs(syn.cubic_two_atom(nao=4, naux=16, nlow=2, kmesh=(3, 3, 1)), 41,
                                           vscale=2e-3),
    "spin": syn.config_spin,
}


@pytest.fixture(scope="module", params=sorted(CASES))
def inp(request):
    return CASES[request.param]()


def test_hamiltonian_and_ks_vectors(inp):
    for R, h in inp.hr.items():
        assert np.isrealobj(h)
        mR = tuple(-x for x in R)
        assert np.array_equal(inp.hr[mR], h.T)
    for eig, occ, wfc in inp.channels():
        nocc = int(round(occ[0].sum()))
        assert eig[:, nocc].min() - eig[:, nocc - 1].max() >= 0.1 - 1e-12
        for k in range(inp.st.nk):
            c = wfc[k]
            assert np.abs(c @ c.conj().T - np.eye(inp.st.nao)).max() < 1e-12
            assert np.all(np.diff(eig[k]) >= 0)
            assert set(np.unique(occ[k])) <= {0.0, 1.0} and occ[k].sum() == nocc


def test_lri_blocks(inp):
    st = inp.st
    seen = set()
    for I, K, R, C in inp.lri:
        d = np.linalg.norm(st.pos[K] + np.array(R) @ st.lat - st.pos[I])
        assert d <= st.r_cut + 1e-9
        assert C.shape == (st.n_aux[I], st.n_ao[I], st.n_ao[K])
        if I == K and not any(R):
            assert np.array_equal(C, C.transpose(0, 2, 1))
        seen.add(I)
    assert seen == set(range(st.natoms))    # every atom has a block (the library requires one)


def test_coulomb_matrices(inp):
    st = inp.st
    mi = syn.minus_index(st.kmesh)
    for q in range(st.nk):
        v = inp.vq[q]
        assert np.array_equal(v, v.conj().T)
        assert np.linalg.eigvalsh(v).min() > 0
        assert np.array_equal(inp.vq[mi[q]], v.conj())
        if mi[q] == q:
            assert np.all(v.imag == 0.0)
