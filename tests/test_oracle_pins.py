"""Pins of the CPU oracle against mathematics (no GPU).

Each test ties the oracle to something other than itself: an independent
route to the same number, a closed form, an invariant or a textbook special
case.  Together they catch a dropped term, a wrong sign, phase or index,
a transposed operand or a wrong normalisation anywhere in the oracle.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2407_19930_gb300 import synthetic as syn
from oracle import energy, freq, green, grid as ogrid, pipeline, screen
from oracle.chi0_matrix import chi0_matrix_form
from oracle.chi0_definition import chi0_definition
from oracle.chi0_sos import chi0_sos


@pytest.fixture(scope="module")
def tiny():
    return syn.config_tiny()


@pytest.fixture(scope="module")
def cubic():
    return syn.config_cubic()


def _green(inp, tau):
    st = inp.st
    return green.green(st.kmesh, inp.kfrac, inp.eig, inp.occ, inp.wfc, inp.efermi, tau)


# ---------------------------------------------------------------- P0: G


def test_green_completeness_and_trace(cubic):
    """sum over all bands at tau = 0: G^occ(R,0) + G^vir(R,0) = delta_R0 I (S = I);
    Tr G^occ(0, 0) = number of occupied bands."""
    st = cubic.st
    go, gv, im = green.green(st.kmesh, cubic.kfrac, cubic.eig, cubic.occ, cubic.wfc,
                             cubic.efermi, [0.0], return_imag=True)
    assert im < 1e-13
    tot = go[0] + gv[0]
    for iR in range(st.nk):
        ref = np.eye(st.nao) if iR == 0 else np.zeros((st.nao, st.nao))
        assert np.abs(tot[iR] - ref).max() < 1e-12
    assert abs(np.trace(go[0, 0]) - st.nocc) < 1e-12


def test_green_matches_bvk_supercell(cubic):
    """G(R, tau) equals the block of the Green's function of the BvK supercell
    Hamiltonian diagonalised at Gamma: pins exp(-i k.R) and 1/N_k."""
    st = cubic.st
    n1, n2, n3 = st.kmesh
    cells = [(a, b, c) for a in range(n1) for b in range(n2) for c in range(n3)]
    nao, nR = st.nao, len(cells)
    hs = np.zeros((nR * nao, nR * nao))
    for ia, Ra in enumerate(cells):
        for ib, Rb in enumerate(cells):
            for R, h in cubic.hr.items():
                d = np.array(R) - (np.array(Rb) - np.array(Ra))
                if d[0] % n1 == 0 and d[1] % n2 == 0 and d[2] % n3 == 0:
                    hs[ia * nao:(ia + 1) * nao, ib * nao:(ib + 1) * nao] += h
    e, v = np.linalg.eigh(0.5 * (hs + hs.T))
    nocc = st.nocc * nR
    tau = np.array([0.0, 0.7, 2.5])
    go, gv = _green(cubic, tau)
    mu = cubic.efermi
    for it, t in enumerate(tau):
        wo = np.where(np.arange(len(e)) < nocc, np.exp(-(mu - e) * t), 0.0)
        wv = np.where(np.arange(len(e)) >= nocc, np.exp(-(e - mu) * t), 0.0)
        gso = (v * wo) @ v.T
        gsv = (v * wv) @ v.T
        for iR in range(nR):
            blk_o = gso[0:nao, iR * nao:(iR + 1) * nao]
            blk_v = gsv[0:nao, iR * nao:(iR + 1) * nao]
            assert np.abs(blk_o - go[it, iR]).max() < 1e-12
            assert np.abs(blk_v - gv[it, iR]).max() < 1e-12


# ---------------------------------------------------------------- P1: exact in tau


@pytest.mark.parametrize("name", ["tiny", "cubic"])
def test_three_routes_agree_in_tau(name, request):
    """Four-term matrix form == plain definition (R space) and == sum over states (q space),
    an algebraic identity with no grid error."""
    inp = request.getfixturevalue(name)
    st = inp.st
    tau = np.array([0.25, 1.3])
    go, gv = _green(inp, tau)
    pts = [(iR, it) for it in range(len(tau)) for iR in range(st.nk)]
    ca = chi0_matrix_form(st, inp.lri, go, gv, pts)
    cd = chi0_definition(st, inp.lri, go, gv, pts)
    scale = np.abs(ca).max()
    assert scale > 1.0
    assert np.abs(ca - cd).max() < 1e-13 * scale
    ca = ca.reshape(len(tau), st.nk, st.naux, st.naux)
    for iq in range(st.nk):
        s = chi0_sos(st, inp.lri, inp.kfrac, inp.eig, inp.occ, inp.wfc, iq, tau=tau)
        for it in range(len(tau)):
            q = freq.r_to_q(ca[it], st.kmesh, inp.kfrac, [iq])[0]
            assert np.abs(q - s[it]).max() < 1e-13 * scale


# ---------------------------------------------------------------- P2..P5: frequency domain


@pytest.fixture(scope="module")
def cubic_run(cubic):
    dmin, dmax = cubic.delta_range
    g = ogrid.make_grid(8, dmin, dmax)
    out = pipeline.rpa_energy(cubic, g)
    return g, out


def test_frequency_form_within_grid_error(cubic, cubic_run):
    """Space-time chi0(q, i omega_k) vs the exact sum over states with the
    Lorentzian kernel: |diff_{mu nu}| <= (s/N_k) sum f(1-f) |rho^mu||rho^nu| eps_k."""
    g, out = cubic_run
    st = cubic.st
    dmin, dmax = cubic.delta_range
    eps = ogrid.transform_error(g, dmin, dmax)
    # |rho| bound: recompute the diagonal of the tau = 0 response (kernel 1)
    for iq in (0, 3):
        exact = chi0_sos(st, cubic.lri, cubic.kfrac, cubic.eig, cubic.occ, cubic.wfc, iq,
                         omega=g["omega"])
        bound0 = -chi0_sos(st, cubic.lri, cubic.kfrac, cubic.eig, cubic.occ, cubic.wfc, iq,
                           tau=[0.0])[0]
        dia = np.sqrt(np.abs(np.diag(bound0)).real)
        for k in range(len(g["omega"])):
            diff = np.abs(out["chi_qw"][iq, k] - exact[k])
            bound = eps[k] * np.outer(dia, dia) * 1.0000001 + 1e-12
            assert np.all(diff <= bound)
    # and the grid is good enough for the bound to mean something
    assert eps.max() < 1e-5


def test_hermitian_and_time_reversal(cubic, cubic_run):
    g, out = cubic_run
    st = cubic.st
    mi = syn.minus_index(st.kmesh)
    cq = out["chi_qw"]
    scale = np.abs(cq).max()
    for iq in range(st.nk):
        for k in range(cq.shape[1]):
            assert np.abs(cq[iq, k] - cq[iq, k].conj().T).max() < 1e-13 * scale
            assert np.abs(cq[mi[iq], k] - cq[iq, k].conj()).max() < 1e-13 * scale


def test_negative_semidefinite_and_energy_sign(cubic, cubic_run):
    """chi0(q, i omega) <= 0 when the grid kernel sum_j Gamma_kj e^{-D tau_j}
    is >= 0 on every transition energy; every integrand and E_c are <= 0."""
    g, out = cubic_run
    st = cubic.st
    nocc = st.nocc
    d = (cubic.eig[:, None, nocc:][..., None] - cubic.eig[None, :, :nocc][..., None, :]).ravel()
    ker = np.exp(-np.outer(d, g["tau"])) @ g["gamma"].T
    assert ker.min() >= 0
    for iq in range(st.nk):
        for k in range(len(g["omega"])):
            ev = np.linalg.eigvalsh(out["chi_qw"][iq, k])
            assert ev.max() <= 1e-12 * np.abs(ev).max()
    assert np.all(out["integrand"] <= 0)
    assert out["ec"] < 0


def test_lu_equals_eigenvalues(cubic, cubic_run):
    """ln det(1 - Pi) + Tr Pi by LU == sum ln(1 - lambda) + lambda over eigenvalues of Pi."""
    g, out = cubic_run
    for iq in (0, 5):
        for k in (0, 4):
            a, phase, _ = energy.integrand_lu(out["chi_qw"][iq, k], cubic.vq[iq])
            b = energy.integrand_eig(out["chi_qw"][iq, k], cubic.vq[iq])
            assert abs(phase) < 1e-10
            assert abs(a - b) < 1e-10 * max(1.0, abs(a))


def test_quadratic_limit(cubic, cubic_run):
    """E_c(lambda V) / lambda^2 -> -(1/4 pi) sum_q w_q sum_k W_k Tr[(chi0 V)^2]."""
    g, out = cubic_run
    cq = out["chi_qw"]
    nq = cq.shape[0]
    lim = 0.0
    for iq in range(nq):
        for k in range(cq.shape[1]):
            p = cq[iq, k] @ cubic.vq[iq]
            lim += g["w_omega"][k] * np.trace(p @ p).real / nq
    lim *= -1.0 / (4 * math.pi)
    vals = []
    for lam in (1e-2, 1e-3):
        ec = energy.correlation_energy(cq, cubic.vq * lam, g["w_omega"])[0]
        vals.append(ec / lam ** 2)
    # O(lambda) correction: Richardson-extrapolate the two values to lambda -> 0
    rich = (vals[1] * 1e-2 - vals[0] * 1e-3) / (1e-2 - 1e-3)
    assert abs(vals[1] - lim) < 2e-2 * abs(lim)
    assert abs(rich - lim) < 1e-5 * abs(lim)


# ---------------------------------------------------------------- P8: two-level closed form


def _two_level(delta, c01, v, n_tau=16):
    """One atom, one k point, two NAOs (one occupied, one virtual), one ABF."""
    st = syn.Structure(lat=np.eye(3) * 50.0, pos=np.zeros((1, 3)), n_ao=np.array([2]),
                       n_aux=np.array([1]), n_low=np.array([1]), kmesh=(1, 1, 1))
    eig = np.array([[-delta / 2, delta / 2]])
    occ = np.array([[1.0, 0.0]])
    wfc = np.eye(2, dtype=np.complex128)[None]
    C = np.array([[[0.0, c01], [c01, 0.0]]])
    inp = syn.Inputs(st=st, kfrac=np.zeros((1, 3)), eig=eig, occ=occ, wfc=wfc, efermi=0.0,
                     lri=[(0, 0, (0, 0, 0), C)], vq=np.array([[[v + 0j]]]))
    g = ogrid.make_grid(n_tau, delta, delta)
    return inp, g


@pytest.mark.parametrize("delta,c01,v", [(0.6, 0.7, 1.3), (1.1, 0.2, 0.5), (0.3, 1.5, 2.0)])
def test_two_level_closed_form(delta, c01, v):
    """E_c = (1/2)(sqrt(D^2 + 2aD) - D - a), a = s rho^2 V, rho = 2 c01 (both
    on-site terms of Eq. LRI), from int_0^inf ln(1 + c/(D^2+w^2)) dw = pi(sqrt(D^2+c) - D)."""
    inp, g = _two_level(delta, c01, v)
    out = pipeline.rpa_energy(inp, g)
    a = 2.0 * (2 * c01) ** 2 * v
    exact = 0.5 * (math.sqrt(delta ** 2 + 2 * a * delta) - delta - a)
    assert out["ec"] < 0
    assert abs(out["ec"] - exact) < 1e-6 * abs(exact)


# ---------------------------------------------------------------- P9: grid


def test_grid_rules():
    """The Gauss-Legendre rule integrates Legendre polynomials exactly; the
    mapped omega rule reproduces int_0^inf 4D^2/(D^2+w^2)^2 dw = pi/D; the
    fitted transform reproduces the exact cosine transform of e^{-D tau}."""
    t, w = ogrid.gauss_legendre(12)
    for deg in range(0, 23):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(w * t ** deg) - exact) < 1e-14
    for n, dmin, dmax, tol_q, tol_t in ((8, 0.7, 1.3, 1e-4, 1e-6), (16, 0.7, 1.3, 1e-9, 1e-8),
                                        (16, 0.5, 5.0, 1e-7, 1e-5)):
        g = ogrid.make_grid(n, dmin, dmax)
        assert ogrid.quadrature_error(g, dmin, dmax) < tol_q
        eps = ogrid.transform_error(g, dmin, dmax)
        scale = 2.0 / dmin
        assert eps.max() < tol_t * scale
        assert np.all(g["w_omega"] > 0) and np.all(np.diff(g["tau"]) > 0)


# ---------------------------------------------------------------- P10: invariances


def _permute(inp, perm):
    """Relabel atoms: new atom a is old atom perm[a]."""
    st = inp.st
    inv = np.argsort(perm)
    ao_off = np.concatenate([[0], np.cumsum(st.n_ao)])
    aux_off = np.concatenate([[0], np.cumsum(st.n_aux)])
    st2 = syn.Structure(lat=st.lat, pos=st.pos[perm], n_ao=st.n_ao[perm], n_aux=st.n_aux[perm],
                        n_low=st.n_low[perm], kmesh=st.kmesh)
    orb = np.concatenate([np.arange(ao_off[p], ao_off[p + 1]) for p in perm])
    aux = np.concatenate([np.arange(aux_off[p], aux_off[p + 1]) for p in perm])
    lri = [(int(inv[I]), int(inv[K]), R, C) for I, K, R, C in inp.lri]
    vq = inp.vq[:, aux][:, :, aux]
    return syn.Inputs(st=st2, kfrac=inp.kfrac, eig=inp.eig, occ=inp.occ, wfc=inp.wfc[:, :, orb],
                      efermi=inp.efermi, lri=lri, vq=vq), aux


def test_atom_permutation_invariance(cubic, cubic_run):
    g, out = cubic_run
    inp2, aux = _permute(cubic, [1, 0])
    out2 = pipeline.rpa_energy(inp2, g)
    assert abs(out2["ec"] - out["ec"]) < 1e-12 * abs(out["ec"])
    assert np.abs(out2["chi_tau"] - out["chi_tau"][:, :, aux][:, :, :, aux]).max() < 1e-12 * np.abs(
        out["chi_tau"]).max()


def test_lattice_shift_invariance(cubic, cubic_run):
    """Moving atom 1 by a lattice vector L relabels its cells: C[I,1,R] -> C[I,1,R-L],
    C[1,K,R] -> C[1,K,R+L], c_i(k) of atom 1 picks up e^{+i k.L}."""
    g, out = cubic_run
    st = cubic.st
    L = np.array([1, 0, -1])
    lri = []
    for I, K, R, C in cubic.lri:
        R = np.array(R)
        if K == 1:
            R = R - L
        if I == 1:
            R = R + L
        lri.append((I, K, tuple(int(x) for x in R), C))
    wfc = cubic.wfc.copy()
    orb1 = slice(int(st.n_ao[0]), st.nao)
    ph = np.exp(2j * np.pi * (cubic.kfrac @ L))
    wfc[:, :, orb1] *= ph[:, None, None]
    st2 = syn.Structure(lat=st.lat, pos=st.pos + np.array([[0, 0, 0], L @ st.lat]), n_ao=st.n_ao,
                        n_aux=st.n_aux, n_low=st.n_low, kmesh=st.kmesh)
    inp2 = syn.Inputs(st=st2, kfrac=cubic.kfrac, eig=cubic.eig, occ=cubic.occ, wfc=wfc,
                      efermi=cubic.efermi, lri=lri, vq=cubic.vq)
    # V(q) in the relabelled ABF cells: V_{mu nu} -> e^{+i q.L_mu} V_{mu nu} e^{-i q.L_nu}
    aux1 = slice(int(st.n_aux[0]), st.naux)
    vq = cubic.vq.copy()
    phq = np.exp(2j * np.pi * (cubic.kfrac @ L))
    for iq in range(st.nk):
        vq[iq][aux1, :] *= phq[iq]
        vq[iq][:, aux1] *= phq[iq].conj()
    inp2.vq = vq
    out2 = pipeline.rpa_energy(inp2, g)
    assert abs(out2["ec"] - out["ec"]) < 1e-12 * abs(out["ec"])


def test_pair_transpose_symmetry(cubic, cubic_run):
    """chi0_{VU}(-R) = chi0_{UV}(R)^T (the U <-> V symmetry of the pair set)."""
    g, out = cubic_run
    st = cubic.st
    ct = out["chi_tau"]
    mi = syn.minus_index(st.kmesh)
    scale = np.abs(ct).max()
    for it in range(ct.shape[0]):
        for iR in range(st.nk):
            assert np.abs(ct[it, mi[iR]] - ct[it, iR].T).max() < 1e-13 * scale


# ---------------------------------------------------------------- spin-polarised requests (nspins = 2)


def test_spin_identical_channels_equal_unpolarised():
    """Two equal spin channels with s = 1 each are the unpolarised problem with s = 2."""
    a = syn.config_cubic()
    b = syn.config_spin(identical=True)
    g = ogrid.make_grid(6, *a.delta_range)
    ra, rb = pipeline.rpa_energy(a, g), pipeline.rpa_energy(b, g)
    assert np.abs(ra["chi_tau"] - rb["chi_tau"]).max() <= 1e-14 * np.abs(ra["chi_tau"]).max()
    assert abs(ra["ec"] - rb["ec"]) <= 1e-14 * abs(ra["ec"])


def test_spin_routes_agree_in_tau():
    """Polarised channels (one more occupied band spin up): the matrix form on each channel's Green's
    functions, summed with s = 1, equals the sum over states of both channels in q space."""
    inp = syn.config_spin()
    st = inp.st
    tau = np.array([0.25, 1.3])
    ct = pipeline.chi0_tau(inp, {"tau": tau})
    scale = np.abs(ct).max()
    assert scale > 1.0
    for iq in range(st.nk):
        s = sum(chi0_sos(st, inp.lri, inp.kfrac, e, o, w, iq, tau=tau, spin=1.0) for e, o, w in inp.channels())
        for it in range(len(tau)):
            q = freq.r_to_q(ct[it], st.kmesh, inp.kfrac, [iq])[0]
            assert np.abs(q - s[it]).max() < 1e-13 * scale
    # and the channels really differ: the up channel alone is not half of the sum
    up = pipeline.chi0_tau(syn.Inputs(st=syn.Structure(**{**st.__dict__, "nspins": 1}), kfrac=inp.kfrac,
                                      eig=inp.eig_s[0], occ=inp.occ_s[0], wfc=inp.wfc_s[0], efermi=inp.efermi,
                                      lri=inp.lri, vq=inp.vq), {"tau": tau})
    assert np.abs(ct - 0.5 * up).max() > 1e-3 * scale


@pytest.mark.parametrize("delta,c01,v", [(0.6, 0.7, 1.3), (1.1, 0.2, 0.5)])
def test_spin_two_level_closed_form(delta, c01, v):
    """One spin channel with the two-level transition, the other without occupied states:
    E_c = (1/2)(sqrt(D^2 + 2aD) - D - a) with a = 1 rho^2 V (spin factor 1 per channel)."""
    st = syn.Structure(lat=np.eye(3) * 50.0, pos=np.zeros((1, 3)), n_ao=np.array([2]), n_aux=np.array([1]),
                       n_low=np.array([1]), kmesh=(1, 1, 1), nspins=2)
    eig = np.array([[-delta / 2, delta / 2]])
    wfc = np.eye(2, dtype=np.complex128)[None]
    occ_up, occ_dn = np.array([[1.0, 0.0]]), np.array([[0.0, 0.0]])
    C = np.array([[[0.0, c01], [c01, 0.0]]])
    inp = syn.Inputs(st=st, kfrac=np.zeros((1, 3)), eig=eig, occ=occ_up, wfc=wfc, efermi=0.0,
                     lri=[(0, 0, (0, 0, 0), C)], vq=np.array([[[v + 0j]]]),
                     eig_s=np.stack([eig, eig]), occ_s=np.stack([occ_up, occ_dn]), wfc_s=np.stack([wfc, wfc]))
    g = ogrid.make_grid(16, delta, delta)
    out = pipeline.rpa_energy(inp, g)
    a = 1.0 * (2 * c01) ** 2 * v
    exact = 0.5 * (math.sqrt(delta ** 2 + 2 * a * delta) - delta - a)
    assert abs(out["ec"] - exact) < 1e-6 * abs(exact)


# ---------------------------------------------------------------- P11: molecular limit


def test_molecule_in_a_box_is_molecular_ri_rpa():
    """P11: one k point and a molecule in a box large enough that no LRI block reaches a
    periodic image is molecular RI-RPA.  Computed here in the MO basis with the exact frequency
    kernel: rho^mu_ia = sum_jk Chat^mu_jk conj(c_ji) c_ka (Chat from Eq. LRI, both terms),
    Pi(i w) = -2 sum_{i occ, a virt} rho_ia rho_ia^H 2D/(D^2 + w^2) V, and
    E_c = (1/2 pi) sum_k W_k [ln det(1 - Pi) + Tr Pi]; the oracle's space-time E_c (G, Algorithm
    1, cosine and Fourier transforms, LU) must agree within the grid's transform error."""
    roh, ang = 1.81, math.radians(104.5)
    o = np.array([20.0, 20.0, 20.0])
    h1 = o + roh * np.array([math.sin(ang / 2), 0.0, -math.cos(ang / 2)])
    h2 = o + roh * np.array([-math.sin(ang / 2), 0.0, -math.cos(ang / 2)])
    st = syn.Structure(lat=np.eye(3) * 40.0, pos=np.array([o, h1, h2]), n_ao=np.array([5, 5, 5]),
                       n_aux=np.array([30, 30, 30]), n_low=np.array([2, 1, 1]), kmesh=(1, 1, 1))
    inp = syn.make_inputs(st, 17, vscale=2e-3)
    g = ogrid.make_grid(16, *inp.delta_range)
    ref = pipeline.rpa_energy(inp, g)["ec"]
    # Eq. LRI pair coefficients of the molecule
    ao = np.concatenate([[0], np.cumsum(st.n_ao)])
    ax = np.concatenate([[0], np.cumsum(st.n_aux)])
    chat = np.zeros((st.naux, st.nao, st.nao))
    for I, K, R, C in inp.lri:
        assert tuple(R) == (0, 0, 0)          # no periodic image within r_cut
        mu, a, b = slice(ax[I], ax[I + 1]), slice(ao[I], ao[I + 1]), slice(ao[K], ao[K + 1])
        chat[mu, a, b] += C                   # [mu in atom(i)] C[I,K]_{mu i k}
        chat[mu, b, a] += C.transpose(0, 2, 1)  # [mu in atom(k)] C[K,I]_{mu k i}
    eps, c, f = inp.eig[0], inp.wfc[0].T, inp.occ[0]   # c[:, n] = MO n in the NAO basis
    occ, vir = np.where(f > 0.5)[0], np.where(f < 0.5)[0]
    rho = np.einsum("mjk,ji,ka->mia", chat, c[:, occ].conj(), c[:, vir])
    delta = eps[vir][None, :] - eps[occ][:, None]
    v = inp.vq[0]
    ec = 0.0
    for w, wk in zip(g["omega"], g["w_omega"]):
        ker = 2.0 * delta / (delta ** 2 + w ** 2)
        chi = -2.0 * np.einsum("mia,ia,nia->mn", rho, ker, rho.conj())
        pi = chi @ v
        sign, logdet = np.linalg.slogdet(np.eye(st.naux) - pi)
        assert sign.real > 0
        ec += wk * (logdet + np.trace(pi).real) / (2.0 * math.pi)
    assert ec < 0
    assert abs(ec - ref) < 1e-6 * abs(ref), (ec, ref)


# ---------------------------------------------------------------- P12: Green's-function screening


def test_screen_hand_fixture():
    """The block rule on a hand-made G (atoms of 1 and 2 NAOs, 2 tau, 2 R): a block whose
    largest |element| equals theta is kept, one just below is dropped, an all-zero block stays
    zero, small elements of a kept block are untouched, and the rule acts per (tau, R, I, J)."""
    th = 1e-3
    G = np.zeros((2, 2, 3, 3))
    G[0, 0, 0, 0] = -0.5                              # (0,0) kept
    G[0, 0, 0, 1:3] = [th, -0.25 * th]                # (0,1) max == theta: kept
    G[0, 0, 1:3, 0] = [0.999 * th, -0.5 * th]         # (1,0) below: dropped
    G[0, 1, 1:3, 1:3] = [[2e-7, -3.0], [1e-9, 0.0]]   # (1,1) kept, tiny entries included
    G[0, 1, 0, 0] = 1e-4                              # (0,0) at R 1: dropped
    G[1, 0, 0, 1:3] = [-2e-3, 5e-4]                   # (0,1) at tau 1: kept
    G[1, 1, 1:3, 0] = [1e-3, 0.0]                     # (1,0) at tau 1, R 1: kept (== theta)
    G[1, 1, 1:3, 1:3] = 9e-4                          # (1,1) at tau 1, R 1: dropped
    want = G.copy()
    want[0, 0, 1:3, 0] = 0.0
    want[0, 1, 0, 0] = 0.0
    want[1, 1, 1:3, 1:3] = 0.0
    keep_want = np.zeros((2, 2, 2, 2), dtype=bool)
    keep_want[0, 0, 0, 0] = keep_want[0, 0, 0, 1] = True
    keep_want[0, 1, 1, 1] = True
    keep_want[1, 0, 0, 1] = True
    keep_want[1, 1, 1, 0] = True
    out, keep = screen.screen_blocks(G, [1, 2], th)
    assert np.array_equal(out, want)
    assert np.array_equal(keep, keep_want)
    out0, keep0 = screen.screen_blocks(G, [1, 2], 0.0)   # theta = 0 keeps everything
    assert np.array_equal(out0, G) and keep0.all()


def test_screen_limits_of_the_energy(cubic):
    """theta above every block maximum drops all of G: chi0 = 0 and E_c = 0 exactly
    (ln det 1 + Tr 0); theta at or below every block maximum keeps all of G and gives the
    unscreened E_c bit for bit; theta in between keeps nested block sets."""
    g = ogrid.make_grid(8, *cubic.delta_range)
    go, gv = pipeline.greens(cubic, g)[0]
    bm = np.concatenate([screen.block_max(go, cubic.st.n_ao).ravel(), screen.block_max(gv, cubic.st.n_ao).ravel()])
    full = pipeline.rpa_energy(cubic, g)
    none = pipeline.rpa_energy(cubic, g, screen=2.0 * bm.max())
    assert np.all(none["chi_tau"] == 0.0) and none["ec"] == 0.0
    same = pipeline.rpa_energy(cubic, g, screen=bm.min())
    assert same["ec"] == full["ec"]
    k1 = screen.screen_blocks(go, cubic.st.n_ao, 1e-3)[1]
    k2 = screen.screen_blocks(go, cubic.st.n_ao, 1e-2)[1]
    assert np.all(k1 | ~k2) and k1.sum() > k2.sum()   # kept(1e-2) is a strict subset of kept(1e-3)


def test_weights_folded_onto_q_leq_minus_q():
    """The integrand of -q equals that of q (chi0(-q) = conj chi0(q) from real chi0(R), and
    V(-q) = conj V(q)): E_c with each pair's weight moved onto q <= -q equals the 1/N_q sum, and
    an irreducible set's weights (star weights on representatives, 0 elsewhere) reproduce it."""
    inp = syn.make_inputs(syn.cubic_two_atom(nao=4, naux=16, nlow=2, kmesh=(3, 3, 1)), 41, vscale=2e-3)
    st = inp.st
    g = ogrid.make_grid(8, *inp.delta_range)
    out = pipeline.rpa_energy(inp, g)
    mi = syn.minus_index(st.kmesh)
    w = np.zeros(st.nk)
    for q in range(st.nk):
        w[min(q, mi[q])] += 1.0 / st.nk
    assert np.count_nonzero(w) < st.nk
    ec_w = energy.correlation_energy(out["chi_qw"], inp.vq, g["w_omega"], wq=w)[0]
    assert abs(ec_w - out["ec"]) < 1e-13 * abs(out["ec"])
