"""Seeded synthetic inputs for the LRI space-time RPA path.

This module only *draws* inputs: crystal geometries, a tight-binding
Kohn-Sham problem solved with ``numpy.linalg.eigh``, localized-RI (LRI)
expansion coefficients and Coulomb matrices V(q).  It holds none of the
method's arithmetic (no Green's function, no response function, no
transform, no determinant), so both the library tests and the CPU oracle
can take their inputs from it.

The inputs stand in for the files a NAO-based DFT code exports (KS
eigenvectors, LRI coefficients C, Coulomb matrix V; Sec. 3.3 "Interface"),
which are not available here.  The shapes follow the paper's workloads:
a cubic test cell, and the graphene 4x4 supercell with a water-shaped
3-atom molecule above it (Sec. 5, 4x4x1 k-mesh, 16 minimax points).

Conventions (shared with every consumer):

* lattice rows ``lat[a]`` are the vectors a1, a2, a3 in bohr; positions are
  Cartesian bohr;
* the Gamma-centred k-mesh point (i1, i2, i3) has fractional coordinates
  (i1/nk1, i2/nk2, i3/nk3) and flat index ``(i1*nk2 + i2)*nk3 + i3``;
  the same flat order enumerates the Born-von-Karman (BvK) cells R and the
  q-mesh;
* ``wfc[k, n, i]`` is the KS coefficient c_{i,n}(k) (S = I, nbands = n_ao);
* H(k) = sum_R exp(+2 pi i k.R) H(R), so that the real-space Green's
  function carries exp(-i k.R) (Eq. green_mat);
* an LRI block ``C[I, K, R]`` has shape [n_aux(I)][n_ao(I)][n_ao(K)] and
  holds C^{mu(0)}_{i(0), k(R)} with mu and i on atom I in the home cell and
  k on atom K in cell R (Eq. LRI); R is a true lattice vector, not folded.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

HARTREE_TO_MEV = 27211.386245988


@dataclasses.dataclass
class Structure:
    """Periodic structure with per-atom NAO / ABF counts."""

    lat: np.ndarray          # (3, 3) rows a1, a2, a3 (bohr)
    pos: np.ndarray          # (nat, 3) Cartesian (bohr)
    n_ao: np.ndarray         # (nat,) NAOs per atom
    n_aux: np.ndarray        # (nat,) ABFs per atom
    n_low: np.ndarray        # (nat,) low-lying (occupied) orbitals per atom
    kmesh: tuple             # (nk1, nk2, nk3), Gamma-centred
    r_cut: float = 6.0       # LRI cutoff (bohr)
    nspins: int = 1

    @property
    def natoms(self) -> int:
        return int(len(self.n_ao))

    @property
    def nao(self) -> int:
        return int(np.sum(self.n_ao))

    @property
    def naux(self) -> int:
        return int(np.sum(self.n_aux))

    @property
    def nk(self) -> int:
        return int(np.prod(self.kmesh))

    @property
    def nocc(self) -> int:
        return int(np.sum(self.n_low))


@dataclasses.dataclass
class Inputs:
    """All inputs of one RPA energy request."""

    st: Structure
    kfrac: np.ndarray        # (nk, 3)
    eig: np.ndarray          # (nk, nb) Ha
    occ: np.ndarray          # (nk, nb) occupation per spin-orbital in [0, 1]
    wfc: np.ndarray          # (nk, nb, nao) complex, wfc[k, n, i] = c_{i n}(k)
    efermi: float            # Ha, mid-gap
    lri: list                # [(I, K, (r1, r2, r3), C[naux_I, nao_I, nao_K])]
    vq: np.ndarray           # (nq, naux, naux) complex Hermitian positive definite
    seed: int = 0
    hr: dict = None          # real-space tight-binding H(R) the KS data came from
    # spin-polarised requests (st.nspins = 2): KS data per channel, [spin][k][...]; eig, occ and
    # wfc above then hold channel 0
    eig_s: np.ndarray = None
    occ_s: np.ndarray = None
    wfc_s: np.ndarray = None

    def channels(self) -> list:
        """[(eig, occ, wfc)] per spin channel."""
        if self.st.nspins == 1:
            return [(self.eig, self.occ, self.wfc)]
        return [(self.eig_s[c], self.occ_s[c], self.wfc_s[c]) for c in range(self.st.nspins)]

    @property
    def gap(self) -> float:
        nocc = self.st.nocc
        return float(self.eig[:, nocc].min() - self.eig[:, nocc - 1].max())

    @property
    def delta_range(self) -> tuple:
        """(smallest, largest) occupied->virtual transition energy within a spin channel, Ha."""
        lo, hi = np.inf, -np.inf
        for eig, occ, _ in self.channels():
            o, v = occ > 0, occ < 1
            if o.any() and v.any():
                lo = min(lo, float(eig[v].min() - eig[o].max()))
                hi = max(hi, float(eig[v].max() - eig[o].min()))
        return (lo, hi)


# ----------------------------------------------------------------------------
# meshes and lattice helpers


def kmesh_frac(kmesh) -> np.ndarray:
    """Fractional coordinates of the Gamma-centred mesh in flat order."""
    n1, n2, n3 = kmesh
    return np.array([(i1 / n1, i2 / n2, i3 / n3)
                     for i1 in range(n1) for i2 in range(n2) for i3 in range(n3)],
                    dtype=np.float64)


def bvk_cells(kmesh) -> np.ndarray:
    """Integer BvK cell vectors (r1, r2, r3), 0 <= r_a < nk_a, flat order."""
    n1, n2, n3 = kmesh
    return np.array([(i1, i2, i3)
                     for i1 in range(n1) for i2 in range(n2) for i3 in range(n3)],
                    dtype=np.int64)


def minus_index(kmesh) -> np.ndarray:
    """Flat index of -k (mod the mesh) for every mesh point."""
    n1, n2, n3 = kmesh
    out = np.empty(n1 * n2 * n3, dtype=np.int64)
    for i1, i2, i3 in itertools.product(range(n1), range(n2), range(n3)):
        out[(i1 * n2 + i2) * n3 + i3] = (((-i1) % n1) * n2 + (-i2) % n2) * n3 + (-i3) % n3
    return out


def lattice_vectors_within(lat: np.ndarray, rmax: float) -> np.ndarray:
    """All integer triples n with |n @ lat| <= rmax + span of the cell."""
    inv = np.linalg.inv(lat)
    # bound on |n_a| from the dual-vector norms
    bounds = [int(math.ceil(rmax * np.linalg.norm(inv[:, a]))) + 1 for a in range(3)]
    rng = [range(-b, b + 1) for b in bounds]
    return np.array(list(itertools.product(*rng)), dtype=np.int64)


# ----------------------------------------------------------------------------
# geometries


def cubic_two_atom(nao=8, naux=24, nlow=2, kmesh=(2, 2, 2)) -> Structure:
    """Cubic cell a = 4 bohr, atoms at (0,0,0) and (a/2, a/2, a/2)."""
    a = 4.0
    return Structure(lat=np.eye(3) * a,
                     pos=np.array([[0.0, 0.0, 0.0], [a / 2, a / 2, a / 2]]),
                     n_ao=np.array([nao, nao]), n_aux=np.array([naux, naux]),
                     n_low=np.array([nlow, nlow]), kmesh=tuple(kmesh))


def graphene_water_slab(nsuper=4, kmesh=(4, 4, 1)) -> Structure:
    """Graphene nsuper x nsuper supercell (a = 4.65 bohr primitive) with a
    water-shaped molecule whose O sits 6 bohr above a hexagon centre.

    C: 13 NAO / 60 ABF, 2 occupied orbitals; O and H: 5 NAO / 30 ABF with
    2 (O) and 1 (H) occupied orbitals; vacuum c = 30 bohr.
    """
    a = 4.65
    a1 = np.array([a, 0.0, 0.0])
    a2 = np.array([a / 2, a * math.sqrt(3) / 2, 0.0])
    c = 30.0
    lat = np.array([nsuper * a1, nsuper * a2, [0.0, 0.0, c]])
    base = [np.zeros(3), (a1 + a2) / 3.0]
    pos, n_ao, n_aux, n_low = [], [], [], []
    z0 = 10.0
    for i, j in itertools.product(range(nsuper), range(nsuper)):
        for b in base:
            pos.append(i * a1 + j * a2 + b + np.array([0.0, 0.0, z0]))
            n_ao.append(13), n_aux.append(60), n_low.append(2)
    # hexagon centre of the primitive cell (0,0): (2/3)(a1+a2)
    hc = (a1 + a2) * 2.0 / 3.0 + np.array([0.0, 0.0, z0])
    o = hc + np.array([0.0, 0.0, 6.0])
    roh, ang = 1.81, math.radians(104.5)
    # two-leg orientation: C2 axis along z, hydrogens pointing to the sheet
    h1 = o + roh * np.array([math.sin(ang / 2), 0.0, -math.cos(ang / 2)])
    h2 = o + roh * np.array([-math.sin(ang / 2), 0.0, -math.cos(ang / 2)])
    for p, nl in ((o, 2), (h1, 1), (h2, 1)):
        pos.append(p), n_ao.append(5), n_aux.append(30), n_low.append(nl)
    return Structure(lat=lat, pos=np.array(pos), n_ao=np.array(n_ao),
                     n_aux=np.array(n_aux), n_low=np.array(n_low), kmesh=tuple(kmesh))


def random_cell(rng: np.random.Generator, natoms: int, kmesh) -> Structure:
    """Random cell at the atom density of the cubic test cell, species drawn
    from {(5 NAO, 20 ABF), (9, 40), (13, 60)}, minimum spacing 2.5 bohr."""
    density = 2.0 / 64.0
    vol = natoms / density
    # slightly skewed box with the volume above
    l = vol ** (1.0 / 3.0)
    lat = np.diag([l, l, l]) + rng.uniform(-0.1, 0.1, size=(3, 3)) * l * np.array(
        [[0, 1, 1], [0, 0, 1], [0, 0, 0]])
    species = [(5, 20, 1), (9, 40, 2), (13, 60, 2)]
    pos, n_ao, n_aux, n_low = [], [], [], []
    cells = lattice_vectors_within(lat, 3.0)
    while len(pos) < natoms:
        f = rng.uniform(0, 1, size=3)
        p = f @ lat
        ok = True
        for q in pos:
            d = np.min(np.linalg.norm(p - q - cells @ lat, axis=1))
            if d < 2.5:
                ok = False
                break
        if not ok:
            continue
        s = species[int(rng.integers(0, 3))]
        pos.append(p), n_ao.append(s[0]), n_aux.append(s[1]), n_low.append(s[2])
    return Structure(lat=lat, pos=np.array(pos), n_ao=np.array(n_ao), n_aux=np.array(n_aux),
                     n_low=np.array(n_low), kmesh=tuple(kmesh))


# ----------------------------------------------------------------------------
# KS problem, LRI coefficients, Coulomb matrices


def tight_binding_hr(st: Structure, rng: np.random.Generator, t0=0.1, decay=1.5, dmax=9.0,
                     e_low=-0.5, e_high=0.5) -> dict:
    """Real H(R) blocks as {R tuple: (nao, nao) array} with H(-R) = H(R)^T.

    On-site: the first n_low orbitals of each atom at e_low, the others at
    e_high.  Hopping between atoms at distance d <= dmax:
    t0 * g * exp(-d / decay) with g ~ N(0, 1).
    """
    nat = st.natoms
    off = np.concatenate([[0], np.cumsum(st.n_ao)])
    nao = st.nao
    hr = {}
    cells = lattice_vectors_within(st.lat, dmax + 1e-9)

    def block(R):
        key = tuple(int(x) for x in R)
        if key not in hr:
            hr[key] = np.zeros((nao, nao))
        return hr[key]

    h0 = block((0, 0, 0))
    for I in range(nat):
        d = np.full(st.n_ao[I], e_high)
        d[: st.n_low[I]] = e_low
        h0[off[I]:off[I + 1], off[I]:off[I + 1]] += np.diag(d)
    for I in range(nat):
        for J in range(I, nat):
            for R in cells:
                Rt = tuple(int(x) for x in R)
                if I == J and Rt <= (0, 0, 0):
                    continue   # on-site and the -R half are set by symmetry
                dist = float(np.linalg.norm(st.pos[J] + R @ st.lat - st.pos[I]))
                if dist > dmax:
                    continue
                t = t0 * rng.standard_normal((st.n_ao[I], st.n_ao[J])) * math.exp(-dist / decay)
                block(Rt)[off[I]:off[I + 1], off[J]:off[J + 1]] += t
                mR = tuple(-x for x in Rt)
                block(mR)[off[J]:off[J + 1], off[I]:off[I + 1]] += t.T
    return hr


def solve_ks(st: Structure, hr: dict):
    kf = kmesh_frac(st.kmesh)
    nao = st.nao
    eig = np.empty((len(kf), nao))
    wfc = np.empty((len(kf), nao, nao), dtype=np.complex128)
    for ik, k in enumerate(kf):
        hk = np.zeros((nao, nao), dtype=np.complex128)
        for R, h in hr.items():
            hk += np.exp(2j * np.pi * float(np.dot(k, R))) * h
        hk = 0.5 * (hk + hk.conj().T)
        w, v = np.linalg.eigh(hk)
        eig[ik] = w
        wfc[ik] = v.T          # wfc[k, n, i] = c_{i n}(k)
    return kf, eig, wfc


def lri_coefficients(st: Structure, rng: np.random.Generator) -> list:
    """C[I, K, R] ~ N(0, 1) exp(-d / 2) for d = |tau_K + R - tau_I| <= r_cut;
    on-site blocks (I = K, R = 0) symmetrised in (i, k)."""
    out = []
    cells = lattice_vectors_within(st.lat, st.r_cut + 1e-9)
    for I in range(st.natoms):
        for K in range(st.natoms):
            for R in cells:
                dist = float(np.linalg.norm(st.pos[K] + R @ st.lat - st.pos[I]))
                if dist > st.r_cut:
                    continue
                c = rng.standard_normal((st.n_aux[I], st.n_ao[I], st.n_ao[K])) * math.exp(-dist / 2.0)
                if I == K and not np.any(R):
                    c = 0.5 * (c + c.transpose(0, 2, 1))
                out.append((I, K, tuple(int(x) for x in R), np.ascontiguousarray(c)))
    return out


def coulomb_q(st: Structure, rng: np.random.Generator, scale=1.0) -> np.ndarray:
    """V(q) = scale * (L L^H + 0.1 I), L ~ N(0, 1/naux); V(-q) = conj V(q).
    Self-conjugate q points (q = -q mod the mesh) get a real L."""
    n = st.naux
    mi = minus_index(st.kmesh)
    vq = np.empty((st.nk, n, n), dtype=np.complex128)
    for iq in range(st.nk):
        p = mi[iq]
        if p < iq:
            vq[iq] = vq[p].conj()
            continue
        if p == iq:
            L = rng.standard_normal((n, n)) / math.sqrt(n)
        else:
            L = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2 * n)
        v = L @ L.conj().T + 0.1 * np.eye(n)
        vq[iq] = scale * 0.5 * (v + v.conj().T)
    return vq


def make_inputs(st: Structure, seed: int, vscale=1.0, t0=0.1, min_gap=0.1) -> Inputs:
    """Draw a full request for structure ``st``.  The KS problem is redrawn
    with seed+1, seed+2, ... until the gap is at least ``min_gap`` Ha."""
    s = seed
    while True:
        rng = np.random.default_rng(s)
        hr = tight_binding_hr(st, rng, t0=t0)
        kf, eig, wfc = solve_ks(st, hr)
        nocc = st.nocc
        gap = eig[:, nocc].min() - eig[:, nocc - 1].max()
        if gap >= min_gap:
            break
        s += 1
    efermi = 0.5 * (eig[:, nocc].min() + eig[:, nocc - 1].max())
    occ = np.zeros_like(eig)
    occ[:, :nocc] = 1.0
    lri = lri_coefficients(st, rng)
    vq = coulomb_q(st, rng, scale=vscale)
    return Inputs(st=st, kfrac=kf, eig=eig, occ=occ, wfc=wfc, efermi=float(efermi),
                  lri=lri, vq=vq, seed=seed, hr=hr)


def make_inputs_spin(st: Structure, seed: int, vscale=1.0, t0=0.1, min_gap=0.1, identical=False) -> Inputs:
    """Spin-polarised request (st.nspins = 2): both channels from one H(R), except that the up
    channel has one more low orbital on atom 0 (its first high on-site level moved to the low
    one), so it holds one more occupied band.  ``identical`` keeps both channels equal to the
    spin-unpolarised problem drawn by ``make_inputs`` with the same seed (same random draws)."""
    assert st.nspins == 2 and st.n_ao[0] > st.n_low[0]
    s = seed
    while True:
        rng = np.random.default_rng(s)
        hr = tight_binding_hr(st, rng, t0=t0)
        hr_up = {R: b.copy() for R, b in hr.items()}
        nocc_up = st.nocc
        if not identical:
            i = int(st.n_low[0])   # first high orbital of atom 0
            hr_up[(0, 0, 0)][i, i] -= 1.0
            nocc_up += 1
        chans, ok = [], True
        for h_c, nocc in ((hr_up, nocc_up), (hr, st.nocc)):
            kf, eig, wfc = solve_ks(st, h_c)
            if eig[:, nocc].min() - eig[:, nocc - 1].max() < min_gap:
                ok = False
            occ = np.zeros_like(eig)
            occ[:, :nocc] = 1.0
            chans.append((eig, occ, wfc, 0.5 * (eig[:, nocc].min() + eig[:, nocc - 1].max())))
        if ok:
            break
        s += 1
    efermi = float(np.mean([c[3] for c in chans]))   # any common level: it cancels within a channel
    lri = lri_coefficients(st, rng)
    vq = coulomb_q(st, rng, scale=vscale)
    return Inputs(st=st, kfrac=kf, eig=chans[0][0], occ=chans[0][1], wfc=chans[0][2], efermi=efermi,
                  lri=lri, vq=vq, seed=seed, hr=hr, eig_s=np.stack([c[0] for c in chans]),
                  occ_s=np.stack([c[1] for c in chans]), wfc_s=np.stack([c[2] for c in chans]))


# ----------------------------------------------------------------------------
# named workloads
#
# ``vscale`` multiplies V(q) so that the largest eigenvalue of -chi0 V at
# q = 0 and the lowest grid frequency is of order one, as for a real
# Coulomb matrix in an ABF basis (measured once per workload with the CPU
# oracle at vscale = 1 and rounded: cubic 992, tiny 87, mixed 1717).


def config_cubic(seed=1001, vscale=1e-3) -> Inputs:
    """Cubic a = 4 bohr, 2 atoms, 2x2x2 k, 8 NAO / 24 ABF per atom, 4 occupied bands."""
    return make_inputs(cubic_two_atom(), seed, vscale=vscale)


def config_graphene(seed=2002, kmesh=(4, 4, 1), vscale=3e-4) -> Inputs:
    """Graphene 4x4 supercell + water-shaped molecule, 4x4x1 k (N_aux = 2010)."""
    return make_inputs(graphene_water_slab(kmesh=kmesh), seed, vscale=vscale)


def config_tiny(seed=7, kmesh=(2, 1, 1), nao=3, naux=4, vscale=1e-2) -> Inputs:
    """Two-atom cubic cell with very few functions, for brute-force checks."""
    return make_inputs(cubic_two_atom(nao=nao, naux=naux, nlow=1, kmesh=kmesh), seed, vscale=vscale)


def config_mixed(seed=11, kmesh=(2, 2, 1), vscale=6e-4) -> Inputs:
    """Four atoms of three species in a skewed cell: ragged block shapes
    (5/9/13 NAO, 20/40/60 ABF) spanning several GEMM tiles."""
    rng = np.random.default_rng(seed)
    st = random_cell(rng, 4, kmesh)
    return make_inputs(st, seed, vscale=vscale)


def config_spin(seed=1001, vscale=1e-3, kmesh=(2, 2, 2), identical=False) -> Inputs:
    """The cubic two-atom cell, spin-polarised (nspins = 2)."""
    st = cubic_two_atom(kmesh=kmesh)
    st.nspins = 2
    return make_inputs_spin(st, seed, vscale=vscale, identical=identical)


def config_request(index, natoms_range=(2, 64), seed_base=4004, vscale=2e-4) -> Inputs:
    """Request ``index`` of the serving and batched workloads: a random cell of
    U{natoms_range} atoms (species as in ``random_cell``), a k-mesh drawn from
    1x1x1, 2x2x1 and 3x3x1, seeded by (seed_base, index).  ``vscale`` is one
    conservative value for every size (the largest calibrated workloads above
    need 3e-4 to 1e-3)."""
    rng = np.random.default_rng([seed_base, index])
    natoms = int(rng.integers(natoms_range[0], natoms_range[1] + 1))
    kmesh = [(1, 1, 1), (2, 2, 1), (3, 3, 1)][int(rng.integers(0, 3))]
    st = random_cell(rng, natoms, kmesh)
    return make_inputs(st, seed_base * 1000 + index, vscale=vscale)
