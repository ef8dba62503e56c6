"""librpa_gpu_ec_noalloc (the ln det stage with its scratch in a static device array) against
librpa_gpu_ec on the same chi0(q, i omega) and V(q), on two calls in a row per q; against the
oracle's LU at the largest size the scratch holds; NaN where a matrix is not positive definite.

Collected last (file name) so that it also runs after every other test in one process."""
import math

import numpy as np
import pytest

from paper_2407_19930_gb300 import librpa_gpu as L
from paper_2407_19930_gb300 import synthetic as syn
from oracle import grid as ogrid

TOL_EC = 1e-8   # Ha, as for the handle-based energy


def test_noalloc_rejects_sizes_beyond_the_scratch():
    """Checked on the host before any CUDA call: runs without a GPU."""
    for n in (0, L.LIBRPA_NOALLOC_MAX_NAUX + 1):
        with pytest.raises(L.LibrpaError) as e:
            L.librpa_gpu_ec_noalloc(n, 1, 16, 16, 16)
        assert e.value.code == L.LIBRPA_E_ARG
        assert "naux" in str(e.value)
    with pytest.raises(L.LibrpaError) as e:
        L.librpa_gpu_ec_noalloc(8, -1, 16, 16, 16)
    assert e.value.code == L.LIBRPA_E_ARG


@pytest.mark.gpu
def test_noalloc_matches_ec():
    torch = pytest.importorskip("torch")
    inp = syn.config_mixed()    # 4 q points
    st = inp.st
    grid = ogrid.make_grid(8, *inp.delta_range)
    nw = len(grid["omega"])
    h = L.librpa_gpu_create()
    try:
        L.set_inputs(h, inp, grid)
        chi = L.librpa_gpu_chi0(h, out=(st.nk, nw, st.naux))
        ec, ec_q, _ = L.librpa_gpu_ec(h, st.nk, nw)
    finally:
        L.librpa_gpu_destroy(h)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    d_chi = [torch.view_as_real(torch.from_numpy(np.ascontiguousarray(chi[q]))).contiguous().to(dev)
             for q in range(st.nk)]
    d_v = [torch.view_as_real(torch.from_numpy(np.ascontiguousarray(inp.vq[q]))).contiguous().to(dev)
           for q in range(st.nk)]
    out = torch.full((nw,), float("nan"), dtype=torch.float64, device=dev)
    w = np.asarray(grid["w_omega"])
    pref = 1.0 / (2.0 * math.pi * st.nk)
    # two calls in a row for every q, visiting the q points in two orders, so that each call
    # follows one on other inputs and one on the same inputs
    for order in (range(st.nk), reversed(range(st.nk))):
        tot = 0.0
        for q in order:
            for _ in range(2):
                out.fill_(float("nan"))
                L.librpa_gpu_ec_noalloc(st.naux, nw, d_v[q].data_ptr(), d_chi[q].data_ptr(), out.data_ptr(),
                                        stream.cuda_stream)
                torch.cuda.synchronize(dev)
                f = out.cpu().numpy()
                assert np.all(np.isfinite(f))
                eq = pref * float(np.dot(w, f))
                assert abs(eq - ec_q[q]) < TOL_EC, (q, eq, ec_q[q])
            tot += eq
        assert abs(tot - ec) < TOL_EC, (tot, ec)


def _hpd(rng, n, shift=0.1):
    x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2 * n)
    return x @ x.conj().T + shift * np.eye(n)


def _nsd(rng, n, scale):
    x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2 * n)
    return -scale * (x @ x.conj().T)


def _dev(torch, a):
    return torch.view_as_real(torch.from_numpy(np.ascontiguousarray(a))).contiguous().to("cuda:0")


def _call(torch, n, d_v, d_chi, nw):
    out = torch.full((nw,), 123.0, dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream()
    L.librpa_gpu_ec_noalloc(n, nw, d_v.data_ptr(), d_chi.data_ptr(), out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_at_the_one_slot_limit_against_the_oracle():
    """naux = LIBRPA_NOALLOC_MAX_NAUX (591: not a multiple of the 32-wide tiles), where exactly one
    scratch slot fits and one CTA walks every frequency: each out[k] against the oracle's LU of
    1 - chi_k V on the host, on two calls in a row."""
    torch = pytest.importorskip("torch")
    from oracle.energy import integrand_lu
    n, nw = L.LIBRPA_NOALLOC_MAX_NAUX, 3
    rng = np.random.default_rng(591)
    v = _hpd(rng, n)
    chi = np.stack([_nsd(rng, n, s) for s in (0.05, 0.5, 2.0)])
    ref = np.array([integrand_lu(chi[k], v)[0] for k in range(nw)])
    d_v, d_chi = _dev(torch, v), _dev(torch, chi)
    for _ in range(2):
        f = _call(torch, n, d_v, d_chi, nw)
        assert np.all(np.isfinite(f))
        assert np.abs(f - ref).max() < 1e-9 * max(1.0, np.abs(ref).max()), (f, ref)


@pytest.mark.gpu
def test_noalloc_not_positive_definite_gives_nan_and_the_next_call_is_right():
    """A V(q) with a negative eigenvalue gives NaN in every slot; a chi that makes one frequency's
    I - L^H chi L indefinite gives NaN in that slot only; the following call on good inputs matches
    the oracle (the scratch left by the failed calls does not leak into it)."""
    torch = pytest.importorskip("torch")
    from oracle.energy import integrand_lu
    n, nw = 77, 4
    rng = np.random.default_rng(77)
    v = _hpd(rng, n)
    chi = np.stack([_nsd(rng, n, 0.3 * (k + 1)) for k in range(nw)])
    ref = np.array([integrand_lu(chi[k], v)[0] for k in range(nw)])
    w, u = np.linalg.eigh(v)
    w_bad = w.copy()
    w_bad[0] = -0.5
    v_bad = (u * w_bad) @ u.conj().T
    f = _call(torch, n, _dev(torch, v_bad), _dev(torch, chi), nw)
    assert np.all(np.isnan(f)), f
    chi_bad = chi.copy()
    chi_bad[2] = (2.0 / w[0]) * np.eye(n)      # L^H chi L >= 2 I: A = I - L^H chi L negative definite
    f = _call(torch, n, _dev(torch, v), _dev(torch, chi_bad), nw)
    assert np.isnan(f[2]) and np.all(np.isfinite(np.delete(f, 2))), f
    assert np.abs(np.delete(f, 2) - np.delete(ref, 2)).max() < 1e-10 * np.abs(ref).max()
    f = _call(torch, n, _dev(torch, v), _dev(torch, chi), nw)
    assert np.abs(f - ref).max() < 1e-10 * np.abs(ref).max(), (f, ref)


@pytest.mark.gpu
def test_noalloc_setup_call():
    """nomega = 0 performs only the per-device set-up (no buffers needed) and succeeds again."""
    pytest.importorskip("torch")
    for _ in range(2):
        L.librpa_gpu_ec_noalloc(8, 0, 0, 0, 0)
