"""librpa_gpu_ec_noalloc (the ln det stage with its scratch in a static device array) against
librpa_gpu_ec on the same chi0(q, i omega) and V(q), on two calls in a row per q.

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
