"""The bounded-wait failure path of the tensor-core GEMM, made to run without a GPU fault.

Every mbarrier wait in the tcgen05 GEMM kernel has a time limit; when one runs out the CTA
records the failure, waits for the copies and MMAs it has already issued, frees its TMEM and
returns, and the call reports LIBRPA_E_TIMEOUT.  The testing option ``test_stall_gemms`` makes
the MMA issuer of every tile of the handle's first GEMM launches wait on a barrier that nothing
arrives at (a 100 us limit), so the path runs deterministically; the same handle must then give
the oracle's energy, and the CUDA context must stay usable."""
import numpy as np
import pytest

from paper_2407_19930_gb300 import librpa_gpu as L
from paper_2407_19930_gb300 import synthetic as syn
from oracle import grid as ogrid, pipeline

TOL_EC = 1e-8


def test_stall_option_is_validated():
    """A negative value is rejected before any CUDA call (runs without a GPU)."""
    o = L.librpa_gpu_default_opts()
    o.test_stall_gemms = -1
    with pytest.raises(L.LibrpaError) as e:
        L.librpa_gpu_create(o)
    assert e.value.code == L.LIBRPA_E_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("stalls", [1, 3])
def test_wait_runs_out_then_the_handle_recovers(stalls):
    inp = syn.config_cubic()
    grid = ogrid.make_grid(8, *inp.delta_range)
    ref = pipeline.rpa_energy(inp, grid)
    o = L.librpa_gpu_default_opts()
    o.precision = L.LIBRPA_FP64_TC
    o.test_stall_gemms = stalls
    h = L.librpa_gpu_create(o)
    try:
        L.set_inputs(h, inp, grid)
        with pytest.raises(L.LibrpaError) as e:
            L.librpa_gpu_chi0(h)
        assert e.value.code == L.LIBRPA_E_TIMEOUT
        assert "bounded wait" in L.librpa_gpu_last_error(h)
        # the handle's later launches run normally
        L.librpa_gpu_chi0(h)
        ec, ec_q, _ = L.librpa_gpu_ec(h, inp.st.nk, None)
    finally:
        L.librpa_gpu_destroy(h)
    assert abs(ec - ref["ec"]) < TOL_EC
    assert np.abs(ec_q - ref["ec_q"]).max() < TOL_EC


@pytest.mark.gpu
def test_wait_runs_out_in_the_energy_stage():
    """The stall reaches the ln det GEMMs when the chi0 stage has no tensor-core GEMM (FP64 chi0,
    5-plane ln det): librpa_gpu_ec reports the timeout, and the next librpa_gpu_ec is right."""
    inp = syn.config_cubic()
    grid = ogrid.make_grid(8, *inp.delta_range)
    ref = pipeline.rpa_energy(inp, grid)
    o = L.librpa_gpu_default_opts()
    o.precision = L.LIBRPA_FP64
    o.ec_slices = 5
    o.test_stall_gemms = 1
    h = L.librpa_gpu_create(o)
    try:
        L.set_inputs(h, inp, grid)
        L.librpa_gpu_chi0(h)
        with pytest.raises(L.LibrpaError) as e:
            L.librpa_gpu_ec(h)
        assert e.value.code == L.LIBRPA_E_TIMEOUT
        ec, _, _ = L.librpa_gpu_ec(h)
    finally:
        L.librpa_gpu_destroy(h)
    assert abs(ec - ref["ec"]) < TOL_EC
    # the context is still usable by a fresh handle
    h2 = L.librpa_gpu_create()
    try:
        L.set_inputs(h2, inp, grid)
        L.librpa_gpu_chi0(h2)
        ec2, _, _ = L.librpa_gpu_ec(h2)
    finally:
        L.librpa_gpu_destroy(h2)
    assert abs(ec2 - ref["ec"]) < TOL_EC
