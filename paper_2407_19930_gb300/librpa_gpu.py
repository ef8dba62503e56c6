"""Python binding of the librpa_gpu C ABI (include/librpa_gpu.h).

Argument marshalling only: every function has the name of the C entry point it
calls, converts numpy arrays to the pointers and sizes the C ABI takes, and
raises ``LibrpaError`` on a non-zero status.  All computation runs in the CUDA
library; there is no Python or CPU fallback, and importing this module without
a built library fails loudly.

PyTorch, when given, supplies the device memory (its caching allocator through
the allocator hooks) and the stream the library runs on.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LIBRPA_OK = 0
LIBRPA_E_ARG = -1
LIBRPA_E_STATE = -2
LIBRPA_E_NOMEM = -3
LIBRPA_E_CUDA = -4
LIBRPA_E_NOT_PD = -5
LIBRPA_E_TIMEOUT = -6
LIBRPA_E_NUMERIC = -7
LIBRPA_FP64 = 0
LIBRPA_FP64_TC = 1
LIBRPA_SPLIT = 2
LIBRPA_BF16 = 3
LIBRPA_TF32 = 4
LIBRPA_TF32X3 = 5
LIBRPA_SPLIT_FAST = 6
LIBRPA_GRID_MINIMAX = 0
LIBRPA_GRID_GAUSS_LEGENDRE = 1
LIBRPA_NOALLOC_SCRATCH_BYTES = 16 << 20
LIBRPA_NOALLOC_MAX_NAUX = 591

_CODES = {v: k for k, v in globals().items() if k.startswith("LIBRPA_E_")}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class librpa_gpu_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("dev_alloc", ALLOC_FN),
                ("dev_free", FREE_FN), ("alloc_ctx", ctypes.c_void_p), ("n_tau", ctypes.c_int),
                ("precision", ctypes.c_int), ("hbm_budget", ctypes.c_size_t), ("check_level", ctypes.c_int),
                ("chi0_slices", ctypes.c_int), ("ec_slices", ctypes.c_int), ("test_stall_gemms", ctypes.c_int),
                ("grid_kind", ctypes.c_int)]


class librpa_gpu_stats(ctypes.Structure):
    _fields_ = [("ms_green", ctypes.c_double), ("ms_chi0", ctypes.c_double), ("ms_freq", ctypes.c_double),
                ("ms_ec", ctypes.c_double), ("flop_chi0", ctypes.c_double), ("flop_ec", ctypes.c_double),
                ("ms_gemm_chi0", ctypes.c_double), ("flop_gemm_chi0", ctypes.c_double),
                ("n_gemm_chi0", ctypes.c_longlong), ("ms_gemm_ec", ctypes.c_double),
                ("flop_gemm_ec", ctypes.c_double), ("n_gemm_ec", ctypes.c_longlong),
                ("launches", ctypes.c_longlong),
                ("bytes_device", ctypes.c_size_t), ("flop_exec_gemm_chi0", ctypes.c_double),
                ("flop_exec_gemm_ec", ctypes.c_double), ("bytes_device_peak", ctypes.c_size_t),
                ("n_points_chi0", ctypes.c_longlong), ("n_points_skipped", ctypes.c_longlong),
                ("n_blocks_kept", ctypes.c_longlong), ("n_blocks_total", ctypes.c_longlong)]


class librpa_gpu_server_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("slots", ctypes.c_int), ("hbm_budget", ctypes.c_size_t)]


class librpa_gpu_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("ec", ctypes.c_double), ("ms_queue", ctypes.c_double),
                ("ms_run", ctypes.c_double), ("ms_total", ctypes.c_double), ("bytes_reserved", ctypes.c_size_t),
                ("bytes_peak", ctypes.c_size_t), ("slot", ctypes.c_int)]


class librpa_gpu_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_queue_ms", ctypes.c_double),
                ("energies_per_s", ctypes.c_double), ("peak_running", ctypes.c_int),
                ("peak_reserved", ctypes.c_size_t), ("hbm_budget", ctypes.c_size_t)]


class librpa_gpu_batch_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_merged", ctypes.c_int), ("graph", ctypes.c_int), ("var_nx", ctypes.c_int),
                ("var_fin", ctypes.c_int), ("failed_index", ctypes.c_int), ("ms_green", ctypes.c_double),
                ("ms_chi0", ctypes.c_double), ("ms_freq", ctypes.c_double), ("ms_ec", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("launches", ctypes.c_longlong), ("n_merged_tc", ctypes.c_int)]


class LibrpaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_CODES.get(code, "?"), code, msg))
        self.code = code


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_H = ctypes.c_void_p

_SIGS = {
    "librpa_gpu_default_opts": (None, [ctypes.POINTER(librpa_gpu_opts)]),
    "librpa_gpu_create": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.POINTER(librpa_gpu_opts)]),
    "librpa_gpu_set_structure": (ctypes.c_int, [_H, ctypes.c_int, _D, _D, _I, _I, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_double]),
    "librpa_gpu_set_lri_coeffs": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, _I, _D]),
    "librpa_gpu_set_green": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D,
                                            ctypes.c_double]),
    "librpa_gpu_set_coulomb": (ctypes.c_int, [_H, ctypes.c_int, _D, _D]),
    "librpa_gpu_set_grid": (ctypes.c_int, [_H, ctypes.c_int, _D, ctypes.c_int, _D, _D, _D]),
    "librpa_gpu_set_screening": (ctypes.c_int, [_H, ctypes.c_double]),
    "librpa_gpu_set_q_weights": (ctypes.c_int, [_H, _D]),
    "librpa_gpu_build_grid": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D]),
    "librpa_gpu_build_grid_minimax": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D,
                                                     _D]),
    "librpa_gpu_get_grid": (ctypes.c_int, [_H, _I, _D, _D, _D, _D]),
    "librpa_gpu_chi0": (ctypes.c_int, [_H, _D, _D]),
    "librpa_gpu_ec": (ctypes.c_int, [_H, _D, _D, _D]),
    "librpa_gpu_get_green": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, _D, _D]),
    "librpa_gpu_get_chi0_tau": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, _D]),
    "librpa_gpu_get_chi0_freq": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, _D, _D]),
    "librpa_gpu_get_stats": (ctypes.c_int, [_H, ctypes.POINTER(librpa_gpu_stats)]),
    "librpa_gpu_last_error": (ctypes.c_char_p, [_H]),
    "librpa_gpu_estimate_bytes": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_size_t)]),
    "librpa_gpu_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p),
                                                ctypes.POINTER(librpa_gpu_server_opts)]),
    "librpa_gpu_server_request": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(librpa_gpu_opts),
                                                 ctypes.POINTER(_H)]),
    "librpa_gpu_server_submit": (ctypes.c_int, [ctypes.c_void_p, _H, ctypes.POINTER(ctypes.c_longlong)]),
    "librpa_gpu_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double,
                                              ctypes.POINTER(librpa_gpu_result)]),
    "librpa_gpu_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(librpa_gpu_server_stats)]),
    "librpa_gpu_server_destroy": (None, [ctypes.c_void_p]),
    "librpa_gpu_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_H), ctypes.c_int]),
    "librpa_gpu_batch_run": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "librpa_gpu_batch_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(librpa_gpu_batch_stats)]),
    "librpa_gpu_batch_destroy": (None, [ctypes.c_void_p]),
    "librpa_gpu_set_green_dev": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                                ctypes.c_void_p, ctypes.c_double]),
    "librpa_gpu_set_coulomb_dev": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p]),
    "librpa_gpu_get_chi0_freq_dev": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "librpa_gpu_ec_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "librpa_gpu_destroy": (None, [_H]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the shared library (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("librpa_gpu.so is not built (run paper_2407_19930_gb300.build.build())")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(h, rc):
    if rc != LIBRPA_OK:
        msg = load().librpa_gpu_last_error(h) if h else b""
        raise LibrpaError(rc, (msg or b"").decode())


# ---------------------------------------------------------------- allocator hooks from torch

class _TorchHooks:
    """Device allocations from torch's caching allocator on a given stream."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream

        def alloc(nbytes, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=self.stream))
            except Exception:
                return None

        def free(ptr, ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


_keepalive = {}


def librpa_gpu_default_opts():
    o = librpa_gpu_opts()
    load().librpa_gpu_default_opts(ctypes.byref(o))
    return o


def librpa_gpu_create(opts=None, torch_stream=None, torch_alloc=False):
    """Create a handle.  ``torch_stream``: a torch.cuda.Stream to run on;
    ``torch_alloc``: take device memory from torch's caching allocator."""
    o = opts if opts is not None else librpa_gpu_default_opts()
    hooks = None
    if torch_stream is not None:
        o.stream = ctypes.c_void_p(torch_stream.cuda_stream)
    if torch_alloc:
        import torch
        stream = torch_stream if torch_stream is not None else torch.cuda.current_stream(o.device)
        hooks = _TorchHooks(o.device, stream)
        o.dev_alloc = hooks.alloc
        o.dev_free = hooks.free
    h = _H()
    rc = load().librpa_gpu_create(ctypes.byref(h), ctypes.byref(o))
    _check(None, rc)
    _keepalive[h.value] = (o, hooks)
    return h


def librpa_gpu_set_structure(h, lat, pos, n_ao, n_aux, kmesh, nspins=1, r_cut=6.0):
    lat = _f64(np.asarray(lat).reshape(9))
    pos = _f64(np.asarray(pos).reshape(-1, 3))
    nao = np.ascontiguousarray(n_ao, dtype=np.int32)
    naux = np.ascontiguousarray(n_aux, dtype=np.int32)
    _check(h, load().librpa_gpu_set_structure(h, len(nao), _dp(lat), _dp(pos), nao.ctypes.data_as(_I),
                                              naux.ctypes.data_as(_I), int(kmesh[0]), int(kmesh[1]),
                                              int(kmesh[2]), int(nspins), float(r_cut)))


def librpa_gpu_set_lri_coeffs(h, I, K, R, C):
    r = np.ascontiguousarray(R, dtype=np.int32)
    c = _f64(C)
    _check(h, load().librpa_gpu_set_lri_coeffs(h, int(I), int(K), r.ctypes.data_as(_I), _dp(c)))


def librpa_gpu_set_green(h, ispin, ik, eig, occ, wfc, efermi):
    """``wfc``: complex [nbands][n_ao_total] with wfc[n][i] = c_{i n}(k)."""
    eig = _f64(eig)
    occ = _f64(occ)
    wfc = np.asarray(wfc)
    wre = _f64(wfc.real)
    wim = _f64(wfc.imag)
    _check(h, load().librpa_gpu_set_green(h, int(ispin), int(ik), len(eig), _dp(eig), _dp(occ), _dp(wre),
                                          _dp(wim), float(efermi)))


def librpa_gpu_set_coulomb(h, iq, V):
    V = np.asarray(V)
    _check(h, load().librpa_gpu_set_coulomb(h, int(iq), _dp(_f64(V.real)), _dp(_f64(V.imag))))


def librpa_gpu_set_grid(h, tau, omega, w_omega, gamma):
    tau, omega, w_omega, gamma = _f64(tau), _f64(omega), _f64(w_omega), _f64(gamma)
    _check(h, load().librpa_gpu_set_grid(h, len(tau), _dp(tau), len(omega), _dp(omega), _dp(w_omega),
                                         _dp(gamma)))


def librpa_gpu_set_q_weights(h, w=None):
    if w is None:
        _check(h, load().librpa_gpu_set_q_weights(h, None))
        return
    w = _f64(w)
    _check(h, load().librpa_gpu_set_q_weights(h, _dp(w)))


def librpa_gpu_set_screening(h, threshold):
    _check(h, load().librpa_gpu_set_screening(h, float(threshold)))


def librpa_gpu_build_grid(n, dmin, dmax):
    tau, omega, w = np.zeros(n), np.zeros(n), np.zeros(n)
    gamma = np.zeros((n, n))
    rc = load().librpa_gpu_build_grid(int(n), float(dmin), float(dmax), _dp(tau), _dp(omega), _dp(w), _dp(gamma))
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, "build_grid")
    return dict(tau=tau, omega=omega, w_omega=w, gamma=gamma)


def librpa_gpu_build_grid_minimax(n, dmin, dmax):
    tau, omega, w = np.zeros(n), np.zeros(n), np.zeros(n)
    gamma, info = np.zeros((n, n)), np.zeros(3)
    rc = load().librpa_gpu_build_grid_minimax(int(n), float(dmin), float(dmax), _dp(tau), _dp(omega), _dp(w),
                                              _dp(gamma), _dp(info))
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, "build_grid_minimax")
    return dict(tau=tau, omega=omega, w_omega=w, gamma=gamma, r_eff=float(info[0]), err_tau=float(info[1]),
                err_omega=float(info[2]))


def librpa_gpu_get_grid(h):
    n = ctypes.c_int(0)
    _check(h, load().librpa_gpu_get_grid(h, ctypes.byref(n), None, None, None, None))
    n = n.value
    tau, omega, w, gamma = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros((n, n))
    nn = ctypes.c_int(0)
    _check(h, load().librpa_gpu_get_grid(h, ctypes.byref(nn), _dp(tau), _dp(omega), _dp(w), _dp(gamma)))
    return dict(tau=tau, omega=omega, w_omega=w, gamma=gamma)


def librpa_gpu_chi0(h, out=None):
    """Runs the response-function stage.  With ``out=(nq, nomega, naux)`` returns
    chi0(q, i omega) as a complex array of that shape (host copy)."""
    if out is None:
        _check(h, load().librpa_gpu_chi0(h, None, None))
        return None
    nq, nw, n = out
    re = np.zeros((nq, nw, n, n))
    im = np.zeros((nq, nw, n, n))
    _check(h, load().librpa_gpu_chi0(h, _dp(re), _dp(im)))
    return re + 1j * im


def librpa_gpu_ec(h, nq=None, nomega=None):
    """Returns (E_c, per-q [nq] or None, per-omega [nomega] or None)."""
    ec = ctypes.c_double(0.0)
    eq = np.zeros(nq) if nq else None
    ew = np.zeros(nomega) if nomega else None
    _check(h, load().librpa_gpu_ec(h, ctypes.byref(ec), _dp(eq), _dp(ew)))
    return ec.value, eq, ew


def librpa_gpu_get_green(h, itau, iR, nao):
    go, gv = np.zeros((nao, nao)), np.zeros((nao, nao))
    _check(h, load().librpa_gpu_get_green(h, int(itau), int(iR), _dp(go), _dp(gv)))
    return go, gv


def librpa_gpu_get_chi0_tau(h, itau, iR, naux):
    out = np.zeros((naux, naux))
    _check(h, load().librpa_gpu_get_chi0_tau(h, int(itau), int(iR), _dp(out)))
    return out


def librpa_gpu_get_chi0_freq(h, iq, iw, naux):
    re, im = np.zeros((naux, naux)), np.zeros((naux, naux))
    _check(h, load().librpa_gpu_get_chi0_freq(h, int(iq), int(iw), _dp(re), _dp(im)))
    return re + 1j * im


def librpa_gpu_set_green_dev(h, ispin, ik, eig, occ, wfc_ptr, efermi):
    """wfc_ptr: device address of [nbands][n_ao] complex128 (e.g. tensor.data_ptr())."""
    eig, occ = _f64(eig), _f64(occ)
    _check(h, load().librpa_gpu_set_green_dev(h, int(ispin), int(ik), len(eig), _dp(eig), _dp(occ), wfc_ptr,
                                              float(efermi)))


def librpa_gpu_set_coulomb_dev(h, iq, v_ptr):
    _check(h, load().librpa_gpu_set_coulomb_dev(h, int(iq), v_ptr))


def librpa_gpu_get_chi0_freq_dev(h, iq, iw, out_ptr):
    _check(h, load().librpa_gpu_get_chi0_freq_dev(h, int(iq), int(iw), out_ptr))


def librpa_gpu_get_stats(h):
    s = librpa_gpu_stats()
    _check(h, load().librpa_gpu_get_stats(h, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in s._fields_}


def librpa_gpu_last_error(h):
    return (load().librpa_gpu_last_error(h) or b"").decode()


def librpa_gpu_ec_noalloc(naux, nomega, V, chi, out, stream=None):
    """ln det(1 - chi_k V) + Re Tr(chi_k V) for k < nomega into ``out`` (device pointers as
    ints: V [naux][naux] and chi [nomega][naux][naux] complex interleaved, out [nomega] doubles),
    enqueued on ``stream`` (a cudaStream_t as int, or None); nothing is allocated."""
    msg = ctypes.create_string_buffer(256)
    rc = load().librpa_gpu_ec_noalloc(int(naux), int(nomega), V, chi, out, stream, msg, len(msg))
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, msg.value.decode())


def librpa_gpu_batch_create(handles):
    arr = (_H * len(handles))(*[h.value if hasattr(h, "value") else h for h in handles])
    b = ctypes.c_void_p()
    rc = load().librpa_gpu_batch_create(ctypes.byref(b), arr, len(handles))
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, "batch_create")
    b._handles = list(handles)
    return b


def librpa_gpu_batch_run(b):
    """E_c of every handle of the batch (numpy array)."""
    ec = np.zeros(len(b._handles))
    rc = load().librpa_gpu_batch_run(b, _dp(ec))
    if rc != LIBRPA_OK:
        st = librpa_gpu_batch_get_stats(b)
        i = st["failed_index"]
        msg = librpa_gpu_last_error(b._handles[i]) if i >= 0 else ""
        raise LibrpaError(rc, "batch handle %d: %s" % (i, msg))
    return ec


def librpa_gpu_batch_get_stats(b):
    st = librpa_gpu_batch_stats()
    rc = load().librpa_gpu_batch_get_stats(b, ctypes.byref(st))
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, "batch_get_stats")
    return {f: getattr(st, f) for f, _ in st._fields_}


def librpa_gpu_batch_destroy(b):
    if b:
        load().librpa_gpu_batch_destroy(b)


def librpa_gpu_estimate_bytes(h):
    b = ctypes.c_size_t(0)
    _check(h, load().librpa_gpu_estimate_bytes(h, ctypes.byref(b)))
    return b.value


def librpa_gpu_server_create(device=0, slots=2, hbm_budget=0):
    o = librpa_gpu_server_opts(device, slots, hbm_budget)
    s = ctypes.c_void_p()
    rc = load().librpa_gpu_server_create(ctypes.byref(s), ctypes.byref(o))
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, "server_create")
    return s


def librpa_gpu_server_request(s, opts=None):
    """A request handle; fill it with the set_* calls (or set_inputs) and submit it."""
    if opts is None:
        opts = librpa_gpu_default_opts()
    h = _H()
    rc = load().librpa_gpu_server_request(s, ctypes.byref(opts), ctypes.byref(h))
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, "server_request")
    return h


def librpa_gpu_server_submit(s, req):
    t = ctypes.c_longlong(0)
    _check(req, load().librpa_gpu_server_submit(s, req, ctypes.byref(t)))
    return t.value


def librpa_gpu_server_wait(s, ticket, timeout_s=-1.0):
    """Returns the result as a dict, or None if it is not ready within timeout_s."""
    r = librpa_gpu_result()
    rc = load().librpa_gpu_server_wait(s, int(ticket), float(timeout_s), ctypes.byref(r))
    if rc == LIBRPA_E_TIMEOUT:
        return None
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, "server_wait")
    return {f: getattr(r, f) for f, _ in r._fields_}


def librpa_gpu_server_get_stats(s):
    st = librpa_gpu_server_stats()
    rc = load().librpa_gpu_server_get_stats(s, ctypes.byref(st))
    if rc != LIBRPA_OK:
        raise LibrpaError(rc, "server_get_stats")
    return {f: getattr(st, f) for f, _ in st._fields_}


def librpa_gpu_server_destroy(s):
    if s:
        load().librpa_gpu_server_destroy(s)


def librpa_gpu_destroy(h):
    if h:
        load().librpa_gpu_destroy(h)
        _keepalive.pop(h.value if hasattr(h, "value") else h, None)


# ---------------------------------------------------------------- convenience


def set_inputs(h, inp, grid=None):
    """Pass every input of a ``synthetic.Inputs`` request through the C ABI."""
    st = inp.st
    librpa_gpu_set_structure(h, st.lat, st.pos, st.n_ao, st.n_aux, st.kmesh, st.nspins, st.r_cut)
    for I, K, R, C in inp.lri:
        librpa_gpu_set_lri_coeffs(h, I, K, R, C)
    for isp, (eig, occ, wfc) in enumerate(inp.channels()):
        for ik in range(st.nk):
            librpa_gpu_set_green(h, isp, ik, eig[ik], occ[ik], wfc[ik], inp.efermi)
    for iq in range(st.nk):
        librpa_gpu_set_coulomb(h, iq, inp.vq[iq])
    if grid is not None:
        librpa_gpu_set_grid(h, grid["tau"], grid["omega"], grid["w_omega"], grid["gamma"])
