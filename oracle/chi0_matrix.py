"""Oracle: Python entry to the plain-C evaluation of chi0(R, tau) from the four-term matrix form of
Sec. 2 (``chi0_matrix.c``).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.oracle_chi0_matrix.restype = ctypes.c_int
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def pack_lri(lri):
    """Flatten [(I, K, R, C)] into the arrays the C routine takes."""
    blk_I = np.array([b[0] for b in lri], dtype=np.int32)
    blk_K = np.array([b[1] for b in lri], dtype=np.int32)
    blk_R = np.array([list(b[2]) for b in lri], dtype=np.int32).reshape(-1)
    sizes = [b[3].size for b in lri]
    blk_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    C = np.concatenate([np.ascontiguousarray(b[3], dtype=np.float64).reshape(-1) for b in lri])
    return blk_I, blk_K, blk_R, blk_off, C


def chi0_matrix_form(st, lri, go, gv, points, pairs=None, spin=2.0, out=None):
    """chi0(R, tau) [len(points)][N_aux][N_aux] for (iR, itau) points.

    ``pairs``: optional list of (U, V) atom pairs; only those blocks are
    computed (the rest of ``out`` is left as given, zeros by default).
    """
    lib = _load()
    n_ao = np.ascontiguousarray(st.n_ao, dtype=np.int32)
    n_aux = np.ascontiguousarray(st.n_aux, dtype=np.int32)
    kmesh = np.array(st.kmesh, dtype=np.int32)
    blk_I, blk_K, blk_R, blk_off, C = pack_lri(lri)
    go = np.ascontiguousarray(go, dtype=np.float64)
    gv = np.ascontiguousarray(gv, dtype=np.float64)
    pts = np.ascontiguousarray(np.array(points, dtype=np.int32).reshape(-1))
    npts = len(pts) // 2
    naux = int(n_aux.sum())
    if out is None:
        out = np.zeros((npts, naux, naux))
    if pairs is None:
        pr = np.zeros(2, dtype=np.int32)
        npairs = 0
    else:
        pr = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1))
        npairs = len(pr) // 2
    rc = lib.oracle_chi0_matrix(
        ctypes.c_int(st.natoms), _ptr(n_ao, ctypes.c_int), _ptr(n_aux, ctypes.c_int),
        _ptr(kmesh, ctypes.c_int), ctypes.c_int(len(lri)), _ptr(blk_I, ctypes.c_int),
        _ptr(blk_K, ctypes.c_int), _ptr(blk_R, ctypes.c_int), _ptr(blk_off, ctypes.c_long),
        _ptr(C, ctypes.c_double), ctypes.c_int(go.shape[0]), _ptr(go, ctypes.c_double),
        _ptr(gv, ctypes.c_double), ctypes.c_double(spin), ctypes.c_int(npts),
        _ptr(pts, ctypes.c_int), ctypes.c_int(npairs), _ptr(pr, ctypes.c_int),
        _ptr(out, ctypes.c_double))
    if rc != 0:
        raise RuntimeError("oracle_chi0_matrix failed: %d" % rc)
    return out
