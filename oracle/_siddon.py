"""ORACLE (test infrastructure): FP64 Siddon system matrix via the plain-C tracer.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siddon.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# -ffp-contract=off: no fused multiply-add, every operation rounds on its own
# (gcc contracts by default on aarch64).  OpenMP spreads the ray-by-ray
# projections (forward, adjoint) over the host cores.
CFLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the C tracer into oracle/liboracle.so (plain gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.orc_trace_ray.restype = ctypes.c_int64
        L.orc_trace_ray.argtypes = [P, P, ctypes.c_int, P, P]
        L.orc_siddon_count.restype = ctypes.c_int64
        L.orc_siddon_count.argtypes = [ctypes.c_int] * 5 + [P, P]
        L.orc_siddon_fill.restype = None
        L.orc_siddon_fill.argtypes = [ctypes.c_int] * 5 + [P, P, P, P]
        L.orc_siddon_row.restype = ctypes.c_int64
        L.orc_siddon_row.argtypes = [ctypes.c_int] * 4 + [P, ctypes.c_int64, P, P]
        L.orc_forward.restype = None
        L.orc_forward.argtypes = [ctypes.c_int] * 5 + [P, P, P]
        L.orc_adjoint.restype = None
        L.orc_adjoint.argtypes = [ctypes.c_int] * 5 + [P, P, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def trace_ray(s, c, n: int):
    """(cols int32, lengths float64) of the ray from s to c in traversal order."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    cols = np.zeros(3 * n + 4, dtype=np.int32)
    vals = np.zeros(3 * n + 4, dtype=np.float64)
    k = lib().orc_trace_ray(_ptr(s), _ptr(c), n, _ptr(cols), _ptr(vals))
    return cols[:k].copy(), vals[:k].copy()


def system_matrix(geom) -> sp.csr_matrix:
    """A (m x N, FP64 CSR, rows in traversal order) for a synth.Geometry."""
    views = np.ascontiguousarray(geom.views, dtype=np.float64)
    m, N = geom.m, geom.N
    counts = np.zeros(m, dtype=np.int64)
    L = lib()
    nnz = L.orc_siddon_count(geom.n, geom.n_views, geom.det_cols, geom.det_rows, geom.kind,
                             _ptr(views), _ptr(counts))
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    assert row_ptr[-1] == nnz
    cols = np.zeros(nnz, dtype=np.int32)
    vals = np.zeros(nnz, dtype=np.float64)
    L.orc_siddon_fill(geom.n, geom.n_views, geom.det_cols, geom.det_rows, geom.kind,
                      _ptr(views), _ptr(row_ptr), _ptr(cols), _ptr(vals))
    # scipy keeps the given order (no sorting, no duplicate summation)
    A = sp.csr_matrix((vals, cols, row_ptr), shape=(m, N))
    return A


def row(geom, i: int):
    """Row i of A computed on the fly (matrix-free)."""
    views = np.ascontiguousarray(geom.views, dtype=np.float64)
    n = geom.n
    cols = np.zeros(3 * n + 4, dtype=np.int32)
    vals = np.zeros(3 * n + 4, dtype=np.float64)
    k = lib().orc_siddon_row(n, geom.det_cols, geom.det_rows, geom.kind, _ptr(views), int(i),
                             _ptr(cols), _ptr(vals))
    return cols[:k].copy(), vals[:k].copy()


def forward(geom, x) -> np.ndarray:
    """A x (FP64) computed ray by ray without storing A."""
    views = np.ascontiguousarray(geom.views, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.size == geom.N
    y = np.zeros(geom.m, dtype=np.float64)
    lib().orc_forward(geom.n, geom.n_views, geom.det_cols, geom.det_rows, geom.kind, _ptr(views),
                      _ptr(x), _ptr(y))
    return y


def adjoint(geom, r) -> np.ndarray:
    """A^T r (FP64) computed ray by ray without storing A."""
    views = np.ascontiguousarray(geom.views, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    assert r.size == geom.m
    z = np.zeros(geom.N, dtype=np.float64)
    lib().orc_adjoint(geom.n, geom.n_views, geom.det_cols, geom.det_rows, geom.kind, _ptr(views),
                      _ptr(r), _ptr(z))
    return z
