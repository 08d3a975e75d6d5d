"""Python front end of the CPU brute-force FRNN oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this module.  The library's product path never does: it runs
the CUDA kernels or fails.

The arithmetic lives in ``frnn_oracle.c`` (plain C, compiled here with gcc,
``-O2 -ffp-contract=off``, no fast-math).  This module only compiles it,
marshals NumPy arrays and returns NumPy arrays.  What the oracle computes is
the paper's Eq. 1 (Sec. 1) by brute force; see the C file's header for the
readings it takes where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "frnn_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

# The FP32 contract depends on these flags: no FMA contraction, no fast-math.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
          "-ffp-contract=off", "-fno-fast-math", "-fno-unsafe-math-optimizations"]

_lock = threading.Lock()
_lib = None
_lib_path = None   # set only by use_library()


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source if it is missing or stale."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def use_library(path: str) -> None:
    """Load the checker from ``path`` instead of building this file.  Only the
    test of the pins calls it (through pytest's ``--oracle-lib`` option), to
    run the pins against a copy of the oracle with one mistake planted; it must
    be called before the first oracle call of the process."""
    global _lib_path
    with _lock:
        if _lib is not None:
            raise RuntimeError("the oracle library is already loaded")
        _lib_path = path


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_lib_path or build())
            i64, f32p = ctypes.c_int64, ctypes.c_void_p
            lib.frnn_oracle_query.argtypes = [f32p, f32p, i64, f32p, i64, ctypes.c_int,
                                              ctypes.c_float, ctypes.c_int,
                                              f32p, f32p, f32p, f32p]
            lib.frnn_oracle_query.restype = ctypes.c_int
            lib.frnn_oracle_degree.argtypes = [f32p, f32p, i64, f32p, i64, ctypes.c_int,
                                               ctypes.c_float, f32p]
            lib.frnn_oracle_degree.restype = ctypes.c_int
            lib.frnn_oracle_fp64_audit.argtypes = [f32p, f32p, i64, f32p, i64, ctypes.c_int,
                                                   ctypes.c_float, f32p, f32p]
            lib.frnn_oracle_fp64_audit.restype = ctypes.c_int64
            lib.frnn_oracle_num_threads.argtypes = []
            lib.frnn_oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(queries, refs, query_ids):
    q = np.ascontiguousarray(queries, dtype=np.float32)
    p = np.ascontiguousarray(refs, dtype=np.float32)
    if q.ndim != 2 or p.ndim != 2 or q.shape[1] != p.shape[1]:
        raise ValueError("queries [M,D] and refs [N,D] must share D")
    ids = None
    if query_ids is not None:
        ids = np.ascontiguousarray(query_ids, dtype=np.int64)
        if ids.shape != (q.shape[0],):
            raise ValueError("query_ids must have shape [M]")
    return q, p, ids


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use (OMP_NUM_THREADS or all cores)."""
    return int(_load().frnn_oracle_num_threads())


def frnn(queries, refs, r: float, K: int, query_ids=None):
    """Brute-force FRNN under the FP32 contract.

    ``query_ids`` gives each query's own index in ``refs`` (self-query: that
    reference is excluded by index); ``None`` means distinct sets.
    Returns ``counts [M] int32, idx [M,K] int32, dist2 [M,K] float32,
    degree [M] int64``.
    """
    q, p, ids = _prep(queries, refs, query_ids)
    M, D = q.shape
    N = p.shape[0]
    counts = np.empty(M, np.int32)
    idx = np.empty((M, K), np.int32)
    dist2 = np.empty((M, K), np.float32)
    degree = np.empty(M, np.int64)
    rc = _load().frnn_oracle_query(_ptr(q), _ptr(ids), M, _ptr(p), N, D,
                                   ctypes.c_float(r), int(K), _ptr(counts), _ptr(idx),
                                   _ptr(dist2), _ptr(degree))
    if rc != 0:
        raise RuntimeError("oracle frnn failed")
    return counts, idx, dist2, degree


def self_query(points, r: float, K: int, rows=None):
    """Self-query of ``points`` against itself; ``rows`` selects a subset of
    query rows (their own index is excluded), default all rows."""
    pts = np.ascontiguousarray(points, dtype=np.float32)
    if rows is None:
        rows = np.arange(pts.shape[0], dtype=np.int64)
    rows = np.asarray(rows, dtype=np.int64)
    return frnn(pts[rows], pts, r, K, query_ids=rows)


def csr(queries, refs, r: float, K: int, query_ids=None):
    """Compact (CSR) form of ``frnn``'s result: row i holds its first
    counts[i] = min(degree_i, K) entries, rows back to back (the paper's
    count-first exact allocation, Sec. 4).  Returns ``offsets [M+1] int64,
    idx [E] int32, dist2 [E] float32, degree [M] int64``."""
    counts, idx, dist2, deg = frnn(queries, refs, r, K, query_ids)
    offsets = np.zeros(len(counts) + 1, np.int64)
    offsets[1:] = np.cumsum(counts, dtype=np.int64)
    keep = np.arange(idx.shape[1])[None, :] < counts[:, None]
    return offsets, idx[keep], dist2[keep], deg


def degree(queries, refs, r: float, query_ids=None):
    """Untruncated degree under the FP32 contract (no sorting)."""
    q, p, ids = _prep(queries, refs, query_ids)
    out = np.empty(q.shape[0], np.int64)
    rc = _load().frnn_oracle_degree(_ptr(q), _ptr(ids), q.shape[0], _ptr(p), p.shape[0],
                                    q.shape[1], ctypes.c_float(r), _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle degree failed")
    return out


def fp64_audit(queries, refs, r: float, query_ids=None):
    """Pairs whose FP32-contract verdict differs from the FP64 verdict.

    Returns ``(crossings, only_fp32, only_fp64)``.
    """
    q, p, ids = _prep(queries, refs, query_ids)
    a32 = ctypes.c_int64(0)
    a64 = ctypes.c_int64(0)
    tot = _load().frnn_oracle_fp64_audit(_ptr(q), _ptr(ids), q.shape[0], _ptr(p), p.shape[0],
                                         q.shape[1], ctypes.c_float(r),
                                         ctypes.byref(a32), ctypes.byref(a64))
    if tot < 0:
        raise RuntimeError("oracle audit failed")
    return int(tot), int(a32.value), int(a64.value)
