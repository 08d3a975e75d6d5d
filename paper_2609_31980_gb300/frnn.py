"""Thin ctypes binding of libfrnn (include/frnn.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  If libfrnn.so is missing the import of this module fails:
there is no other implementation to fall back on.

Low-level functions carry the C names (``frnn_create``, ``frnn_build_grid``,
``frnn_query``, ``frnn_query_batched``, ``frnn_sync`` ...); ``Context`` wraps
them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfrnn.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libfrnn.so not built ({LIB_PATH}); run "
                      "`python -m paper_2609_31980_gb300.build` (needs nvcc)")

_lib = ctypes.CDLL(LIB_PATH)

FRNN_OK = 0
STATUS_NAMES = {
    0: "FRNN_OK", -1: "FRNN_ERR_INVALID_ARG", -2: "FRNN_ERR_UNSUPPORTED",
    -3: "FRNN_ERR_OUT_OF_MEMORY", -4: "FRNN_ERR_BUDGET", -5: "FRNN_ERR_NONFINITE",
    -6: "FRNN_ERR_CUDA", -7: "FRNN_ERR_TIMEOUT", -8: "FRNN_ERR_CAPACITY",
}
FRNN_SELF_QUERY = 0x1
FRNN_PATH_AUTO = 0x0
FRNN_PATH_GRID = 0x2
FRNN_PATH_TC = 0x4
PATHS = {"auto": FRNN_PATH_AUTO, "grid": FRNN_PATH_GRID, "tc": FRNN_PATH_TC}

FRNN_OPT_CELL_MULT = 1
FRNN_OPT_GRID_AXES = 2
FRNN_OPT_EXIT_DIMS = 3
FRNN_OPT_USE_GRAPH = 4
FRNN_OPT_AUTOTUNE = 5
FRNN_OPT_AUTO_TC = 6
FRNN_OPT_TC_SURVIVORS = 7
FRNN_OPT_TC_ACCEPTED = 8
FRNN_OPT_KERNEL_TIMING = 9
FRNN_ERR_CAPACITY = -8
FRNN_ERR_TIMEOUT = -7
FRNN_ERR_INVALID_ARG = -1
FRNN_OPT_GRID_NAXES = 10
FRNN_OPT_STAGING = 11

EXPORTED = ["frnn_version", "frnn_create", "frnn_destroy", "frnn_build_grid",
            "frnn_grid_destroy", "frnn_query", "frnn_query_batched", "frnn_self_query_host",
            "frnn_sync", "frnn_last_error", "frnn_set_option", "frnn_get_option",
            "frnn_autotune", "frnn_serve_run", "frnn_self_query_noalloc",
            "frnn_kernel_times", "frnn_query_csr_count", "frnn_query_csr_fill",
            "frnn_self_query_host_csr", "frnn_check_wait_timeout", "frnn_grid_params"]


class frnn_tune_result(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("cell_mult", ctypes.c_int), ("exit_dims", ctypes.c_int),
                ("ms", ctypes.c_float), ("grid_axes", ctypes.c_int), ("staging", ctypes.c_int)]


class frnn_grid_info(ctypes.Structure):
    _fields_ = [("naxes", ctypes.c_int), ("cell_mult", ctypes.c_int), ("axes", ctypes.c_int * 5),
                ("dims", ctypes.c_int * 5), ("cell_edge", ctypes.c_float), ("cells", ctypes.c_int64),
                ("kernel", ctypes.c_int), ("valid", ctypes.c_int)]


class frnn_request(ctypes.Structure):
    _fields_ = [("pts", ctypes.c_void_p), ("n", ctypes.c_int64), ("counts", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("dist2", ctypes.c_void_p), ("arrival_s", ctypes.c_double)]


class frnn_serve_stats(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("events_per_s", ctypes.c_double),
                ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("peak_inflight_bytes", ctypes.c_int64), ("peak_inflight_batches", ctypes.c_int)]


class frnn_event(ctypes.Structure):
    _fields_ = [("pts", ctypes.c_void_p), ("n", ctypes.c_int64), ("counts", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("dist2", ctypes.c_void_p)]


_vp, _i64, _int, _f32, _u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_uint
_sigs = {
    "frnn_version": ([], ctypes.c_char_p),
    "frnn_create": ([ctypes.POINTER(_vp), _vp, ctypes.c_size_t], _int),
    "frnn_destroy": ([_vp], _int),
    "frnn_build_grid": ([_vp, _vp, _i64, _int, _f32, ctypes.POINTER(_vp)], _int),
    "frnn_grid_destroy": ([_vp], _int),
    "frnn_grid_params": ([_vp, ctypes.c_void_p], _int),
    "frnn_query": ([_vp, _vp, _vp, _i64, _f32, _int, _u32, _vp, _vp, _vp], _int),
    "frnn_query_batched": ([_vp, ctypes.POINTER(frnn_event), _int, _int, _f32, _int, _u32], _int),
    "frnn_self_query_host": ([_vp, _vp, _i64, _int, _f32, _int, _u32, _vp, _vp, _vp], _int),
    "frnn_sync": ([_vp], _int),
    "frnn_last_error": ([_vp], ctypes.c_char_p),
    "frnn_set_option": ([_vp, _int, _i64], _int),
    "frnn_get_option": ([_vp, _int, ctypes.POINTER(_i64)], _int),
    "frnn_kernel_times": ([_vp, ctypes.POINTER(_f32), _int, ctypes.POINTER(_int)], _int),
    "frnn_query_csr_count": ([_vp, _vp, _vp, _i64, _f32, _int, _u32, _vp, _vp,
                              ctypes.POINTER(_i64)], _int),
    "frnn_query_csr_fill": ([_vp, _vp, _vp], _int),
    "frnn_check_wait_timeout": ([_vp, ctypes.c_uint64], _int),
    "frnn_self_query_host_csr": ([_vp, _vp, _i64, _int, _f32, _int, _u32, _vp, _vp, _vp, _i64,
                                  ctypes.POINTER(_i64)], _int),
    "frnn_autotune": ([_vp, _vp, _i64, _int, _f32, _int, _u32, ctypes.POINTER(frnn_tune_result)],
                      _int),
    "frnn_self_query_noalloc": ([_vp, _i64, _int, _f32, _int, _vp, _vp, _vp, _vp], _int),
    "frnn_serve_run": ([_vp, ctypes.POINTER(frnn_request), _int, _int, _f32, _int, ctypes.c_size_t,
                        _int, _int, ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(frnn_serve_stats)], _int),
}
for _name, (_args, _res) in _sigs.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res
    globals()[_name] = _fn


class FrnnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(ctx, status: int):
    if status != FRNN_OK:
        msg = frnn_last_error(ctx)
        raise FrnnError(status, msg.decode() if msg else "")


def version() -> str:
    return frnn_version().decode()


def _torch():
    import torch
    return torch


def _dev_f32(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or t.dim() != 2 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 [N, D] tensor")
    return t


class Grid:
    """A built grid (owns the library's frnn_grid)."""

    def __init__(self, ctx: "Context", handle, points, r: float):
        self.ctx = ctx
        self.handle = handle
        self.points = points   # keeps the caller's tensor alive for self-queries
        self.r = r

    def params(self) -> dict:
        """frnn_grid_params: the parameters the build gave this grid."""
        info = frnn_grid_info()
        _check(self.ctx.handle, frnn_grid_params(self.handle, ctypes.byref(info)))
        n = info.naxes
        return {"naxes": n, "cell_mult": info.cell_mult, "axes": list(info.axes)[:n],
                "dims": list(info.dims)[:n], "cell_edge": info.cell_edge, "cells": info.cells,
                "kernel": "rows" if info.kernel == 1 else "chunks", "valid": bool(info.valid)}

    def close(self):
        if self.handle:
            frnn_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A library context bound to a CUDA stream (default: torch's current)."""

    def __init__(self, stream=None, budget_bytes: int = 0):
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _vp()
        rc = frnn_create(ctypes.byref(h), _vp(stream.cuda_stream), budget_bytes)
        _check(None, rc)
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            frnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, opt: int, value: int):
        _check(self.handle, frnn_set_option(self.handle, opt, int(value)))

    def get_option(self, opt: int) -> int:
        v = _i64(0)
        _check(self.handle, frnn_get_option(self.handle, opt, ctypes.byref(v)))
        return int(v.value)

    def build_grid(self, points, r: float, grid: Grid | None = None) -> Grid:
        """frnn_build_grid on a [N, D] float32 CUDA tensor (rebuilds ``grid``
        in place when given and large enough)."""
        _dev_f32(points, "points")
        old = grid.handle.value if (grid is not None and grid.handle) else None
        h = _vp(old)
        rc = frnn_build_grid(self.handle, _vp(points.data_ptr()), points.shape[0],
                             points.shape[1], float(r), ctypes.byref(h))
        _check(self.handle, rc)
        if old is not None and h.value == old:
            grid.points, grid.r = points, r
            return grid
        return Grid(self, h, points, r)

    def query(self, grid: Grid, queries, r: float, K: int, self_query: bool = True,
              path: str = "auto", out=None):
        """frnn_query; returns (counts [M] int32, idx [M,K] int32, dist2 [M,K] f32)."""
        torch = _torch()
        _dev_f32(queries, "queries")
        M = queries.shape[0]
        if out is None:
            dev = queries.device
            out = (torch.empty(M, dtype=torch.int32, device=dev),
                   torch.empty((M, K), dtype=torch.int32, device=dev),
                   torch.empty((M, K), dtype=torch.float32, device=dev))
        counts, idx, dist2 = out
        flags = PATHS[path] | (FRNN_SELF_QUERY if self_query else 0)
        rc = frnn_query(self.handle, grid.handle, _vp(queries.data_ptr()), M, float(r), int(K),
                        flags, _vp(counts.data_ptr()), _vp(idx.data_ptr()),
                        _vp(dist2.data_ptr()))
        _check(self.handle, rc)
        return counts, idx, dist2

    def query_csr(self, grid: Grid, queries, r: float, K: int, self_query: bool = True,
                  path: str = "auto", degree: bool = False):
        """frnn_query_csr_count + frnn_query_csr_fill (compact rows, exact
        allocation); returns (offsets [M+1] int64, idx [E] int32,
        dist2 [E] f32, degree [M] int32 or None)."""
        torch = _torch()
        _dev_f32(queries, "queries")
        M = queries.shape[0]
        dev = queries.device
        offsets = torch.empty(M + 1, dtype=torch.int64, device=dev)
        deg = torch.empty(M, dtype=torch.int32, device=dev) if degree else None
        n_edges = _i64(0)
        flags = PATHS[path] | (FRNN_SELF_QUERY if self_query else 0)
        rc = frnn_query_csr_count(self.handle, grid.handle, _vp(queries.data_ptr()), M, float(r),
                                  int(K), flags, _vp(offsets.data_ptr()),
                                  _vp(deg.data_ptr()) if deg is not None else None,
                                  ctypes.byref(n_edges))
        _check(self.handle, rc)
        E = int(n_edges.value)
        idx = torch.empty(E, dtype=torch.int32, device=dev)
        dist2 = torch.empty(E, dtype=torch.float32, device=dev)
        rc = frnn_query_csr_fill(self.handle, _vp(idx.data_ptr()) if E else None,
                                 _vp(dist2.data_ptr()) if E else None)
        _check(self.handle, rc)
        return offsets, idx, dist2, deg

    def self_query(self, points, r: float, K: int, path: str = "auto", out=None):
        """Build a grid on ``points`` and self-query it (one call each)."""
        g = self.build_grid(points, r)
        res = self.query(g, points, r, K, True, path, out)
        self._last_grid = g
        return res

    def query_batched(self, events, r: float, K: int, path: str = "auto", outs=None):
        """frnn_query_batched over a list of [n_e, D] tensors (self-queries)."""
        torch = _torch()
        n = len(events)
        if n == 0:
            return []
        D = events[0].shape[1]
        if outs is None:
            outs = []
            for p in events:
                _dev_f32(p, "event points")
                m = p.shape[0]
                outs.append((torch.empty(m, dtype=torch.int32, device=p.device),
                             torch.empty((m, K), dtype=torch.int32, device=p.device),
                             torch.empty((m, K), dtype=torch.float32, device=p.device)))
        arr = (frnn_event * n)()
        for e, (p, (c, i, d)) in enumerate(zip(events, outs)):
            _dev_f32(p, "event points")
            arr[e] = frnn_event(p.data_ptr(), p.shape[0], c.data_ptr(), i.data_ptr(), d.data_ptr())
        self._batch_keep = (events, outs)
        rc = frnn_query_batched(self.handle, arr, n, D, float(r), int(K), PATHS[path])
        _check(self.handle, rc)
        return outs

    def self_query_host(self, points_np, r: float, K: int, path: str = "auto", out=None):
        """frnn_self_query_host on NumPy arrays (copies in and out, synchronous)."""
        import numpy as np
        p = np.ascontiguousarray(points_np, dtype=np.float32)
        N, D = p.shape
        if out is None:
            out = (np.empty(N, np.int32), np.empty((N, K), np.int32),
                   np.empty((N, K), np.float32))
        c, i, d = out
        rc = frnn_self_query_host(self.handle, _vp(p.ctypes.data), N, D, float(r), int(K),
                                  PATHS[path], _vp(c.ctypes.data), _vp(i.ctypes.data),
                                  _vp(d.ctypes.data))
        _check(self.handle, rc)
        return out

    def self_query_host_csr(self, points_np, r: float, K: int, path: str = "auto", out=None):
        """frnn_self_query_host_csr on NumPy arrays: returns (offsets [N+1],
        idx [E], dist2 [E]) views; ``out`` = (offsets, idx, dist2) buffers,
        idx/dist2 of any capacity (retried larger if too small)."""
        import numpy as np
        p = np.ascontiguousarray(points_np, dtype=np.float32)
        N, D = p.shape
        if out is None:
            cap = N * min(K, 32)
            out = (np.empty(N + 1, np.int64), np.empty(cap, np.int32), np.empty(cap, np.float32))
        off, idx, d2 = out
        ne = _i64(0)
        for _ in range(2):
            rc = frnn_self_query_host_csr(self.handle, _vp(p.ctypes.data), N, D, float(r), int(K),
                                          PATHS[path], _vp(off.ctypes.data),
                                          _vp(idx.ctypes.data) if len(idx) else None,
                                          _vp(d2.ctypes.data) if len(d2) else None, len(idx),
                                          ctypes.byref(ne))
            if rc == FRNN_ERR_CAPACITY and ne.value > len(idx):
                idx = np.empty(ne.value, np.int32)
                d2 = np.empty(ne.value, np.float32)
                continue
            _check(self.handle, rc)
            break
        E = int(ne.value)
        return off, idx[:E], d2[:E]

    def autotune(self, points, r: float, K: int, path: str = "auto") -> dict:
        """frnn_autotune on a representative [N, D] CUDA tensor; returns the
        winning configuration (cached in the context for its size class)."""
        _dev_f32(points, "points")
        res = frnn_tune_result()
        rc = frnn_autotune(self.handle, _vp(points.data_ptr()), points.shape[0], points.shape[1],
                           float(r), int(K), PATHS[path], ctypes.byref(res))
        _check(self.handle, rc)
        return {"path": {FRNN_PATH_GRID: "grid", FRNN_PATH_TC: "tc"}.get(res.path, res.path),
                "cell_mult": res.cell_mult, "exit_dims": res.exit_dims, "ms": res.ms,
                "grid_axes": res.grid_axes, "staging": res.staging}

    def serve(self, events, arrivals, r: float, K: int, budget_bytes: int = 0, slots: int = 4,
              max_batch: int = 16, outs=None):
        """frnn_serve_run over host (NumPy, ideally page-locked) events with
        arrival times in seconds; returns (outputs, latencies_ms, stats)."""
        import numpy as np
        n = len(events)
        D = events[0].shape[1] if n else 1
        if outs is None:
            outs = [(np.empty(len(p), np.int32), np.empty((len(p), K), np.int32),
                     np.empty((len(p), K), np.float32)) for p in events]
        arr = (frnn_request * max(n, 1))()
        for i, (p, (c, ix, d)) in enumerate(zip(events, outs)):
            if p.dtype != np.float32 or not p.flags.c_contiguous:
                raise TypeError("events must be contiguous float32 [n, D] arrays")
            arr[i] = frnn_request(p.ctypes.data, len(p), c.ctypes.data, ix.ctypes.data,
                                  d.ctypes.data, float(arrivals[i]))
        lat = (ctypes.c_double * max(n, 1))()
        st = frnn_serve_stats()
        rc = frnn_serve_run(self.handle, arr, n, D, float(r), int(K), int(budget_bytes),
                            int(slots), int(max_batch), lat, ctypes.byref(st))
        _check(self.handle, rc)
        stats = {f: getattr(st, f) for f, _ in frnn_serve_stats._fields_}
        return outs, np.array(lat[:n]), stats

    def kernel_times(self) -> list:
        """frnn_kernel_times: main query kernel durations (ms) recorded since
        the last read, when FRNN_OPT_KERNEL_TIMING is on."""
        cap = 4096
        buf = (_f32 * cap)()
        n = _int(0)
        _check(self.handle, frnn_kernel_times(self.handle, buf, cap, ctypes.byref(n)))
        return [float(buf[i]) for i in range(min(n.value, cap))]

    def sync(self):
        """frnn_sync: wait and raise the device status (non-finite input, ...)."""
        _check(self.handle, frnn_sync(self.handle))
