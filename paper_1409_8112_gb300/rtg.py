"""Python binding of the RTG C ABI (include/rtg.h).

Argument marshalling only: every step of a build runs in the CUDA library
``_build/librtg.so``.  The functions ``rtg_*`` mirror the C entry points one to one;
``Context`` is a small convenience wrapper over them.  If the library cannot be loaded the
import fails loudly: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

RTG_OK = 0
RTG_E_INVALID = 1
RTG_E_NOMEM = 2
RTG_E_BUDGET = 3
RTG_E_KEY_OVERFLOW = 4
RTG_E_CUDA = 5
RTG_E_TIMEOUT = 6
RTG_PENDING = 7
RTG_E_UNKNOWN_TICKET = 8
RTG_E_INTERNAL = 9

RTG_FLAG_SHIFT_ONLY = 1
RTG_FLAG_SYMMETRIC = 2
RTG_FLAG_TIMING = 4
RTG_FLAG_TWO_PASS = 8
RTG_FLAG_TC_FP16 = 16
RTG_FLAG_TC_BF16 = 32
RTG_FLAG_BITSET = 64

RTG_INJECT_SORT_WAIT = 1
RTG_INJECT_SCAN_WAIT = 2
RTG_INJECT_TC_WAIT = 4

RTG_DTYPE_F64 = 0
RTG_DTYPE_F32 = 1

RTG_MAX_DIM = 16
RTG_MAX_GRIDS = 64

PHASES = ("prep", "keys", "sort", "pairs", "scan", "scatter", "rowsort", "total")


class rtg_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class rtg_stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64 * RTG_MAX_GRIDS),
                ("total_candidates", ctypes.c_int64), ("owned_candidates", ctypes.c_int64),
                ("near_wall", ctypes.c_int64), ("near_r", ctypes.c_int64),
                ("key_rechecks", ctypes.c_int64), ("dist_rechecks", ctypes.c_int64),
                ("large_cells", ctypes.c_int64), ("max_cell", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("key_bits", ctypes.c_int32),
                ("sort_passes", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("attempts", ctypes.c_int32), ("sort_digit_bits", ctypes.c_int32),
                ("sort_tile_keys", ctypes.c_int32), ("sort_lookback", ctypes.c_int32),
                ("sort_tuned", ctypes.c_int32), ("phase_us", ctypes.c_double * 8),
                ("max_abs_err_d2", ctypes.c_double), ("band", ctypes.c_double),
                ("phase_bytes", ctypes.c_int64 * 8), ("bytes_moved", ctypes.c_int64),
                ("pairs_spans_per_warp", ctypes.c_int32), ("dense_cell_min", ctypes.c_int32),
                ("pairs_tuned", ctypes.c_int32), ("mem_estimate", ctypes.c_int64),
                ("mem_peak", ctypes.c_int64), ("sort_cell_major", ctypes.c_int32),
                ("sort_key_bits", ctypes.c_int32)]


class rtg_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("symmetric", ctypes.c_int32), ("handle", ctypes.c_uint64),
                ("stats", rtg_stats)]


class rtg_param_choice(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("cell_side", ctypes.c_double), ("c_factor", ctypes.c_double),
                ("recall", ctypes.c_double), ("build_us", ctypes.c_double),
                ("sample_n", ctypes.c_int64), ("sample_exact", ctypes.c_int64),
                ("candidates", ctypes.c_int)]


class rtg_instance(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int),
                ("r", ctypes.c_double), ("cell_side", ctypes.c_double),
                ("transforms", ctypes.c_void_p)]


class rtg_request(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("dtype", ctypes.c_int), ("n", ctypes.c_int64),
                ("d", ctypes.c_int), ("r", ctypes.c_double), ("cell_side", ctypes.c_double),
                ("transforms", ctypes.c_void_p), ("m", ctypes.c_int), ("flags", ctypes.c_uint32)]


class RTGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_lib = None

# Every function the header declares, with its ctypes signature.
_SIGNATURES = {
    "rtg_create": (ctypes.c_int, [ctypes.POINTER(rtg_config), ctypes.POINTER(ctypes.c_void_p)]),
    "rtg_destroy": (None, [ctypes.c_void_p]),
    "rtg_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "rtg_get_stream": (ctypes.c_void_p, [ctypes.c_void_p]),
    "rtg_tune_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.POINTER(rtg_param_choice)]),
    "rtg_query_neighbors": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(rtg_csr),
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                           ctypes.POINTER(rtg_csr)]),
    "rtg_index_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]),
    "rtg_index_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_int64, ctypes.POINTER(rtg_csr)]),
    "rtg_index_destroy": (None, [ctypes.c_void_p, ctypes.c_void_p]),
    "rtg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rtg_transforms_generate": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_uint32,
                                               ctypes.c_void_p]),
    "rtg_all_pairs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_uint32,
                                     ctypes.POINTER(rtg_csr)]),
    "rtg_batch_all_pairs": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(rtg_instance),
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_uint32, ctypes.POINTER(rtg_csr),
                                           ctypes.c_void_p]),
    "rtg_brute_force": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_uint32, ctypes.c_int,
                                       ctypes.POINTER(rtg_csr)]),
    "rtg_brute_count_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                               ctypes.POINTER(ctypes.c_uint64)]),
    "rtg_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(rtg_request),
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "rtg_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(rtg_csr)]),
    "rtg_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64,
                                ctypes.POINTER(rtg_csr)]),
    "rtg_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(rtg_csr)]),
    "rtg_set_test_hooks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int64]),
    "rtg_csr_download": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(rtg_csr),
                                        ctypes.c_void_p, ctypes.c_void_p]),
}


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"RTG CUDA library missing: {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def status_name(s: int) -> str:
    return lib().rtg_status_string(s).decode()


def _check(status: int, ctx=None):
    if status != RTG_OK:
        msg = lib().rtg_last_error(ctx).decode(errors="replace")
        raise RTGError(status, msg)


# ---- thin 1:1 wrappers ---------------------------------------------------------------------

def rtg_create(device: int = 0, mem_budget_bytes: int = 0, stream: int | None = None):
    cfg = rtg_config(device, mem_budget_bytes, stream or None, 0)
    out = ctypes.c_void_p()
    _check(lib().rtg_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out


def rtg_destroy(ctx) -> None:
    lib().rtg_destroy(ctx)


def rtg_transforms_generate(seed: int, d: int, m: int, cell_side: float,
                            flags: int = 0) -> np.ndarray:
    out = np.zeros((m, d * d + d), dtype=np.float64)
    _check(lib().rtg_transforms_generate(seed, d, m, cell_side, flags, out.ctypes.data))
    return out


def rtg_all_pairs(ctx, points_ptr: int, dtype: int, on_device: bool, n: int, d: int, r: float,
                  transforms: np.ndarray, m: int, cell_side: float, flags: int = 0) -> rtg_csr:
    T = np.ascontiguousarray(transforms, dtype=np.float64)
    out = rtg_csr()
    st = lib().rtg_all_pairs(ctx, points_ptr, dtype, 1 if on_device else 0, n, d, r,
                             T.ctypes.data, m, cell_side, flags, ctypes.byref(out))
    _check(st, ctx)
    return out


def rtg_batch_all_pairs(ctx, items, m: int, dtype: int, on_device: bool, flags: int = 0):
    """items: sequence of rtg_instance; returns (block-diagonal csr, row_offsets)."""
    arr = (rtg_instance * len(items))(*items)
    offs = np.zeros(len(items) + 1, dtype=np.int64)
    out = rtg_csr()
    st = lib().rtg_batch_all_pairs(ctx, arr, len(items), m, dtype, 1 if on_device else 0, flags,
                                   ctypes.byref(out), offs.ctypes.data)
    _check(st, ctx)
    return out, offs


def rtg_brute_force(ctx, points_ptr: int, dtype: int, on_device: bool, n: int, d: int,
                    r: float, flags: int = 0, count_only: bool = False) -> rtg_csr:
    out = rtg_csr()
    st = lib().rtg_brute_force(ctx, points_ptr, dtype, 1 if on_device else 0, n, d, r, flags,
                               1 if count_only else 0, ctypes.byref(out))
    _check(st, ctx)
    return out


def rtg_brute_count_noalloc(points_ptr: int, dtype: int, n: int, d: int, r: float,
                            stream: int | None = None) -> int:
    """Exact pair count with no device allocation (static scratch; n <= 65536)."""
    out = ctypes.c_uint64(0)
    _check(lib().rtg_brute_count_noalloc(points_ptr, dtype, n, d, r, stream or None,
                                         ctypes.byref(out)))
    return int(out.value)


def rtg_submit(ctx, points: np.ndarray, r: float, transforms: np.ndarray, cell_side: float,
               flags: int = 0) -> int:
    p = np.ascontiguousarray(points)
    code = RTG_DTYPE_F64 if p.dtype == np.float64 else RTG_DTYPE_F32
    if p.dtype not in (np.float64, np.float32):
        raise TypeError("points must be float64 or float32")
    n, d = p.shape
    T = np.ascontiguousarray(transforms, dtype=np.float64).reshape(-1)
    m = T.size // (d * d + d)
    req = rtg_request(p.ctypes.data, code, n, d, float(r), float(cell_side), T.ctypes.data, m, flags)
    t = ctypes.c_uint64(0)
    _check(lib().rtg_submit(ctx, ctypes.byref(req), ctypes.byref(t)), ctx)
    return int(t.value)


def rtg_poll(ctx, ticket: int):
    """None while pending, else the CSR (raises on a failed request)."""
    out = rtg_csr()
    st = lib().rtg_poll(ctx, ticket, ctypes.byref(out))
    if st == RTG_PENDING:
        return None
    _check(st, ctx)
    return out


def rtg_wait(ctx, ticket: int, timeout_us: int = -1) -> rtg_csr:
    out = rtg_csr()
    _check(lib().rtg_wait(ctx, ticket, timeout_us, ctypes.byref(out)), ctx)
    return out


def rtg_set_test_hooks(ctx, inject: int = 0, wait_limit: int = 0,
                       fail_alloc_after: int = 0) -> None:
    _check(lib().rtg_set_test_hooks(ctx, inject, wait_limit, fail_alloc_after), ctx)


def rtg_release(ctx, csr: rtg_csr) -> None:
    _check(lib().rtg_release(ctx, ctypes.byref(csr)), ctx)


def rtg_csr_download(ctx, csr: rtg_csr, out=None):
    """Copies the CSR to host arrays: new ones, or out = (row_ptr, col), contiguous int64 and
    int32 arrays of at least n + 1 and nnz entries (pinned ones make the copy a direct DMA);
    returns views of the copied length."""
    if out is None:
        # every element is written by the copy (fresh zeroed pages would fault during it)
        row_ptr = np.empty(csr.n + 1, dtype=np.int64)
        col = np.empty(max(csr.nnz, 0), dtype=np.int32)
    else:
        row_ptr, col = out
        if (row_ptr.dtype != np.int64 or col.dtype != np.int32 or
                not row_ptr.flags.c_contiguous or not col.flags.c_contiguous or
                row_ptr.size < csr.n + 1 or col.size < max(csr.nnz, 0)):
            raise ValueError("out must be contiguous int64 / int32 arrays of n + 1 / nnz entries")
        row_ptr, col = row_ptr[:csr.n + 1], col[:max(csr.nnz, 0)]
    _check(lib().rtg_csr_download(ctx, ctypes.byref(csr), row_ptr.ctypes.data,
                                  col.ctypes.data if csr.nnz > 0 else None), ctx)
    return row_ptr, col


# ---- convenience -----------------------------------------------------------------------------

def stats_dict(s: rtg_stats, m: int) -> dict:
    return {
        "candidates": [int(s.candidates[t]) for t in range(m)],
        "total_candidates": int(s.total_candidates),
        "owned_candidates": int(s.owned_candidates),
        "near_wall": int(s.near_wall), "near_r": int(s.near_r),
        "key_rechecks": int(s.key_rechecks), "dist_rechecks": int(s.dist_rechecks),
        "large_cells": int(s.large_cells), "max_cell": int(s.max_cell),
        "pairs": int(s.pairs), "key_bits": int(s.key_bits), "sort_passes": int(s.sort_passes),
        "launches": int(s.launches), "attempts": int(s.attempts),
        "sort": {"digit_bits": int(s.sort_digit_bits), "tile_keys": int(s.sort_tile_keys),
                 "lookback": int(s.sort_lookback), "tuned": int(s.sort_tuned),
                 "cell_major": int(s.sort_cell_major), "sorted_bits": int(s.sort_key_bits)},
        "phase_us": {p: float(s.phase_us[i]) for i, p in enumerate(PHASES)},
        "max_abs_err_d2": float(s.max_abs_err_d2), "band": float(s.band),
        "phase_bytes": {p: int(s.phase_bytes[i]) for i, p in enumerate(PHASES)},
        "bytes_moved": int(s.bytes_moved),
        "enumeration": {"spans_per_warp": int(s.pairs_spans_per_warp),
                  "dense_cell_min": int(s.dense_cell_min), "tuned": int(s.pairs_tuned)},
        "mem_estimate": int(s.mem_estimate), "mem_peak": int(s.mem_peak),
    }


def _points_arg(points):
    """(pointer, dtype code, on_device, n, d, keepalive) for a numpy array or CUDA tensor."""
    if hasattr(points, "data_ptr") and hasattr(points, "is_cuda"):
        import torch
        if points.dim() != 2:
            raise ValueError("points must be (n, d)")
        if points.dtype == torch.float64:
            code = RTG_DTYPE_F64
        elif points.dtype == torch.float32:
            code = RTG_DTYPE_F32
        else:
            raise TypeError("points must be float64 or float32")
        p = points.contiguous()
        if not p.is_cuda:
            p = p.numpy()
            return p.ctypes.data, code, False, p.shape[0], p.shape[1], p
        return p.data_ptr(), code, True, p.shape[0], p.shape[1], p
    p = np.ascontiguousarray(points)
    if p.ndim != 2:
        raise ValueError("points must be (n, d)")
    if p.dtype == np.float64:
        code = RTG_DTYPE_F64
    elif p.dtype == np.float32:
        code = RTG_DTYPE_F32
    else:
        raise TypeError("points must be float64 or float32")
    return p.ctypes.data, code, False, p.shape[0], p.shape[1], p


class Result:
    """A device CSR owned by the library; ``download()`` copies it to numpy."""

    def __init__(self, ctx: "Context", csr: rtg_csr, m: int):
        self._ctx = ctx
        self.csr = csr
        self.m = m

    @property
    def n(self) -> int:
        return int(self.csr.n)

    @property
    def nnz(self) -> int:
        return int(self.csr.nnz)

    @property
    def stats(self) -> dict:
        return stats_dict(self.csr.stats, self.m)

    def download(self, out=None):
        """(row_ptr, col) on the host; out = (row_ptr, col) arrays to fill (see
        rtg_csr_download)."""
        return rtg_csr_download(self._ctx.handle, self.csr, out)

    def release(self):
        if self.csr.handle:
            rtg_release(self._ctx.handle, self.csr)

    def __del__(self):
        try:
            if self._ctx.handle is not None and self.csr.handle:
                lib().rtg_release(self._ctx.handle, ctypes.byref(self.csr))
        except Exception:
            pass


class Index:
    """Device index of one point set's m grids (``Context.index``); ``query`` answers r-NN
    queries of new points.  ``close()`` frees it (also on garbage collection)."""

    def __init__(self, ctx: "Context", handle: int, d: int, dtype_code: int):
        self._ctx = ctx
        self.handle = handle
        self.d = d
        self.dtype_code = dtype_code

    def query(self, queries) -> "Result":
        """Row k of the result lists, ascending, the indexed points within r of queries[k]
        that share a cell with it in some grid.  queries: (nq, d) array of the index's dtype,
        numpy or CUDA tensor."""
        ptr, code, on_dev, nq, d, keep = _points_arg(queries)
        if nq > 0 and (d != self.d or code != self.dtype_code):
            raise ValueError("queries must be (nq, d) with the indexed points' d and dtype")
        self._ctx._after_producer(keep)
        out = rtg_csr()
        st = lib().rtg_index_query(self._ctx.handle, self.handle, ptr if nq > 0 else None,
                                   on_dev, nq, ctypes.byref(out))
        del keep
        _check(st, self._ctx.handle)
        return Result(self._ctx, out, 0)

    def close(self):
        if self.handle and self._ctx.handle is not None:
            lib().rtg_index_destroy(self._ctx.handle, self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream: int | None = None):
        self.handle = rtg_create(device, mem_budget_bytes, stream)
        self.stream = lib().rtg_get_stream(self.handle) or 0

    def _after_producer(self, points):
        """Orders the library's stream after torch's current stream when the points are a
        CUDA tensor produced there (a device-side wait; the host does not block)."""
        if hasattr(points, "is_cuda") and points.is_cuda:
            import torch
            cur = torch.cuda.current_stream(points.device)
            if cur.cuda_stream != self.stream:
                ext = getattr(self, "_ext_stream", None)
                if ext is None or ext.device != points.device:
                    ext = torch.cuda.ExternalStream(self.stream, device=points.device)
                    self._ext_stream = ext
                ext.wait_stream(cur)

    def close(self):
        if self.handle is not None:
            rtg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def all_pairs(self, points, r: float, transforms: np.ndarray, cell_side: float,
                  symmetric: bool = False, timing: bool = False, two_pass: bool = False,
                  bitset: bool = False, tensor: str | None = None) -> Result:
        """Alg. 1 over the grids of `transforms`; tensor = "fp16" or "bf16" takes the
        distances of cells of more than 256 points from tensor-core tiles (a filter; the
        reported set is the same)."""
        ptr, code, on_dev, n, d, keep = _points_arg(points)
        self._after_producer(keep)
        T = np.ascontiguousarray(transforms, dtype=np.float64).reshape(-1)
        if T.size % (d * d + d) != 0:
            raise ValueError("transforms must hold m * (d*d + d) values")
        m = T.size // (d * d + d)
        flags = ((RTG_FLAG_SYMMETRIC if symmetric else 0) | (RTG_FLAG_TIMING if timing else 0) |
                 (RTG_FLAG_TWO_PASS if two_pass else 0) | (RTG_FLAG_BITSET if bitset else 0))
        if tensor == "fp16":
            flags |= RTG_FLAG_TC_FP16
        elif tensor == "bf16":
            flags |= RTG_FLAG_TC_BF16
        elif tensor is not None:
            raise ValueError("tensor must be 'fp16', 'bf16' or None")
        csr = rtg_all_pairs(self.handle, ptr, code, on_dev, n, d, float(r), T, m,
                            float(cell_side), flags)
        del keep
        return Result(self, csr, m)

    def batch_all_pairs(self, instances, m: int, symmetric: bool = False, timing: bool = False,
                        two_pass: bool = False, bitset: bool = False):
        """instances: list of (points, r, transforms, cell_side); points all numpy (host) or
        all CUDA tensors, one dtype.  Returns (Result over the block-diagonal CSR, offsets)."""
        items, keep, codes, devs = [], [], set(), set()
        ordered = set()  # devices whose current stream the library's stream already follows
        for pts, r, T, c in instances:
            ptr, code, on_dev, n, d, kp = _points_arg(pts)
            if on_dev and kp.device not in ordered:
                self._after_producer(kp)  # one wait covers every tensor of that stream
                ordered.add(kp.device)
            Tc = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
            if Tc.size != m * (d * d + d):
                raise ValueError("each instance needs m * (d*d + d) transform values")
            keep += [kp, Tc]
            codes.add(code)
            devs.add(on_dev)
            items.append(rtg_instance(ptr, n, d, float(r), float(c), Tc.ctypes.data))
        if len(codes) != 1 or len(devs) != 1:
            raise ValueError("all instances need the same dtype and the same location")
        flags = ((RTG_FLAG_SYMMETRIC if symmetric else 0) | (RTG_FLAG_TIMING if timing else 0) |
                 (RTG_FLAG_TWO_PASS if two_pass else 0) | (RTG_FLAG_BITSET if bitset else 0))
        csr, offs = rtg_batch_all_pairs(self.handle, items, m, codes.pop(), devs.pop(), flags)
        del keep
        return Result(self, csr, m), offs

    def submit(self, points: np.ndarray, r: float, transforms: np.ndarray, cell_side: float,
               symmetric: bool = False) -> int:
        return rtg_submit(self.handle, points, r, transforms, cell_side,
                          RTG_FLAG_SYMMETRIC if symmetric else 0)

    def poll(self, ticket: int, m: int = 0):
        csr = rtg_poll(self.handle, ticket)
        return None if csr is None else Result(self, csr, m)

    def wait(self, ticket: int, timeout_us: int = -1, m: int = 0) -> Result:
        return Result(self, rtg_wait(self.handle, ticket, timeout_us), m)

    def tune_params(self, points, r: float, target_recall: float, seed: int = 0,
                    shift_only: bool = False) -> dict:
        """c and m for a target recall (Sec. III-A): the fastest measured (c, m) whose grids
        report at least target_recall of a prefix sample's exact pairs.  The grids are
        gen.transforms(seed, d, m, c, flags) with the same shift-only flag."""
        ptr, code, on_dev, n, d, keep = _points_arg(points)
        self._after_producer(keep)
        out = rtg_param_choice()
        st = lib().rtg_tune_params(self.handle, ptr, code, on_dev, n, d, float(r),
                                   float(target_recall), int(seed),
                                   RTG_FLAG_SHIFT_ONLY if shift_only else 0, ctypes.byref(out))
        del keep
        _check(st, self.handle)
        return {f: getattr(out, f) for f, _ in rtg_param_choice._fields_}

    def query_neighbors(self, graph: "Result", queries) -> "Result":
        """Multiple r-NN queries (Sec. II): row k of the result is the neighbour list of
        queries[k], read from `graph` (a symmetric result of this context).  queries: int32
        numpy array or CUDA tensor."""
        if hasattr(queries, "is_cuda") and queries.is_cuda:
            import torch
            q = queries.to(torch.int32).contiguous()
            self._after_producer(q)
            ptr, on_dev, nq, keep = q.data_ptr(), 1, q.numel(), q
        else:
            q = np.ascontiguousarray(queries, dtype=np.int32).reshape(-1)
            ptr, on_dev, nq, keep = (q.ctypes.data if q.size else None), 0, q.size, q
        out = rtg_csr()
        st = lib().rtg_query_neighbors(self.handle, ctypes.byref(graph.csr), ptr, nq, on_dev,
                                       ctypes.byref(out))
        del keep
        _check(st, self.handle)
        return Result(self, out, 0)

    def index(self, points, r: float, transforms: np.ndarray, cell_side: float) -> "Index":
        """The m grids of `points` kept on the device for r-NN queries of new points (Sec. V).
        points: (n, d) float64/float32 numpy array or CUDA tensor."""
        ptr, code, on_dev, n, d, keep = _points_arg(points)
        self._after_producer(keep)
        T = np.ascontiguousarray(transforms, dtype=np.float64).reshape(-1)
        if T.size % (d * d + d) != 0:
            raise ValueError("transforms must hold m * (d*d + d) values")
        m = T.size // (d * d + d)
        h = ctypes.c_void_p()
        st = lib().rtg_index_create(self.handle, ptr, code, on_dev, n, d, float(r),
                                    T.ctypes.data, m, float(cell_side), ctypes.byref(h))
        del keep
        _check(st, self.handle)
        return Index(self, h.value, d, code)

    def brute_force(self, points, r: float, symmetric: bool = False,
                    count_only: bool = False, tensor: str | None = None,
                    timing: bool = False) -> Result:
        """Exact set of Sec. I on the device (all pairs checked); tensor = "fp16" or "bf16"
        takes the distances from tensor-core tiles with an FP64 band check."""
        ptr, code, on_dev, n, d, keep = _points_arg(points)
        self._after_producer(keep)
        flags = (RTG_FLAG_SYMMETRIC if symmetric else 0) | (RTG_FLAG_TIMING if timing else 0)
        if tensor == "fp16":
            flags |= RTG_FLAG_TC_FP16
        elif tensor == "bf16":
            flags |= RTG_FLAG_TC_BF16
        elif tensor is not None:
            raise ValueError("tensor must be 'fp16', 'bf16' or None")
        csr = rtg_brute_force(self.handle, ptr, code, on_dev, n, d, float(r), flags, count_only)
        del keep
        return Result(self, csr, 0)
