"""CPU oracle for randomly transformed grids (RTG) all-pairs r-NN.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
leg are the only callers.  The GPU library never imports this package.

Python side of ``rtg_oracle.cpp``: ``build()`` compiles it with gcc (FP contraction off)
and the wrappers return plain numpy arrays.  Each wrapper names the passage of
arXiv:1409.8112 that its C function follows (see the header of ``rtg_oracle.cpp``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtg_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (optionally with planted mistake ``mutant``) and return its path."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-pthread", "-shared", f"-DORACLE_MUTANT={mutant}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("col", ctypes.POINTER(ctypes.c_int32))]


class _GridStats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64), ("nonempty_cells", ctypes.c_int64),
                ("multi_cells", ctypes.c_int64), ("max_cell", ctypes.c_int64),
                ("near_wall", ctypes.c_int64), ("reported", ctypes.c_int64)]


@dataclass
class CSR:
    row_ptr: np.ndarray  # int64, n + 1
    col: np.ndarray      # int32, nnz; ascending per row, col > row

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def pairs(self) -> np.ndarray:
        """(nnz, 2) int64 array of (i, j), i < j, in CSR order."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        return np.stack([rows, self.col.astype(np.int64)], axis=1)

    def pair_keys(self) -> np.ndarray:
        """Pairs packed as i * 2^32 + j (uint64), sorted ascending."""
        p = self.pairs()
        return (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)


_libs: dict[int, ctypes.CDLL] = {}


def _lib(mutant: int = 0) -> ctypes.CDLL:
    if mutant in _libs:
        return _libs[mutant]
    lib = ctypes.CDLL(build(mutant))
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    csrp = ctypes.POINTER(_CSR)
    lib.oracle_brute.argtypes = [vp, i32, i64, i32, dbl, csrp]
    lib.oracle_exact_grid.argtypes = [vp, i32, i64, i32, dbl, csrp]
    lib.oracle_cells.argtypes = [vp, i32, i64, i32, vp, i32, dbl, vp, vp]
    lib.oracle_rtg.argtypes = [vp, i32, i64, i32, dbl, vp, i32, dbl, csrp, vp, vp]
    lib.oracle_rtg_query.argtypes = [vp, i32, i64, i32, dbl, vp, i32, dbl, vp, i64, csrp]
    lib.oracle_rtg_threads.argtypes = [vp, i32, i64, i32, dbl, vp, i32, dbl, i32, csrp]
    lib.oracle_free.argtypes = [csrp]
    for f in (lib.oracle_brute, lib.oracle_exact_grid, lib.oracle_cells, lib.oracle_rtg,
              lib.oracle_rtg_query, lib.oracle_rtg_threads):
        f.restype = ctypes.c_int
    lib.oracle_mutant.restype = ctypes.c_int
    _libs[mutant] = lib
    return lib


def _points(points: np.ndarray):
    if points.dtype == np.float64:
        dtype = 0
    elif points.dtype == np.float32:
        dtype = 1
    else:
        raise TypeError("points must be float64 or float32")
    p = np.ascontiguousarray(points)
    if p.ndim != 2:
        raise ValueError("points must be (n, d)")
    return p, dtype


def _take(lib, c: _CSR) -> CSR:
    n, nnz = c.n, c.nnz
    row_ptr = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy()
    col = (np.ctypeslib.as_array(c.col, shape=(nnz,)).copy() if nnz > 0
           else np.zeros(0, dtype=np.int32))
    lib.oracle_free(ctypes.byref(c))
    return CSR(row_ptr, col)


def brute(points: np.ndarray, r: float, mutant: int = 0) -> CSR:
    """Exact all-pairs r-NN set (Sec. I problem statement) by checking every pair."""
    lib = _lib(mutant)
    p, dt = _points(points)
    c = _CSR()
    rc = lib.oracle_brute(p.ctypes.data, dt, p.shape[0], p.shape[1], float(r), ctypes.byref(c))
    if rc != 0:
        raise ValueError("oracle_brute: invalid arguments")
    return _take(lib, c)


def exact_grid(points: np.ndarray, r: float, mutant: int = 0) -> CSR:
    """Exact all-pairs r-NN set through a side-r grid and its adjacent cells (Sec. II-B)."""
    lib = _lib(mutant)
    p, dt = _points(points)
    c = _CSR()
    rc = lib.oracle_exact_grid(p.ctypes.data, dt, p.shape[0], p.shape[1], float(r),
                               ctypes.byref(c))
    if rc != 0:
        raise ValueError("oracle_exact_grid: invalid arguments")
    return _take(lib, c)


def cells(points: np.ndarray, transforms: np.ndarray, cell_side: float, mutant: int = 0):
    """The point-to-cell step of Alg. 1 for each grid: (m, n, d) int64 cell coordinates and
    near-wall counts."""
    lib = _lib(mutant)
    p, dt = _points(points)
    n, d = p.shape
    T = np.ascontiguousarray(transforms, dtype=np.float64).reshape(-1)
    m = T.size // (d * d + d)
    q = np.zeros((m, n, d), dtype=np.int64)
    near = np.zeros(m, dtype=np.int64)
    rc = lib.oracle_cells(p.ctypes.data, dt, n, d, T.ctypes.data, m, float(cell_side),
                          q.ctypes.data, near.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_cells: invalid arguments")
    return q, near


@dataclass
class RTGResult:
    csr: CSR
    stats: list  # one dict per grid
    near_r: int


def rtg(points: np.ndarray, r: float, transforms: np.ndarray, cell_side: float,
        mutant: int = 0) -> RTGResult:
    """Alg. 1 with the Sec. III-B unordered-set dedupe; returns the CSR and per-grid stats."""
    lib = _lib(mutant)
    p, dt = _points(points)
    n, d = p.shape
    T = np.ascontiguousarray(transforms, dtype=np.float64).reshape(-1)
    if T.size % (d * d + d) != 0:
        raise ValueError("transforms must hold m * (d*d + d) values")
    m = T.size // (d * d + d)
    st = (_GridStats * m)()
    near_r = ctypes.c_int64(0)
    c = _CSR()
    rc = lib.oracle_rtg(p.ctypes.data, dt, n, d, float(r), T.ctypes.data, m, float(cell_side),
                        ctypes.byref(c), st, ctypes.byref(near_r))
    if rc != 0:
        raise ValueError("oracle_rtg: invalid arguments")
    stats = [{f: int(getattr(st[t], f)) for f, _ in _GridStats._fields_} for t in range(m)]
    return RTGResult(_take(lib, c), stats, int(near_r.value))


def rtg_threads(points: np.ndarray, r: float, transforms: np.ndarray, cell_side: float,
                threads: int = 0, mutant: int = 0) -> CSR:
    """Alg. 1 with the Sec. III-B dedupe on several host threads (grids in parallel, then the
    merge by row ranges); the same CSR as ``rtg``.  ``threads`` = 0 takes one per hardware
    thread."""
    lib = _lib(mutant)
    p, dt = _points(points)
    n, d = p.shape
    T = np.ascontiguousarray(transforms, dtype=np.float64).reshape(-1)
    if T.size % (d * d + d) != 0:
        raise ValueError("transforms must hold m * (d*d + d) values")
    m = T.size // (d * d + d)
    c = _CSR()
    rc = lib.oracle_rtg_threads(p.ctypes.data, dt, n, d, float(r), T.ctypes.data, m,
                                float(cell_side), int(threads), ctypes.byref(c))
    if rc != 0:
        raise ValueError("oracle_rtg_threads: invalid arguments")
    return _take(lib, c)


def rtg_query(points: np.ndarray, r: float, transforms: np.ndarray, cell_side: float,
              queries: np.ndarray, mutant: int = 0) -> CSR:
    """r-NN queries of new points from the m stored grids (the single-query use of the grids,
    Sec. V): row k lists the points of P within r of query k that share a cell with it in
    some grid, ascending."""
    lib = _lib(mutant)
    p, dt = _points(points)
    x, dq = _points(queries)
    n, d = p.shape
    if x.ndim != 2 or x.shape[1] != d or dq != dt:
        raise ValueError("queries must be nq x d with the points' dtype")
    T = np.ascontiguousarray(transforms, dtype=np.float64).reshape(-1)
    if T.size % (d * d + d) != 0:
        raise ValueError("transforms must hold m * (d*d + d) values")
    m = T.size // (d * d + d)
    c = _CSR()
    rc = lib.oracle_rtg_query(p.ctypes.data, dt, n, d, float(r), T.ctypes.data, m,
                              float(cell_side), x.ctypes.data, x.shape[0], ctypes.byref(c))
    if rc != 0:
        raise ValueError("oracle_rtg_query: invalid arguments")
    return _take(lib, c)


def recall(rtg_csr: CSR, exact: CSR) -> float:
    """Success rate of Sec. IV-A: reported pairs / ground-truth pairs (1 if there are none)."""
    return 1.0 if exact.nnz == 0 else rtg_csr.nnz / exact.nnz
