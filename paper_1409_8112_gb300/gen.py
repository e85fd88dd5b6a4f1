"""Seeded synthetic inputs (points, random grid transforms, radii, request traces).

A module of its own: it draws random numbers and holds none of the method's arithmetic,
so the oracle's tests and the GPU library's callers use the same inputs.  The C code is in
``csrc/gen/rtg_gen.c`` (SplitMix64-seeded xoshiro256**, Box-Muller, Householder QR for
Haar rotations); this file builds it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "gen", "rtg_gen.c")
_OUT = os.path.join(_HERE, "_build", "librtg_gen.so")

SHIFT_ONLY = 1  # rotation = identity: the shift-only grids of Alg. 1

_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                   check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _l():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i64, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_void_p)
        lib.rtg_gen_transforms.argtypes = [u64, i32, i32, dbl, ctypes.c_uint32, vp]
        lib.rtg_gen_points_uniform.argtypes = [u64, i64, i32, i32, vp]
        lib.rtg_gen_points_mixture.argtypes = [u64, i64, i32, i32, dbl, dbl, dbl, i32, vp]
        lib.rtg_gen_radius_for_degree.argtypes = [i64, i32, dbl]
        lib.rtg_gen_radius_for_degree.restype = dbl
        _lib = lib
    return _lib


def transforms(seed: int, d: int, m: int, cell_side: float, flags: int = 0) -> np.ndarray:
    """(m, d*d + d) float64: row-major Haar rotation R then shift s ~ U[0, cell_side)^d."""
    out = np.zeros((m, d * d + d), dtype=np.float64)
    if _l().rtg_gen_transforms(seed, d, m, float(cell_side), flags, out.ctypes.data) != 0:
        raise ValueError("invalid transform arguments")
    return out


def points_uniform(seed: int, n: int, d: int, dtype=np.float64) -> np.ndarray:
    """(n, d) points i.i.d. uniform in [0,1)^d (the paper's unit-hypercube workloads)."""
    dt = np.dtype(dtype)
    out = np.zeros((n, d), dtype=dt)
    code = 0 if dt == np.float64 else 1
    if _l().rtg_gen_points_uniform(seed, n, d, code, out.ctypes.data) != 0:
        raise ValueError("invalid point arguments")
    return out


def points_mixture(seed: int, n: int, d: int, k: int = 8, sigma: float = 0.05, lo: float = 0.1,
                   hi: float = 0.9, dtype=np.float32) -> np.ndarray:
    """(n, d) points from k Gaussians (means uniform in [lo,hi]^d), clipped to [0,1]."""
    dt = np.dtype(dtype)
    out = np.zeros((n, d), dtype=dt)
    code = 0 if dt == np.float64 else 1
    if _l().rtg_gen_points_mixture(seed, n, d, k, sigma, lo, hi, code, out.ctypes.data) != 0:
        raise ValueError("invalid mixture arguments")
    return out


def radius_for_degree(n: int, d: int, degree: float | None = None) -> float:
    """r with expected ball population `degree` (default 2 ln n) for uniform density."""
    if degree is None:
        degree = 2.0 * math.log(n)
    return float(_l().rtg_gen_radius_for_degree(n, d, float(degree)))


def radius_fmt(n: int, d: int, eta: float = 0.0, mu: float = 1.0) -> float:
    """Eq. 2 radius 2(1+eta)[(1/d)(mu/zeta_d)(log n / n)]^(1/d), natural log."""
    zeta = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
    return 2.0 * (1.0 + eta) * ((1.0 / d) * (mu / zeta) * (math.log(n) / n)) ** (1.0 / d)


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int, size: int) -> np.ndarray:
    """floor(exp(U[ln lo, ln hi])) integers (the batched and served size mixes)."""
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size))).astype(np.int64)
