"""Seeded, counter-based Bernoulli bit matrices (inputs only; see bitgen.h).

The CPU generator (``libbitgen.so``, plain C) feeds the oracle and the tests;
the GPU generator (``libbitgen_cuda.so``) fills device buffers for the bench.
Both implement the same SplitMix64-based definition and are checked against
each other bit for bit. Nothing here computes a matrix product.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CPU_SO = os.path.join(_HERE, "libbitgen.so")
_CUDA_SO = os.path.join(_HERE, "libbitgen_cuda.so")

DENSE = 0
THRESHOLD = 1
GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def build_cpu() -> str:
    cmd = ["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", _CPU_SO,
           os.path.join(_HERE, "bitgen.c")]
    subprocess.run(cmd, check=True)
    return _CPU_SO


def build_cuda_cmd() -> list[str]:
    return ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
            "-Xcompiler", "-fPIC", "-shared", "-o", _CUDA_SO, os.path.join(_HERE, "bitgen.cu")]


_cpu = None
_cuda = None


def _lib_cpu():
    global _cpu
    if _cpu is None:
        if not os.path.exists(_CPU_SO):
            build_cpu()
        lib = ctypes.CDLL(_CPU_SO)
        lib.bitgen_fill_rows.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_uint64, ctypes.c_int]
        lib.bitgen_fill_rows.restype = None
        lib.bitgen_draw.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64]
        lib.bitgen_draw.restype = ctypes.c_uint64
        _cpu = lib
    return _cpu


def _lib_cuda():
    global _cuda
    if _cuda is None:
        if not os.path.exists(_CUDA_SO):
            raise RuntimeError("libbitgen_cuda.so is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(_CUDA_SO)
        lib.bitgen_fill_rows_device.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]
        lib.bitgen_fill_rows_device.restype = ctypes.c_int
        _cuda = lib
    return _cuda


# ---------------------------------------------------------------- thresholds
def theta_pow2(a: int) -> int:
    """theta for p = 2^-a (a >= 1): floor(2^64 * 2^-a)."""
    return 1 << (64 - a)


def theta_pow2_half(a: int) -> int:
    """theta for p = 2^-(a + 1/2): floor(2^(64 - a - 1/2)) = isqrt(2^(127 - 2a))."""
    return math.isqrt(1 << (127 - 2 * a))


def theta_inv_sqrt(k: int) -> int:
    """theta for p = 1/sqrt(k): floor(2^64 / sqrt(k)) = isqrt(floor(2^128 / k))."""
    return math.isqrt((1 << 128) // k)


def spec(p: str | float | None):
    """(mode, theta) for a density spec: None or 0.5 -> dense; '2^-7.5' etc."""
    if p is None or p == 0.5 or p == "0.5":
        return DENSE, 0
    if isinstance(p, str) and p.startswith("2^-"):
        e = float(p[3:])
        a = int(math.floor(e))
        if e == a:
            return THRESHOLD, theta_pow2(a)
        if abs(e - a - 0.5) < 1e-12:
            return THRESHOLD, theta_pow2_half(a)
        raise ValueError(p)
    if isinstance(p, str) and p.startswith("1/sqrt("):
        return THRESHOLD, theta_inv_sqrt(int(p[7:-1]))
    if isinstance(p, str) and p.startswith("1/"):
        d = int(p[2:])
        return THRESHOLD, ((1 << 64) // d)
    raise ValueError(f"unsupported density spec {p!r}")


# ---------------------------------------------------------------- reference draw
def draw_py(seed: int, matrix_id: int, counter: int) -> int:
    """Pure-Python draw, written from the definition (used to pin the C code)."""
    z = (((seed << 32) ^ (matrix_id << 62)) + (counter + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def draw(seed: int, matrix_id: int, counter: int) -> int:
    return int(_lib_cpu().bitgen_draw(seed, matrix_id, counter))


# ---------------------------------------------------------------- fills
def fill_cpu(rows: int, cols: int, seed: int, matrix_id: int, p=None, row0: int = 0,
             nrows: int | None = None, nthreads: int | None = None) -> np.ndarray:
    """Rows [row0, row0+nrows) of the matrix as an (nrows, cols//64) uint64 array."""
    if cols % 64:
        raise ValueError("cols must be a multiple of 64")
    if nrows is None:
        nrows = rows - row0
    mode, theta = spec(p)
    out = np.empty((nrows, cols // 64), dtype=np.uint64)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    _lib_cpu().bitgen_fill_rows(out.ctypes.data, cols, row0, nrows, seed, matrix_id, mode,
                                theta, nthreads)
    return out


def fill_device(t, cols: int, seed: int, matrix_id: int, p=None, row0: int = 0,
                stream: int = 0) -> None:
    """Fill a contiguous device tensor t (nrows x cols//64 words) on the GPU."""
    mode, theta = spec(p)
    nrows = t.numel() // (cols // 64)
    rc = _lib_cuda().bitgen_fill_rows_device(t.data_ptr(), cols, row0, nrows, seed, matrix_id,
                                             mode, theta, stream)
    if rc != 0:
        raise RuntimeError(f"bitgen_fill_rows_device failed: cudaError {rc}")


# ---------------------------------------------------------------- batched shapes
def batched_shapes(count: int, seed: int, lo: int = 256, hi: int = 8192, mult: int = 64):
    """Per-problem (m, k, n) drawn log-uniform in [lo, hi], rounded to a multiple of
    `mult`, plus an op flag (0 = GF(2), 1 = Boolean) alternating for a 50/50 mix.
    Draws come from matrix_id 3 of the same generator (counter 4*i + axis)."""
    out = []
    llo, lhi = math.log(lo), math.log(hi)
    for i in range(count):
        dims = []
        for axis in range(3):
            u = (draw_py(seed, 3, 4 * i + axis) >> 11) * (1.0 / (1 << 53))
            v = math.exp(llo + u * (lhi - llo))
            r = int(round(v / mult)) * mult
            dims.append(min(max(r, lo), hi))
        out.append((dims[0], dims[1], dims[2], i % 2))
    return out
