"""CPU oracle for the Boolean and GF(2) bit-matrix products — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``bmm_oracle.c`` (plain C,
built with gcc) and adds tiny pure-Python/numpy helpers for brute force.
It shares no code with the GPU path in ``paper_1909_01554_gb300``.

Layout everywhere: row-major, bit j of row i is bit (j % 64) of uint64 word
i*(cols/64) + j/64 (least significant index in the bits of a word, as in the
paper's linearisation convention, Sec. 3.4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

GF2 = 0
BOOL = 1

SW, SELF_INVERSE, CHAINING = 0, 1, 2
PHI, PSI, CHI, ALPHA, BETA, GAMMA = 0, 1, 2, 3, 4, 5


class Counts(ctypes.Structure):
    _fields_ = [("basis_bitops", ctypes.c_uint64), ("lincomb_bitops", ctypes.c_uint64),
                ("mult_bitops", ctypes.c_uint64), ("leaf_products", ctypes.c_uint64)]


def build() -> str:
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", _SO,
                    os.path.join(_HERE, "bmm_oracle.c")], check=True)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            build()
        L = ctypes.CDLL(_SO)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.oracle_cubic.argtypes = [i32, vp, vp, vp, i64, i64, i64, i32]
        L.oracle_rows.argtypes = [i32, vp, vp, vp, i64, i64, i64, i32]
        L.oracle_extract_column.argtypes = [vp, i64, i64, i64, vp]
        L.oracle_column.argtypes = [i32, vp, vp, vp, i64, i64]
        L.oracle_matvec_gf2.argtypes = [vp, vp, vp, i64, i64]
        L.oracle_level_probe.argtypes = [i32, i32, vp, vp]
        L.oracle_basis_change.argtypes = [i32, i32, vp, i64, i64, i32, vp]
        L.oracle_strassen_gf2.argtypes = [i32, vp, vp, vp, i64, i64, i64, i32,
                                          ctypes.POINTER(Counts)]
        L.oracle_strassen_gf2.restype = ctypes.c_int
        L.oracle_transpose.argtypes = [vp, vp, i64, i64]
        L.oracle_alt_product.argtypes = [i32, vp, vp, vp, i64, i64, i64, i32]
        L.oracle_alt_product.restype = ctypes.c_int
        for f in (L.oracle_cubic, L.oracle_rows, L.oracle_extract_column, L.oracle_column,
                  L.oracle_matvec_gf2, L.oracle_level_probe, L.oracle_basis_change,
                  L.oracle_transpose):
            f.restype = None
        _lib = L
    return _lib


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def threads() -> int:
    return os.cpu_count() or 1


# ------------------------------------------------------------ products
def cubic(op: int, A: np.ndarray, B: np.ndarray, m: int, k: int, n: int,
          nthreads: int | None = None) -> np.ndarray:
    """C = A B (op GF2: XOR of ANDs; op BOOL: OR of ANDs), packed (m, n/64)."""
    A, B = _c(A), _c(B)
    assert A.size == m * k // 64 and B.size == k * n // 64
    C = np.empty((m, n // 64), dtype=np.uint64)
    lib().oracle_cubic(op, A.ctypes.data, B.ctypes.data, C.ctypes.data, m, k, n,
                       nthreads or threads())
    return C


def rows(op: int, Arows: np.ndarray, B: np.ndarray, k: int, n: int,
         nthreads: int | None = None) -> np.ndarray:
    """The rows of C for the given rows of A (Arows: (r, k/64))."""
    Arows, B = _c(Arows), _c(B)
    r = Arows.size // (k // 64)
    out = np.empty((r, n // 64), dtype=np.uint64)
    lib().oracle_rows(op, Arows.ctypes.data, B.ctypes.data, out.ctypes.data, r, k, n,
                      nthreads or threads())
    return out


def column(op: int, A: np.ndarray, B: np.ndarray, j: int, m: int, k: int, n: int) -> np.ndarray:
    """Column j of C as a uint8 vector of length m."""
    A, B = _c(A), _c(B)
    bcol = np.empty(k // 64, dtype=np.uint64)
    lib().oracle_extract_column(B.ctypes.data, k, n, j, bcol.ctypes.data)
    out = np.empty(m, dtype=np.uint8)
    lib().oracle_column(op, A.ctypes.data, bcol.ctypes.data, out.ctypes.data, m, k)
    return out


def matvec_gf2(M: np.ndarray, x: np.ndarray, rows_: int, cols: int) -> np.ndarray:
    """y = M x over GF(2); x packed (cols/64 words), y packed (ceil(rows/64) words)."""
    M, x = _c(M), _c(x)
    y = np.empty((rows_ + 63) // 64, dtype=np.uint64)
    lib().oracle_matvec_gf2(M.ctypes.data, x.ctypes.data, y.ctypes.data, rows_, cols)
    return y


def transpose(P: np.ndarray, rows_: int, cols: int) -> np.ndarray:
    P = _c(P)
    out = np.empty((cols, rows_ // 64), dtype=np.uint64)
    lib().oracle_transpose(P.ctypes.data, out.ctypes.data, rows_, cols)
    return out


def strassen_gf2(variant: int, A: np.ndarray, B: np.ndarray, m: int, k: int, n: int,
                 depth: int):
    """GF(2) product through `depth` levels of the chosen 2x2 recursion.
    Returns (C, counts dict)."""
    A, B = _c(A), _c(B)
    C = np.empty((m, n // 64), dtype=np.uint64)
    cnt = Counts()
    rc = lib().oracle_strassen_gf2(variant, A.ctypes.data, B.ctypes.data, C.ctypes.data, m, k, n,
                                   depth, ctypes.byref(cnt))
    if rc != 0:
        raise ValueError("sizes not divisible by 64 * 2^depth")
    return C, {f: int(getattr(cnt, f)) for f, _ in Counts._fields_}


def alt_product(variant: int, Ah: np.ndarray, Bh: np.ndarray, m: int, k: int, n: int,
                depth: int) -> np.ndarray:
    """Hat C from operands already in the alternative basis (no basis changes)."""
    Ah, Bh = _c(Ah), _c(Bh)
    Ch = np.empty((m, n // 64), dtype=np.uint64)
    if lib().oracle_alt_product(variant, Ah.ctypes.data, Bh.ctypes.data, Ch.ctypes.data, m, k,
                                n, depth) != 0:
        raise ValueError("sizes not divisible by 64 * 2^depth")
    return Ch


def basis_change(variant: int, inverse: bool, X: np.ndarray, rows_: int, cols: int,
                 depth: int):
    """Basis change of a copy of X over `depth` levels (phi, or chi when inverse)."""
    Y = _c(X).copy()
    ops = ctypes.c_uint64(0)
    lib().oracle_basis_change(variant, int(inverse), Y.ctypes.data, rows_, cols, depth,
                              ctypes.byref(ops))
    return Y, int(ops.value)


def level_matrix(variant: int, which: int) -> np.ndarray:
    """The 0/1 matrix that one level's straight-line program implements, read
    off by feeding unit vectors (lane 0 of each word)."""
    n_in = 7 if which == GAMMA else 4
    n_out = 7 if which in (ALPHA, BETA) else 4
    M = np.zeros((n_out, n_in), dtype=np.uint8)
    for c in range(n_in):
        inp = np.zeros(7, dtype=np.uint64)
        inp[c] = 1
        out = np.zeros(7, dtype=np.uint64)
        lib().oracle_level_probe(variant, which, inp.ctypes.data, out.ctypes.data)
        M[:, c] = (out[:n_out] & np.uint64(1)).astype(np.uint8)
    return M


# ------------------------------------------------------------ bit helpers (numpy)
def unpack(P: np.ndarray, rows_: int, cols: int) -> np.ndarray:
    """Packed (rows, cols/64) uint64 -> (rows, cols) uint8 of 0/1."""
    b = np.ascontiguousarray(P, dtype=np.uint64).reshape(rows_, cols // 64).view(np.uint8)
    return np.unpackbits(b, axis=1, bitorder="little")[:, :cols]


def pack(M: np.ndarray) -> np.ndarray:
    """(rows, cols) 0/1 -> packed (rows, cols/64) uint64."""
    rows_, cols = M.shape
    assert cols % 64 == 0
    b = np.packbits(np.asarray(M, dtype=np.uint8), axis=1, bitorder="little")
    return np.ascontiguousarray(b).view(np.uint64).reshape(rows_, cols // 64)


def brute_force(op: int, Abits: np.ndarray, Bbits: np.ndarray) -> np.ndarray:
    """Per-bit quadruple loop straight from the definition (tiny inputs only)."""
    m, k = Abits.shape
    k2, n = Bbits.shape
    assert k == k2
    C = np.zeros((m, n), dtype=np.uint8)
    for i in range(m):
        for j in range(n):
            acc = 0
            for t in range(k):
                term = int(Abits[i, t]) & int(Bbits[t, j])
                acc = (acc ^ term) if op == GF2 else (acc | term)
            C[i, j] = acc
    return C
