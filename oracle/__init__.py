"""Plain CPU oracle for the modular BLAS and the NTT -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The CUDA library never imports, links or executes it.

This module is a thin ctypes wrapper over ``oracle.c`` (u32-limb bignum, binary long division,
textbook iterative NTT); see that file's header for what each function computes and which passage
of the paper it follows.  Arrays are numpy ``uint64``: shape ``(n,)`` for width 1 (q < 2^64) and
``(n, w)`` -- low word first -- for width w = 2, 3, 4.  Widths 1 and 2 use the default build of
oracle.c; widths 3 and 4 use its wide build (the same source with longer integers).

ctypes releases the GIL for the duration of each foreign call, so callers may run independent
jobs on a thread pool (the CPU baseline does).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "oracle.c")
LIBRARY = os.path.join(_HERE, "liboracle.so")
LIBRARY_WIDE = os.path.join(_HERE, "liboracle_wide.so")
WIDE_LIMBS = 18  # 32-bit limbs of the wide build: residues of up to four 64-bit words
_lock = threading.Lock()

VADD, VSUB, VMUL, AXPY = 0, 1, 2, 3
CYCLIC, BITREV = 1, 2

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(src: str = SOURCE, out: str = LIBRARY, force: bool = False, bn_limbs: int | None = None) -> str:
    """Compile oracle.c into a shared object (plain -O2, no tuning); bn_limbs selects the wide build."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        defs = [f"-DBN_LIMBS={bn_limbs}"] if bn_limbs else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", *defs, "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def build_all(force: bool = False):
    """Both builds: widths 1-2 and widths 3-4."""
    return build(force=force), build(out=LIBRARY_WIDE, force=force, bn_limbs=WIDE_LIMBS)


def _words(v: int, width: int = 2) -> np.ndarray:
    """v as max(width, 2) 64-bit words, low word first."""
    n = max(width, 2)
    return np.array([(v >> (64 * k)) & (2**64 - 1) for k in range(n)], dtype=np.uint64)


def _int(words: np.ndarray, width: int) -> int:
    return sum(int(words[k]) << (64 * k) for k in range(width))


def _shape(N: int, width: int):
    return (-1, N) if width == 1 else (-1, N, width)


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments")


class Oracle:
    """The oracle functions bound to one compiled copy of oracle.c."""

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        L.oracle_blas.argtypes = [ctypes.c_int, _u64p, _u64p, _u64p, _u64p, ctypes.c_size_t, _u64p, ctypes.c_int]
        L.oracle_ntt_work_bytes.argtypes = [ctypes.c_uint]
        L.oracle_ntt_work_bytes.restype = ctypes.c_size_t
        L.oracle_ntt.argtypes = [_u64p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_uint, _u64p, _u64p,
                                 ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.c_void_p]
        L.oracle_dft.argtypes = [_u64p, _u64p, ctypes.c_uint, _u64p, _u64p, ctypes.c_int, ctypes.c_uint,
                                 ctypes.c_int]
        L.oracle_ntt_point.argtypes = [_u64p, _u64p, ctypes.c_uint, _u64p, _u64p, ctypes.c_int, ctypes.c_uint,
                                       ctypes.c_uint64]
        L.oracle_intt_point.argtypes = L.oracle_ntt_point.argtypes
        L.oracle_negacyclic_mul.argtypes = [_u64p, _u64p, _u64p, ctypes.c_uint, _u64p, ctypes.c_int]
        L.oracle_powmod.argtypes = [_u64p, _u64p, _u64p, _u64p]
        for f in ("oracle_blas", "oracle_ntt", "oracle_dft", "oracle_ntt_point", "oracle_intt_point",
                  "oracle_negacyclic_mul", "oracle_powmod", "oracle_max_width"):
            getattr(L, f).restype = ctypes.c_int
        self.L = L
        self.max_width = L.oracle_max_width()

    def blas(self, op: int, a: np.ndarray, b: np.ndarray, q: int, width: int, s: int = 0) -> np.ndarray:
        """Element-wise op over n residues; axpy computes s*a + b (x = a, y = b)."""
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.empty_like(a)
        _check(self.L.oracle_blas(op, _p(out), _p(a), _p(b), _p(_words(s, width)), a.shape[0], _p(_words(q, width)),
                                  width), "blas")
        return out

    def ntt(self, x: np.ndarray, log2n: int, q: int, root: int, width: int, flags: int = 0,
            inverse: bool = False) -> np.ndarray:
        """Transform of each polynomial in x: shape (N,)/(N,2) or (batch, N)/(batch, N, 2)."""
        x = np.array(x, dtype=np.uint64, copy=True, order="C")
        N = 1 << log2n
        xb = x.reshape(_shape(N, width))
        work = ctypes.create_string_buffer(self.L.oracle_ntt_work_bytes(log2n))
        _check(self.L.oracle_ntt(_p(xb), xb.shape[0], N, log2n, _p(_words(q, width)), _p(_words(root, width)),
                                 width, flags, int(inverse), work), "ntt")
        return xb.reshape(x.shape)

    def ntt_strided(self, x: np.ndarray, batch: int, stride: int, log2n: int, q: int, root: int, width: int,
                    flags: int = 0, inverse: bool = False) -> np.ndarray:
        """Transform `batch` polynomials stored `stride` residues apart in a flat array (gaps untouched)."""
        x = np.array(x, dtype=np.uint64, copy=True, order="C")
        work = ctypes.create_string_buffer(self.L.oracle_ntt_work_bytes(log2n))
        _check(self.L.oracle_ntt(_p(x), batch, stride, log2n, _p(_words(q, width)), _p(_words(root, width)),
                                 width, flags, int(inverse), work), "ntt")
        return x

    def dft(self, x: np.ndarray, log2n: int, q: int, root: int, width: int, flags: int = 0,
            inverse: bool = False) -> np.ndarray:
        """The same transform from its O(N^2) definition (N <= 4096)."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = np.empty_like(x)
        _check(self.L.oracle_dft(_p(out), _p(x), log2n, _p(_words(q, width)), _p(_words(root, width)), width,
                                 flags, int(inverse)), "dft")
        return out

    def ntt_point(self, x: np.ndarray, log2n: int, q: int, root: int, width: int, k: int,
                  flags: int = 0) -> int:
        """Forward output k (natural order) of one polynomial, from the definition, O(N)."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        out = np.zeros(max(width, 2), dtype=np.uint64)
        _check(self.L.oracle_ntt_point(_p(out), _p(x), log2n, _p(_words(q, width)), _p(_words(root, width)), width,
                                       flags, k), "ntt_point")
        return _int(out, width)

    def intt_point(self, y: np.ndarray, log2n: int, q: int, root: int, width: int, j: int,
                   flags: int = 0) -> int:
        """Inverse output j of one natural-order spectrum, from the definition, O(N)."""
        y = np.ascontiguousarray(y, dtype=np.uint64)
        out = np.zeros(max(width, 2), dtype=np.uint64)
        _check(self.L.oracle_intt_point(_p(out), _p(y), log2n, _p(_words(q, width)), _p(_words(root, width)), width,
                                        flags, j), "intt_point")
        return _int(out, width)

    def negacyclic_mul(self, a: np.ndarray, b: np.ndarray, log2n: int, q: int, width: int) -> np.ndarray:
        """Schoolbook product of two polynomials modulo x^N + 1 (N <= 16384)."""
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.empty_like(a)
        _check(self.L.oracle_negacyclic_mul(_p(out), _p(a), _p(b), log2n, _p(_words(q, width)), width),
               "negacyclic_mul")
        return out

    def powmod(self, g: int, e: int, q: int) -> int:
        out = np.zeros(2, dtype=np.uint64)
        _check(self.L.oracle_powmod(_p(out), _p(_words(g)), _p(_words(e)), _p(_words(q))), "powmod")
        return int(out[0]) | (int(out[1]) << 64)


_default = None
_wide = None


def default() -> Oracle:
    """The oracle compiled from this directory's oracle.c (built on first use): widths 1 and 2."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def wide() -> Oracle:
    """The wide build of the same source: widths 1 to 4."""
    global _wide
    with _lock:
        if _wide is None:
            _wide = Oracle(build(out=LIBRARY_WIDE, bn_limbs=WIDE_LIMBS))
    return _wide


def _for(args, kwargs) -> Oracle:
    """The build that takes the call's width (the fifth argument of every function below)."""
    width = kwargs.get("width", args[4] if len(args) > 4 else 1)
    return wide() if width > 2 else default()


def blas(*a, **k):
    return _for(a, k).blas(*a, **k)


def ntt(*a, **k):
    return _for(a, k).ntt(*a, **k)


def dft(*a, **k):
    return _for(a, k).dft(*a, **k)


def ntt_point(*a, **k):
    return _for(a, k).ntt_point(*a, **k)


def intt_point(*a, **k):
    return _for(a, k).intt_point(*a, **k)


def negacyclic_mul(*a, **k):
    return _for(a, k).negacyclic_mul(*a, **k)


def powmod(*a, **k):
    return default().powmod(*a, **k)
