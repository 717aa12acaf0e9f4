"""FP64 reference (oracle) of OpenFFT's 3-D C2C method: ctypes binding.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import this package.  The library it loads is
built from ``oracle/oracle.c`` alone and shares no code with the CUDA path.

Every function cites the passage of Duy & Ozaki, "Performance Tuning of a
Parallel 3-D FFT Package OpenFFT", that it follows (see ``oracle.c``).
Arrays are numpy complex128 (re, im interleaved), C-contiguous.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

FORWARD = -1
BACKWARD = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain gcc, portable flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if force or not fresh:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    """Argument and result types of the library's entry points."""
    i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    p64 = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_f.restype = i64
    lib.oracle_f.argtypes = [i64] * 5
    lib.oracle_boundaries.restype = i32
    lib.oracle_boundaries.argtypes = [i64] * 4 + [p64]
    lib.oracle_box.restype = i32
    lib.oracle_box.argtypes = [i64] * 5 + [p64, p64, p64, p64]
    lib.oracle_degree.restype = i32
    lib.oracle_degree.argtypes = [i64] * 3
    lib.oracle_fft1d.restype = None
    lib.oracle_fft1d.argtypes = [i64, vp, vp, i32]
    lib.oracle_dft1d_brute.restype = None
    lib.oracle_dft1d_brute.argtypes = [i64, vp, vp, i32]
    lib.oracle_dft3d_brute.restype = None
    lib.oracle_dft3d_brute.argtypes = [i64, i64, i64, vp, vp, i32]
    lib.oracle_dft3d_line.restype = None
    lib.oracle_dft3d_line.argtypes = [i64, i64, i64, vp, i32, i64, i64, vp]
    lib.oracle_redistribute.restype = i32
    lib.oracle_redistribute.argtypes = [i64] * 4 + [i32, vp, vp, vp]
    lib.oracle_fft3d.restype = i32
    lib.oracle_fft3d.argtypes = [i64] * 4 + [i32, vp, vp, vp, vp]
    lib.oracle_rfft3d.restype = i32
    lib.oracle_rfft3d.argtypes = [i64] * 4 + [i32, vp, vp, vp, vp]
    lib.oracle_nd_boundaries.restype = i32
    lib.oracle_nd_boundaries.argtypes = [i32, p64, i32, i64, p64]
    lib.oracle_nd_redistribute.restype = i32
    lib.oracle_nd_redistribute.argtypes = [i32, p64, i64, i32, i32, vp, vp, vp]
    lib.oracle_fftnd.restype = i32
    lib.oracle_fftnd.argtypes = [i32, p64, i64, i32, vp, vp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------- Eqs. 2-9 --

def f(N1: int, N2: int, N3: int, Np: int, myid: int) -> int:
    """Eq. 2: start offset of process ``myid``; -1 where Eq. 2 is undefined."""
    return int(_load().oracle_f(N1, N2, N3, Np, myid))


def boundaries(N1: int, N2: int, N3: int, Np: int) -> np.ndarray:
    """Eqs. 3-4 for every rank: array xs[0..Np], rank r owns [xs[r], xs[r+1])."""
    xs = np.zeros(Np + 1, dtype=np.int64)
    rc = _load().oracle_boundaries(N1, N2, N3, Np, xs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise ValueError("decomposition undefined for Np=%d with N1=%d, N2=%d" % (Np, N1, N2))
    return xs


def box(N1: int, N2: int, N3: int, Np: int, myid: int):
    """Eqs. 3-7: (x^s, x^e, start (a,b,c), end (a,b,c)) of rank ``myid``."""
    xs = ctypes.c_int64()
    xe = ctypes.c_int64()
    s3 = (ctypes.c_int64 * 3)()
    e3 = (ctypes.c_int64 * 3)()
    rc = _load().oracle_box(N1, N2, N3, Np, myid, ctypes.byref(xs), ctypes.byref(xe), s3, e3)
    if rc != 0:
        raise ValueError("decomposition undefined")
    return xs.value, xe.value, tuple(s3), tuple(e3)


def degree(N1: int, N2: int, Np: int) -> int:
    """Eqs. 2, 8-9: 1 (slabs) if Np <= N1, 2 (pencils) if N1 < Np <= N1*N2, else -1."""
    return int(_load().oracle_degree(N1, N2, Np))


# ------------------------------------------------------------ transforms --

def fft1d(x, sign: int = FORWARD) -> np.ndarray:
    """Recursive mixed-radix 1-D DFT (the oracle's local FFT engine)."""
    x = _c128(x)
    y = np.empty_like(x)
    _load().oracle_fft1d(x.size, _ptr(x), _ptr(y), sign)
    return y


def dft1d_brute(x, sign: int = FORWARD) -> np.ndarray:
    """O(n^2) DFT by definition, long-double accumulation."""
    x = _c128(x)
    y = np.empty_like(x)
    _load().oracle_dft1d_brute(x.size, _ptr(x), _ptr(y), sign)
    return y


def dft3d_brute(A, sign: int = FORWARD) -> np.ndarray:
    """O(N^2) 3-D DFT by definition; A and the result are [Na][Nb][Nc]."""
    A = _c128(A)
    Na, Nb, Nc = A.shape
    X = np.empty_like(A)
    _load().oracle_dft3d_brute(Na, Nb, Nc, _ptr(A), _ptr(X), sign)
    return X


def dft3d_line(A, kb: int, kc: int, sign: int = FORWARD) -> np.ndarray:
    """X[:, kb, kc] of the 3-D DFT of A[Na][Nb][Nc] by its definition, O(N)."""
    A = _c128(A)
    Na, Nb, Nc = A.shape
    line = np.empty(Na, dtype=np.complex128)
    _load().oracle_dft3d_line(Na, Nb, Nc, _ptr(A), sign, kb, kc, _ptr(line))
    return line


REDIST = {"abc->cab": 1, "cab->cba": 2, "cba->cab": -2, "cab->abc": -1}


def redistribute(Na: int, Nb: int, Nc: int, Np: int, which: str, src):
    """Steps (4)-(6) of one transpose: returns (dst, count matrix [Np][Np])."""
    src = _c128(src).reshape(-1)
    dst = np.full_like(src, np.nan + 1j * np.nan)
    C = np.zeros((Np, Np), dtype=np.int64)
    rc = _load().oracle_redistribute(Na, Nb, Nc, Np, REDIST[which], _ptr(src), _ptr(dst), _ptr(C))
    if rc != 0:
        raise ValueError("redistribution undefined or inconsistent")
    return dst, C


def fft3d(A, Na: int, Nb: int, Nc: int, Np: int, direction: int = FORWARD, counts: bool = False):
    """Full 3-D C2C transform under the decomposition over Np ranks.

    forward: A is the abc-ordered array, result is cba-ordered (flat, N);
    backward: A is cba-ordered, result is abc-ordered and divided by N.
    With ``counts`` also returns the two Np x Np count matrices."""
    A = _c128(A).reshape(-1)
    if A.size != Na * Nb * Nc:
        raise ValueError("size mismatch")
    out = np.empty_like(A)
    C1 = np.zeros((Np, Np), dtype=np.int64)
    C2 = np.zeros((Np, Np), dtype=np.int64)
    rc = _load().oracle_fft3d(Na, Nb, Nc, Np, direction, _ptr(A), _ptr(out), _ptr(C1), _ptr(C2))
    if rc != 0:
        raise ValueError("decomposition undefined for this (Na, Nb, Nc, Np)")
    if counts:
        return out, C1, C2
    return out


def rfft3d(A, Na: int, Nb: int, Nc: int, Np: int, direction: int = FORWARD, counts: bool = False):
    """Real 3-D transform under the decomposition over Np ranks.

    forward: A is the real abc-ordered array (N doubles); the result is the
    half spectrum kc <= Nc/2 in cba order, [Nc//2 + 1][Nb][Na] flat complex.
    backward: A is that half spectrum; the result is the real abc array
    divided by N (the real part of the inverse of the Hermitian-extended
    spectrum).  With ``counts`` also returns the count matrices of the two
    transposes of the half array."""
    Nch = Nc // 2 + 1
    M = Na * Nb * Nch
    if direction == FORWARD:
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(-1))
        if A.size != Na * Nb * Nc:
            raise ValueError("size mismatch")
        out = np.empty(M, dtype=np.complex128)
    else:
        A = _c128(A).reshape(-1)
        if A.size != M:
            raise ValueError("size mismatch")
        out = np.empty(Na * Nb * Nc, dtype=np.float64)
    C1 = np.zeros((Np, Np), dtype=np.int64)
    C2 = np.zeros((Np, Np), dtype=np.int64)
    rc = _load().oracle_rfft3d(Na, Nb, Nc, Np, direction, _ptr(A), _ptr(out), _ptr(C1), _ptr(C2))
    if rc != 0:
        raise ValueError("decomposition undefined for this (Na, Nb, Nc, Np)")
    if counts:
        return out, C1, C2
    return out


def abc_to_cba(X_abc: np.ndarray) -> np.ndarray:
    """Reorder a [Na][Nb][Nc] array into flat cba order (index (c*Nb+b)*Na+a)."""
    return np.ascontiguousarray(np.transpose(X_abc, (2, 1, 0))).reshape(-1)


def rel_l2(y, y_ref) -> float:
    """Relative L2 error ||y - y_ref|| / ||y_ref||, accumulated in long double."""
    y = np.asarray(y, dtype=np.complex128).reshape(-1)
    y_ref = np.asarray(y_ref, dtype=np.complex128).reshape(-1)
    d = (y - y_ref)
    num = np.sum(np.longdouble(d.real) ** 2 + np.longdouble(d.imag) ** 2)
    den = np.sum(np.longdouble(y_ref.real) ** 2 + np.longdouble(y_ref.imag) ** 2)
    return float(np.sqrt(num / den))


# ------------------------------------------------------ D-dimensional --

def _dims64(dims):
    return (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])


def nd_boundaries(dims, Np: int, s: int) -> np.ndarray:
    """Eqs. 2-4 of ordering s (1..D) of a D-dimensional array: xs[0..Np].

    Ordering s is (d_D, ..., d_{D-s+2}, d_1, ..., d_{D-s+1}) (slowest first),
    decomposed with (N1, N2, N3) = (first dim, second dim, product of the rest)."""
    xs = np.zeros(Np + 1, dtype=np.int64)
    rc = _load().oracle_nd_boundaries(len(dims), _dims64(dims), s, Np,
                                      xs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise ValueError("decomposition undefined")
    return xs


def nd_redistribute(dims, Np: int, s: int, forward: bool, src):
    """Steps (4)-(6) from ordering s to s+1 (forward) or s+1 to s: (dst, counts)."""
    src = _c128(src).reshape(-1)
    dst = np.full_like(src, np.nan + 1j * np.nan)
    C = np.zeros((Np, Np), dtype=np.int64)
    rc = _load().oracle_nd_redistribute(len(dims), _dims64(dims), Np, s, 1 if forward else 0,
                                        _ptr(src), _ptr(dst), _ptr(C))
    if rc != 0:
        raise ValueError("redistribution undefined or inconsistent")
    return dst, C


def fftnd(A, dims, Np: int, direction: int = FORWARD) -> np.ndarray:
    """D-dimensional C2C transform under the decomposition over Np ranks (D = 3..8).

    forward: A is the array as given (ordering 1), the result is in ordering D
    (the axes reversed, d_D slowest); backward: the reverse, divided by N."""
    A = _c128(A).reshape(-1)
    if A.size != int(np.prod(dims)):
        raise ValueError("size mismatch")
    out = np.empty_like(A)
    rc = _load().oracle_fftnd(len(dims), _dims64(dims), Np, direction, _ptr(A), _ptr(out))
    if rc != 0:
        raise ValueError("decomposition undefined for these dims and Np")
    return out
