"""CPU oracle for the dual-select FMA radix-2 FFT — TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it, and
it shares no code with the CUDA path: the arithmetic lives in the plain C file
``dsfft_oracle.c`` next to this module (FP64 reference transforms, the
twiddle tables of Algorithm 1 / Eqs. 4-9, and an op-by-op emulation of the
6-FMA Stockham FFT with correctly rounded FP32/FP16/BF16 operations).  This
module only compiles that file with gcc and marshals numpy arrays.

Array conventions: complex signals are numpy ``complex128`` arrays of shape
``(batch, N)`` (or ``(N,)``) whose values are exactly representable in the
format being emulated.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

FP64, FP32, FP16, BF16 = 0, 1, 2, 3
LF, COS, DS = 0, 1, 2          # Linzer-Feig clamped, cosine, dual-select
PATH_COS, PATH_SIN = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsfft_oracle.c")
_LIB = os.path.join(_HERE, "libdsfft_oracle.so")
_lock = threading.Lock()
_lib = None

FORMATS = {"fp64": FP64, "fp32": FP32, "fp16": FP16, "bf16": BF16}
FACTORIZATIONS = {"linzer_feig_clamped": LF, "cosine": COS, "dual_select": DS}


def build(force: bool = False) -> str:
    """Compile the C oracle into ``libdsfft_oracle.so`` (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-ffp-contract=off",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            P = ctypes.c_void_p
            lib.orc_round.restype = d
            lib.orc_round.argtypes = [d, i32]
            lib.orc_fma.restype = d
            lib.orc_fma.argtypes = [d, d, d, i32]
            lib.orc_mul.restype = d
            lib.orc_mul.argtypes = [d, d, i32]
            lib.orc_dft.argtypes = [i64, P, P, i32]
            lib.orc_dft_bin.argtypes = [i64, P, i64, i32, P]
            lib.orc_fft_fp64.argtypes = [i64, P, P, i64, i32]
            lib.orc_table.argtypes = [i64, i32, d, i32, i32, i32, P, P, P]
            lib.orc_table_range.argtypes = [i64, i64, i32, d, i32, i32, d, P, P, P]
            lib.orc_emulate_fft_r4.argtypes = [i64, i32, i32, i32, P, P, P, d, d, i32, P, P, i64]
            lib.orc_butterfly.argtypes = [i32, i32, d, d, i32, P, P, P, P]
            lib.orc_emulate_fft.argtypes = [i64, i32, i32, P, P, P, P, P, i64]
            lib.orc_round_array.argtypes = [P, P, i64, i32]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as_c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


# --------------------------------------------------------------------------
# scalar arithmetic of the formats
def round_to(x: float, fmt: int) -> float:
    """Round an FP64 value to the nearest value of ``fmt`` (ties to even)."""
    return _load().orc_round(float(x), int(fmt))


def fma(a: float, b: float, c: float, fmt: int) -> float:
    """Correctly rounded ``a*b + c`` in ``fmt`` (operands must be values of fmt)."""
    return _load().orc_fma(float(a), float(b), float(c), int(fmt))


def mul(a: float, b: float, fmt: int) -> float:
    return _load().orc_mul(float(a), float(b), int(fmt))


def round_array(x, fmt: int) -> np.ndarray:
    """Elementwise RN-even rounding of a real or complex array to ``fmt``."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        v = _as_c128(x)
        flat = v.view(np.float64).ravel()
        out = np.empty_like(flat)
        _load().orc_round_array(_ptr(flat), _ptr(out), flat.size, int(fmt))
        return out.view(np.complex128).reshape(v.shape)
    v = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(v)
    _load().orc_round_array(_ptr(v), _ptr(out), v.size, int(fmt))
    return out


# --------------------------------------------------------------------------
# FP64 references (Eq. 1 definition and the 10-op radix-2 FFT of Eqs. 2-3)
def dft(x, sign: int = -1) -> np.ndarray:
    """Direct O(N^2) DFT in FP64 of each row of ``x``."""
    x = _as_c128(x)
    rows = x.reshape(-1, x.shape[-1])
    out = np.empty_like(rows)
    N = rows.shape[1]
    lib = _load()
    for r in range(rows.shape[0]):
        xi = np.ascontiguousarray(rows[r])
        yo = np.empty_like(xi)
        lib.orc_dft(N, _ptr(xi), _ptr(yo), int(sign))
        out[r] = yo
    return out.reshape(x.shape)


def dft_bin(x, k: int, sign: int = -1) -> complex:
    """One bin X[k] of the FP64 DFT of a single signal ``x`` (shape (N,))."""
    x = _as_c128(x)
    o = np.empty(2, dtype=np.float64)
    _load().orc_dft_bin(x.shape[-1], _ptr(x), int(k), int(sign), _ptr(o))
    return complex(o[0], o[1])


def fft_fp64(x, sign: int = -1) -> np.ndarray:
    """Radix-2 Stockham FFT in FP64 (10-op butterflies) of each row of ``x``."""
    x = _as_c128(x)
    N = x.shape[-1]
    batch = x.size // N
    y = np.empty_like(x)
    _load().orc_fft_fp64(N, _ptr(x), _ptr(y), batch, int(sign))
    return y


# --------------------------------------------------------------------------
# twiddle tables (Algorithm 1 and the two single factorizations)
def table(N: int, fac: int, fmt: int, direction: int = -1, scaled: bool = False,
          eps: float = 1e-7):
    """Return ``(t, m, path)`` for k in [0, N/2): ratio and multiplier rounded
    once to ``fmt`` (as float64 arrays) and the path flag (0 cos, 1 sin)."""
    h = N // 2
    t = np.empty(h, dtype=np.float64)
    m = np.empty(h, dtype=np.float64)
    p = np.empty(h, dtype=np.int32)
    _load().orc_table(int(N), int(fac), float(eps), 1 if direction > 0 else -1, int(fmt),
                      1 if scaled else 0, _ptr(t), _ptr(m), _ptr(p))
    return t, m, p


def table_range(N: int, count: int, fac: int, fmt: int, direction: int = -1, mscale: float = 1.0,
                eps: float = 1e-7):
    """The rules of :func:`table` for k in [0, count) (k may exceed N/2),
    multiplier times ``mscale`` (a power of two) before the rounding."""
    t = np.empty(count, dtype=np.float64)
    m = np.empty(count, dtype=np.float64)
    p = np.empty(count, dtype=np.int32)
    _load().orc_table_range(int(N), int(count), int(fac), float(eps), 1 if direction > 0 else -1, int(fmt),
                            float(mscale), _ptr(t), _ptr(m), _ptr(p))
    return t, m, p


def table4(N: int, fac: int, fmt: int, direction: int = -1, scaled: bool = False, eps: float = 1e-7):
    """Radix-4 table: k in [0, 3N/4), multipliers RN(m/4) when scaled."""
    return table_range(N, 3 * N // 4, fac, fmt, direction, 0.25 if scaled else 1.0, eps)


def butterfly(fmt: int, scaled: bool, t: float, m: float, path: int, a: complex, b: complex):
    """One 6-FMA butterfly (branched on ``path``) — returns (A, B)."""
    av = np.array([a.real, a.imag], dtype=np.float64)
    bv = np.array([b.real, b.imag], dtype=np.float64)
    A = np.empty(2, dtype=np.float64)
    B = np.empty(2, dtype=np.float64)
    _load().orc_butterfly(int(fmt), 1 if scaled else 0, float(t), float(m), int(path),
                          _ptr(av), _ptr(bv), _ptr(A), _ptr(B))
    return complex(A[0], A[1]), complex(B[0], B[1])


def emulate_fft(x, fmt: int, t, m, path, scaled: bool = False, threads: int = 1) -> np.ndarray:
    """Op-by-op emulation of the 6-FMA Stockham FFT on each row of ``x``.

    ``t, m, path`` are the table entries the transform uses (length N/2),
    already rounded to ``fmt``.  ``threads > 1`` splits the batch over host
    threads (ctypes releases the GIL)."""
    x = _as_c128(x)
    N = x.shape[-1]
    batch = x.size // N
    xs = x.reshape(batch, N)
    y = np.empty_like(xs)
    t = np.ascontiguousarray(t, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    path = np.ascontiguousarray(path, dtype=np.int32)
    assert t.shape == (N // 2,) and m.shape == (N // 2,) and path.shape == (N // 2,)
    lib = _load()

    def run(lo, hi):
        if hi > lo:
            lib.orc_emulate_fft(N, int(fmt), 1 if scaled else 0, _ptr(t), _ptr(m), _ptr(path),
                                xs[lo:hi].ctypes.data_as(ctypes.c_void_p),
                                y[lo:hi].ctypes.data_as(ctypes.c_void_p), hi - lo)

    if threads <= 1 or batch < 2:
        run(0, batch)
    else:
        th = min(threads, batch)
        cuts = [batch * i // th for i in range(th + 1)]
        ws = [threading.Thread(target=run, args=(cuts[i], cuts[i + 1])) for i in range(th)]
        for w in ws:
            w.start()
        for w in ws:
            w.join()
    return y.reshape(x.shape)


def emulate_fft_r4(x, fmt: int, t4, m4, path4, e0, scaled: bool = False, inverse: bool = False,
                   threads: int = 1) -> np.ndarray:
    """Op-by-op emulation of the radix-4 dual-select FFT (orc_emulate_fft_r4)
    on each row of ``x``.  ``t4, m4, path4``: the radix-4 table (k < 3N/4);
    ``e0 = (t, m, path)``: the radix-2 entry k = 0 (used when log2 N is odd)."""
    x = _as_c128(x)
    N = x.shape[-1]
    batch = x.size // N
    xs = x.reshape(batch, N)
    y = np.empty_like(xs)
    t4 = np.ascontiguousarray(t4, dtype=np.float64)
    m4 = np.ascontiguousarray(m4, dtype=np.float64)
    path4 = np.ascontiguousarray(path4, dtype=np.int32)
    need = max(1, 3 * N // 4)
    assert t4.shape[0] >= need and m4.shape[0] >= need and path4.shape[0] >= need
    lib = _load()

    def run(lo, hi):
        if hi > lo:
            lib.orc_emulate_fft_r4(N, int(fmt), 1 if scaled else 0, 1 if inverse else 0, _ptr(t4), _ptr(m4),
                                   _ptr(path4), float(e0[0]), float(e0[1]), int(e0[2]),
                                   xs[lo:hi].ctypes.data_as(ctypes.c_void_p),
                                   y[lo:hi].ctypes.data_as(ctypes.c_void_p), hi - lo)

    if threads <= 1 or batch < 2:
        run(0, batch)
    else:
        th = min(threads, batch)
        cuts = [batch * i // th for i in range(th + 1)]
        ws = [threading.Thread(target=run, args=(cuts[i], cuts[i + 1])) for i in range(th)]
        for w in ws:
            w.start()
        for w in ws:
            w.join()
    return y.reshape(x.shape)


def rel_l2(y, ref) -> float:
    """Relative L2 error ||y - ref|| / ||ref|| over all elements."""
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.linalg.norm((y - ref).ravel()) / np.linalg.norm(ref.ravel()))
