"""CPU oracle for the TTC permute-scale-add (arXiv 1607.01249, section 1 Eq. 1).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.

The arithmetic lives in ``ttc_oracle.c`` (plain C, one element at a time, see
that file's header for the readings it takes).  This module only compiles it
with gcc, loads it with ctypes and marshals numpy arrays.  Arrays are passed as
flat buffers holding the column-major tensors (or the larger "outer" tensors
they live in, section 2.1 Table 1 --lda/--ldb).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ttc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# The oracle's own dtype numbering (independent of the product's enum).
F32, F64, BF16, E4M3, C64, C128 = 0, 1, 2, 3, 4, 5
NP_DTYPE = {F32: np.float32, F64: np.float64, BF16: np.uint16, E4M3: np.uint8, C64: np.complex64,
            C128: np.complex128}
NAMES = {"f32": F32, "f64": F64, "bf16": BF16, "e4m3": E4M3, "c64": C64, "c128": C128}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i64p = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        L.oracle_permute.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, i64p, i64p,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     vp, vp, ctypes.c_float]
        L.oracle_permute.restype = ctypes.c_int
        L.oracle_permute_exact.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, i64p,
                                           i64p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, vp, vp, vp, vp]
        L.oracle_permute_exact.restype = ctypes.c_int
        L.oracle_fp8_scale.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, ctypes.c_double, vp,
                                       ctypes.POINTER(ctypes.c_float)]
        L.oracle_fp8_scale.restype = ctypes.c_float
        L.oracle_permute_complex.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, i64p, i64p,
                                             ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [vp, vp]
        L.oracle_permute_complex.restype = ctypes.c_int
        L.oracle_permute_complex_exact.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, i64p, i64p,
                                                   ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [vp] * 4
        L.oracle_permute_complex_exact.restype = ctypes.c_int
        for name in ("oracle_bf16_from_f32_n", "oracle_e4m3_from_f32_n", "oracle_e4m3_to_f32_n"):
            getattr(L, name).argtypes = [vp, vp, ctypes.c_int64]
            getattr(L, name).restype = None
        L.oracle_fmaf_n.argtypes = [vp, vp, vp, vp, ctypes.c_int64]
        L.oracle_fmaf_n.restype = None
        _lib = L
    return _lib


def _i64(a):
    if a is None:
        return None
    arr = (ctypes.c_int64 * len(a))(*[int(x) for x in a])
    return arr


def _ptr(x: np.ndarray):
    return ctypes.c_void_p(x.ctypes.data)


def _span(sizes, outer) -> int:
    """1 + the largest element offset of a column-major (sub-)tensor."""
    if any(int(s) == 0 for s in sizes):
        return 0
    span, stride = 1, 1
    for s, o in zip(sizes, outer):
        span += (int(s) - 1) * stride
        stride *= int(o)
    return span


def _check_buf(x: np.ndarray, dt: int, sizes, outer, name: str):
    need = _span(sizes, outer)
    if x.dtype != NP_DTYPE[dt] or not x.flags.c_contiguous or x.size < need:
        raise ValueError(f"{name}: need a contiguous {NP_DTYPE[dt].__name__} buffer of >= {need}")


def dims(perm, sizes, outerA=None, outerB=None):
    n = len(sizes)
    oA = list(outerA) if outerA is not None else list(sizes)
    sB = [sizes[p] for p in perm]
    oB = list(outerB) if outerB is not None else sB
    return n, oA, sB, oB


def permute(perm, sizes, A, B, alpha=1.0, beta=0.0, dtA=F32, dtB=F32, outerA=None,
            outerB=None, fp8_scale=1.0):
    """B <- alpha*A + beta*B under perm (in place on the numpy buffer B)."""
    n, oA, sB, oB = dims(perm, sizes, outerA, outerB)
    _check_buf(A, dtA, sizes, oA, "A")
    _check_buf(B, dtB, sB, oB, "B")
    rc = lib().oracle_permute(n, (ctypes.c_int * n)(*perm), _i64(sizes), _i64(outerA),
                              _i64(outerB), dtA, dtB, float(alpha), float(beta), _ptr(A),
                              _ptr(B), float(fp8_scale))
    if rc:
        raise ValueError(f"oracle_permute rejected the problem (code {rc})")
    return B


def permute_exact(perm, sizes, A, B, alpha=1.0, beta=0.0, dtA=F32, dtB=F32, outerA=None,
                  outerB=None):
    """Exact value (rounded once to double) and tolerance scale, in B's layout."""
    n, oA, sB, oB = dims(perm, sizes, outerA, outerB)
    _check_buf(A, dtA, sizes, oA, "A")
    _check_buf(B, dtB, sB, oB, "B")
    vol = B.size
    R = np.full(vol, np.nan)
    S = np.full(vol, np.nan)
    rc = lib().oracle_permute_exact(n, (ctypes.c_int * n)(*perm), _i64(sizes), _i64(outerA),
                                    _i64(outerB), dtA, dtB, float(alpha), float(beta), _ptr(A),
                                    _ptr(B), _ptr(R), _ptr(S))
    if rc:
        raise ValueError(f"oracle_permute_exact rejected the problem (code {rc})")
    return R, S


def permute_complex(perm, sizes, A, B, alpha=1.0, beta=0.0, dtA=C64, dtB=C64, outerA=None, outerB=None):
    """Complex B <- alpha*A + beta*B under perm (in place on the numpy buffer
    B); alpha and beta may be complex."""
    n, oA, sB, oB = dims(perm, sizes, outerA, outerB)
    _check_buf(A, dtA, sizes, oA, "A")
    _check_buf(B, dtB, sB, oB, "B")
    a, b = complex(alpha), complex(beta)
    rc = lib().oracle_permute_complex(n, (ctypes.c_int * n)(*perm), _i64(sizes), _i64(outerA), _i64(outerB),
                                      dtA, dtB, a.real, a.imag, b.real, b.imag, _ptr(A), _ptr(B))
    if rc:
        raise ValueError(f"oracle_permute_complex rejected the problem (code {rc})")
    return B


def permute_complex_exact(perm, sizes, A, B, alpha=1.0, beta=0.0, dtA=C64, dtB=C64, outerA=None, outerB=None):
    """Exact complex value (each part rounded once to double) as a complex128
    array in B's layout, and the tolerance scale of each part as an (n, 2)
    float64 array (NaN where B has no element)."""
    n, oA, sB, oB = dims(perm, sizes, outerA, outerB)
    _check_buf(A, dtA, sizes, oA, "A")
    _check_buf(B, dtB, sB, oB, "B")
    vol = B.size
    R = np.full(2 * vol, np.nan)
    S = np.full(2 * vol, np.nan)
    a, b = complex(alpha), complex(beta)
    rc = lib().oracle_permute_complex_exact(n, (ctypes.c_int * n)(*perm), _i64(sizes), _i64(outerA),
                                            _i64(outerB), dtA, dtB, a.real, a.imag, b.real, b.imag, _ptr(A),
                                            _ptr(B), _ptr(R), _ptr(S))
    if rc:
        raise ValueError(f"oracle_permute_complex_exact rejected the problem (code {rc})")
    return R.view(np.complex128), S.reshape(vol, 2)


def fp8_scale(sizes, A, alpha=1.0, dtA=F32, outerA=None):
    """(scale, amax) of the FP8 E4M3 output for A's sub-tensor."""
    n = len(sizes)
    oA = list(outerA) if outerA is not None else list(sizes)
    _check_buf(A, dtA, sizes, oA, "A")
    amax = ctypes.c_float(0)
    s = lib().oracle_fp8_scale(n, _i64(sizes), _i64(outerA), dtA, float(alpha), _ptr(A),
                               ctypes.byref(amax))
    return float(np.float32(s)), float(np.float32(amax.value))


def bf16_from_f32(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(x.shape, np.uint16)
    lib().oracle_bf16_from_f32_n(_ptr(x), _ptr(y), x.size)
    return y


def e4m3_from_f32(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(x.shape, np.uint8)
    lib().oracle_e4m3_from_f32_n(_ptr(x), _ptr(y), x.size)
    return y


def e4m3_to_f32(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint8)
    y = np.empty(x.shape, np.float32)
    lib().oracle_e4m3_to_f32_n(_ptr(x), _ptr(y), x.size)
    return y


def fmaf(a, b, c) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    c = np.ascontiguousarray(c, dtype=np.float32)
    y = np.empty(a.shape, np.float32)
    lib().oracle_fmaf_n(_ptr(a), _ptr(b), _ptr(c), _ptr(y), a.size)
    return y


# ------------------------------------------------------------ contraction

def contract(modes_a, A, sizes_a, modes_b, B, sizes_b, modes_c, C, sizes_c, alpha=1.0, beta=0.0, absolute=False):
    """Tensor contraction by its definition (section 1: the operation TTGT
    computes), in float64: C[modes_c] = alpha * sum over the labels of A and B
    missing from C of A * B + beta * C, every tensor a flat column-major
    buffer.  numpy.einsum evaluates the sum of products (a library primitive
    serving as one step).  With absolute=True it returns the same contraction
    of |A|, |B| with |alpha|, |beta| and |C|: the scale of the GEMM's error
    bound.  B is read only when beta != 0."""
    letters = {}
    for m in list(modes_a) + list(modes_b) + list(modes_c):
        letters.setdefault(m, "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"[len(letters)])
    spec = "".join(letters[m] for m in modes_a) + "," + "".join(letters[m] for m in modes_b) + "->" + \
        "".join(letters[m] for m in modes_c)
    a = np.asarray(A, dtype=np.float64).reshape(tuple(sizes_a), order="F")
    b = np.asarray(B, dtype=np.float64).reshape(tuple(sizes_b), order="F")
    if absolute:
        a, b, alpha, beta = np.abs(a), np.abs(b), abs(alpha), abs(beta)
    r = alpha * np.einsum(spec, a, b).reshape(-1, order="F")
    if beta != 0.0:
        c = np.asarray(C, dtype=np.float64)
        r = r + beta * (np.abs(c) if absolute else c)
    return r
