"""Thin ctypes binding of libttc (include/ttc.h).

Argument marshalling only: every step of the permute-scale-add runs in the
library's CUDA kernels.  Tensors may be passed as torch tensors (their
``data_ptr()`` is used) or as raw integer device pointers; streams as
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers, or None (the
current torch stream when torch is loaded, else the legacy default stream).

There is no fallback: if ``libttc.so`` is missing or fails to load, ``lib()``
raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttc.so")

DTYPES = {"f32": 0, "f64": 1, "bf16": 2, "e4m3": 3, "c64": 4, "c128": 5}
DTYPE_BYTES = {"f32": 4, "f64": 8, "bf16": 2, "e4m3": 1, "c64": 8, "c128": 16}
COMPLEX_DTYPES = ("c64", "c128")
MAX_DIM = 16
STATUS = {0: "TTC_OK", 1: "TTC_ERR_INVALID_PERM", 2: "TTC_ERR_INVALID_SIZE", 3: "TTC_ERR_INVALID_OUTER",
          4: "TTC_ERR_UNSUPPORTED_DTYPE", 5: "TTC_ERR_ALIAS", 6: "TTC_ERR_ALIGN", 7: "TTC_ERR_OOM",
          8: "TTC_ERR_CUDA", 9: "TTC_ERR_TIMEOUT", 10: "TTC_ERR_BUDGET", 11: "TTC_ERR_INVALID_ARG",
          12: "TTC_ERR_NOT_READY"}
STATUS_CODE = {v: k for k, v in STATUS.items()}


class TTCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class PlanInfo(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("perm", ctypes.c_int * MAX_DIM),
                ("sizes", ctypes.c_int64 * MAX_DIM), ("stride_A", ctypes.c_int64 * MAX_DIM),
                ("stride_B", ctypes.c_int64 * MAX_DIM), ("n", ctypes.c_int64),
                ("algorithmic_bytes", ctypes.c_int64), ("variant", ctypes.c_int),
                ("tile_c", ctypes.c_int), ("tile_a", ctypes.c_int), ("tile_b", ctypes.c_int),
                ("ntiles", ctypes.c_int64), ("vec_in", ctypes.c_int), ("vec_out", ctypes.c_int),
                ("candidate", ctypes.c_int), ("ncandidates", ctypes.c_int),
                ("lanes_a", ctypes.c_int), ("lanes_b", ctypes.c_int), ("slot_tables", ctypes.c_int),
                ("packed_threads", ctypes.c_int), ("packed_rows", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("epochs", ctypes.c_int64), ("launches", ctypes.c_int64), ("bytes", ctypes.c_int64),
                ("p50_us", ctypes.c_double), ("p90_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("first_submit_s", ctypes.c_double), ("last_complete_s", ctypes.c_double),
                ("peak_inflight_bytes", ctypes.c_int64)]


# Every symbol include/ttc.h declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "ttc_plan": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _i64p,
                                _i64p, _i64p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "ttc_plan_complex": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _i64p,
                                        _i64p, _i64p, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4),
    "ttc_execute": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "ttc_plan_destroy": (ctypes.c_int, [_vp]),
    "ttc_plan_set_fp8_scale": (ctypes.c_int, [_vp, _vp]),
    "ttc_plan_get_fp8_scale": (ctypes.c_int, [_vp, _vp, _vp]),
    "ttc_plan_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(PlanInfo)]),
    "ttc_plan_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_float)]),
    "ttc_plan_select_candidate": (ctypes.c_int, [_vp, ctypes.c_int]),
    "ttc_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "ttc_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "ttc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ttc_last_error": (ctypes.c_char_p, []),
    "ttc_launch_count": (ctypes.c_int64, []),
    "ttc_execute_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ttc_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp)]),
    "ttc_batch_add": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "ttc_batch_execute": (ctypes.c_int, [_vp, _vp]),
    "ttc_batch_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "ttc_batch_destroy": (ctypes.c_int, [_vp]),
    "ttc_batch_info": (ctypes.c_int, [_vp, _i64p, _i64p]),
    "ttc_batch_set_direct_threshold": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "ttc_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int64)]),
    "ttc_contraction_plan": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _i64p,
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_int), _i64p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int), _i64p, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double]),
    "ttc_contraction_execute": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ttc_contraction_check": (ctypes.c_int, [_vp]),
    "ttc_contraction_info": (ctypes.c_int, [_vp, _i64p, _i64p, _i64p, ctypes.POINTER(ctypes.c_int)]),
    "ttc_contraction_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "ttc_contraction_destroy": (ctypes.c_int, [_vp]),
    "ttc_packed_gemm_plan": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _i64p,
                                            _i64p, ctypes.c_int, ctypes.c_int64, ctypes.c_double]),
    "ttc_packed_gemm_execute": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ttc_packed_gemm_check": (ctypes.c_int, [_vp]),
    "ttc_packed_gemm_info": (ctypes.c_int, [_vp, _i64p, _i64p, _i64p]),
    "ttc_packed_gemm_destroy": (ctypes.c_int, [_vp]),
    "ttc_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_int, ctypes.c_int64]),
    "ttc_server_submit": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64p]),
    "ttc_server_poll": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64]),
    "ttc_server_drain": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "ttc_server_stats": (ctypes.c_int, [_vp, _vp]),
    "ttc_server_destroy": (ctypes.c_int, [_vp]),
    "ttc_server_times": (ctypes.c_int, [_vp, ctypes.c_int64] + [ctypes.POINTER(ctypes.c_double)] * 4),
    # include/ttc_debug.h
    "ttc_debug_verify_schedule": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]),
    "ttc_debug_describe_candidate": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]),
    "ttc_debug_slot_tables": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                             _i64p]),
    "ttc_debug_packed_gemm_skip_mma": (ctypes.c_int, [_vp, ctypes.c_int]),
    "ttc_debug_contraction_use_cublas": (ctypes.c_int, [_vp, ctypes.c_int]),
    "ttc_debug_packed_gemm_classic": (ctypes.c_int, [_vp, ctypes.c_int]),
    "ttc_packed_gemm_set_fp8": (ctypes.c_int, [_vp, _vp, _vp]),
    "ttc_debug_contraction_gemm_variant": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ttc_debug_server_set_watchdog": (ctypes.c_int, [_vp, ctypes.c_double]),
    "ttc_debug_server_submit_delay": (ctypes.c_int, [_vp, ctypes.c_int64, _i64p]),
}

_lib = None


def lib():
    """Load libttc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1607_01249_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise TTCError(status, lib().ttc_last_error().decode(errors="replace"))


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int:
    if s is None:
        try:
            import sys
            if "torch" in sys.modules:
                import torch
                if torch.cuda.is_available() and torch.cuda.is_initialized():
                    return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _i64arr(vals):
    if vals is None:
        return None
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


class Plan:
    """A planned permute-scale-add B <- alpha*A + beta*B under `perm` (Eq. 1).
    For the complex dtypes alpha and beta may be complex numbers."""

    def __init__(self, perm, sizes, dtype_in="f32", dtype_out=None, alpha=1.0, beta=0.0,
                 outer_a=None, outer_b=None):
        dtype_out = dtype_out or dtype_in
        self.perm = tuple(int(p) for p in perm)
        self.sizes = tuple(int(s) for s in sizes)
        self.dtype_in, self.dtype_out = dtype_in, dtype_out
        a, b = complex(alpha), complex(beta)
        cplx = dtype_in in COMPLEX_DTYPES or a.imag != 0 or b.imag != 0
        self.alpha, self.beta = (a, b) if cplx else (a.real, b.real)
        self.outer_a = tuple(outer_a) if outer_a is not None else None
        self.outer_b = tuple(outer_b) if outer_b is not None else None
        h = ctypes.c_void_p()
        n = len(self.perm)
        if len(self.sizes) != n:
            raise ValueError("perm and sizes differ in length")
        args = (ctypes.byref(h), n, (ctypes.c_int * n)(*self.perm), _i64arr(self.sizes), _i64arr(self.outer_a),
                _i64arr(self.outer_b), DTYPES[dtype_in], DTYPES[dtype_out])
        if cplx:
            _check(lib().ttc_plan_complex(*args, a.real, a.imag, b.real, b.imag))
        else:
            _check(lib().ttc_plan(*args, a.real, b.real))
        self._h = h

    @property
    def handle(self):
        return self._h

    def execute(self, A, B, stream=None):
        _check(lib().ttc_execute(self._h, _ptr(A), _ptr(B), _stream(stream)))
        return B

    __call__ = execute

    def execute_noalloc(self, A, B, d_scale_out=None, stream=None):
        """ttc_execute_noalloc: the same work with the device scratch in the
        library's static array (no device-memory allocation)."""
        _check(lib().ttc_execute_noalloc(self._h, _ptr(A), _ptr(B), _ptr(d_scale_out), _stream(stream)))
        return B

    def info(self) -> dict:
        inf = PlanInfo()
        _check(lib().ttc_plan_get_info(self._h, ctypes.byref(inf)))
        N = inf.ndim
        return {"ndim": N, "perm": list(inf.perm[:N]), "sizes": list(inf.sizes[:N]),
                "stride_A": list(inf.stride_A[:N]), "stride_B": list(inf.stride_B[:N]), "n": inf.n,
                "algorithmic_bytes": inf.algorithmic_bytes,
                "variant": {0: "empty", 1: "copy", 2: "tile", 3: "rowcopy", 4: "tma_tile"}[inf.variant],
                "tile": (inf.tile_c, inf.tile_a, inf.tile_b), "ntiles": inf.ntiles,
                "vec": (inf.vec_in, inf.vec_out), "candidate": inf.candidate,
                "ncandidates": inf.ncandidates, "lanes": (inf.lanes_a, inf.lanes_b),
                "slot_tables": bool(inf.slot_tables), "packed_threads": inf.packed_threads,
                "packed_rows": inf.packed_rows,
                "kernel": ({0: "empty", 1: "copy_kernel", 3: "rowcopy_vec_kernel" if inf.vec_in > 1 else "rowcopy_kernel",
                            4: "tma2d_kernel"}.get(inf.variant) or
                           ("tile2_kernel" if inf.lanes_a else "tilep_kernel" if inf.packed_threads else
                            "rowsp_kernel" if inf.packed_rows else
                            "tile_slots_kernel" if inf.slot_tables else "tile_kernel"))}

    def autotune(self, max_candidates=8, stream=None) -> float:
        ms = ctypes.c_float(0)
        _check(lib().ttc_plan_autotune(self._h, int(max_candidates), _stream(stream), ctypes.byref(ms)))
        return float(ms.value)

    def verify_schedule(self, candidate=None) -> str:
        """Host-side check of a schedule's index arithmetic (no GPU); returns
        "" when it is sound, else a description of the first violation.
        candidate=-1-j checks the batched body's schedule j for this plan (0:
        its default, then the candidates the batch autotuner may pick)."""
        if candidate is None:
            candidate = self.info()["candidate"]
        buf = ctypes.create_string_buffer(512)
        st = lib().ttc_debug_verify_schedule(self._h, int(candidate), buf, 512)
        return "" if st == 0 else buf.value.decode(errors="replace") or "failed"

    def describe(self, candidate=None) -> str:
        """The planner's description of a candidate schedule (kernel, tile
        groups, lanes, grid order, estimate)."""
        if candidate is None:
            candidate = self.info()["candidate"]
        buf = ctypes.create_string_buffer(1024)
        _check(lib().ttc_debug_describe_candidate(self._h, int(candidate), buf, 1024))
        return buf.value.decode(errors="replace")

    def slot_tables(self, candidate=None):
        """The slot tables of a tile_slots_kernel candidate, as a list of
        int32 (layout of TileParams::slots)."""
        if candidate is None:
            candidate = self.info()["candidate"]
        need = ctypes.c_int64(0)
        lib().ttc_debug_slot_tables(self._h, int(candidate), None, 0, ctypes.byref(need))
        if need.value <= 0:
            raise TTCError(STATUS_CODE["TTC_ERR_INVALID_ARG"], "candidate has no slot tables")
        buf = (ctypes.c_int32 * need.value)()
        _check(lib().ttc_debug_slot_tables(self._h, int(candidate), buf, need.value, ctypes.byref(need)))
        return list(buf)

    def select(self, index: int):
        _check(lib().ttc_plan_select_candidate(self._h, int(index)))

    def set_fp8_scale(self, d_scale=None):
        _check(lib().ttc_plan_set_fp8_scale(self._h, _ptr(d_scale)))

    def get_fp8_scale(self, d_out, stream=None):
        _check(lib().ttc_plan_get_fp8_scale(self._h, _ptr(d_out), _stream(stream)))
        return d_out

    def close(self):
        if getattr(self, "_h", None):
            lib().ttc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Contraction:
    """C[modes_c] <- alpha * sum A[modes_a] * B[modes_b] + beta * C[modes_c]
    by Transpose-Transpose-GEMM-Transpose (ttc_contraction_*).  Modes are
    integer labels, sizes the extents of each tensor's indices (column-major).
    dtype f32 (gemm_dtype f32 or bf16) or f64."""

    def __init__(self, modes_a, sizes_a, modes_b, sizes_b, modes_c, sizes_c, dtype="f32", gemm_dtype=None,
                 alpha=1.0, beta=0.0):
        gemm_dtype = gemm_dtype or dtype
        self.modes = (tuple(modes_a), tuple(modes_b), tuple(modes_c))
        self.sizes = (tuple(sizes_a), tuple(sizes_b), tuple(sizes_c))
        self.dtype, self.gemm_dtype, self.alpha, self.beta = dtype, gemm_dtype, float(alpha), float(beta)
        h = ctypes.c_void_p()
        args = []
        for m, sz in zip(self.modes, self.sizes):
            if len(m) != len(sz):
                raise ValueError("modes and sizes differ in length")
            args += [len(m), (ctypes.c_int * max(len(m), 1))(*m), _i64arr(sz) if sz else None]
        _check(lib().ttc_contraction_plan(ctypes.byref(h), *args, DTYPES[dtype], DTYPES[gemm_dtype], self.alpha,
                                          self.beta))
        self._h = h

    def execute(self, A, B, C, stream=None):
        _check(lib().ttc_contraction_execute(self._h, _ptr(A), _ptr(B), _ptr(C), _stream(stream)))
        return C

    __call__ = execute

    def check(self):
        """ttc_contraction_check: raises TTCError(TTC_ERR_TIMEOUT) once after a
        tensor-core wait of the BF16 GEMM gave up."""
        _check(lib().ttc_contraction_check(self._h))

    def use_cublas(self, use: bool = True):
        """Testing hook: the BF16 GEMM on cuBLAS (a timed comparison)."""
        _check(lib().ttc_debug_contraction_use_cublas(self._h, 1 if use else 0))
        return self

    def autotune(self, max_candidates=8, stream=None):
        """Autotune the contraction's permute plans (before its first
        execution on the device)."""
        _check(lib().ttc_contraction_autotune(self._h, int(max_candidates), _stream(stream)))
        return self

    GEMM_VARIANTS = {0: "auto", 1: "single 128x256", 2: "pair 256x256", 3: "pair 256x128", 4: "single 128x192",
                     5: "single 128x128", 6: "pair 256x192"}

    def gemm_variant(self, variant: int = -1) -> int:
        """Testing hook: force the BF16 GEMM's tile shape (GEMM_VARIANTS; 0
        lets the library pick, -1 keeps the setting); returns the shape the
        last execution ran."""
        used = ctypes.c_int()
        _check(lib().ttc_debug_contraction_gemm_variant(self._h, int(variant), ctypes.byref(used)))
        return used.value

    def info(self) -> dict:
        m, n, k, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().ttc_contraction_info(self._h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(k),
                                          ctypes.byref(t)))
        return {"m": m.value, "n": n.value, "k": k.value, "permuted": {"A": bool(t.value & 1),
                                                                       "B": bool(t.value & 2),
                                                                       "C": bool(t.value & 4)}}

    def close(self):
        if getattr(self, "_h", None):
            lib().ttc_contraction_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PackedGemm:
    """C = alpha * P * Bm on the tensor cores, P the BF16 panel of the
    permutation (perm, sizes, outer_a) viewed as M x K (first rank_m indices
    form m), Bm a K x N BF16 column-major matrix (ttc_packed_gemm_*)."""

    def __init__(self, perm, sizes, rank_m, n, alpha=1.0, outer_a=None):
        self.perm, self.sizes = tuple(int(p) for p in perm), tuple(int(s) for s in sizes)
        self.outer_a = tuple(outer_a) if outer_a is not None else None
        h = ctypes.c_void_p()
        k = len(self.perm)
        _check(lib().ttc_packed_gemm_plan(ctypes.byref(h), k, (ctypes.c_int * k)(*self.perm), _i64arr(self.sizes),
                                          _i64arr(self.outer_a), int(rank_m), int(n), float(alpha)))
        self._h = h

    def execute(self, A, B, C, stream=None):
        _check(lib().ttc_packed_gemm_execute(self._h, _ptr(A), _ptr(B), _ptr(C), _stream(stream)))
        return C

    __call__ = execute

    def check(self):
        _check(lib().ttc_packed_gemm_check(self._h))

    def skip_mma(self, skip: bool = True):
        """Testing hook: executions issue no MMA, so their bounded waits run
        out and check() reports TTC_ERR_TIMEOUT."""
        _check(lib().ttc_debug_packed_gemm_skip_mma(self._h, int(bool(skip))))

    def set_fp8(self, scale_p=None, scale_b=None):
        """E4M3 operands: P packed as codes of alpha * a / scale_p, Bm given
        as E4M3 codes standing for scale_b * code (device float tensors of
        one element; None for both restores BF16)."""
        _check(lib().ttc_packed_gemm_set_fp8(self._h, _ptr(scale_p) if scale_p is not None else None,
                                             _ptr(scale_b) if scale_b is not None else None))
        self._scales = (scale_p, scale_b)
        return self

    def classic(self, on: bool = True):
        """Testing hook: run the register-staged kernel even when the
        warp-specialised one applies (K a multiple of 8)."""
        _check(lib().ttc_debug_packed_gemm_classic(self._h, 1 if on else 0))
        return self

    def info(self) -> dict:
        m, n, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ttc_packed_gemm_info(self._h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(k)))
        return {"m": m.value, "n": n.value, "k": k.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().ttc_packed_gemm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many permute-scale-adds launched together (ttc_batch_*): one kernel
    launch per class of problems (dtype pair, beta, body), one CTA per tile,
    with the large problems as their own kernels on a side stream; all of it
    one CUDA graph with graph_launch.  The batch keeps references to its
    plans so that they outlive it."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().ttc_batch_create(ctypes.byref(h)))
        self._h = h
        self._keep = []

    def add(self, plan: Plan, A, B):
        _check(lib().ttc_batch_add(self._h, plan.handle, _ptr(A), _ptr(B)))
        self._keep.append((plan, A, B))
        return self

    def execute(self, stream=None):
        _check(lib().ttc_batch_execute(self._h, _stream(stream)))

    def graph_launch(self, stream=None):
        _check(lib().ttc_batch_graph_launch(self._h, _stream(stream)))

    def info(self):
        p, t = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().ttc_batch_info(self._h, ctypes.byref(p), ctypes.byref(t)))
        return {"problems": p.value, "tiles": t.value}

    DIRECT_MIN_DEFAULT = 0     # off

    def set_direct_threshold(self, min_elements: int):
        """Problems of at least this many elements run as their own kernels
        beside the batch kernels (<= 0: none, the default)."""
        _check(lib().ttc_batch_set_direct_threshold(self._h, int(min_elements)))
        return self

    def autotune(self, max_candidates: int = 4, stream=None) -> int:
        """Time up to max_candidates batch-body schedules of each distinct
        plan and keep the fastest (ttc_batch_autotune); returns how many
        plans changed schedule."""
        n = ctypes.c_int64(0)
        _check(lib().ttc_batch_autotune(self._h, int(max_candidates), _stream(stream), ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().ttc_batch_destroy(self._h)
            self._h = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of requests (ttc_server_*).  The binding keeps a
    reference to each request's plan and tensors until the request is seen
    complete (poll or drain), so that they outlive it."""

    def __init__(self, budget_bytes: int, nstreams: int = 4, small_tiles: int = 4096):
        h = ctypes.c_void_p()
        _check(lib().ttc_server_create(ctypes.byref(h), int(budget_bytes), int(nstreams), int(small_tiles)))
        self._h = h
        self._keep = {}

    def submit(self, plan: Plan, A, B) -> int:
        t = ctypes.c_int64(-1)
        _check(lib().ttc_server_submit(self._h, plan.handle, _ptr(A), _ptr(B), ctypes.byref(t)))
        self._keep[t.value] = (plan, A, B)
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0) -> bool:
        """True once the request completed, False while it has not; raises
        if it failed."""
        st = lib().ttc_server_poll(self._h, int(ticket), int(timeout_us))
        if st == STATUS_CODE["TTC_ERR_NOT_READY"]:
            return False
        self._keep.pop(int(ticket), None)
        _check(st)
        return True

    def drain(self, timeout_us: int = 60_000_000):
        _check(lib().ttc_server_drain(self._h, int(timeout_us)))
        self._keep.clear()

    def times(self, ticket: int):
        """(submit_s, admit_s, launch_s, complete_s) of a completed request,
        host steady clock."""
        v = [ctypes.c_double(0) for _ in range(4)]
        _check(lib().ttc_server_times(self._h, int(ticket), *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_watchdog(self, seconds: float):
        """Testing hook: give up epochs unseen for this long."""
        _check(lib().ttc_debug_server_set_watchdog(self._h, float(seconds)))

    def submit_delay(self, microseconds: int) -> int:
        """Testing hook: a request that keeps one thread busy for the given
        time on a large-class stream (ends on its own)."""
        t = ctypes.c_int64(-1)
        _check(lib().ttc_debug_server_submit_delay(self._h, int(microseconds), ctypes.byref(t)))
        return t.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().ttc_server_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().ttc_server_destroy(self._h)
            self._h = None
        self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    return int(lib().ttc_launch_count())


def tune_cache_save(path: str):
    _check(lib().ttc_tune_cache_save(path.encode()))


def tune_cache_load(path: str):
    _check(lib().ttc_tune_cache_load(path.encode()))
