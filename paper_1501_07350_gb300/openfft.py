"""Thin ctypes binding of the C ABI in include/openfft_gb.h.

Argument marshalling only: every step of the transform runs in the CUDA
kernels of libopenfft_gb.so.  Device buffers are passed as torch CUDA tensors
(or raw integer device pointers); torch provides memory and streams only.
There is no fallback: if the shared library has not been built, loading
raises an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

OK = 0
ERR_INVALID_ARG, ERR_P_TOO_LARGE, ERR_UNSUPPORTED_RADIX, ERR_CUDA, ERR_NOMEM = 1, 2, 3, 4, 5
ERR_TIMEOUT, ERR_ALIAS, ERR_UNSUPPORTED, ERR_BOUNDS = 6, 7, 8, 9

C2C_F64, C2C_F32, C2C_SPLIT_BF16, C2C_SPLIT_TF32 = 0, 1, 2, 3
R2C_F64, R2C_F32 = 4, 5
FORWARD, BACKWARD = -1, 1
VARIANT_PACK_EXCHANGE_UNPACK, VARIANT_PACK_UNPACK, VARIANT_FUSED = 0, 1, 2
VARIANT_ISEND_WAITALL, VARIANT_ISEND_WAITALL_BLOCK, VARIANT_ISEND_WAITSOME_BLOCK, VARIANT_SENDRECV = 3, 4, 5, 6
# the paper's methods (Sec. 3.2.1) by name
METHODS = {"Alltoallv": 0, "Isend_Waitsome": 1, "fused": 2, "Isend_Waitall": 3, "Isend_Waitall_Block": 4,
           "Isend_Waitsome_Block": 5, "Sendrecv": 6}
ARITH_NATIVE, ARITH_DOUBLE_FLOAT, ARITH_TC_TF32, ARITH_TC_BF16 = 0, 1, 2, 3
TUNE_DEFAULT, TUNE_EXHAUSTIVE, TUNE_LEARNED, TUNE_USER, TUNE_SAVED = 0, 1, 2, 3, 4
LAYOUT_ABC, LAYOUT_CAB, LAYOUT_CBA = 0, 1, 2
KERNEL_AUTO, KERNEL_WARP, KERNEL_TILE, KERNEL_GENERIC = 0, 1, 2, 3

# every symbol declared in include/openfft_gb.h
EXPORTS = [
    "openfft_plan", "openfft_exec_c2c", "openfft_exec_c2c_host", "openfft_destroy", "openfft_sync",
    "openfft_set_stream", "openfft_last_error", "openfft_last_status", "openfft_box", "openfft_counts",
    "openfft_decomp_box", "openfft_decomp_counts", "openfft_decomp_degree", "openfft_set_tuning",
    "openfft_num_candidates", "openfft_candidate", "openfft_current_candidate", "openfft_redistribute",
    "openfft_set_timing", "openfft_get_timing", "openfft_exec_c2c_noalloc",
    "openfft_plan_many", "openfft_exec_many", "openfft_batch_debug",
    "openfft_mlp_num_params", "openfft_mlp_predict", "openfft_mlp_loss_grad", "openfft_mlp_train",
    "openfft_num_features", "openfft_candidate_features", "openfft_tune_times", "openfft_set_cost_model",
    "openfft_tc_gemm", "openfft_exec_r2c", "openfft_exec_c2r", "openfft_tc_debug", "openfft_set_host_chunks",
    "openfft_exec_c2c_host_async", "openfft_set_copy_streams",
    "openfft_debug_alloc_fail", "openfft_checked_build", "openfft_tuning_save", "openfft_tuning_load",
    "openfft_tuning_lookup", "openfft_tuning_clear", "openfft_debug_bounds_status", "openfft_nd_plan", "openfft_nd_exec", "openfft_nd_destroy", "openfft_nd_set_stream",
    "openfft_nd_box", "openfft_nd_decomp_box", "openfft_nd_decomp_counts", "openfft_dist_rows", "openfft_dist_counts", "openfft_dist_pack_host", "openfft_dist_unpack_host",
    "openfft_dist_plan", "openfft_dist_destroy", "openfft_dist_set_stream", "openfft_dist_elem_bytes",
    "openfft_dist_exchange_counts", "openfft_dist_stage", "openfft_dist_pack", "openfft_dist_unpack",
]

_lock = threading.Lock()
_lib = None


class OpenFFTError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("openfft status %d: %s" % (status, message))
        self.status = status


def checked() -> bool:
    """OPENFFT_GB_CHECKED=1 in the environment selects the bounds-checked
    library (libopenfft_gb_checked.so, built by _build.build(checked=True))."""
    return os.environ.get("OPENFFT_GB_CHECKED", "") == "1"


def library_path() -> str:
    return _build.CHECKED_LIB_PATH if checked() else _build.LIB_PATH


def load():
    """Load libopenfft_gb.so (build it first with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libopenfft_gb.so is not built (%s); run `python -c \"import "
                               "__graft_entry__ as g; g.build()\"`" % path)
        lib = ctypes.CDLL(path)
        i32, i64, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        p64 = ctypes.POINTER(ctypes.c_int64)
        pi32 = ctypes.POINTER(ctypes.c_int)
        pf = ctypes.POINTER(ctypes.c_float)
        sig = {
            "openfft_plan": (vp, [i32, i32, i32, i32, i32]),
            "openfft_exec_c2c": (i32, [vp, vp, vp, i32]),
            "openfft_exec_r2c": (i32, [vp, vp, vp]),
            "openfft_tc_debug": (i32, [i32, ctypes.c_longlong]),
            "openfft_exec_c2r": (i32, [vp, vp, vp]),
            "openfft_exec_c2c_host": (i32, [vp, vp, vp, i32]),
            "openfft_set_host_chunks": (i32, [vp, i32]),
            "openfft_exec_c2c_host_async": (i32, [vp, vp, vp, i32]),
            "openfft_set_copy_streams": (i32, [vp, vp, vp]),
            "openfft_destroy": (None, [vp]),
            "openfft_sync": (i32, [vp]),
            "openfft_set_stream": (i32, [vp, vp]),
            "openfft_last_error": (ctypes.c_char_p, []),
            "openfft_last_status": (i32, []),
            "openfft_box": (i32, [vp, i32, i32, p64, p64, p64, p64]),
            "openfft_counts": (i32, [vp, i32, p64]),
            "openfft_decomp_box": (i32, [i32, i32, i32, i32, i32, i32, p64, p64, p64, p64]),
            "openfft_decomp_counts": (i32, [i32, i32, i32, i32, i32, p64]),
            "openfft_decomp_degree": (i32, [i32, i32, i32, i32, i32]),
            "openfft_set_tuning": (i32, [vp, i32, i32]),
            "openfft_num_candidates": (i32, [vp]),
            "openfft_candidate": (i32, [vp, i32, pi32, pi32, pi32, pi32]),
            "openfft_current_candidate": (i32, [vp]),
            "openfft_redistribute": (i32, [vp, i32, i32, vp, vp]),
            "openfft_set_timing": (i32, [vp, i32]),
            "openfft_get_timing": (i32, [vp, ctypes.POINTER(ctypes.c_double), p64]),
            "openfft_exec_c2c_noalloc": (i32, [i32, i32, i32, i32, i32, vp, vp, i32, vp]),
            "openfft_plan_many": (vp, [i32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), i32]),
            "openfft_exec_many": (i32, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32]),
            "openfft_batch_debug": (i32, [vp, i32, ctypes.c_longlong]),
            "openfft_mlp_num_params": (i32, [i32, i32]),
            "openfft_mlp_predict": (i32, [i32, i32, pf, pf, i32, pf]),
            "openfft_mlp_loss_grad": (i32, [i32, i32, pf, pf, pf, i32, pf, pf]),
            "openfft_mlp_train": (i32, [i32, i32, pf, pf, i32, i32, ctypes.c_float, pf, pf]),
            "openfft_num_features": (i32, []),
            "openfft_candidate_features": (i32, [vp, i32, pf]),
            "openfft_tune_times": (i32, [vp, pf]),
            "openfft_set_cost_model": (i32, [i32, i32, i32, pf]),
            "openfft_tc_gemm": (i32, [i32, i32, i32, i32, i32, pf, pf, pf]),
            "openfft_debug_alloc_fail": (i32, [ctypes.c_longlong]),
            "openfft_checked_build": (i32, []),
            "openfft_tuning_save": (i32, [ctypes.c_char_p]),
            "openfft_tuning_load": (i32, [ctypes.c_char_p]),
            "openfft_tuning_lookup": (i32, [i32, i32, i32, i32, i32, pi32, pi32]),
            "openfft_tuning_clear": (i32, []),
            "openfft_debug_bounds_status": (i32, [pi32]),
            "openfft_nd_plan": (vp, [i32, pi32, i32, i32]),
            "openfft_nd_exec": (i32, [vp, vp, vp, i32]),
            "openfft_nd_destroy": (None, [vp]),
            "openfft_nd_set_stream": (i32, [vp, vp]),
            "openfft_nd_box": (i32, [vp, i32, i32, p64, p64]),
            "openfft_nd_decomp_box": (i32, [i32, pi32, i32, i32, i32, p64, p64]),
            "openfft_nd_decomp_counts": (i32, [i32, pi32, i32, i32, p64]),
            "openfft_dist_rows": (i32, [i32, i32, i32, i32, i32, i32, i32, p64, p64]),
            "openfft_dist_counts": (i32, [i32, i32, i32, i32, i32, i32, p64]),
            "openfft_dist_pack_host": (i32, [i32, i32, i32, i32, i32, i32, i32, i32, vp, vp]),
            "openfft_dist_unpack_host": (i32, [i32, i32, i32, i32, i32, i32, i32, i32, vp, vp]),
            "openfft_dist_plan": (vp, [i32, i32, i32, i32, i32, i32, i32]),
            "openfft_dist_destroy": (None, [vp]),
            "openfft_dist_set_stream": (i32, [vp, vp]),
            "openfft_dist_elem_bytes": (i32, [vp]),
            "openfft_dist_exchange_counts": (i32, [vp, i32, p64, p64]),
            "openfft_dist_stage": (i32, [vp, i32, i32, vp, vp]),
            "openfft_dist_pack": (i32, [vp, i32, vp, vp]),
            "openfft_dist_unpack": (i32, [vp, i32, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def last_error() -> str:
    return load().openfft_last_error().decode()


def _check(status: int):
    if status != OK:
        raise OpenFFTError(status, last_error())


def _ptr(x) -> int:
    """Device pointer of a torch tensor (or an int passed through)."""
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


# ------------------------------------------------ same names as the C ABI --

def openfft_plan(Na: int, Nb: int, Nc: int, P: int, dtype: int) -> int:
    h = load().openfft_plan(Na, Nb, Nc, P, dtype)
    if not h:
        raise OpenFFTError(load().openfft_last_status(), last_error())
    return h


def openfft_exec_c2c(plan: int, inp, out, direction: int) -> None:
    _check(load().openfft_exec_c2c(plan, _ptr(inp), _ptr(out), direction))


def openfft_tc_debug(what: int, value: int) -> None:
    """Test controls of the DFT-GEMM stages: 1 = wait budget (cycles), 2 = skip the MMAs."""
    _check(load().openfft_tc_debug(what, value))


def openfft_exec_r2c(plan: int, inp, out) -> None:
    """Real abc array (float64 / float32) -> half spectrum [Nc//2+1][Nb][Na] (complex)."""
    _check(load().openfft_exec_r2c(plan, _ptr(inp), _ptr(out)))


def openfft_exec_c2r(plan: int, inp, out) -> None:
    """Half spectrum [Nc//2+1][Nb][Na] -> real abc array, divided by N."""
    _check(load().openfft_exec_c2r(plan, _ptr(inp), _ptr(out)))


def openfft_exec_c2c_host(plan: int, host_in: np.ndarray, host_out: np.ndarray, direction: int) -> None:
    _check(load().openfft_exec_c2c_host(plan, host_in.ctypes.data, host_out.ctypes.data, direction))


def openfft_exec_c2c_host_async(plan: int, host_in: np.ndarray, host_out: np.ndarray, direction: int) -> None:
    """Enqueue only; the buffers belong to the call until openfft_sync(plan)."""
    _check(load().openfft_exec_c2c_host_async(plan, host_in.ctypes.data, host_out.ctypes.data, direction))


def openfft_set_copy_streams(plan: int, h2d=None, d2h=None) -> None:
    """Upload / download streams of the host-buffer calls (torch streams, raw
    handles or None for the plan's own)."""
    def handle(s):
        return None if s is None else (s.cuda_stream if hasattr(s, "cuda_stream") else s)
    _check(load().openfft_set_copy_streams(plan, handle(h2d), handle(d2h)))


def openfft_set_host_chunks(plan: int, chunks: int) -> None:
    """Line ranges of the host-buffer exec's copy / compute overlap (0 = by size, 1..32)."""
    _check(load().openfft_set_host_chunks(plan, chunks))


def openfft_destroy(plan: int) -> None:
    load().openfft_destroy(plan)


def openfft_sync(plan: int) -> None:
    _check(load().openfft_sync(plan))


def openfft_set_stream(plan: int, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().openfft_set_stream(plan, raw))


def openfft_box(plan: int, which: int, rank: int):
    s = (ctypes.c_int64 * 3)()
    e = (ctypes.c_int64 * 3)()
    off, cnt = ctypes.c_int64(), ctypes.c_int64()
    _check(load().openfft_box(plan, which, rank, s, e, ctypes.byref(off), ctypes.byref(cnt)))
    return tuple(s), tuple(e), off.value, cnt.value


def openfft_counts(plan: int, exchange: int, P: int) -> np.ndarray:
    C = np.zeros((P, P), dtype=np.int64)
    _check(load().openfft_counts(plan, exchange, C.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return C


def openfft_decomp_box(Na, Nb, Nc, P, layout, rank):
    s = (ctypes.c_int64 * 3)()
    e = (ctypes.c_int64 * 3)()
    off, cnt = ctypes.c_int64(), ctypes.c_int64()
    _check(load().openfft_decomp_box(Na, Nb, Nc, P, layout, rank, s, e, ctypes.byref(off), ctypes.byref(cnt)))
    return tuple(s), tuple(e), off.value, cnt.value


def openfft_decomp_counts(Na, Nb, Nc, P, exchange) -> np.ndarray:
    C = np.zeros((P, P), dtype=np.int64)
    _check(load().openfft_decomp_counts(Na, Nb, Nc, P, exchange, C.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return C


def openfft_decomp_degree(Na, Nb, Nc, P, layout) -> int:
    return int(load().openfft_decomp_degree(Na, Nb, Nc, P, layout))


def openfft_set_tuning(plan: int, mode: int, candidate: int = 0) -> None:
    _check(load().openfft_set_tuning(plan, mode, candidate))


def openfft_num_candidates(plan: int) -> int:
    return int(load().openfft_num_candidates(plan))


def openfft_candidate(plan: int, index: int):
    v, a, g, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().openfft_candidate(plan, index, ctypes.byref(v), ctypes.byref(a), ctypes.byref(g), ctypes.byref(t)))
    return {"variant": v.value, "arith": a.value, "lines_per_cta": g.value, "kernel": t.value}


def openfft_current_candidate(plan: int) -> int:
    return int(load().openfft_current_candidate(plan))


def openfft_redistribute(plan: int, exchange: int, variant: int, inp, out) -> None:
    _check(load().openfft_redistribute(plan, exchange, variant, _ptr(inp), _ptr(out)))


def openfft_set_timing(plan: int, enable: bool) -> None:
    _check(load().openfft_set_timing(plan, 1 if enable else 0))


PHASES = ("fft", "buffer_comm", "communication", "exec")


def openfft_get_timing(plan: int) -> dict:
    """Per-phase milliseconds and launch counts since the previous call."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int64 * 4)()
    _check(load().openfft_get_timing(plan, ms, n))
    return {name: {"ms": ms[i], "launches": n[i]} for i, name in enumerate(PHASES)}


def openfft_exec_c2c_noalloc(Na: int, Nb: int, Nc: int, P: int, dtype: int, inp, out, direction: int,
                             stream=None) -> None:
    """Plan-free transform that allocates nothing (static device scratch, 16 MiB)."""
    raw = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().openfft_exec_c2c_noalloc(Na, Nb, Nc, P, dtype, _ptr(inp), _ptr(out), direction, raw))


def openfft_debug_alloc_fail(nth: int) -> None:
    """Test control: the nth device allocation from now on fails (0 = off)."""
    _check(load().openfft_debug_alloc_fail(nth))


def openfft_tuning_save(path: str) -> None:
    """Write the process-wide table of tuned choices to a text file."""
    _check(load().openfft_tuning_save(os.fsencode(path)))


def openfft_tuning_load(path: str) -> None:
    """Merge a file of tuned choices into the process-wide table."""
    _check(load().openfft_tuning_load(os.fsencode(path)))


def openfft_tuning_lookup(Na: int, Nb: int, Nc: int, P: int, dtype: int):
    """The recorded choice of a problem as (variant, arith, lines_per_cta,
    kernel), or None."""
    found = ctypes.c_int(0)
    choice = (ctypes.c_int * 4)()
    _check(load().openfft_tuning_lookup(Na, Nb, Nc, P, dtype, ctypes.byref(found), choice))
    return tuple(int(v) for v in choice) if found.value else None


def openfft_tuning_clear() -> None:
    _check(load().openfft_tuning_clear())


def openfft_checked_build() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(load().openfft_checked_build())


def openfft_debug_bounds_status() -> int:
    """Checked build: the per-device bounds status word (0 or OPENFFT_ERR_BOUNDS),
    read after synchronising the device, then cleared."""
    st = ctypes.c_int(0)
    _check(load().openfft_debug_bounds_status(ctypes.byref(st)))
    return st.value


# ------------------------------------------------- 4-D and 5-D transforms --

def _dims32(dims):
    return (ctypes.c_int * len(dims))(*[int(v) for v in dims])


def openfft_nd_plan(dims, P: int, dtype: int) -> int:
    h = load().openfft_nd_plan(len(dims), _dims32(dims), P, dtype)
    if not h:
        raise OpenFFTError(load().openfft_last_status(), last_error())
    return h


def openfft_nd_exec(plan: int, inp, out, direction: int) -> None:
    _check(load().openfft_nd_exec(plan, _ptr(inp), _ptr(out), direction))


def openfft_nd_destroy(plan: int) -> None:
    load().openfft_nd_destroy(plan)


def openfft_nd_set_stream(plan: int, stream) -> None:
    raw = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().openfft_nd_set_stream(plan, raw))


def openfft_nd_box(plan: int, which: int, rank: int):
    off, cnt = ctypes.c_int64(), ctypes.c_int64()
    _check(load().openfft_nd_box(plan, which, rank, ctypes.byref(off), ctypes.byref(cnt)))
    return off.value, cnt.value


def openfft_nd_decomp_box(dims, P: int, ordering: int, rank: int):
    off, cnt = ctypes.c_int64(), ctypes.c_int64()
    _check(load().openfft_nd_decomp_box(len(dims), _dims32(dims), P, ordering, rank, ctypes.byref(off),
                                        ctypes.byref(cnt)))
    return off.value, cnt.value


def openfft_nd_decomp_counts(dims, P: int, exchange: int) -> np.ndarray:
    out = np.zeros((P, P), dtype=np.int64)
    _check(load().openfft_nd_decomp_counts(len(dims), _dims32(dims), P, exchange,
                                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out


# ------------------------------------------- transform over several devices --

def openfft_dist_rows(Na, Nb, Nc, P, G, layout, g):
    """(offset, count) of device g's slice of `layout` (host only)."""
    off, cnt = ctypes.c_int64(), ctypes.c_int64()
    _check(load().openfft_dist_rows(Na, Nb, Nc, P, G, layout, g, ctypes.byref(off), ctypes.byref(cnt)))
    return off.value, cnt.value


def openfft_dist_counts(Na, Nb, Nc, P, G, exchange) -> np.ndarray:
    """G x G device count matrix of one transpose (host only)."""
    out = np.zeros((G, G), dtype=np.int64)
    _check(load().openfft_dist_counts(Na, Nb, Nc, P, G, exchange,
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out


def openfft_dist_pack_host(Na, Nb, Nc, P, G, exchange, g, src: np.ndarray, send: np.ndarray) -> None:
    _check(load().openfft_dist_pack_host(Na, Nb, Nc, P, G, exchange, g, src.itemsize,
                                         src.ctypes.data, send.ctypes.data))


def openfft_dist_unpack_host(Na, Nb, Nc, P, G, exchange, g, recv: np.ndarray, dst: np.ndarray) -> None:
    _check(load().openfft_dist_unpack_host(Na, Nb, Nc, P, G, exchange, g, recv.itemsize,
                                           recv.ctypes.data, dst.ctypes.data))


def openfft_dist_plan(Na, Nb, Nc, P, G, g, dtype) -> int:
    h = load().openfft_dist_plan(Na, Nb, Nc, P, G, g, dtype)
    if not h:
        raise OpenFFTError(load().openfft_last_status(), last_error())
    return h


def openfft_dist_destroy(plan: int) -> None:
    load().openfft_dist_destroy(plan)


def openfft_dist_set_stream(plan: int, stream) -> None:
    raw = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().openfft_dist_set_stream(plan, raw))


def openfft_dist_elem_bytes(plan: int) -> int:
    return int(load().openfft_dist_elem_bytes(plan))


def openfft_dist_exchange_counts(plan: int, exchange: int, G: int):
    """(send_counts[G], recv_counts[G]) of this device in one transpose."""
    sc = np.zeros(G, dtype=np.int64)
    rc = np.zeros(G, dtype=np.int64)
    p64 = ctypes.POINTER(ctypes.c_int64)
    _check(load().openfft_dist_exchange_counts(plan, exchange, sc.ctypes.data_as(p64), rc.ctypes.data_as(p64)))
    return sc, rc


def openfft_dist_stage(plan: int, stage: int, direction: int, inp, out) -> None:
    _check(load().openfft_dist_stage(plan, stage, direction, _ptr(inp), _ptr(out)))


def openfft_dist_pack(plan: int, exchange: int, src, send) -> None:
    _check(load().openfft_dist_pack(plan, exchange, _ptr(src), _ptr(send)))


def openfft_dist_unpack(plan: int, exchange: int, recv, dst) -> None:
    _check(load().openfft_dist_unpack(plan, exchange, _ptr(recv), _ptr(dst)))


def openfft_plan_many(shapes, Ps, dtype: int) -> int:
    """Batched plan of len(shapes) transforms; shapes: [(Na, Nb, Nc)], Ps: [P]."""
    count = len(shapes)
    dims = (ctypes.c_int * (3 * count))(*[int(v) for sh in shapes for v in sh])
    ps = (ctypes.c_int * count)(*[int(p) for p in Ps])
    h = load().openfft_plan_many(count, dims, ps, dtype)
    if not h:
        raise OpenFFTError(load().openfft_last_status(), last_error())
    return h


def openfft_exec_many(plan: int, inputs, outputs, direction: int) -> None:
    count = len(inputs)
    ins = (ctypes.c_void_p * count)(*[_ptr(x) for x in inputs])
    outs = (ctypes.c_void_p * count)(*[_ptr(x) for x in outputs])
    _check(load().openfft_exec_many(plan, ins, outs, direction))


def openfft_batch_debug(plan: int, what: int, value: int) -> None:
    _check(load().openfft_batch_debug(plan, what, value))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _pf(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def openfft_mlp_num_params(d: int, hidden: int) -> int:
    return int(load().openfft_mlp_num_params(d, hidden))


def openfft_mlp_predict(d: int, hidden: int, params, X) -> np.ndarray:
    params, X = _f32(params), _f32(X)
    n = X.shape[0]
    yhat = np.empty(n, dtype=np.float32)
    _check(load().openfft_mlp_predict(d, hidden, _pf(params), _pf(X), n, _pf(yhat)))
    return yhat


def openfft_mlp_loss_grad(d: int, hidden: int, params, X, y):
    params, X, y = _f32(params), _f32(X), _f32(y)
    loss = np.zeros(1, dtype=np.float32)
    grad = np.empty_like(params)
    _check(load().openfft_mlp_loss_grad(d, hidden, _pf(params), _pf(X), _pf(y), X.shape[0], _pf(loss), _pf(grad)))
    return float(loss[0]), grad


def openfft_mlp_train(d: int, hidden: int, X, y, steps: int, lr: float, params):
    """Returns (trained params, loss before each step)."""
    X, y = _f32(X), _f32(y)
    p = _f32(params).copy()
    losses = np.empty(steps, dtype=np.float32)
    _check(load().openfft_mlp_train(d, hidden, _pf(X), _pf(y), X.shape[0], steps, lr, _pf(p), _pf(losses)))
    return p, losses


def openfft_num_features() -> int:
    return int(load().openfft_num_features())


def openfft_candidate_features(plan: int, index: int) -> np.ndarray:
    f = np.empty(openfft_num_features(), dtype=np.float32)
    _check(load().openfft_candidate_features(plan, index, _pf(f)))
    return f


def openfft_tune_times(plan: int) -> np.ndarray:
    ms = np.empty(openfft_num_candidates(plan), dtype=np.float32)
    _check(load().openfft_tune_times(plan, _pf(ms)))
    return ms


def openfft_set_cost_model(d: int, hidden: int, params, count: int = 1) -> None:
    """Install an ensemble of `count` networks (params: count parameter sets
    back to back), or remove the model with params=None."""
    if params is None:
        _check(load().openfft_set_cost_model(0, d, hidden, None))
    else:
        p = _f32(params)
        _check(load().openfft_set_cost_model(count, d, hidden, _pf(p)))


def openfft_tc_gemm(A, B, tf32: bool = True, split: bool = True) -> np.ndarray:
    """D = A B^T on the tensor cores (split precision, fp32 accumulation)."""
    A, B = _f32(A), _f32(B)
    M, K = A.shape
    N = B.shape[0]
    D = np.empty((M, N), dtype=np.float32)
    _check(load().openfft_tc_gemm(1 if tf32 else 0, 1 if split else 0, M, N, K, _pf(A), _pf(B), _pf(D)))
    return D


# ------------------------------------------------------- convenience ----

class Plan:
    """RAII wrapper: ``with Plan(Na, Nb, Nc, P, dtype) as p: p.exec(x, y, FORWARD)``.

    Uses torch's current CUDA stream unless ``stream`` is given."""

    def __init__(self, Na, Nb, Nc, P, dtype=C2C_F64, stream=None):
        import torch
        self.shape = (Na, Nb, Nc)
        self.P = P
        self.dtype = dtype
        self.handle = openfft_plan(Na, Nb, Nc, P, dtype)
        openfft_set_stream(self.handle, stream if stream is not None else torch.cuda.current_stream())

    def exec(self, inp, out, direction=FORWARD):
        openfft_exec_c2c(self.handle, inp, out, direction)

    def close(self):
        if self.handle:
            openfft_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
