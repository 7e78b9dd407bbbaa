"""Python binding of the liftblas C-ABI (``include/lift.h``).

Argument marshalling only: every function has the name of its C entry
point, takes the same arguments in the same order, and passes device
pointers, sizes and a CUDA stream straight through.  Array arguments may be
torch tensors (their ``data_ptr()`` is passed) or integer addresses; the
stream defaults to torch's current stream.  A non-OK status raises
``LiftError``.  There is no fallback: if the shared library is missing, the
first call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liftblas.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_NO_MEMORY, ERR_TIMEOUT, ERR_NOT_INITIALIZED = range(7)
F32, BF16, FP8_E4M3 = 0, 1, 2
(OP_ASUM, OP_DOT, OP_SCAL, OP_GEMV, OP_ASUM_BF16, OP_DOT_BF16, OP_ASUM_FP8, OP_DOT_FP8, OP_NRM2,
 OP_SUM, OP_AXPY, OP_GEMV_T, OP_BLACKSCHOLES, OP_ASUM_COMP, OP_DOT_COMP) = range(15)
NUM_OPS = 15
MLP_OPS = 15    # op ids a cost model can cover (all of them)
NUM_FEATURES = 12   # lift_features output length
OP_NAMES = ["asum", "dot", "scal", "gemv", "asum_bf16", "dot_bf16", "asum_fp8", "dot_fp8", "nrm2",
            "sum", "axpy", "gemv_t", "blackscholes", "asum_comp", "dot_comp"]
POLICY_FIXED, POLICY_TABLE, POLICY_MLP, POLICY_MLP_TUNE = 0, 1, 2, 3


class LiftError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({status_string(status)}) {detail}".strip())


class OpDesc(ctypes.Structure):
    """lift_op_desc"""
    _fields_ = [("op", ctypes.c_int), ("variant", ctypes.c_int), ("n", ctypes.c_int64),
                ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("A", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class VariantInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("op", "id", "tile", "vw", "threads", "stride", "tree",
                                           "cluster", "passes", "stages", "rows", "lanes",
                                           "final_threads", "grid")] + [("name", ctypes.c_char * 64)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "lift_init": ([ctypes.c_int], ctypes.c_int),
    "lift_finalize": ([], ctypes.c_int),
    "lift_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "lift_last_error": ([], ctypes.c_char_p),
    "lift_sm_count": ([], ctypes.c_int),
    "lift_read_status": ([ctypes.c_int], ctypes.c_int),
    "lift_asum": ([_P, _I64, _P, _P], ctypes.c_int),
    "lift_dot": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "lift_scal": ([_I64, ctypes.c_float, _P, _P, _P], ctypes.c_int),
    "lift_gemv": ([_I64, _I64, ctypes.c_float, _P, _I64, _P, ctypes.c_float, _P, _P], ctypes.c_int),
    "lift_asum_v": ([ctypes.c_int, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_dot_v": ([ctypes.c_int, _P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_scal_v": ([ctypes.c_int, _I64, ctypes.c_float, _P, _P, _P], ctypes.c_int),
    "lift_gemv_v": ([ctypes.c_int, _I64, _I64, ctypes.c_float, _P, _I64, _P, ctypes.c_float, _P, _P],
                    ctypes.c_int),
    "lift_variant_count": ([ctypes.c_int], ctypes.c_int),
    "lift_variant_describe": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(VariantInfo)], ctypes.c_int),
    "lift_variant_grid": ([ctypes.c_int, ctypes.c_int, _I64, ctypes.POINTER(_I64)], ctypes.c_int),
    "lift_asum_ex": ([ctypes.c_int, _P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_dot_ex": ([ctypes.c_int, _P, _P, _P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_asum_ex_v": ([ctypes.c_int, ctypes.c_int, _P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_dot_ex_v": ([ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_set_policy": ([ctypes.c_int, ctypes.c_char_p], ctypes.c_int),
    "lift_set_variant": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "lift_pick": ([ctypes.c_int, _I64, _I64, _I64, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "lift_features": ([ctypes.c_int, _I64, _I64, _I64, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "lift_asum_noalloc": ([_P, _I64, _P, _P], ctypes.c_int),
    "lift_nrm2": ([_P, _I64, _P, _P], ctypes.c_int),
    "lift_gemv_t": ([_I64, _I64, ctypes.c_float, _P, _I64, _P, ctypes.c_float, _P, _P], ctypes.c_int),
    "lift_wait_probe": ([ctypes.c_uint32, _P], ctypes.c_int),
    "lift_set_wait_polls": ([ctypes.c_uint32], ctypes.c_int),
    "lift_tune_stats": ([ctypes.POINTER(_I64), ctypes.POINTER(_I64)], ctypes.c_int),
    "lift_asum_partial": ([_P, _I64, _P, _P], ctypes.c_int),
    "lift_dot_partial": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "lift_combine_partials": ([_P, _I64, _P, _P], ctypes.c_int),
    "lift_asum_comp": ([_P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_dot_comp": ([_P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_asum_comp_v": ([ctypes.c_int, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_dot_comp_v": ([ctypes.c_int, _P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_blackscholes": ([_I64, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           _P, _P, _P], ctypes.c_int),
    "lift_blackscholes_v": ([ctypes.c_int, _I64, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, _P, _P, _P], ctypes.c_int),
    "lift_gemv_t_v": ([ctypes.c_int, _I64, _I64, ctypes.c_float, _P, _I64, _P, ctypes.c_float, _P,
                       _P], ctypes.c_int),
    "lift_gemv_t_blocks": ([ctypes.c_int, _I64, _I64, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
                           ctypes.c_int),
    "lift_gemv_segments": ([ctypes.c_int, _I64, _I64, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
                           ctypes.c_int),
    "lift_sum": ([_P, _I64, _P, _P], ctypes.c_int),
    "lift_axpy": ([_I64, ctypes.c_float, _P, _P, _P], ctypes.c_int),
    "lift_nrm2_v": ([ctypes.c_int, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_sum_v": ([ctypes.c_int, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_axpy_v": ([ctypes.c_int, _I64, ctypes.c_float, _P, _P, _P], ctypes.c_int),
    "lift_batch_create": ([ctypes.c_void_p, _I64, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "lift_batch_run": ([_P, _P], ctypes.c_int),
    "lift_batch_set_schedule": ([_P, ctypes.c_int], ctypes.c_int),
    "lift_batch_schedule": ([_P], ctypes.c_int),
    "lift_batch_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
                        ctypes.c_int),
    "lift_batch_op_choice": ([_P, _I64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(_I64)], ctypes.c_int),
    "lift_batch_destroy": ([_P], ctypes.c_int),
    "lift_mlp_param_count": ([ctypes.c_int] * 4, _I64),
    "lift_mlp_work_count": ([_I64, ctypes.c_int, ctypes.c_int], _I64),
    "lift_mlp_forward": ([ctypes.c_int] * 4 + [_P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "lift_mlp_loss": ([_P, _P, _P, _I64, ctypes.c_float, _P, _P, _P], ctypes.c_int),
    "lift_mlp_backward": ([ctypes.c_int] * 4 + [_P, _P, _I64, _P, _P, _P, _P], ctypes.c_int),
    "lift_mlp_adam": ([_P, _P, _P, _P, _I64, ctypes.c_int] + [ctypes.c_float] * 4 + [_P], ctypes.c_int),
}

_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Load liftblas.so (built in-tree by ``paper_1502_02389_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_1502_02389_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols() -> List[str]:
    return list(_SIGS)


def status_string(s: int) -> str:
    try:
        return lib().lift_status_string(s).decode()
    except Exception:  # the library itself may be what is missing
        return "unknown"


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s) -> Optional[int]:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc: int, where: str) -> None:
    if rc != OK:
        raise LiftError(rc, where, lib().lift_last_error().decode())


# ---------------------------------------------------------------------------
# entry points (same names and argument order as include/lift.h)
# ---------------------------------------------------------------------------
def lift_init(device: Optional[int] = None) -> None:
    if device is None:
        import torch
        device = torch.cuda.current_device()
    _check(lib().lift_init(device), "lift_init")


def lift_finalize() -> None:
    _check(lib().lift_finalize(), "lift_finalize")


def lift_sm_count() -> int:
    return lib().lift_sm_count()


def lift_read_status(clear: bool = True) -> int:
    return lib().lift_read_status(1 if clear else 0)


def lift_asum(x, n, result, stream=None):
    _check(lib().lift_asum(_ptr(x), n, _ptr(result), _stream(stream)), "lift_asum")


def lift_dot(x, y, n, result, stream=None):
    _check(lib().lift_dot(_ptr(x), _ptr(y), n, _ptr(result), _stream(stream)), "lift_dot")


def lift_scal(n, alpha, x, y, stream=None):
    _check(lib().lift_scal(n, alpha, _ptr(x), _ptr(y), _stream(stream)), "lift_scal")


def lift_gemv(M, N, alpha, A, lda, x, beta, y, stream=None):
    _check(lib().lift_gemv(M, N, alpha, _ptr(A), lda, _ptr(x), beta, _ptr(y), _stream(stream)),
           "lift_gemv")


def lift_asum_v(variant, x, n, result, result_f64=None, stream=None):
    _check(lib().lift_asum_v(variant, _ptr(x), n, _ptr(result), _ptr(result_f64), _stream(stream)),
           "lift_asum_v")


def lift_dot_v(variant, x, y, n, result, result_f64=None, stream=None):
    _check(lib().lift_dot_v(variant, _ptr(x), _ptr(y), n, _ptr(result), _ptr(result_f64),
                            _stream(stream)), "lift_dot_v")


def lift_scal_v(variant, n, alpha, x, y, stream=None):
    _check(lib().lift_scal_v(variant, n, alpha, _ptr(x), _ptr(y), _stream(stream)), "lift_scal_v")


def lift_gemv_v(variant, M, N, alpha, A, lda, x, beta, y, stream=None):
    _check(lib().lift_gemv_v(variant, M, N, alpha, _ptr(A), lda, _ptr(x), beta, _ptr(y),
                             _stream(stream)), "lift_gemv_v")


def lift_asum_partial(x, n, partial, stream=None):
    _check(lib().lift_asum_partial(_ptr(x), n, _ptr(partial), _stream(stream)), "lift_asum_partial")


def lift_dot_partial(x, y, n, partial, stream=None):
    _check(lib().lift_dot_partial(_ptr(x), _ptr(y), n, _ptr(partial), _stream(stream)),
           "lift_dot_partial")


def lift_combine_partials(partials) -> tuple:
    """Host combine of gathered FP64 partials (a sequence of floats):
    (fp32 result, FP64 sum)."""
    arr = (ctypes.c_double * len(partials))(*[float(p) for p in partials])
    r, r64 = ctypes.c_float(), ctypes.c_double()
    _check(lib().lift_combine_partials(arr, len(partials), ctypes.byref(r), ctypes.byref(r64)),
           "lift_combine_partials")
    return r.value, r64.value


def lift_wait_probe(polls, stream=None):
    _check(lib().lift_wait_probe(polls, _stream(stream)), "lift_wait_probe")


def lift_tune_stats() -> tuple:
    """(shapes with a cached timed winner, launches timed so far)."""
    a, b = _I64(), _I64()
    _check(lib().lift_tune_stats(ctypes.byref(a), ctypes.byref(b)), "lift_tune_stats")
    return a.value, b.value


def lift_set_wait_polls(polls):
    _check(lib().lift_set_wait_polls(polls), "lift_set_wait_polls")


def lift_asum_comp(x, n, result, result_f64=None, stream=None):
    _check(lib().lift_asum_comp(_ptr(x), n, _ptr(result), _ptr(result_f64), _stream(stream)),
           "lift_asum_comp")


def lift_dot_comp(x, y, n, result, result_f64=None, stream=None):
    _check(lib().lift_dot_comp(_ptr(x), _ptr(y), n, _ptr(result), _ptr(result_f64),
                               _stream(stream)), "lift_dot_comp")


def lift_asum_comp_v(variant, x, n, result, result_f64=None, stream=None):
    _check(lib().lift_asum_comp_v(variant, _ptr(x), n, _ptr(result), _ptr(result_f64),
                                  _stream(stream)), "lift_asum_comp_v")


def lift_dot_comp_v(variant, x, y, n, result, result_f64=None, stream=None):
    _check(lib().lift_dot_comp_v(variant, _ptr(x), _ptr(y), n, _ptr(result), _ptr(result_f64),
                                 _stream(stream)), "lift_dot_comp_v")


def lift_blackscholes(n, s, strike, rate, volatility, years, call, put, stream=None):
    _check(lib().lift_blackscholes(n, _ptr(s), strike, rate, volatility, years, _ptr(call),
                                   _ptr(put), _stream(stream)), "lift_blackscholes")


def lift_blackscholes_v(variant, n, s, strike, rate, volatility, years, call, put, stream=None):
    _check(lib().lift_blackscholes_v(variant, n, _ptr(s), strike, rate, volatility, years,
                                     _ptr(call), _ptr(put), _stream(stream)), "lift_blackscholes_v")


def lift_gemv_t(M, N, alpha, A, lda, x, beta, y, stream=None):
    _check(lib().lift_gemv_t(M, N, alpha, _ptr(A), lda, _ptr(x), beta, _ptr(y), _stream(stream)),
           "lift_gemv_t")


def lift_gemv_t_v(variant, M, N, alpha, A, lda, x, beta, y, stream=None):
    _check(lib().lift_gemv_t_v(variant, M, N, alpha, _ptr(A), lda, _ptr(x), beta, _ptr(y),
                               _stream(stream)), "lift_gemv_t_v")


def lift_gemv_t_blocks(variant, M, N):
    """(rows per block, blocks) of a gemv-T variant for an M x N call."""
    b, rb = _I64(), _I64()
    _check(lib().lift_gemv_t_blocks(variant, M, N, ctypes.byref(b), ctypes.byref(rb)),
           "lift_gemv_t_blocks")
    return b.value, rb.value


def lift_gemv_segments(variant, M, N):
    """(segment length, segments per row) of a gemv variant for an M x N
    call; (N, 1) for the variants that give a row to one warp or CTA."""
    L, S = _I64(), _I64()
    _check(lib().lift_gemv_segments(variant, M, N, ctypes.byref(L), ctypes.byref(S)),
           "lift_gemv_segments")
    return L.value, S.value


def lift_nrm2(x, n, result, stream=None):
    _check(lib().lift_nrm2(_ptr(x), n, _ptr(result), _stream(stream)), "lift_nrm2")


def lift_sum(x, n, result, stream=None):
    _check(lib().lift_sum(_ptr(x), n, _ptr(result), _stream(stream)), "lift_sum")


def lift_axpy(n, alpha, x, y, stream=None):
    _check(lib().lift_axpy(n, alpha, _ptr(x), _ptr(y), _stream(stream)), "lift_axpy")


def lift_nrm2_v(variant, x, n, result, result_f64=None, stream=None):
    _check(lib().lift_nrm2_v(variant, _ptr(x), n, _ptr(result), _ptr(result_f64), _stream(stream)),
           "lift_nrm2_v")


def lift_sum_v(variant, x, n, result, result_f64=None, stream=None):
    _check(lib().lift_sum_v(variant, _ptr(x), n, _ptr(result), _ptr(result_f64), _stream(stream)),
           "lift_sum_v")


def lift_axpy_v(variant, n, alpha, x, y, stream=None):
    _check(lib().lift_axpy_v(variant, n, alpha, _ptr(x), _ptr(y), _stream(stream)), "lift_axpy_v")


def lift_asum_ex(dtype, x, xscale, n, result, result_f64=None, stream=None):
    _check(lib().lift_asum_ex(dtype, _ptr(x), _ptr(xscale), n, _ptr(result), _ptr(result_f64),
                              _stream(stream)), "lift_asum_ex")


def lift_dot_ex(dtype, x, xscale, y, yscale, n, result, result_f64=None, stream=None):
    _check(lib().lift_dot_ex(dtype, _ptr(x), _ptr(xscale), _ptr(y), _ptr(yscale), n, _ptr(result),
                             _ptr(result_f64), _stream(stream)), "lift_dot_ex")


def lift_asum_ex_v(variant, dtype, x, xscale, n, result, result_f64=None, stream=None):
    _check(lib().lift_asum_ex_v(variant, dtype, _ptr(x), _ptr(xscale), n, _ptr(result),
                                _ptr(result_f64), _stream(stream)), "lift_asum_ex_v")


def lift_dot_ex_v(variant, dtype, x, xscale, y, yscale, n, result, result_f64=None, stream=None):
    _check(lib().lift_dot_ex_v(variant, dtype, _ptr(x), _ptr(xscale), _ptr(y), _ptr(yscale), n,
                               _ptr(result), _ptr(result_f64), _stream(stream)), "lift_dot_ex_v")


def lift_variant_count(op: int) -> int:
    return lib().lift_variant_count(op)


def lift_variant_describe(op: int, vid: int) -> Dict:
    info = VariantInfo()
    _check(lib().lift_variant_describe(op, vid, ctypes.byref(info)), "lift_variant_describe")
    d = {k: getattr(info, k) for k, _ in VariantInfo._fields_ if k != "name"}
    d["name"] = info.name.decode()
    return d


def lift_variant_grid(op: int, vid: int, n: int) -> int:
    g = _I64()
    _check(lib().lift_variant_grid(op, vid, n, ctypes.byref(g)), "lift_variant_grid")
    return g.value


def lift_set_policy(policy: int, path: Optional[str] = None) -> None:
    _check(lib().lift_set_policy(policy, path.encode() if path else None), "lift_set_policy")


def lift_set_variant(op: int, variant: int) -> None:
    _check(lib().lift_set_variant(op, variant), "lift_set_variant")


def lift_pick(op: int, n: int, M: int = 0, N: int = 0) -> int:
    v = ctypes.c_int()
    _check(lib().lift_pick(op, n, M, N, ctypes.byref(v)), "lift_pick")
    return v.value


def lift_features(op: int, n: int, M: int = 0, N: int = 0) -> List[float]:
    out = (ctypes.c_float * NUM_FEATURES)()
    _check(lib().lift_features(op, n, M, N, out), "lift_features")
    return list(out)


def lift_asum_noalloc(x, n, result, stream=None):
    _check(lib().lift_asum_noalloc(_ptr(x), n, _ptr(result), _stream(stream)), "lift_asum_noalloc")


def lift_batch_create(descs) -> int:
    """descs: a ctypes array of OpDesc (or a list of dicts with its fields);
    returns the opaque batch handle."""
    if not isinstance(descs, ctypes.Array):
        arr = (OpDesc * len(descs))()
        for i, d in enumerate(descs):
            for k, v in d.items():
                setattr(arr[i], k, _ptr(v) if k in ("x", "y", "A", "out") else v)
        descs = arr
    h = ctypes.c_void_p()
    _check(lib().lift_batch_create(ctypes.cast(descs, ctypes.c_void_p), len(descs), ctypes.byref(h)),
           "lift_batch_create")
    return h.value


def lift_batch_run(batch, stream=None):
    _check(lib().lift_batch_run(batch, _stream(stream)), "lift_batch_run")


BATCH_QUEUE = 0
BATCH_PER_ITEM = 1


def lift_batch_set_schedule(batch, schedule: int):
    _check(lib().lift_batch_set_schedule(batch, int(schedule)), "lift_batch_set_schedule")


def lift_batch_schedule(batch) -> int:
    return int(lib().lift_batch_schedule(batch))


def lift_batch_info(batch):
    it, by, gr = _I64(), _I64(), _I64()
    _check(lib().lift_batch_info(batch, ctypes.byref(it), ctypes.byref(by), ctypes.byref(gr)),
           "lift_batch_info")
    return {"items": it.value, "bytes": by.value, "grid": gr.value}


def lift_batch_op_choice(batch, i):
    """(variant, mode, item length) of op i."""
    v, m, it = ctypes.c_int(), ctypes.c_int(), _I64()
    _check(lib().lift_batch_op_choice(batch, i, ctypes.byref(v), ctypes.byref(m), ctypes.byref(it)),
           "lift_batch_op_choice")
    return v.value, m.value, it.value


def lift_batch_destroy(batch):
    _check(lib().lift_batch_destroy(batch), "lift_batch_destroy")


def lift_mlp_param_count(d_in, h1, h2, V) -> int:
    return lib().lift_mlp_param_count(d_in, h1, h2, V)


def lift_mlp_work_count(B, h1, h2) -> int:
    return lib().lift_mlp_work_count(B, h1, h2)


def lift_mlp_forward(d_in, h1, h2, V, params, X, B, work, P, stream=None):
    _check(lib().lift_mlp_forward(d_in, h1, h2, V, _ptr(params), _ptr(X), B, _ptr(work), _ptr(P),
                                  _stream(stream)), "lift_mlp_forward")


def lift_mlp_loss(P, T, mask, count, inv_measured, dP, loss, stream=None):
    _check(lib().lift_mlp_loss(_ptr(P), _ptr(T), _ptr(mask), count, inv_measured, _ptr(dP),
                               _ptr(loss), _stream(stream)), "lift_mlp_loss")


def lift_mlp_backward(d_in, h1, h2, V, params, X, B, work, dP, grads, stream=None):
    _check(lib().lift_mlp_backward(d_in, h1, h2, V, _ptr(params), _ptr(X), B, _ptr(work), _ptr(dP),
                                   _ptr(grads), _stream(stream)), "lift_mlp_backward")


def lift_mlp_adam(params, grads, m, v, count, t, lr, beta1, beta2, eps, stream=None):
    _check(lib().lift_mlp_adam(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), count, t, lr, beta1,
                               beta2, eps, _stream(stream)), "lift_mlp_adam")


def variants(op: int) -> List[Dict]:
    return [lift_variant_describe(op, i) for i in range(lift_variant_count(op))]
