"""ctypes mirror of include/sage.h (argument marshalling only).

Every step of the hot path runs in libsage.so's kernels; this module only
declares the C structs and function signatures.  Importing it fails loudly when
the library has not been built: there is no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsage.so")

SAGE_OK, SAGE_PENDING = 0, 1
SAGE_ERR_INVALID, SAGE_ERR_NOMEM, SAGE_ERR_CUDA, SAGE_ERR_TIMEOUT = -1, -2, -3, -4
SAGE_ERR_BUSY, SAGE_ERR_STAGING, SAGE_ERR_BOUNDS, SAGE_ERR_DEVICE = -5, -6, -7, -8
STATUS_NAMES = {0: "SAGE_OK", 1: "SAGE_PENDING", -1: "SAGE_ERR_INVALID", -2: "SAGE_ERR_NOMEM",
                -3: "SAGE_ERR_CUDA", -4: "SAGE_ERR_TIMEOUT", -5: "SAGE_ERR_BUSY", -6: "SAGE_ERR_STAGING",
                -7: "SAGE_ERR_BOUNDS", -8: "SAGE_ERR_DEVICE"}
SAGE_READONLY, SAGE_WRITABLE = 0, 1
SAGE_F32, SAGE_BF16 = 0, 1

DEV_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
DEV_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FILL_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p)


class PoolConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("budget_bytes", ctypes.c_size_t),
                ("staging_chunk_bytes", ctypes.c_size_t), ("staging_chunks", ctypes.c_int),
                ("producer_threads", ctypes.c_int), ("serial_setup", ctypes.c_int),
                ("dev_alloc", ctypes.c_void_p), ("dev_free", ctypes.c_void_p), ("alloc_ctx", ctypes.c_void_p),
                ("host_cache_bytes", ctypes.c_size_t), ("graphs", ctypes.c_int), ("exportable", ctypes.c_int)]


class DataDesc(ctypes.Structure):
    _fields_ = [("key", ctypes.c_char_p), ("access", ctypes.c_int), ("bytes", ctypes.c_size_t),
                ("host_src", ctypes.c_void_p), ("fill", ctypes.c_void_p), ("fill_ctx", ctypes.c_void_p)]


class FnDesc(ctypes.Structure):
    _fields_ = [("fn_key", ctypes.c_char_p), ("dtype", ctypes.c_int), ("num_tables", ctypes.c_int),
                ("rows", ctypes.POINTER(ctypes.c_int64)), ("dim", ctypes.c_int), ("n_dense", ctypes.c_int),
                ("n_bot", ctypes.c_int), ("bot_dims", ctypes.POINTER(ctypes.c_int)),
                ("n_top", ctypes.c_int), ("top_dims", ctypes.POINTER(ctypes.c_int)),
                ("max_batch", ctypes.c_int), ("workspace_slots", ctypes.c_int),
                ("tables", DataDesc), ("weights", DataDesc)]


class Invocation(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("dense", ctypes.c_void_p), ("indices", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("out", ctypes.c_void_p), ("num_indices", ctypes.c_int64)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("work", ctypes.c_double)]


class HostInvocation(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("dense", ctypes.c_void_p), ("indices", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("num_indices", ctypes.c_int64), ("out", ctypes.c_void_p)]


class Request(ctypes.Structure):
    _fields_ = [("fn", ctypes.c_int), ("arrival_s", ctypes.c_double), ("inv", HostInvocation)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("max_batch_invocations", ctypes.c_int), ("max_batch_rows", ctypes.c_int64),
                ("lanes_per_fn", ctypes.c_int), ("linger_s", ctypes.c_double), ("timeout_s", ctypes.c_double),
                ("sm_partition", ctypes.c_int)]


class RequestResult(ctypes.Structure):
    _fields_ = [("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double), ("service_ms", ctypes.c_double),
                ("cold", ctypes.c_int), ("batch_invocations", ctypes.c_int), ("status", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("prepares", ctypes.c_int64), ("evictions", ctypes.c_int64), ("cold_requests", ctypes.c_int64),
                ("max_inflight_batches", ctypes.c_int64), ("invocations_per_s", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("warm_p50_ms", ctypes.c_double), ("warm_p99_ms", ctypes.c_double),
                ("cold_p50_ms", ctypes.c_double), ("cold_p99_ms", ctypes.c_double)]


class PoolStats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("resident_bytes", ctypes.c_size_t),
                ("readonly_bytes", ctypes.c_size_t), ("functions", ctypes.c_int64), ("refs", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("prepares", ctypes.c_int64), ("hits", ctypes.c_int64),
                ("misses", ctypes.c_int64), ("invocations", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("ctx_ms", ctypes.c_double), ("last_stage_ms", ctypes.c_double),
                ("last_fill_ms", ctypes.c_double), ("last_module_ms", ctypes.c_double),
                ("last_workspace_ms", ctypes.c_double), ("last_prepare_ms", ctypes.c_double),
                ("host_cache_bytes", ctypes.c_size_t), ("host_cache_entries", ctypes.c_int64),
                ("host_cache_hits", ctypes.c_int64), ("demotions", ctypes.c_int64)]


class ShareStats(ctypes.Structure):
    _fields_ = [("connections", ctypes.c_int64), ("grants", ctypes.c_int64), ("rejects", ctypes.c_int64),
                ("ready", ctypes.c_int64), ("releases", ctypes.c_int64), ("active", ctypes.c_int64)]


# (name, restype, argtypes) of every exported entry point of include/sage.h
_vp, _i, _i64, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = [
    ("sage_pool_create", _i, [ctypes.POINTER(PoolConfig), ctypes.POINTER(_vp)]),
    ("sage_prepare", _i, [_vp, ctypes.POINTER(FnDesc), ctypes.POINTER(_vp)]),
    ("sage_fn_data", _i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    ("sage_fn_query", _i, [_vp]),
    ("sage_wait", _i, [_vp, _i64]),
    ("sage_invoke", _i, [_vp, ctypes.POINTER(Invocation), _vp]),
    ("sage_invoke_batch", _i, [_vp, ctypes.POINTER(Invocation), _i, _vp]),
    ("sage_invoke_batch_host", _i, [_vp, ctypes.POINTER(HostInvocation), _i, _vp]),
    ("sage_invoke_batch_host_async", _i, [_vp, ctypes.POINTER(HostInvocation), _i, _vp]),
    ("sage_fn_check", _i, [_vp]),
    ("sage_fn_debug_copy", _i, [_vp, _i, _i, _vp, _sz, ctypes.POINTER(_i)]),
    ("sage_release", _i, [_vp]),
    ("sage_pool_destroy", _i, [_vp]),
    ("sage_pool_stats", _i, [_vp, ctypes.POINTER(PoolStats)]),
    ("sage_last_error", ctypes.c_char_p, []),
    ("sage_host_alloc", _i, [_sz, ctypes.POINTER(_vp)]),
    ("sage_host_free", _i, [_vp]),
    ("sage_kernel_launches", _i64, []),
    ("sage_profile_enable", _i, [_i]),
    ("sage_profile_read", _i, [ctypes.POINTER(KernelTime), _i]),
    ("sage_autotune", _i, [_vp, _i, _vp]),
    ("sage_tuning_set", _i, [_i, _i, _i, _i, _i, _i]),
    ("sage_tuning_save", _i, [ctypes.c_char_p]),
    ("sage_tuning_load", _i, [ctypes.c_char_p]),
    ("sage_serve", _i, [_vp, ctypes.POINTER(FnDesc), _i, ctypes.POINTER(Request), _i, ctypes.POINTER(ServeConfig),
                        ctypes.POINTER(RequestResult), ctypes.POINTER(ServeStats)]),
    ("sage_invoke_noalloc", _i, [ctypes.POINTER(FnDesc), _vp, _vp, ctypes.POINTER(Invocation), _vp]),
    ("sage_noalloc_check", _i, [_vp]),
    ("sage_embedding_bag_sum", _i, [_i, _vp, _vp, _i, _i, _i, _vp, _vp, _vp, _i, _vp, _vp]),
    ("sage_linear", _i, [_i, _i, _i, _i, _vp, _i, _vp, _vp, _i, _vp, _i, _vp, _vp]),
    ("sage_share_start", _i, [_vp, ctypes.c_char_p, ctypes.POINTER(_vp)]),
    ("sage_share_register", _i, [_vp, ctypes.POINTER(FnDesc)]),
    ("sage_share_stats_get", _i, [_vp, ctypes.POINTER(ShareStats)]),
    ("sage_share_stop", _i, [_vp]),
    ("sage_attach_begin", _i, [ctypes.c_char_p, ctypes.POINTER(FnDesc), ctypes.POINTER(_vp)]),
    ("sage_attach_end", _i, [_vp, _vp, ctypes.POINTER(_vp)]),
    ("sage_attach_cancel", _i, [_vp]),
    ("sage_partition_create", _i, [_i, _i, _i, ctypes.POINTER(_vp)]),
    ("sage_partition_groups", _i, [_vp]),
    ("sage_partition_stream", _i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_i)]),
    ("sage_partition_destroy", _i, [_vp]),
    ("sage_linear_tiled", _i, [_i, _i, _i, _i, _vp, _i, _vp, _vp, _i, _vp, _i, _i, _i, _vp, _vp]),
]

_lib = None


def lib():
    """Load libsage.so (raises if it is missing: the product path has no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsage.so is not built; run `python -m paper_2404_14691_b300.build` "
                              "(or __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SageError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().sage_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))


def check(status: int, where: str) -> int:
    if status < 0:
        raise SageError(status, where)
    return status
