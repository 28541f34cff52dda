"""B300-native runtime for many concurrent invocations of one GPU function that
share one reference-counted device copy of its read-only data (SAGE,
arXiv 2404.14691), with hand-written sm_103a kernels for the function itself
(an embedding-bag gather-sum and bottom/top MLPs).

This package is a thin ctypes binding over libsage.so (include/sage.h): it
marshals arguments and holds Python-side references; every step of the hot
path runs in the library's CUDA kernels.  PyTorch is used only for device
memory (optional allocator hooks) and streams.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

from ._native import (DEV_ALLOC_FN, DEV_FREE_FN, SAGE_BF16, SAGE_ERR_BUSY, SAGE_F32, SAGE_OK, SAGE_PENDING,
                      SAGE_READONLY, STATUS_NAMES, DataDesc, FnDesc, HostInvocation, Invocation, KernelTime,
                      PoolConfig, PoolStats, Request, RequestResult, SageError, ServeConfig, ServeStats, ShareStats,
                      check, lib)

__all__ = ["Pool", "Function", "SageError", "SAGE_F32", "SAGE_BF16", "embedding_bag_sum", "linear",
           "kernel_launches", "profile_enable", "profile_read", "torch_allocator_hooks", "serve", "Share",
           "attach_begin", "Partition"]


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def kernel_launches() -> int:
    """Kernels launched by libsage.so in this process."""
    return int(lib().sage_kernel_launches())


def profile_enable(on: bool) -> None:
    """Bracket every kernel of sage_invoke* with timing events on its stream."""
    check(lib().sage_profile_enable(1 if on else 0), "sage_profile_enable")


def profile_read() -> dict:
    """{kind: (launches, total_ms, work)} of the kernels timed since the last read."""
    buf = (KernelTime * 8)()
    n = check(lib().sage_profile_read(buf, 8), "sage_profile_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms), float(buf[i].work))
            for i in range(n)}


class _HostBlock:
    def __init__(self, nbytes: int):
        p = ctypes.c_void_p()
        check(lib().sage_host_alloc(int(nbytes), ctypes.byref(p)), "sage_host_alloc")
        self.ptr = p.value

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().sage_host_free(self.ptr)
            self.ptr = None


def host_empty(shape, dtype):
    """A numpy array in page-locked, huge-page-backed host memory (sage_host_alloc)."""
    import numpy as np
    dt = np.dtype(dtype)
    n = int(np.prod(shape)) if np.ndim(shape) else int(shape)
    blk = _HostBlock(max(1, n * dt.itemsize))
    buf = (ctypes.c_char * max(1, n * dt.itemsize)).from_address(blk.ptr)
    buf._block = blk  # the array's base (buf) keeps the block alive
    return np.frombuffer(buf, dtype=dt, count=n).reshape(shape)


def host_copy(a):
    """A copy of numpy array `a` in memory from host_empty."""
    out = host_empty(a.shape, a.dtype)
    out[...] = a
    return out


def torch_allocator_hooks(device: int = 0):
    """(alloc, free) C callbacks routing the pool's device memory through PyTorch's
    caching allocator."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
        except Exception:  # out of memory -> NULL, reported as SAGE_ERR_NOMEM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return DEV_ALLOC_FN(_alloc), DEV_FREE_FN(_free)


def fn_desc(key: str, dtype: int, rows: Sequence[int], dim: int, n_dense: int, bot_dims: Sequence[int],
            top_dims: Sequence[int], tables_bytes: int, weights_bytes: int, tables_src: Optional[int] = None,
            tables_fill: Optional[int] = None, tables_ctx=None, weights_src: Optional[int] = None,
            max_batch: int = 0, workspace_slots: int = 0, keep=None):
    """A sage_fn_desc and the Python objects it points into.  tables_src / weights_src:
    host addresses of the data items; or tables_fill: address of a C producer
    (sage_fill_fn) with tables_ctx."""
    T = len(rows)
    rows_a = (ctypes.c_int64 * T)(*rows)
    bot_a = (ctypes.c_int * len(bot_dims))(*bot_dims)
    top_a = (ctypes.c_int * len(top_dims))(*top_dims)
    kb = key.encode()
    ctx_ptr = ctypes.cast(ctypes.byref(tables_ctx), ctypes.c_void_p) if tables_ctx is not None else None
    tdesc = DataDesc(kb, SAGE_READONLY, tables_bytes, tables_src, tables_fill, ctx_ptr)
    wdesc = DataDesc(kb, SAGE_READONLY, weights_bytes, weights_src, None, None)
    d = FnDesc(kb, dtype, T, rows_a, dim, n_dense, len(bot_dims), bot_a, len(top_dims), top_a,
               max_batch, workspace_slots, tdesc, wdesc)
    return d, (rows_a, bot_a, top_a, kb, tables_ctx, keep)


def serve(pool: "Pool", functions: Sequence[dict], requests: Sequence[tuple], max_batch_invocations: int = 0,
          max_batch_rows: int = 0, lanes_per_fn: int = 0, linger_s: float = -1.0, timeout_s: float = 0.0,
          sm_partition: bool = False):
    """Replay a request trace with continuous batching (sage_serve).

    functions: fn_desc keyword dicts; requests: (fn, arrival_s, batch, dense, indices, offsets,
    num_indices, out) with host addresses.  Returns (results, stats): results is a list of
    dicts per request, stats a dict."""
    descs = [fn_desc(**kw) for kw in functions]
    arr = (FnDesc * len(descs))(*[d for d, _ in descs])
    reqs = (Request * len(requests))(*[Request(int(f), float(t), HostInvocation(int(b), d, i, o, int(ni), u))
                                       for (f, t, b, d, i, o, ni, u) in requests])
    res = (RequestResult * max(1, len(requests)))()
    st = ServeStats()
    cfg = ServeConfig(max_batch_invocations, max_batch_rows, lanes_per_fn, linger_s, timeout_s,
                      1 if sm_partition else 0)
    check(lib().sage_serve(pool.handle, arr, len(descs), reqs, len(requests), ctypes.byref(cfg), res,
                           ctypes.byref(st)), "sage_serve")
    out = [{name: getattr(res[k], name) for name, _ in RequestResult._fields_} for k in range(len(requests))]
    return out, {name: getattr(st, name) for name, _ in ServeStats._fields_}


def host_invocations(invs: Sequence[tuple]):
    """A reusable C array of sage_host_invocation from (batch, dense, indices, offsets, num_indices, out)."""
    return (HostInvocation * len(invs))(*[HostInvocation(int(b), d, i, o, int(n), u) for (b, d, i, o, n, u) in invs])


class Function:
    """A reference to a prepared function (sage_fn)."""

    def __init__(self, pool: "Pool", handle: int, keep):
        self.pool = pool
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep

    def data(self):
        """(tables, weights) device addresses of the read-only items."""
        t, w = ctypes.c_void_p(), ctypes.c_void_p()
        check(lib().sage_fn_data(self.handle, ctypes.byref(t), ctypes.byref(w)), "sage_fn_data")
        return t.value, w.value

    def query(self) -> int:
        return check(lib().sage_fn_query(self.handle), "sage_fn_query")

    def wait(self, timeout_us: int = -1) -> None:
        check(lib().sage_wait(self.handle, int(timeout_us)), "sage_wait")

    def invoke(self, batch: int, dense: int, indices: int, offsets: int, out: int, stream=None,
               num_indices: int = 0) -> None:
        inv = Invocation(int(batch), dense, indices, offsets, out, int(num_indices))
        check(lib().sage_invoke(self.handle, ctypes.byref(inv), _stream_handle(stream)), "sage_invoke")

    def invoke_batch(self, invs: Sequence[tuple], stream=None) -> None:
        """invs: (batch, dense_ptr, indices_ptr, offsets_ptr, out_ptr[, num_indices]) per invocation
        (device pointers)."""
        arr = (Invocation * len(invs))(*[Invocation(int(v[0]), v[1], v[2], v[3], v[4], int(v[5]) if len(v) > 5 else 0)
                                         for v in invs])
        check(lib().sage_invoke_batch(self.handle, arr, len(invs), _stream_handle(stream)), "sage_invoke_batch")

    def invoke_batch_host(self, invs: Sequence[tuple], stream=None) -> None:
        """invs: (batch, dense_ptr, indices_ptr, offsets_ptr, num_indices, out_ptr) per invocation (host
        pointers), or an array built by host_invocations()."""
        arr = invs if isinstance(invs, ctypes.Array) else host_invocations(invs)
        check(lib().sage_invoke_batch_host(self.handle, arr, len(arr), _stream_handle(stream)),
              "sage_invoke_batch_host")

    def autotune(self, rows: int, stream=None) -> None:
        """Time the tile configurations of this function's tensor-core layers for a batch
        of `rows` samples and keep the fastest (process-wide)."""
        check(lib().sage_autotune(self.handle, int(rows), _stream_handle(stream)), "sage_autotune")

    def invoke_batch_host_async(self, invs, stream=None) -> None:
        """As invoke_batch_host without waiting; synchronise `stream` before reading outputs.
        invs: a list of tuples, or an array built once by host_invocations()."""
        arr = invs if isinstance(invs, ctypes.Array) else host_invocations(invs)
        check(lib().sage_invoke_batch_host_async(self.handle, arr, len(arr), _stream_handle(stream)),
              "sage_invoke_batch_host_async")

    def debug_copy(self, which: int, width: int, bf16: bool, plane: int = 0):
        """Copy an activation buffer of the most recent batch (sage_fn_debug_copy):
        which 0 = concat [M, width = T*dim + bot], 1 + l = top hidden layer l [M,
        width = top_dims[l]].  Returns a numpy array [M, width]: float32, or the
        uint16 bit patterns of bf16 values when bf16 is true."""
        import numpy as np
        rows = ctypes.c_int(0)
        check(lib().sage_fn_debug_copy(self.handle, which, plane, None, 0, ctypes.byref(rows)), "sage_fn_debug_copy")
        out = np.empty((rows.value, int(width)), dtype=np.uint16 if bf16 else np.float32)
        check(lib().sage_fn_debug_copy(self.handle, which, plane, out.ctypes.data, out.nbytes, None),
              "sage_fn_debug_copy")
        return out

    def check_errors(self) -> None:
        """Raise SageError if a kernel saw an out-of-range row or a timed-out wait."""
        check(lib().sage_fn_check(self.handle), "sage_fn_check")

    def release(self) -> None:
        if self.handle is not None:
            # the library releases the handle even when it reports a device failure
            h, self.handle = self.handle, None
            st = lib().sage_release(h)
            self._keep = None
            check(st, "sage_release")


class Pool:
    """A per-GPU pool of read-only function data (sage_pool)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, staging_chunk_bytes: int = 0,
                 staging_chunks: int = 0, producer_threads: int = 0, serial_setup: bool = False,
                 torch_allocator: bool = False, host_cache_bytes: int = 0, graphs: bool = False,
                 exportable: bool = False):
        self._hooks = torch_allocator_hooks(device) if torch_allocator else None
        cfg = PoolConfig(device, budget_bytes, staging_chunk_bytes, staging_chunks, producer_threads,
                         1 if serial_setup else 0,
                         ctypes.cast(self._hooks[0], ctypes.c_void_p) if self._hooks else None,
                         ctypes.cast(self._hooks[1], ctypes.c_void_p) if self._hooks else None, None,
                         int(host_cache_bytes), 1 if graphs else 0, 1 if exportable else 0)
        h = ctypes.c_void_p()
        check(lib().sage_pool_create(ctypes.byref(cfg), ctypes.byref(h)), "sage_pool_create")
        self.handle = h

    def prepare(self, **kw) -> Function:
        """Prepare a function (keyword arguments of fn_desc)."""
        d, keep = fn_desc(**kw)
        h = ctypes.c_void_p()
        check(lib().sage_prepare(self.handle, ctypes.byref(d), ctypes.byref(h)), "sage_prepare")
        return Function(self, h.value, keep)

    def attach(self, ticket: "Ticket") -> Function:
        """Complete an attach begun with attach_begin (sage_attach_end): map the
        owner's read-only copy into this process; returns before it is complete."""
        h = ctypes.c_void_p()
        t, ticket.handle = ticket.handle, None
        if t is None:
            raise ValueError("ticket already used")
        check(lib().sage_attach_end(self.handle, t, ctypes.byref(h)), "sage_attach_end")
        return Function(self, h.value, ticket._keep)

    def stats(self) -> dict:
        s = PoolStats()
        check(lib().sage_pool_stats(self.handle, ctypes.byref(s)), "sage_pool_stats")
        return {name: getattr(s, name) for name, _ in PoolStats._fields_}

    def destroy(self) -> None:
        if self.handle is not None:
            st = lib().sage_pool_destroy(self.handle)
            if st != SAGE_ERR_BUSY:      # destroyed, also when it reports a device failure
                self.handle = None
            check(st, "sage_pool_destroy")


def tuning_set(kind: int, rows: int, N: int, K: int, bn: int, stages: int) -> None:
    """Pin a tensor-core tile configuration for a GEMM shape (see sage_tuning_set)."""
    check(lib().sage_tuning_set(kind, rows, N, K, bn, stages), "sage_tuning_set")


def tuning_save(path: str) -> None:
    check(lib().sage_tuning_save(path.encode()), "sage_tuning_save")


def tuning_load(path: str) -> None:
    check(lib().sage_tuning_load(path.encode()), "sage_tuning_load")


def embedding_bag_sum(dtype: int, tables: int, table_rows: Sequence[int], dim: int, batch: int, indices: int,
                      offsets: int, out: int, ldo: int, err_word: Optional[int] = None, stream=None) -> None:
    """sage_embedding_bag_sum on device pointers."""
    T = len(table_rows)
    rows_a = (ctypes.c_int64 * T)(*table_rows)
    check(lib().sage_embedding_bag_sum(dtype, tables, rows_a, T, dim, batch, indices, offsets, out, ldo, err_word,
                                       _stream_handle(stream)), "sage_embedding_bag_sum")


def linear(dtype: int, M: int, N: int, K: int, x: int, ldx: int, W: int, bias: int, relu: bool, y: int, ldy: int,
           err_word: Optional[int] = None, stream=None, tile=None) -> None:
    """sage_linear on device pointers; tile=(bn, stages) pins the tensor-core tile configuration."""
    if tile is None:
        check(lib().sage_linear(dtype, M, N, K, x, ldx, W, bias, 1 if relu else 0, y, ldy, err_word,
                                _stream_handle(stream)), "sage_linear")
    else:
        check(lib().sage_linear_tiled(dtype, M, N, K, x, ldx, W, bias, 1 if relu else 0, y, ldy, int(tile[0]),
                                      int(tile[1]), err_word, _stream_handle(stream)), "sage_linear_tiled")


class Share:
    """Serve an exportable pool's functions to other processes (sage_share_start)."""

    def __init__(self, pool: Pool, socket_path: str):
        h = ctypes.c_void_p()
        check(lib().sage_share_start(pool.handle, socket_path.encode(), ctypes.byref(h)), "sage_share_start")
        self.handle = h
        self._keep = []

    def register(self, **kw) -> None:
        """Make a function attachable (keyword arguments of fn_desc, with its data sources,
        which stay referenced until stop())."""
        d, keep = fn_desc(**kw)
        check(lib().sage_share_register(self.handle, ctypes.byref(d)), "sage_share_register")
        self._keep.append((d, keep))

    def stats(self) -> dict:
        s = ShareStats()
        check(lib().sage_share_stats_get(self.handle, ctypes.byref(s)), "sage_share_stats_get")
        return {name: getattr(s, name) for name, _ in ShareStats._fields_}

    def stop(self) -> None:
        if self.handle is not None:
            check(lib().sage_share_stop(self.handle), "sage_share_stop")
            self.handle = None
            self._keep = []


class Ticket:
    """An attach request in flight (sage_attach_begin); completed by Pool.attach."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def cancel(self) -> None:
        """Drop the request without completing it (sage_attach_cancel)."""
        if self.handle is not None:
            h, self.handle = self.handle, None
            check(lib().sage_attach_cancel(h), "sage_attach_cancel")

    def __del__(self):
        if getattr(self, "handle", None) is not None:
            lib().sage_attach_cancel(self.handle)
            self.handle = None


def attach_begin(socket_path: str, **kw) -> Ticket:
    """Send an attach request for a function shape to the owner at socket_path.  Makes no
    CUDA call, so a new process can send it before creating its context."""
    d, keep = fn_desc(**kw)
    h = ctypes.c_void_p()
    check(lib().sage_attach_begin(socket_path.encode(), ctypes.byref(d), ctypes.byref(h)), "sage_attach_begin")
    return Ticket(h, keep)


class Partition:
    """SM partition of a GPU (sage_partition_create): `groups` green contexts, each
    with a stream whose kernels run on the group's SMs only."""

    def __init__(self, device: int = 0, groups: int = 2, min_sms: int = 0):
        h = ctypes.c_void_p()
        check(lib().sage_partition_create(device, groups, min_sms, ctypes.byref(h)), "sage_partition_create")
        self.handle = h
        self.groups = lib().sage_partition_groups(h)

    def stream(self, group: int):
        """(stream handle, SM count) of a group."""
        s, n = ctypes.c_void_p(), ctypes.c_int()
        check(lib().sage_partition_stream(self.handle, group, ctypes.byref(s), ctypes.byref(n)),
              "sage_partition_stream")
        return s.value, n.value

    def destroy(self) -> None:
        if self.handle is not None:
            h, self.handle = self.handle, None
            check(lib().sage_partition_destroy(h), "sage_partition_destroy")
