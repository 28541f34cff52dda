"""CPU oracle of the hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and its
reference arm) may import this package.  The product path (the C-ABI library and
its Python binding) never does, and it shares no code with it.

Contents
  * sage_oracle.c (fp64 C loops, built into liboracle.so): embedding-bag sum,
    linear layer, whole function per invocation with magnitude bounds.
  * pack_invocations: the plain definition of fusing several invocations of one
    function into one batch (concatenate samples; rebase each table's CSR
    offsets by the running index count).
  * PoolModel: the refcount / budget model of read-only sharing (Sec. 6.2 of the
    paper: read-only data is loaded on the first invocation and shared by the
    concurrent ones; it is released when no invocation holds it).
  * check_close: the componentwise tolerance used by every parity test.

What is pinned and how: see tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

F64P = ctypes.POINTER(ctypes.c_double)


def build_lib(force: bool = False) -> str:
    src = os.path.join(_HERE, "sage_oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleFn(ctypes.Structure):
    _fields_ = [("n_tables", ctypes.c_int), ("dim", ctypes.c_int), ("n_dense", ctypes.c_int),
                ("n_bot", ctypes.c_int), ("n_top", ctypes.c_int),
                ("bot_dims", ctypes.POINTER(ctypes.c_int)), ("top_dims", ctypes.POINTER(ctypes.c_int)),
                ("bot_W", ctypes.POINTER(F64P)), ("bot_b", ctypes.POINTER(F64P)),
                ("top_W", ctypes.POINTER(F64P)), ("top_b", ctypes.POINTER(F64P)),
                ("tables", ctypes.POINTER(F64P)), ("table_rows", ctypes.POINTER(ctypes.c_int64))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build_lib())
            L.oracle_bag_sum.restype = ctypes.c_int
            L.oracle_bag_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(F64P),
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
            L.oracle_linear.restype = None
            L.oracle_linear.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            L.oracle_sigmoid.restype = ctypes.c_double
            L.oracle_sigmoid.argtypes = [ctypes.c_double]
            L.oracle_forward.restype = ctypes.c_int
            L.oracle_forward.argtypes = [ctypes.POINTER(OracleFn), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------- primitives

def bag_sum(tables: Sequence[np.ndarray], indices: np.ndarray, offsets: np.ndarray, batch: int,
            with_mag: bool = True):
    """pooled [batch, T*D] (fp64) and its magnitude bound, by plain index-order sums."""
    T = len(tables)
    D = int(tables[0].shape[1])
    tabs = [_f64(t) for t in tables]
    arr = (F64P * T)(*[t.ctypes.data_as(F64P) for t in tabs])
    rows = np.array([t.shape[0] for t in tabs], dtype=np.int64)
    idx = np.ascontiguousarray(indices, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    assert off.size == T * batch + 1
    pooled = np.zeros((batch, T * D))
    mag = np.zeros((batch, T * D)) if with_mag else None
    rc = lib().oracle_bag_sum(T, batch, D, arr, rows.ctypes.data, idx.ctypes.data, off.ctypes.data,
                              pooled.ctypes.data, T * D, _ptr(mag))
    if rc != 0:
        raise IndexError("bag index out of range")
    return pooled, mag


def linear(x: np.ndarray, W: np.ndarray, b: np.ndarray, relu: bool, xmag: Optional[np.ndarray] = None):
    """act(x W^T + b) in fp64; returns (y, ymag) -- ymag is None unless xmag is given."""
    x = _f64(x)
    W = _f64(W)
    b = _f64(b)
    m, k = x.shape
    n = W.shape[0]
    assert W.shape[1] == k and b.shape == (n,)
    y = np.zeros((m, n))
    ym = None
    xm = None
    if xmag is not None:
        xm = _f64(xmag)
        ym = np.zeros((m, n))
    lib().oracle_linear(m, k, n, x.ctypes.data, k, W.ctypes.data, b.ctypes.data, 1 if relu else 0,
                        y.ctypes.data, n, _ptr(xm), _ptr(ym))
    return y, ym


def sigmoid(z: float) -> float:
    return lib().oracle_sigmoid(float(z))


# ---------------------------------------------------------------- whole function

class _FnHandle:
    """fp64 copies of one function's weights and (compact) tables, laid out for oracle_forward."""

    def __init__(self, spec, weights, tables: Sequence[np.ndarray]):
        self.spec = spec
        nb, nt = len(spec.bot_dims), len(spec.top_dims)
        self.W = [_f64(w) for (w, _) in weights]
        self.b = [_f64(bb) for (_, bb) in weights]
        self.tabs = [_f64(t) for t in tables]
        self.rows = np.array([t.shape[0] for t in self.tabs], dtype=np.int64)
        self.bot_dims = (ctypes.c_int * nb)(*spec.bot_dims)
        self.top_dims = (ctypes.c_int * nt)(*spec.top_dims)
        mk = lambda arrs: (F64P * len(arrs))(*[a.ctypes.data_as(F64P) for a in arrs])
        self.bW, self.bb = mk(self.W[:nb]), mk(self.b[:nb])
        self.tW, self.tb = mk(self.W[nb:]), mk(self.b[nb:])
        self.tp = mk(self.tabs)
        self.fn = OracleFn(spec.n_tables, spec.dim, spec.n_dense, nb, nt, self.bot_dims, self.top_dims,
                           self.bW, self.bb, self.tW, self.tb, self.tp,
                           self.rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))


def compact_tables(spec, inv, b0: int, b1: int, row_source):
    """Tables holding only the rows that samples [b0, b1) reference, plus remapped
    indices/offsets for that sample range (a renaming of rows, not arithmetic).

    row_source(t, rows) -> float32 [len(rows), D] values of table t."""
    T, B = spec.n_tables, inv["batch"]
    off, idx = inv["offsets"], inv["indices"]
    nb = b1 - b0
    new_off = np.zeros(T * nb + 1, dtype=np.int64)
    parts = []
    tables = []
    pos = 0
    for t in range(T):
        lo, hi = int(off[t * B + b0]), int(off[t * B + b1])
        seg = idx[lo:hi].astype(np.int64)
        uniq, inv_map = np.unique(seg, return_inverse=True)
        tables.append(row_source(t, uniq) if uniq.size else np.zeros((1, spec.dim), np.float32))
        parts.append(inv_map.astype(np.int32))
        local = off[t * B + b0:t * B + b1 + 1] - lo + pos
        new_off[t * nb:t * nb + nb + 1] = local
        pos += hi - lo
    new_idx = np.concatenate(parts) if parts else np.zeros(0, np.int32)
    return tables, new_idx, new_off


def forward(spec, weights, inv, row_source=None, tables=None, b0: int = 0, b1: Optional[int] = None,
            n_threads: int = 1, want_pooled: bool = True) -> Dict[str, np.ndarray]:
    """Oracle of one invocation for samples [b0, b1).

    Either `tables` (full float32 tables) or `row_source(t, rows)` must be given;
    with row_source only the referenced rows are read.  Returns fp64 arrays
    out, out_mag [n] and (if want_pooled) pooled, pooled_mag [n, T*D]."""
    B = inv["batch"]
    b1 = B if b1 is None else b1
    n = b1 - b0
    T, D = spec.n_tables, spec.dim
    if tables is not None and (b0, b1) == (0, B):
        tabs, idx, off = tables, inv["indices"], inv["offsets"]
    else:
        src = row_source if row_source is not None else (lambda t, rows: tables[t][rows])
        tabs, idx, off = compact_tables(spec, inv, b0, b1, src)
    h = _FnHandle(spec, weights, tabs)
    dense = _f64(inv["dense"][b0:b1])
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    out = np.zeros(n)
    out_mag = np.zeros(n)
    pooled = np.zeros((n, T * D)) if want_pooled else None
    pmag = np.zeros((n, T * D)) if want_pooled else None
    rc = lib().oracle_forward(ctypes.byref(h.fn), n, dense.ctypes.data, idx.ctypes.data, off.ctypes.data,
                              0, n, out.ctypes.data, out_mag.ctypes.data, _ptr(pooled), _ptr(pmag),
                              int(n_threads))
    if rc != 0:
        raise RuntimeError("oracle_forward failed: %d" % rc)
    res = {"out": out, "out_mag": out_mag}
    if want_pooled:
        res["pooled"] = pooled
        res["pooled_mag"] = pmag
    return res


# ---------------------------------------------------------------- batching

def pack_invocations(invs: Sequence[dict], n_tables: int) -> dict:
    """Fuse invocations of one function into one batch by the plain definition.

    Samples are concatenated in invocation order (invocation i's sample b becomes
    packed row row_base[i] + b); for each table t the bags of all invocations
    follow each other, and each invocation's offsets are rebased by the number
    of indices already placed.  Returns dense, offsets [T*M+1], indices,
    row_base [n+1]."""
    T = n_tables
    sizes = [int(v["batch"]) for v in invs]
    row_base = [0]
    for s in sizes:
        row_base.append(row_base[-1] + s)
    M = row_base[-1]
    dense = np.concatenate([v["dense"] for v in invs], axis=0) if invs else np.zeros((0, 13), np.float32)
    offsets = [0]
    indices = []
    for t in range(T):
        for v, B in zip(invs, sizes):
            off = v["offsets"]
            for b in range(B):
                lo, hi = int(off[t * B + b]), int(off[t * B + b + 1])
                indices.append(v["indices"][lo:hi])
                offsets.append(offsets[-1] + (hi - lo))
    return {"batch": M, "dense": dense, "offsets": np.array(offsets, dtype=np.int64),
            "indices": np.concatenate(indices).astype(np.int32) if indices else np.zeros(0, np.int32),
            "row_base": np.array(row_base, dtype=np.int64)}


# ---------------------------------------------------------------- sharing model

class PoolModel:
    """Refcount/budget model of read-only sharing (Sec. 6.2).

    The first prepare of a key loads its bytes (counted as H2D bytes) if the
    budget allows; later prepares of a resident key only take a reference;
    release drops one reference and frees the key's bytes at zero."""

    def __init__(self, budget: int):
        self.budget = budget
        self.resident: Dict[str, List[int]] = {}   # key -> [refcount, bytes]
        self.h2d_bytes = 0
        self.hits = 0
        self.misses = 0

    @property
    def used(self) -> int:
        return sum(v[1] for v in self.resident.values())

    def prepare(self, key: str, nbytes: int) -> str:
        if key in self.resident:
            if self.resident[key][1] != nbytes:
                return "INVALID"
            self.resident[key][0] += 1
            self.hits += 1
            return "OK"
        if self.used + nbytes > self.budget:
            return "NOMEM"
        self.resident[key] = [1, nbytes]
        self.h2d_bytes += nbytes
        self.misses += 1
        return "OK"

    def release(self, key: str) -> str:
        if key not in self.resident:
            return "INVALID"
        self.resident[key][0] -= 1
        if self.resident[key][0] == 0:
            del self.resident[key]
        return "OK"

    def refcount(self, key: str) -> int:
        return self.resident.get(key, [0, 0])[0]


# ---------------------------------------------------------------- tolerance

def check_close(got, ref, mag, rtol: float) -> dict:
    """Componentwise check |got - ref| <= rtol * mag (mag = the oracle's magnitude bound).

    Also reports the plain relative error |got-ref|/|ref| (max and median over
    elements with |ref| > 0)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mag = np.asarray(mag, dtype=np.float64)
    err = np.abs(got - ref)
    ok = err <= rtol * mag
    # an exactly-zero bound (e.g. an empty bag) demands an exact zero
    ok |= (mag == 0) & (err == 0)
    nz = np.abs(ref) > 0
    rel = err[nz] / np.abs(ref[nz]) if nz.any() else np.zeros(1)
    scaled = np.where(mag > 0, err / np.where(mag > 0, mag, 1), np.where(err > 0, np.inf, 0))
    worst = int(np.argmax(scaled)) if scaled.size else -1
    return {"ok": bool(ok.all()), "n": int(err.size), "n_bad": int((~ok).sum()),
            "max_scaled_err": float(scaled.max()) if scaled.size else 0.0,
            "max_rel_err": float(rel.max()) if rel.size else 0.0,
            "median_rel_err": float(np.median(rel)) if rel.size else 0.0,
            "worst_index": worst}


def check_output(got, ref, mag, rtol: float) -> dict:
    """The function's final outputs (sigmoids, in (0, 1)): the componentwise bound of
    check_close and, in addition, the plain relative error |got - ref| <= rtol * |ref|
    of every output, the tolerance read literally."""
    c = check_close(got, ref, mag, rtol)
    err = np.abs(np.asarray(got, dtype=np.float64) - np.asarray(ref, dtype=np.float64))
    plain_ok = err <= rtol * np.abs(np.asarray(ref, dtype=np.float64))
    c["n_bad_plain"] = int((~plain_ok).sum())
    c["ok"] = c["ok"] and bool(plain_ok.all())
    return c


# ---------------------------------------------------------------- setup-time model

def setup_latency_model(stages: Dict[str, float], parallel: bool = True) -> float:
    """End-to-end latency of one invocation from its stage durations (Sec. 5.1).

    Serial setup runs every stage one after another.  The parallelised setup
    runs GPU-context preparation beside data preparation (CPU data, then GPU
    data, which depends on it), so the two overlap:
        e2e = cpu_ctx + max(gpu_ctx, cpu_data + gpu_data) + compute + return.
    Keys: cpu_ctx, gpu_ctx, cpu_data, gpu_data, compute, return_data."""
    s = stages
    if not parallel:
        return s["cpu_ctx"] + s["gpu_ctx"] + s["cpu_data"] + s["gpu_data"] + s["compute"] + s["return_data"]
    return s["cpu_ctx"] + max(s["gpu_ctx"], s["cpu_data"] + s["gpu_data"]) + s["compute"] + s["return_data"]


def throughput_perf(throughput_app: float, t_period: float, t_comp: float) -> float:
    """Eq. throughput-theo (Sec. 3.2): Throughput_theo = T_period / T_comp and
    Throughput_perf = Throughput_app / Throughput_theo."""
    return throughput_app / (t_period / t_comp)
