"""Seeded synthetic inputs for the recommendation-style GPU function.

This module is shared by the CUDA path (benchmarks, tests) and the CPU oracle.
It defines *what the inputs are* -- embedding tables, MLP weights, dense
features, bag indices/offsets, batch sizes, arrival times -- and holds none of
the method's arithmetic (no pooling, no MLP, no packing).

Recipe (how the workload descriptions are read):
  * tables: uniform on [-0.05, 0.05), counter-based SplitMix64 values (gen.c);
    BF16 functions store them rounded to nearest-even.
  * weights: Xavier-uniform, bound sqrt(6/(fan_in+fan_out)); biases uniform
    with bound 1/sqrt(fan_in) (the PyTorch Linear default); biases stay fp32.
  * dense features: N(0,1) fp32, 13 per sample.
  * bag indices: bounded Zipf over ranks 1..N, p(k) ~ k^-alpha, sampled by
    inverse CDF on an fp64 CDF, then mapped to rows by the per-table affine
    bijection row = (a*(k-1) + c) mod N with gcd(a, N) = 1, so that hot rows are
    scattered over the table.  Sampling is with replacement.
  * bag lengths: drawn per bag (per sample, per table), uniform integers in
    [l_min, l_max] (fixed when l_min == l_max).
  * batch sizes: uniform integers in [lo, hi], or round(LogNormal(ln 256, 1.0))
    clamped to [1, 4096].
  * CSR layout of one invocation: table-major, offsets int64 [T*B + 1] with
    offsets[0] == 0; bag (t, b) is indices[offsets[t*B+b] : offsets[t*B+b+1]];
    indices are int32 rows of table t.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading
from functools import lru_cache
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 2404146910
_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libworkload.so")
_lib = None
_lib_lock = threading.Lock()

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def build_lib(force: bool = False) -> str:
    """Compile gen.c into libworkload.so (plain C, -O2, no fast-math)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class TablesCtx(ctypes.Structure):
    _fields_ = [("n_tables", ctypes.c_int), ("dim", ctypes.c_int), ("dtype", ctypes.c_int),
                ("bound", ctypes.c_float), ("rows", ctypes.POINTER(ctypes.c_int64)),
                ("seeds", ctypes.POINTER(ctypes.c_uint64)), ("fail_at_call", ctypes.c_int),
                ("calls", ctypes.c_int)]


class WeightsCtx(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("dtype", ctypes.c_int),
                ("in_dims", ctypes.POINTER(ctypes.c_int)), ("out_dims", ctypes.POINTER(ctypes.c_int)),
                ("w_seeds", ctypes.POINTER(ctypes.c_uint64)), ("b_seeds", ctypes.POINTER(ctypes.c_uint64))]


FILL_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p)


def lib():
    global _lib
    with _lib_lock:
        if _lib is None:
            L = ctypes.CDLL(build_lib())
            L.wl_mix64.restype = ctypes.c_uint64
            L.wl_mix64.argtypes = [ctypes.c_uint64]
            L.wl_draw.restype = ctypes.c_uint64
            L.wl_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.wl_fill_stream.restype = None
            L.wl_fill_stream.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_float,
                                         ctypes.c_uint64, ctypes.c_size_t]
            L.wl_fill_tables.restype = ctypes.c_int
            L.wl_fill_tables.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p]
            L.wl_weights_bytes.restype = ctypes.c_size_t
            L.wl_weights_bytes.argtypes = [ctypes.POINTER(WeightsCtx)]
            L.wl_fill_weights_full.restype = ctypes.c_int
            L.wl_fill_weights_full.argtypes = [ctypes.c_void_p, ctypes.POINTER(WeightsCtx)]
            L.wl_fill_rows.restype = None
            L.wl_fill_rows.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_float,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]
            _lib = L
    return _lib


# ---------------------------------------------------------------- seeds

def mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood 2014)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def draw(seed: int, e: int) -> int:
    """(e+1)-th output of the SplitMix64 sequence started at `seed`."""
    return mix64(seed + (e + 1) * GAMMA)


def _tag(x) -> int:
    if isinstance(x, int):
        return x & MASK64
    h = 0
    for ch in str(x).encode():
        h = mix64(h ^ ch)
    return h


def sub_seed(*parts) -> int:
    """Derive a 64-bit sub-seed from the base seed and a path of tags."""
    h = BASE_SEED
    for p in parts:
        h = mix64(h ^ _tag(p))
    return h


# ---------------------------------------------------------------- function specs

@dataclasses.dataclass
class FunctionSpec:
    key: str
    dtype: str                     # "f32" or "bf16"
    rows: List[int]                # rows per table
    dim: int
    bot_dims: List[int]            # bottom MLP output sizes (input is n_dense)
    top_dims: List[int]            # top MLP output sizes (last is 1: sigmoid head)
    n_dense: int = 13
    alpha: float = 1.05
    l_min: int = 20
    l_max: int = 20
    table_bound: float = 0.05

    @property
    def n_tables(self) -> int:
        return len(self.rows)

    @property
    def dtype_code(self) -> int:
        return 0 if self.dtype == "f32" else 1

    @property
    def elem_bytes(self) -> int:
        return 4 if self.dtype == "f32" else 2

    @property
    def concat_dim(self) -> int:
        return self.n_tables * self.dim + self.bot_dims[-1]

    def layer_dims(self):
        """[(in, out)] for bottom layers then top layers."""
        dims = []
        prev = self.n_dense
        for o in self.bot_dims:
            dims.append((prev, o))
            prev = o
        prev = self.concat_dim
        for o in self.top_dims:
            dims.append((prev, o))
            prev = o
        return dims

    def table_seeds(self) -> List[int]:
        return [sub_seed(self.key, "table", t) for t in range(self.n_tables)]

    def table_bytes(self) -> int:
        return sum(self.rows) * self.dim * self.elem_bytes


def spec_c1(key: str = "c1_f32_8x100k_d64") -> FunctionSpec:
    """8 tables x 100,000 rows x 64 fp32, L = 20, Zipf 1.05; MLPs 13-512-256-64 / 576-512-256-1."""
    return FunctionSpec(key=key, dtype="f32", rows=[100_000] * 8, dim=64,
                        bot_dims=[512, 256, 64], top_dims=[512, 256, 1], alpha=1.05, l_min=20, l_max=20)


def spec_c2(key: str = "c1_f32_8x100k_d64") -> FunctionSpec:
    """The same function as C1 with L uniform in [1, 40] (batching workload)."""
    s = spec_c1(key)
    s.l_min, s.l_max = 1, 40
    return s


def spec_c3(key: str = "c3_bf16_26x1m_d128", rows: int = 1_000_000) -> FunctionSpec:
    """26 tables x 1M rows x 128 bf16, L uniform in [1, 100], Zipf 1.1; MLPs 13-512-256-128 / 3456-1024-512-256-1."""
    return FunctionSpec(key=key, dtype="bf16", rows=[rows] * 26, dim=128,
                        bot_dims=[512, 256, 128], top_dims=[1024, 512, 256, 1], alpha=1.1, l_min=1, l_max=100)


def spec_c4_functions() -> List[FunctionSpec]:
    """The four serving functions (BF16; MLP shapes as C1 for D=64 and C3 for D=128)."""
    f = []
    f.append(FunctionSpec(key="c4_fn0_8x1m_d64", dtype="bf16", rows=[1_000_000] * 8, dim=64,
                          bot_dims=[512, 256, 64], top_dims=[512, 256, 1], alpha=1.1, l_min=1, l_max=100))
    f.append(spec_c3("c4_fn1_26x1m_d128"))
    f.append(spec_c3("c4_fn2_26x4m_d128", rows=4_000_000))
    f.append(FunctionSpec(key="c4_fn3_52x2m_d64", dtype="bf16", rows=[2_000_000] * 52, dim=64,
                          bot_dims=[512, 256, 64], top_dims=[1024, 512, 256, 1], alpha=1.1, l_min=1, l_max=100))
    return f


def spec_c5_function(i: int) -> FunctionSpec:
    s = spec_c3("c5_fn%02d_26x2m_d128" % i, rows=2_000_000)
    s.l_min = s.l_max = 80
    return s


def spec_tiny(key="tiny", dtype="f32", n_tables=3, rows=50, dim=8, bot=(16, 8), top=(16, 1),
              l_min=0, l_max=5, alpha=1.05) -> FunctionSpec:
    return FunctionSpec(key=key, dtype=dtype, rows=[rows] * n_tables, dim=dim, bot_dims=list(bot),
                        top_dims=list(top), alpha=alpha, l_min=l_min, l_max=l_max)


# ---------------------------------------------------------------- read-only data

def tables_ctx(spec: FunctionSpec, fail_at_call: int = 0):
    """ctypes context for wl_fill_tables (the producer callback of the tables blob).

    Returns (ctx, keepalive); keep `keepalive` referenced while the ctx is used."""
    rows = (ctypes.c_int64 * spec.n_tables)(*spec.rows)
    seeds = (ctypes.c_uint64 * spec.n_tables)(*spec.table_seeds())
    ctx = TablesCtx(spec.n_tables, spec.dim, spec.dtype_code, spec.table_bound, rows, seeds, fail_at_call, 0)
    return ctx, (rows, seeds)


def fill_tables_fnptr():
    """Address of the C producer callback wl_fill_tables."""
    return ctypes.cast(lib().wl_fill_tables, ctypes.c_void_p).value


def tables_blob(spec: FunctionSpec) -> np.ndarray:
    """The whole tables blob as bytes (only for small functions)."""
    ctx, keep = tables_ctx(spec)
    out = np.empty(spec.table_bytes(), dtype=np.uint8)
    rc = lib().wl_fill_tables(out.ctypes.data, 0, out.nbytes, ctypes.byref(ctx))
    assert rc == 0
    return out


def _weights_ctx(spec: FunctionSpec):
    dims = spec.layer_dims()
    n = len(dims)
    ins = (ctypes.c_int * n)(*[d[0] for d in dims])
    outs = (ctypes.c_int * n)(*[d[1] for d in dims])
    ws = (ctypes.c_uint64 * n)(*[sub_seed(spec.key, "W", l) for l in range(n)])
    bs = (ctypes.c_uint64 * n)(*[sub_seed(spec.key, "b", l) for l in range(n)])
    return WeightsCtx(n, spec.dtype_code, ins, outs, ws, bs), (ins, outs, ws, bs)


def weights_blob(spec: FunctionSpec) -> np.ndarray:
    ctx, keep = _weights_ctx(spec)
    nbytes = lib().wl_weights_bytes(ctypes.byref(ctx))
    out = np.empty(nbytes, dtype=np.uint8)
    lib().wl_fill_weights_full(out.ctypes.data, ctypes.byref(ctx))
    return out


def _align256(x: int) -> int:
    return (x + 255) & ~255


def weights_layout(spec: FunctionSpec):
    """[(w_off, b_off)] byte offsets of W_l and b_l inside the weights blob."""
    es = spec.elem_bytes
    o = 0
    lay = []
    for (i, n) in spec.layer_dims():
        o = _align256(o)
        wo = o
        o += n * i * es
        o = _align256(o)
        bo = o
        o += n * 4
        lay.append((wo, bo))
    return lay


def bf16_bits_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def weights_arrays(spec: FunctionSpec, blob: Optional[np.ndarray] = None):
    """[(W [out,in] float32, b [out] float32)] -- BF16 weights widened exactly to fp32."""
    blob = weights_blob(spec) if blob is None else blob
    res = []
    for (wo, bo), (i, n) in zip(weights_layout(spec), spec.layer_dims()):
        if spec.dtype == "f32":
            W = blob[wo:wo + 4 * n * i].view(np.float32).reshape(n, i).copy()
        else:
            W = bf16_bits_to_f32(blob[wo:wo + 2 * n * i].view(np.uint16)).reshape(n, i)
        b = blob[bo:bo + 4 * n].view(np.float32).copy()
        res.append((W, b))
    return res


def table_rows(spec: FunctionSpec, t: int, rows: np.ndarray) -> np.ndarray:
    """Values of the given rows of table t as float32 [len(rows), dim] (BF16 widened exactly)."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n = rows.size
    if spec.dtype == "f32":
        out = np.empty((n, spec.dim), dtype=np.float32)
    else:
        out = np.empty((n, spec.dim), dtype=np.uint16)
    lib().wl_fill_rows(out.ctypes.data, spec.dtype_code, spec.table_seeds()[t], spec.table_bound,
                       spec.dim, rows.ctypes.data, n)
    return out if spec.dtype == "f32" else bf16_bits_to_f32(out)


def full_table(spec: FunctionSpec, t: int) -> np.ndarray:
    return table_rows(spec, t, np.arange(spec.rows[t], dtype=np.int64))


# ---------------------------------------------------------------- per-invocation data

@lru_cache(maxsize=16)
def zipf_cdf(n: int, alpha: float) -> np.ndarray:
    """Unnormalised fp64 CDF of the bounded Zipf law p(k) ~ k^-alpha on ranks 1..n."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return np.cumsum(k ** (-alpha))


def affine_map(spec: FunctionSpec, t: int):
    """(a, c) of the rank -> row bijection row = (a*rank0 + c) mod N for table t."""
    n = spec.rows[t]
    s = sub_seed(spec.key, "affine", t)
    a = (s % (1 << 31)) | 1
    while math.gcd(a, n) != 1:
        a += 2
    c = mix64(s) % n
    return a % n if n > 1 else 0, c


def zipf_ranks(rng: np.random.Generator, n_rows: int, alpha: float, count: int) -> np.ndarray:
    """0-based Zipf ranks (rank 0 is the most popular)."""
    cdf = zipf_cdf(n_rows, alpha)
    u = rng.random(count) * cdf[-1]
    r = np.searchsorted(cdf, u, side="right")
    return np.minimum(r, n_rows - 1)


def make_invocation(spec: FunctionSpec, batch: int, seed: int, uniform_rows: bool = False):
    """One invocation's inputs: dict(dense [B, n_dense] f32, offsets int64 [T*B+1], indices int32).

    uniform_rows=True draws rows uniformly instead of Zipf (the no-reuse control)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T, B = spec.n_tables, batch
    dense = rng.standard_normal((B, spec.n_dense), dtype=np.float32)
    lengths = rng.integers(spec.l_min, spec.l_max + 1, size=T * B, dtype=np.int64)
    offsets = np.zeros(T * B + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    indices = np.empty(int(offsets[-1]), dtype=np.int32)
    for t in range(T):
        lo, hi = int(offsets[t * B]), int(offsets[(t + 1) * B])
        n_rows = spec.rows[t]
        if uniform_rows:
            rows = rng.integers(0, n_rows, size=hi - lo, dtype=np.int64)
        else:
            ranks = zipf_ranks(rng, n_rows, spec.alpha, hi - lo)
            a, c = affine_map(spec, t)
            rows = (a * ranks + c) % n_rows
        indices[lo:hi] = rows.astype(np.int32)
    return {"batch": B, "dense": dense, "offsets": offsets, "indices": indices}


def batch_sizes_uniform(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=count, dtype=np.int64)


def batch_sizes_lognormal(count: int, seed: int, median: float = 256.0, sigma: float = 1.0,
                          lo: int = 1, hi: int = 4096) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.lognormal(mean=math.log(median), sigma=sigma, size=count)
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


# ---------------------------------------------------------------- C-ABI arguments

def prepare_kwargs(spec: FunctionSpec, fail_at_call: int = 0, tables_in_host_memory: bool = False):
    """Keyword arguments of paper_2404_14691_b300.Pool.prepare for this function's
    read-only data: the tables come from the C producer wl_fill_tables (or from a
    host image when tables_in_host_memory), the weights from a host image."""
    wblob = weights_blob(spec)
    kw = dict(key=spec.key, dtype=spec.dtype_code, rows=list(spec.rows), dim=spec.dim, n_dense=spec.n_dense,
              bot_dims=list(spec.bot_dims), top_dims=list(spec.top_dims), tables_bytes=spec.table_bytes(),
              weights_bytes=int(wblob.nbytes), weights_src=wblob.ctypes.data)
    keep = [wblob]
    if tables_in_host_memory:
        tb = tables_blob(spec)
        kw["tables_src"] = tb.ctypes.data
        keep.append(tb)
    else:
        ctx, k2 = tables_ctx(spec, fail_at_call=fail_at_call)
        kw["tables_fill"] = fill_tables_fnptr()
        kw["tables_ctx"] = ctx
        keep.append(k2)
    kw["keep"] = keep
    return kw
