"""sage_invoke_noalloc: the invocation entry point for callers that may not
allocate device memory (for example a host thread that must never enter the
device allocator, or a runtime that owns every device byte and only lends the
library its buffers).  It keeps its activations in a static device array
instead of a pool workspace, so it needs no prepared function handle.

The tests call it through the C-ABI on the read-only data of a prepared
function and check two calls in a row against sage_invoke, the existing entry
point, within the tolerances of the other parity tests; sage_noalloc_check
reports a clean error word after each.  A bag row outside its table is reported
by sage_noalloc_check and the other rows still match the oracle; oversized
batches and misaligned buffers are refused before anything is launched.  This
file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, prepare, to_f64

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")

SCRATCH_BYTES = 64 << 20      # the documented size of the no-alloc scratch array
SAGE_ERR_INVALID, SAGE_ERR_BOUNDS = -1, -7


def _shape_desc(spec):
    from paper_2404_14691_b300 import _native as N
    rows = (ctypes.c_int64 * spec.n_tables)(*spec.rows)
    bot = (ctypes.c_int * len(spec.bot_dims))(*spec.bot_dims)
    top = (ctypes.c_int * len(spec.top_dims))(*spec.top_dims)
    empty = N.DataDesc(None, 0, 0, None, None, None)
    d = N.FnDesc(spec.key.encode(), spec.dtype_code, spec.n_tables, rows, spec.dim, spec.n_dense,
                 len(spec.bot_dims), bot, len(spec.top_dims), top, 0, 0, empty, empty)
    return d, (rows, bot, top)


def _noalloc(spec, tables, weights, dinv, stream=None):
    from paper_2404_14691_b300 import _native as N
    d, keep = _shape_desc(spec)
    inv = N.Invocation(dinv.batch, dinv.dense.data_ptr(), dinv.indices.data_ptr(), dinv.offsets.data_ptr(),
                       dinv.out.data_ptr(), int(dinv.inv["indices"].size))
    return N.lib().sage_invoke_noalloc(ctypes.byref(d), tables, weights, ctypes.byref(inv), stream)


def _check(stream=None):
    from paper_2404_14691_b300 import _native as N
    return N.lib().sage_noalloc_check(stream)


def _specs(dtype):
    if dtype == "f32":
        return workload.spec_tiny(key="na_f32", dtype="f32", n_tables=4, rows=3000, dim=64,
                                  bot=(128, 64), top=(128, 64, 1), l_min=0, l_max=40)
    return workload.FunctionSpec(key="na_bf16", dtype="bf16", rows=[4000, 2500, 6000], dim=128,
                                 bot_dims=[256, 128], top_dims=[256, 128, 1], alpha=1.1, l_min=0, l_max=60)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_noalloc_matches_sage_invoke_on_two_calls_in_a_row(dtype):
    import torch
    spec = _specs(dtype)
    pool = sage.Pool(device=0)
    fn = prepare(pool, spec)
    try:
        fn.wait()
        tables, weights = fn.data()
        w = workload.weights_arrays(spec)
        full = [workload.full_table(spec, t) for t in range(spec.n_tables)]
        for call, (B, seed) in enumerate([(300, 21), (57, 22)]):
            inv = workload.make_invocation(spec, B, seed=seed)
            ref = DevInvocation(inv)
            fn.invoke(*ref.args())
            got = DevInvocation(inv)
            st = _noalloc(spec, tables, weights, got)
            assert st == 0, sage._native.lib().sage_last_error()
            assert _check() == 0, sage._native.lib().sage_last_error()
            torch.cuda.synchronize()
            a, b = to_f64(ref.out)[:B], to_f64(got.out)[:B]
            # against the existing entry point, within the parity tolerance
            res = oracle.forward(spec, w, inv, tables=full, want_pooled=False)
            scale = np.maximum(res["out_mag"], np.abs(a))
            assert np.all(np.abs(a - b) <= RTOL[dtype] * scale), ("call", call)
            # and both against the oracle
            assert oracle.check_output(b, res["out"], res["out_mag"], RTOL[dtype])["ok"]
            assert oracle.check_output(a, res["out"], res["out_mag"], RTOL[dtype])["ok"]
    finally:
        fn.release()
        pool.destroy()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_noalloc_reports_an_out_of_range_row_and_skips_it(dtype):
    """One index past its table's end: sage_noalloc_check returns SAGE_ERR_BOUNDS,
    the row is skipped (the bag sums the rest), every output matches the oracle of
    the same invocation with that index removed, and the next clean call reports OK."""
    import torch
    spec = _specs(dtype)
    pool = sage.Pool(device=0)
    fn = prepare(pool, spec)
    try:
        fn.wait()
        tables, weights = fn.data()
        w = workload.weights_arrays(spec)
        full = [workload.full_table(spec, t) for t in range(spec.n_tables)]
        B = 120
        inv = workload.make_invocation(spec, B, seed=31)
        t, b = 1, 17                                  # bag (t, b) gets the bad row
        lo, hi = int(inv["offsets"][t * B + b]), int(inv["offsets"][t * B + b + 1])
        assert hi > lo
        bad = dict(inv, indices=inv["indices"].copy())
        bad["indices"][lo] = spec.rows[t]             # one past the end of table t
        got = DevInvocation(bad)
        assert _noalloc(spec, tables, weights, got) == 0
        assert _check() == SAGE_ERR_BOUNDS
        assert "outside" in sage._native.lib().sage_last_error().decode()
        torch.cuda.synchronize()
        # the oracle of the invocation without that index (the skip, by definition)
        dropped = dict(inv, indices=np.delete(inv["indices"], lo), offsets=inv["offsets"].copy())
        dropped["offsets"][t * B + b + 1:] -= 1
        res = oracle.forward(spec, w, dropped, tables=full, want_pooled=False)
        c = oracle.check_output(to_f64(got.out)[:B], res["out"], res["out_mag"], RTOL[dtype])
        assert c["ok"], c
        # the error word was cleared: a clean call reports OK
        clean = DevInvocation(inv)
        assert _noalloc(spec, tables, weights, clean) == 0
        assert _check() == 0
    finally:
        fn.release()
        pool.destroy()


def test_noalloc_rejects_a_batch_beyond_its_scratch():
    """A batch whose activations exceed the 64 MiB array is refused on the host; the
    buffers are real (and aligned) device buffers, so nothing could launch on a bad
    address even if the checks were reordered."""
    import torch
    spec = workload.spec_c1()
    per_sample = 4 * (sum(spec.bot_dims[:-1]) + spec.n_tables * spec.dim + spec.bot_dims[-1]
                      + sum(spec.top_dims[:-1]))
    B = SCRATCH_BYTES // per_sample + 1
    assert B * per_sample > SCRATCH_BYTES
    d, keep = _shape_desc(spec)
    from paper_2404_14691_b300 import _native as N
    tables = torch.zeros(64, dtype=torch.float32, device="cuda")
    weights = torch.zeros(64, dtype=torch.float32, device="cuda")
    dense = torch.zeros(16, dtype=torch.float32, device="cuda")
    idx = torch.zeros(16, dtype=torch.int32, device="cuda")
    off = torch.zeros(16, dtype=torch.int64, device="cuda")
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    inv = N.Invocation(B, dense.data_ptr(), idx.data_ptr(), off.data_ptr(), out.data_ptr(), 0)
    st = N.lib().sage_invoke_noalloc(ctypes.byref(d), tables.data_ptr(), weights.data_ptr(), ctypes.byref(inv), None)
    assert st == SAGE_ERR_INVALID
    msg = N.lib().sage_last_error().decode()
    assert "scratch" in msg and str(SCRATCH_BYTES) in msg


def test_noalloc_refuses_misaligned_buffers():
    """Misaligned tables, weights, dense or out pointers are refused with
    SAGE_ERR_INVALID before any launch (offsets into real device buffers)."""
    import torch
    spec = _specs("f32")
    d, keep = _shape_desc(spec)
    from paper_2404_14691_b300 import _native as N
    buf = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")
    base = buf.data_ptr()
    assert base % 256 == 0
    ok = dict(tables=base, weights=base + 4096, dense=base + 8192, idx=base + 12288, off=base + 16384,
              out=base + 20480)
    for name, delta in (("tables", 16), ("weights", 64), ("dense", 4), ("out", 8), ("idx", 2), ("off", 4)):
        p = dict(ok)
        p[name] += delta
        inv = N.Invocation(4, p["dense"], p["idx"], p["off"], p["out"], 0)
        st = N.lib().sage_invoke_noalloc(ctypes.byref(d), p["tables"], p["weights"], ctypes.byref(inv), None)
        assert st == SAGE_ERR_INVALID, name
        assert "aligned" in N.lib().sage_last_error().decode(), name
    torch.cuda.synchronize()
