"""sage_invoke_noalloc: the invocation entry point for callers that may not
allocate device memory (for example a host thread that must never enter the
device allocator, or a runtime that owns every device byte and only lends the
library its buffers).  It keeps its activations in a static device array
instead of a pool workspace, so it needs no prepared function handle.

The test calls it through the C-ABI on the read-only data of a prepared
function and checks two calls in a row against sage_invoke, the existing entry
point, within the tolerances of the other parity tests.  This file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, prepare, to_f64

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


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


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_noalloc_matches_sage_invoke_on_two_calls_in_a_row(dtype):
    import torch
    if dtype == "f32":
        spec = workload.spec_tiny(key="na_f32", dtype="f32", n_tables=4, rows=3000, dim=64,
                                  bot=(128, 64), top=(128, 64, 1), l_min=0, l_max=40)
    else:
        spec = workload.FunctionSpec(key="na_bf16", dtype="bf16", rows=[4000, 2500, 6000], dim=128,
                                     bot_dims=[256, 128], top_dims=[256, 128, 1], alpha=1.1, l_min=0, l_max=60)
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


def test_noalloc_rejects_a_batch_beyond_its_scratch():
    spec = workload.spec_c1()
    d, keep = _shape_desc(spec)
    from paper_2404_14691_b300 import _native as N
    # 8.4 KB of fp32 activations per sample: 10,000 samples exceed the 64 MiB scratch
    inv = N.Invocation(10_000, 16, 16, 16, 16, 0)
    st = N.lib().sage_invoke_noalloc(ctypes.byref(d), 16, 16, ctypes.byref(inv), None)
    assert st == -1
    msg = N.lib().sage_last_error().decode()
    assert "scratch" in msg and "67108864" in msg
