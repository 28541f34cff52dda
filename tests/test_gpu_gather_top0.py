"""The gather fused with the first top layer (fp32 functions with 64-column tables):
the pooled bags are summed straight into the GEMM's shared-memory A tiles and never
written.  Through the runtime (sage_invoke_batch), the fused kernel's first hidden
layer equals the separate gather + GEMM bit for bit (both planes), the outputs are
identical and match the oracle, over one and several tiles per CTA, ragged last
tiles, empty bags, 256- and 512-wide layers and a bottom output of two or four
k-blocks; an out-of-range row is reported and skipped as in the separate gather."""
import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, prepare, to_f64

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")

KIND = 5      # tuning kind: gather + first top layer (256, 2) fused, (1, 1) separate


def _specs():
    return {
        "n256": workload.FunctionSpec(key="g0_n256", dtype="f32", rows=[3000, 2000, 5000], dim=64,
                                      bot_dims=[128, 64], top_dims=[256, 64, 1], alpha=1.05, l_min=0, l_max=40),
        "n512": workload.FunctionSpec(key="g0_n512", dtype="f32", rows=[4000] * 8, dim=64,
                                      bot_dims=[512, 256, 64], top_dims=[512, 256, 1], alpha=1.05, l_min=0,
                                      l_max=40),
        "n512_bot128": workload.FunctionSpec(key="g0_b128", dtype="f32", rows=[2500] * 5, dim=64,
                                             bot_dims=[128, 128], top_dims=[512, 128, 1], alpha=1.05, l_min=1,
                                             l_max=30),
    }


def _run(fn, spec, invs, fused):
    import torch
    M = sum(v["batch"] for v in invs)
    sage.tuning_set(KIND, M, spec.top_dims[0], spec.concat_dim, 256 if fused else 1, 2 if fused else 1)
    d = [DevInvocation(v) for v in invs]
    fn.invoke_batch([x.args() for x in d])
    torch.cuda.synchronize()
    hi = fn.debug_copy(1, spec.top_dims[0], bf16=False, plane=0)
    lo = fn.debug_copy(1, spec.top_dims[0], bf16=False, plane=1)
    if fused:
        with pytest.raises(sage.SageError):
            fn.debug_copy(0, spec.concat_dim, bf16=False)
    return d, hi, lo


@pytest.mark.parametrize("name,sizes", [("n256", [37]), ("n256", [1, 129, 300, 5]), ("n512", [256] * 80),
                                        ("n512", [333, 1, 900, 128]), ("n512_bot128", [1000, 77, 2500])])
def test_fused_equals_separate_bitwise_and_matches_the_oracle(name, sizes):
    import torch
    spec = _specs()[name]
    pool = sage.Pool(device=0)
    fn = prepare(pool, spec, max_batch=sum(sizes))
    try:
        invs = [workload.make_invocation(spec, B, seed=700 + i) for i, B in enumerate(sizes)]
        ds, hs, ls = _run(fn, spec, invs, fused=False)
        df, hf, lf = _run(fn, spec, invs, fused=True)
        fn.check_errors()
        assert np.array_equal(hs.view(np.uint32), hf.view(np.uint32))
        assert np.array_equal(ls.view(np.uint32), lf.view(np.uint32))
        for a, b in zip(ds, df):
            assert torch.equal(a.out, b.out)
        w = workload.weights_arrays(spec)
        tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
        for v, b in zip(invs, df):
            res = oracle.forward(spec, w, v, tables=tables, want_pooled=False, n_threads=8)
            c = oracle.check_output(to_f64(b.out)[:v["batch"]], res["out"], res["out_mag"], RTOL["f32"])
            assert c["ok"], c
    finally:
        fn.release()
        pool.destroy()


def test_fused_reports_and_skips_an_out_of_range_row():
    import torch
    spec = _specs()["n512"]
    pool = sage.Pool(device=0)
    fn = prepare(pool, spec, max_batch=4096)
    try:
        invs = [workload.make_invocation(spec, B, seed=900 + i) for i, B in enumerate([300, 200])]
        B = invs[1]["batch"]
        t, b = 3, 11
        lo = int(invs[1]["offsets"][t * B + b])
        assert int(invs[1]["offsets"][t * B + b + 1]) > lo
        invs[1] = dict(invs[1], indices=invs[1]["indices"].copy())
        invs[1]["indices"][lo] = spec.rows[t] + 5
        ds, hs, ls = _run(fn, spec, invs, fused=False)
        with pytest.raises(sage.SageError, match="BOUNDS"):
            fn.check_errors()
        df, hf, lf = _run(fn, spec, invs, fused=True)
        with pytest.raises(sage.SageError, match="BOUNDS"):
            fn.check_errors()
        assert np.array_equal(hs.view(np.uint32), hf.view(np.uint32))
        for a, c in zip(ds, df):
            assert torch.equal(a.out, c.out)
        fn.check_errors()          # cleared by the report
    finally:
        fn.release()
        pool.destroy()


def test_many_tiles_per_cta():
    """More row tiles than SMs: each CTA runs several tiles in turn."""
    import torch
    spec = _specs()["n512"]
    sizes = [4096, 4096, 4096, 4096, 3000]            # 19,384 rows = 152 tiles
    pool = sage.Pool(device=0)
    fn = prepare(pool, spec, max_batch=sum(sizes))
    try:
        invs = [workload.make_invocation(spec, B, seed=1100 + i) for i, B in enumerate(sizes)]
        ds, hs, ls = _run(fn, spec, invs, fused=False)
        df, hf, lf = _run(fn, spec, invs, fused=True)
        fn.check_errors()
        assert np.array_equal(hs.view(np.uint32), hf.view(np.uint32))
        assert np.array_equal(ls.view(np.uint32), lf.view(np.uint32))
        for a, b in zip(ds, df):
            assert torch.equal(a.out, b.out)
    finally:
        fn.release()
        pool.destroy()
