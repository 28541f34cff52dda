"""Element-wise parity of the benchmark's fused batches at full size.

The fused batch runs exactly as the benchmark times it (a CUDA-graph pool, tiles
autotuned for the batch, the runtime's claimed-work gather, the persistent GEMMs
with the head in the last hidden layer's epilogue).  Its workspace is then read
back through sage_fn_debug_copy and compared with the oracle element by element:

  * the concat buffer: every pooled bag column (the gather's output) of the
    checked invocations, against the oracle's index-order fp64 sums -- at the
    stated tolerance and at the bound the arithmetic fixes (one rounding of an fp32
    sum), which also catches a dropped or repeated row of a 100-row bf16 bag; and
    the bottom MLP's output columns at the stated tolerance;
  * the first top hidden layer, computed by the oracle from its own concat.

The per-invocation definition is what read-only sharing must reproduce (Sec. 6.2).
Errors against the fp64 oracle are printed per result."""
import numpy as np
import pytest

import oracle
import workload
from helpers import (RTOL, DevInvocation, check_rounded_bag_sums, oracle_bottom, oracle_pooled, oracle_top0,
                     prepare, to_f64)

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


def _fused_batch(name, gather_top0=None):
    """The workload's fused batch as the benchmark runs it; gather_top0 True / False
    pins the gather + first-top-layer fusion on / off (fp32 functions), None leaves
    the default."""
    import bench
    import torch
    spec, invs, _ = bench.make_workload(name)
    M = int(sum(v["batch"] for v in invs))
    pool = sage.Pool(device=0, graphs=True)
    fn = prepare(pool, spec, max_batch=max(4096, M), workspace_slots=2)
    fn.autotune(M)
    if gather_top0 is not None:
        sage.tuning_set(5, M, spec.top_dims[0], spec.concat_dim, 256 if gather_top0 else 1, 2 if gather_top0 else 1)
    dinv = [DevInvocation(v) for v in invs]
    fn.invoke_batch([d.args() + (int(v["indices"].size),) for v, d in zip(invs, dinv)])
    torch.cuda.synchronize()
    fn.check_errors()
    return pool, fn, spec, invs, dinv, M


def _read(fn, spec, which, width):
    if spec.dtype == "bf16":
        return workload.bf16_bits_to_f32(fn.debug_copy(which, width, bf16=True)).astype(np.float64)
    # fp32 functions on the tensor cores keep hi (tf32) and lo planes; value = hi + lo exactly
    hi = fn.debug_copy(which, width, bf16=False, plane=0).astype(np.float64)
    lo = fn.debug_copy(which, width, bf16=False, plane=1).astype(np.float64)
    return hi + lo


def _check_invocation(spec, w, inv, concat_rows, rtol, bits, report):
    T, D = spec.n_tables, spec.dim
    pooled, pmag = oracle_pooled(spec, inv)
    got = concat_rows[:, :T * D]
    c = oracle.check_close(got, pooled, pmag, rtol)
    r = check_rounded_bag_sums(got, pooled, pmag, bits)
    assert c["ok"] and r["ok"], (c, r)
    bot, bmag = oracle_bottom(spec, w, inv["dense"])
    cb = oracle.check_close(concat_rows[:, T * D:], bot, bmag, rtol)
    assert cb["ok"], cb
    report["pooled_max_scaled"] = max(report.get("pooled_max_scaled", 0.0), c["max_scaled_err"])
    report["pooled_max_over_rounding_bound"] = max(report.get("pooled_max_over_rounding_bound", 0.0),
                                                   r["max_err_over_bound"])
    report["bottom_max_scaled"] = max(report.get("bottom_max_scaled", 0.0), cb["max_scaled_err"])
    report["elements"] = report.get("elements", 0) + got.size + cb["n"]
    return np.concatenate([pooled, bot], axis=1), np.concatenate([pmag, bmag], axis=1)


def _check_outputs(spec, w, inv, dinv, rtol, report, threads=16):
    """Every final output (sigmoid) of one invocation against the oracle's, at the
    componentwise bound and at the tolerance read literally."""
    res = oracle.forward(spec, w, inv, row_source=lambda t, r: workload.table_rows(spec, t, r),
                         n_threads=threads, want_pooled=False)
    c = oracle.check_output(to_f64(dinv.out)[:inv["batch"]], res["out"], res["out_mag"], rtol)
    assert c["ok"], c
    report["out_max_rel"] = max(report.get("out_max_rel", 0.0), c["max_rel_err"])
    report["outputs"] = report.get("outputs", 0) + c["n"]


def _check_top0(spec, w, fn, M, row0, B, ref_concat, ref_mag, rtol, report):
    W0 = spec.top_dims[0]
    top0 = _read(fn, spec, 1, W0)
    assert top0.shape == (M, W0)
    h, hm = oracle_top0(spec, w, ref_concat, ref_mag)
    c = oracle.check_close(top0[row0:row0 + B], h, hm, rtol)
    assert c["ok"], c
    report["top0_max_scaled"] = max(report.get("top0_max_scaled", 0.0), c["max_scaled_err"])
    report["top0_elements"] = report.get("top0_elements", 0) + c["n"]


def test_batching_fp32_64_invocations_every_element():
    """8 x 100,000 x 64 fp32, 64 invocations (~16k samples), the gather as its own
    kernel: every pooled and bottom column of every invocation, the first top hidden
    layer of every row, and every output."""
    pool, fn, spec, invs, dinv, M = _fused_batch("c2", gather_top0=False)
    try:
        w = workload.weights_arrays(spec)
        concat = _read(fn, spec, 0, spec.concat_dim)
        assert concat.shape == (M, spec.concat_dim)
        report = {}
        refs, mags = [], []
        row0 = 0
        for v in invs:
            B = v["batch"]
            rc, rm = _check_invocation(spec, w, v, concat[row0:row0 + B], RTOL["f32"], 24, report)
            refs.append(rc)
            mags.append(rm)
            row0 += B
        _check_top0(spec, w, fn, M, 0, M, np.concatenate(refs), np.concatenate(mags), RTOL["f32"], report)
        for v, d in zip(invs, dinv):
            _check_outputs(spec, w, v, d, RTOL["f32"], report)
        print("fp32 batching, error vs fp64 oracle:", report)
    finally:
        fn.release()
        pool.destroy()


def test_batching_fp32_gather_fused_with_top0_every_element():
    """The same batch with the gather fused into the first top layer (the pooled
    columns never leave the chip): the first top hidden layer of every row against
    the oracle, bitwise equal to the unfused chain's, and the outputs identical."""
    import torch
    pool, fn, spec, invs, dinv, M = _fused_batch("c2", gather_top0=True)
    try:
        w = workload.weights_arrays(spec)
        hi = fn.debug_copy(1, spec.top_dims[0], bf16=False, plane=0)
        report = {}
        refs, mags = [], []
        for v in invs:
            pooled, pmag = oracle_pooled(spec, v)
            bot, bmag = oracle_bottom(spec, w, v["dense"])
            refs.append(np.concatenate([pooled, bot], axis=1))
            mags.append(np.concatenate([pmag, bmag], axis=1))
        _check_top0(spec, w, fn, M, 0, M, np.concatenate(refs), np.concatenate(mags), RTOL["f32"], report)
        print("fp32 batching, gather fused with top layer 0, error vs fp64 oracle:", report)
        fn.release()
        pool.destroy()
        pool2, fn2, _, _, dinv2, _ = _fused_batch("c2", gather_top0=False)
        try:
            assert np.array_equal(hi.view(np.uint32),
                                  fn2.debug_copy(1, spec.top_dims[0], bf16=False, plane=0).view(np.uint32))
            for a, b in zip(dinv, dinv2):
                assert torch.equal(a.out, b.out)
        finally:
            fn2.release()
            pool2.destroy()
        fn = pool = None
    finally:
        if fn is not None:
            fn.release()
            pool.destroy()


def test_precision_bf16_full_size_every_element_of_16_invocations():
    """26 x 1,000,000 x 128 bf16 (6.7 GB), 128 lognormal invocations (~57k samples) in one
    fused batch: every pooled and bottom column and every output of 16 whole invocations
    (every eighth), and the first top hidden layer (3456 -> 1024) of two of them."""
    pool, fn, spec, invs, dinv, M = _fused_batch("c3")
    try:
        w = workload.weights_arrays(spec)
        concat = _read(fn, spec, 0, spec.concat_dim)
        assert concat.shape == (M, spec.concat_dim)
        base = np.concatenate([[0], np.cumsum([v["batch"] for v in invs])])
        report = {}
        checked = list(range(0, len(invs), 8))
        for i in checked:
            v = invs[i]
            rc, rm = _check_invocation(spec, w, v, concat[base[i]:base[i + 1]], RTOL["bf16"], 8, report)
            if i in checked[:2]:
                _check_top0(spec, w, fn, M, int(base[i]), v["batch"], rc, rm, RTOL["bf16"], report)
            _check_outputs(spec, w, v, dinv[i], RTOL["bf16"], report)
        report["invocations"] = len(checked)
        report["samples"] = int(sum(invs[i]["batch"] for i in checked))
        print("bf16 precision, error vs fp64 oracle:", report)
    finally:
        fn.release()
        pool.destroy()


def test_debug_copy_refuses_what_was_not_written():
    """The last hidden layer is not written when the head runs in its epilogue, and a
    function with no batch yet has nothing to copy."""
    import torch
    spec = workload.spec_tiny(key="dbg_f32", dtype="f32", n_tables=2, rows=500, dim=64, bot=(64, 64),
                              top=(128, 64, 1), l_min=1, l_max=8)
    pool = sage.Pool(device=0)
    fn = prepare(pool, spec)
    try:
        with pytest.raises(sage.SageError):
            fn.debug_copy(0, spec.concat_dim, bf16=False)
        d = DevInvocation(workload.make_invocation(spec, 300, seed=3))
        fn.invoke(*d.args())
        torch.cuda.synchronize()
        c = fn.debug_copy(0, spec.concat_dim, bf16=False)
        assert c.shape == (300, spec.concat_dim)
        with pytest.raises(sage.SageError):
            fn.debug_copy(5, 10, bf16=False)
        with pytest.raises(sage.SageError):
            fn.debug_copy(0, spec.concat_dim, bf16=False, plane=2)
    finally:
        fn.release()
        pool.destroy()
