"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times (fused batches through sage_invoke_batch), on sampled outputs
that the oracle computes one by one."""
import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, dev, oracle_rows, prepare, to_f64

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


def _torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def pool():
    p = sage.Pool(device=0)
    yield p
    p.destroy()


def _sample_rows(B, rng, k=3):
    rows = {0, B - 1}
    rows.update(int(x) for x in rng.integers(0, B, size=k))
    return sorted(rows)


def test_plain_fp32_invocation_full_oracle(pool):
    """8 x 100,000 x 64 fp32, B = 256, L = 20: every output against the oracle."""
    spec = workload.spec_c1()
    fn = prepare(pool, spec)
    try:
        inv = workload.make_invocation(spec, 256, seed=1234)
        d = DevInvocation(inv)
        fn.invoke(*d.args())
        _torch().cuda.synchronize()
        fn.check_errors()
        w = workload.weights_arrays(spec)
        res = oracle.forward(spec, w, inv, row_source=lambda t, r: workload.table_rows(spec, t, r), n_threads=8,
                             want_pooled=False)
        c = oracle.check_output(to_f64(d.out), res["out"], res["out_mag"], RTOL["f32"])
        assert c["ok"], c
    finally:
        fn.release()


def test_batching_fp32_64_invocations_sampled():
    """The benchmark's default workload: 64 invocations fused into one batch."""
    import bench
    torch = _torch()
    spec, invs, _ = bench.make_workload("c2")
    p = sage.Pool(device=0)
    fn = prepare(p, spec, max_batch=20000)
    try:
        fused = [DevInvocation(v) for v in invs]
        fn.invoke_batch([d.args() for d in fused])
        plain = [DevInvocation(v) for v in invs]
        for d in plain:
            fn.invoke(*d.args())
        torch.cuda.synchronize()
        fn.check_errors()
        for a, b in zip(fused, plain):
            assert torch.equal(a.out, b.out)
        w = workload.weights_arrays(spec)
        rng = np.random.default_rng(0)
        for v, d in zip(invs, fused):
            rows = _sample_rows(v["batch"], rng, 2)
            ref, mag = oracle_rows(spec, w, v, rows)
            c = oracle.check_output(to_f64(d.out)[rows], ref, mag, RTOL["f32"])
            assert c["ok"], c
    finally:
        fn.release()
        p.destroy()


def test_precision_bf16_full_size_sampled(pool):
    """26 x 1,000,000 x 128 bf16 tables (6.7 GB staged), 128 lognormal invocations."""
    import bench
    torch = _torch()
    spec, invs, _ = bench.make_workload("c3")
    M = sum(v["batch"] for v in invs)
    fn = prepare(pool, spec, max_batch=M)
    try:
        fused = [DevInvocation(v) for v in invs]
        fn.invoke_batch([d.args() for d in fused])
        torch.cuda.synchronize()
        fn.check_errors()
        w = workload.weights_arrays(spec)
        rng = np.random.default_rng(1)
        worst = 0.0
        for v, d in list(zip(invs, fused))[::4]:
            rows = _sample_rows(v["batch"], rng, 1)
            ref, mag = oracle_rows(spec, w, v, rows)
            c = oracle.check_output(to_f64(d.out)[rows], ref, mag, RTOL["bf16"])
            assert c["ok"], c
            worst = max(worst, c["max_rel_err"])
        # gather at full size through the building block on the function's own device tables
        tables, _ = fn.data()
        v = max(invs, key=lambda x: x["batch"])
        B = v["batch"]
        out = torch.empty((B, spec.n_tables * spec.dim), dtype=torch.bfloat16, device="cuda")
        idx, off = dev(v["indices"]), dev(v["offsets"])
        sage.embedding_bag_sum(spec.dtype_code, tables, spec.rows, spec.dim, B, idx.data_ptr(), off.data_ptr(),
                               out.data_ptr(), spec.n_tables * spec.dim)
        torch.cuda.synchronize()
        rows = _sample_rows(B, rng, 6)
        got = to_f64(out)[rows]
        for j, r in enumerate(rows):
            for t in range(spec.n_tables):
                lo, hi = v["offsets"][t * B + r], v["offsets"][t * B + r + 1]
                sel = v["indices"][lo:hi].astype(np.int64)
                vals = workload.table_rows(spec, t, sel)
                ref, mag = oracle.bag_sum([vals], np.arange(sel.size, dtype=np.int32),
                                          np.array([0, sel.size], dtype=np.int64), 1)
                c = oracle.check_close(got[j, t * 128:(t + 1) * 128], ref[0], mag[0], RTOL["bf16"])
                assert c["ok"], (r, t, c)
    finally:
        fn.release()
