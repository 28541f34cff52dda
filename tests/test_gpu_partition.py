"""SM partitions (green contexts): a launch chain on a partition's stream stays on
the partition's SMs, gives the same bits as on the whole GPU, and the serving
loop can give each function its own partition."""
import time

import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, prepare

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


def _spec(dtype):
    if dtype == "f32":
        return workload.spec_tiny(key="pt_f32", dtype="f32", n_tables=4, rows=50000, dim=32, bot=(64, 32),
                                  top=(64, 32, 1), l_min=1, l_max=30)
    return workload.FunctionSpec(key="pt_bf16", dtype="bf16", rows=[200000] * 8, dim=64, bot_dims=[128, 64],
                                 top_dims=[128, 64, 1], alpha=1.05, l_min=20, l_max=60)


def test_partition_groups_and_bounds():
    p = sage.Partition(device=0, groups=4)
    try:
        assert p.groups == 4
        sms = [p.stream(g)[1] for g in range(4)]
        assert all(s >= 8 and s % 8 == 0 for s in sms) and sum(sms) <= 148
        with pytest.raises(sage.SageError):
            p.stream(4)
    finally:
        p.destroy()
    with pytest.raises(sage.SageError) as e:
        sage.Partition(device=0, groups=2, min_sms=100)        # 2 x 100 > 148
    assert e.value.status == -1


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_confined_chain_is_bitwise_equal(dtype):
    """The same fused batch on the whole GPU (CUDA graph, branch stream) and on a
    16-SM partition (direct launches on one stream)."""
    import torch
    spec = _spec(dtype)
    pool = sage.Pool(device=0, graphs=True)
    part = sage.Partition(device=0, groups=1, min_sms=16)
    f = prepare(pool, spec)
    try:
        invs = [workload.make_invocation(spec, B, seed=40 + i) for i, B in enumerate([1, 77, 400, 0, 129])]
        a = [DevInvocation(v) for v in invs]
        b = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in a])
        s, n = part.stream(0)
        f.invoke_batch([d.args() for d in b], stream=s)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x.out[:x.batch], y.out[:y.batch])
        w = workload.weights_arrays(spec)
        ref = oracle.forward(spec, w, invs[2], row_source=lambda t, r: workload.table_rows(spec, t, r),
                             want_pooled=False)
        got = b[2].out[:400].double().cpu().numpy()
        assert oracle.check_output(got, ref["out"], ref["out_mag"], RTOL[dtype])["ok"]
    finally:
        f.release()
        pool.destroy()
        part.destroy()


def test_partition_confines_the_work():
    """A gather-bound batch on 16 SMs takes several times longer than on all SMs."""
    import torch
    spec = _spec("bf16")
    pool = sage.Pool(device=0)
    part = sage.Partition(device=0, groups=1, min_sms=16)
    f = prepare(pool, spec, max_batch=16384)
    try:
        invs = [DevInvocation(workload.make_invocation(spec, 2048, seed=60 + i)) for i in range(4)]
        args = [d.args() for d in invs]
        s16, n16 = part.stream(0)
        full = torch.cuda.Stream()

        def timed(stream):
            f.invoke_batch(args, stream=stream)
            torch.cuda.synchronize()
            t = []
            for _ in range(5):
                t0 = time.perf_counter()
                f.invoke_batch(args, stream=stream)
                torch.cuda.synchronize()
                t.append(time.perf_counter() - t0)
            return sorted(t)[2]

        t_full = timed(full.cuda_stream)
        t_part = timed(s16)
        assert n16 == 16
        assert t_part > 3.0 * t_full, (t_part, t_full)
    finally:
        f.release()
        pool.destroy()
        part.destroy()


def test_serve_with_sm_partitions_matches_isolated():
    import torch
    from test_gpu_serve import Trace, _functions
    specs = _functions()
    tr = Trace(specs, 60, rate=400.0, seed=15)
    pool = sage.Pool(device=0)
    try:
        res, st = sage.serve(pool, [workload.prepare_kwargs(s) for s in specs], tr.requests(), sm_partition=True)
        assert st["completed"] == 60 and all(r["status"] == 0 for r in res)
        fns = [prepare(pool, s) for s in specs]
        for k, (fi, v, o) in enumerate(zip(tr.fns, tr.invs, tr.outs)):
            d = DevInvocation(v)
            fns[fi].invoke(*d.args())
            torch.cuda.synchronize()
            assert np.array_equal(d.out[:v["batch"]].cpu().numpy(), o), k
        for f in fns:
            f.release()
    finally:
        pool.destroy()
