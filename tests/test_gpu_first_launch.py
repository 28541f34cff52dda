"""First launches from several host threads at once, in a fresh process: every
kernel launcher sets its function attributes and reads its occupancy once per
device, guarded for concurrent first use.  Four threads start fused batches of two
functions (fp32 on the tensor cores, bf16) at the same moment, each on its own
stream; their outputs must equal, bit for bit, the same batches run one after the
other afterwards, and no kernel may report an error."""
import pytest

import workload
from helpers import DevInvocation, prepare

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


def _specs():
    f32 = workload.spec_tiny(key="fl_f32", dtype="f32", n_tables=4, rows=5000, dim=64, bot=(128, 64),
                             top=(128, 64, 1), l_min=1, l_max=30)
    bf16 = workload.FunctionSpec(key="fl_bf16", dtype="bf16", rows=[6000, 4000, 8000], dim=64,
                                 bot_dims=[128, 64], top_dims=[128, 64, 1], alpha=1.1, l_min=0, l_max=40)
    return [f32, bf16]


def _child(q):
    import threading

    import torch
    try:
        torch.cuda.set_device(0)
        pool = sage.Pool(device=0, graphs=False)
        specs = _specs()
        fns = [prepare(pool, s, workspace_slots=3) for s in specs]
        for f in fns:
            f.wait()
        # thread k: function k % 2, a fused batch of three invocations
        jobs = []
        for k in range(4):
            s = specs[k % 2]
            invs = [workload.make_invocation(s, 40 + 70 * j + 9 * k, seed=900 + 10 * k + j) for j in range(3)]
            jobs.append((fns[k % 2], invs))
        got = [[DevInvocation(v) for v in invs] for _, invs in jobs]
        streams = [torch.cuda.Stream() for _ in range(4)]
        start = threading.Barrier(4)
        errors = []

        def work(k):
            try:
                start.wait()
                jobs[k][0].invoke_batch([d.args() for d in got[k]], stream=streams[k].cuda_stream)
            except Exception as e:       # reported to the parent below
                errors.append(repr(e))

        th = [threading.Thread(target=work, args=(k,)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        for f in fns:
            f.check_errors()
        # the same batches again, one after the other
        ref = [[DevInvocation(v) for v in invs] for _, invs in jobs]
        for k in range(4):
            jobs[k][0].invoke_batch([d.args() for d in ref[k]])
        torch.cuda.synchronize()
        for f in fns:
            f.check_errors()
        same = all(torch.equal(a.out, b.out) for k in range(4) for a, b in zip(got[k], ref[k]))
        finite = all(bool(torch.isfinite(a.out[:a.batch]).all()) for k in range(4) for a in got[k])
        for f in fns:
            f.release()
        pool.destroy()
        q.put((errors, same, finite))
    except Exception as e:
        q.put(([repr(e)], False, False))


def test_first_launches_from_four_threads_in_a_fresh_process():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_child, args=(q,))
    p.start()
    errors, same, finite = q.get(timeout=300)
    p.join(timeout=60)
    assert p.exitcode == 0
    assert errors == []
    assert finite and same
