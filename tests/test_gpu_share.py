"""Cross-process sharing on one GPU: an owner process stages a function's read-only
copy once and other processes map it (Sec. 4.1 / 5.1 daemon process, Sec. 6.2 sharing).

Processes are started with `spawn`; none of their kernels waits on another's."""
import os
import tempfile
import time

import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, prepare, to_f64

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


def _specs():
    return {
        "sh_f32": workload.spec_tiny(key="sh_f32", dtype="f32", n_tables=4, rows=20000, dim=32, bot=(64, 32),
                                     top=(64, 32, 1), l_min=1, l_max=30),
        "sh_bf16": workload.FunctionSpec(key="sh_bf16", dtype="bf16", rows=[30000, 20000, 50000], dim=64,
                                         bot_dims=[128, 64], top_dims=[128, 64, 1], alpha=1.1, l_min=0, l_max=40),
        # every hidden layer tiles by 64: the fp32 tensor-core path, whose split weight planes
        # the attaching process computes itself once the owner reports the data complete
        "sh_f32p": workload.spec_tiny(key="sh_f32p", dtype="f32", n_tables=4, rows=20000, dim=64, bot=(128, 64),
                                      top=(128, 64, 1), l_min=1, l_max=30),
    }


def _sizes():
    return [(1, 11), (37, 12), (300, 13)]


def _owner(path, keys, fail_at_call, q_cmd, q_out):
    pool = sage.Pool(device=0, exportable=True)
    share = sage.Share(pool, path)
    specs = _specs()
    for k in keys:
        share.register(**workload.prepare_kwargs(specs[k], fail_at_call=fail_at_call))
    q_out.put("listening")
    while True:
        cmd = q_cmd.get(timeout=300)
        if cmd == "stats":
            q_out.put((share.stats(), pool.stats()))
        elif cmd == "stop":
            share.stop()
            st = pool.stats()
            pool.destroy()
            q_out.put(st)
            return


def _client(path, key, q_out):
    t0 = time.perf_counter()
    spec = _specs()[key]
    ticket = sage.attach_begin(path, **workload.prepare_kwargs(spec))   # before any CUDA call
    pool = sage.Pool(device=0)
    f = pool.attach(ticket)
    first = f.query()
    import torch
    outs = []
    for B, seed in _sizes():
        d = DevInvocation(workload.make_invocation(spec, B, seed=seed))
        f.invoke(*d.args())
        torch.cuda.synchronize()
        outs.append(d.out[:B].cpu().numpy().copy())
    f.check_errors()
    st = pool.stats()
    f.release()
    pool.destroy()
    q_out.put((key, outs, first, st["h2d_bytes"], time.perf_counter() - t0))


def _client_expect_error(path, key, shape_override, q_out):
    spec = _specs()[key]
    kw = workload.prepare_kwargs(spec)
    kw.update(shape_override)
    try:
        ticket = sage.attach_begin(path, **kw)
        pool = sage.Pool(device=0)
        try:
            f = pool.attach(ticket)
        except sage.SageError as e:
            q_out.put(("attach", e.status))
            return
        import torch
        B = 8
        d = DevInvocation(workload.make_invocation(spec, B, seed=5))
        try:
            f.invoke(*d.args())
            torch.cuda.synchronize()
            q_out.put(("invoke", 0))
        except sage.SageError as e:
            q_out.put(("invoke", e.status))
        f.release()
        pool.destroy()
    except sage.SageError as e:
        q_out.put(("begin", e.status))


def _start_owner(ctx, keys, fail_at_call=0):
    path = os.path.join(tempfile.mkdtemp(prefix="sage_share_"), "owner.sock")
    q_cmd, q_out = ctx.Queue(), ctx.Queue()
    p = ctx.Process(target=_owner, args=(path, keys, fail_at_call, q_cmd, q_out))
    p.start()
    assert q_out.get(timeout=180) == "listening"
    return path, p, q_cmd, q_out


def _stop_owner(p, q_cmd, q_out):
    q_cmd.put("stop")
    st = q_out.get(timeout=120)
    p.join(timeout=60)
    assert p.exitcode == 0
    return st


def _local_outputs(spec):
    import torch
    pool = sage.Pool(device=0)
    f = prepare(pool, spec)
    outs = []
    for B, seed in _sizes():
        d = DevInvocation(workload.make_invocation(spec, B, seed=seed))
        f.invoke(*d.args())
        torch.cuda.synchronize()
        outs.append(d.out[:B].cpu().numpy().copy())
    f.release()
    pool.destroy()
    return outs


@pytest.mark.parametrize("key", ["sh_f32", "sh_bf16", "sh_f32p"])
def test_two_processes_map_one_staged_copy(key):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    path, owner, q_cmd, q_out = _start_owner(ctx, [key])
    q_res = ctx.Queue()
    clients = [ctx.Process(target=_client, args=(path, key, q_res)) for _ in range(2)]
    for c in clients:
        c.start()
    res = [q_res.get(timeout=300) for _ in clients]
    for c in clients:
        c.join(timeout=60)
        assert c.exitcode == 0
    q_cmd.put("stats")
    share_st, pool_st = q_out.get(timeout=60)
    owner_final = _stop_owner(owner, q_cmd, q_out)

    spec = _specs()[key]
    ro = spec.table_bytes() + workload.prepare_kwargs(spec)["weights_bytes"]
    # the owner staged the key once; the second attach shared it
    assert pool_st["misses"] == 1 and pool_st["hits"] == 1
    assert pool_st["h2d_bytes"] == ro
    assert share_st["grants"] == 2 and share_st["ready"] == 2 and share_st["rejects"] == 0
    assert share_st["releases"] == 2 and share_st["active"] == 0
    assert owner_final["functions"] == 0                      # every reference came back
    # the clients copied no read-only bytes themselves
    assert all(r[3] == 0 for r in res)
    # identical results in both processes and in a process that staged locally
    local = _local_outputs(spec)
    for r in res:
        for a, b in zip(r[1], local):
            assert np.array_equal(a, b)
    # and against the oracle
    w = workload.weights_arrays(spec)
    tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
    for (B, seed), got in zip(_sizes(), res[0][1]):
        ref = oracle.forward(spec, w, workload.make_invocation(spec, B, seed=seed), tables=tables, want_pooled=False)
        c = oracle.check_output(got.astype(np.float64), ref["out"], ref["out_mag"], RTOL[spec.dtype])
        assert c["ok"], c


def test_attach_refusals():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    path, owner, q_cmd, q_out = _start_owner(ctx, ["sh_f32"])
    q_res = ctx.Queue()
    cases = [("sh_bf16", {}),                                              # not registered
             ("sh_f32", {"rows": [20000, 20000, 20000, 19999],             # other shape, same key
                         "tables_bytes": (80000 - 1) * 32 * 4})]
    for key, over in cases:
        c = ctx.Process(target=_client_expect_error, args=(path, key, over, q_res))
        c.start()
        where, status = q_res.get(timeout=300)
        c.join(timeout=60)
        assert (where, status) == ("attach", -1)
    q_cmd.put("stats")
    share_st, pool_st = q_out.get(timeout=60)
    assert share_st["rejects"] == 2 and share_st["grants"] == 0 and pool_st["misses"] == 0
    _stop_owner(owner, q_cmd, q_out)


def test_owner_staging_failure_reaches_the_attached_process():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    path, owner, q_cmd, q_out = _start_owner(ctx, ["sh_bf16"], fail_at_call=2)
    q_res = ctx.Queue()
    c = ctx.Process(target=_client_expect_error, args=(path, "sh_bf16", {}, q_res))
    c.start()
    where, status = q_res.get(timeout=300)
    c.join(timeout=60)
    assert (where, status) == ("invoke", -6)                  # SAGE_ERR_STAGING, sticky
    st = _stop_owner(owner, q_cmd, q_out)
    assert st["functions"] == 0


def test_share_needs_an_exportable_pool():
    pool = sage.Pool(device=0)
    try:
        with pytest.raises(sage.SageError) as e:
            sage.Share(pool, os.path.join(tempfile.mkdtemp(), "x.sock"))
        assert e.value.status == -1
    finally:
        pool.destroy()


def test_attach_within_one_process_and_local_sharing():
    """Owner and function pool in one process: the attached handle reads the owner's
    memory; a second attach of the key in the same pool is shared locally."""
    import torch
    spec = _specs()["sh_f32"]
    owner = sage.Pool(device=0, exportable=True)
    path = os.path.join(tempfile.mkdtemp(), "owner.sock")
    share = sage.Share(owner, path)
    share.register(**workload.prepare_kwargs(spec))
    user = sage.Pool(device=0)
    try:
        f1 = user.attach(sage.attach_begin(path, **workload.prepare_kwargs(spec)))
        f2 = user.attach(sage.attach_begin(path, **workload.prepare_kwargs(spec)))
        f1.wait()
        st = user.stats()
        assert st["functions"] == 1 and st["hits"] == 1 and st["h2d_bytes"] == 0
        B = 50
        d1 = DevInvocation(workload.make_invocation(spec, B, seed=21))
        d2 = DevInvocation(workload.make_invocation(spec, B, seed=21))
        f1.invoke(*d1.args())
        f2.invoke(*d2.args())
        torch.cuda.synchronize()
        assert torch.equal(d1.out[:B], d2.out[:B])
        got = to_f64(d1.out)[:B]
        ref = oracle.forward(spec, workload.weights_arrays(spec), d1.inv,
                             tables=[workload.full_table(spec, t) for t in range(spec.n_tables)], want_pooled=False)
        assert oracle.check_output(got, ref["out"], ref["out_mag"], RTOL["f32"])["ok"]
        f1.release()
        f2.release()
        assert user.stats()["functions"] == 0
        time.sleep(0.2)
        assert share.stats()["active"] == 0          # the owner got its references back
    finally:
        user.destroy()
        share.stop()
        owner.destroy()
