"""The runtime through the C-ABI on a GPU: whole function vs the oracle, fused
batches vs isolated invocations, read-only sharing and refcounts, staging
failures, budget, readiness gate, host-buffer invocations, concurrency."""
import ctypes
import threading
import time

import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, oracle_rows, prepare, to_f64

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


def _torch():
    import torch
    return torch


def spec_small(dtype, key=None):
    if dtype == "f32":
        return workload.spec_tiny(key=key or "rt_f32", dtype="f32", n_tables=4, rows=2000, dim=32,
                                  bot=(64, 32), top=(64, 32, 1), l_min=0, l_max=30)
    return workload.FunctionSpec(key=key or "rt_bf16", dtype="bf16", rows=[3000, 2000, 5000], dim=64,
                                 bot_dims=[128, 64], top_dims=[128, 64, 1], alpha=1.1, l_min=0, l_max=40)


@pytest.fixture(scope="module")
def pool():
    p = sage.Pool(device=0, staging_chunk_bytes=1 << 20, staging_chunks=3)
    yield p
    p.destroy()


def _check_inv(spec, weights, dinv, rtol):
    _torch().cuda.synchronize()
    got = to_f64(dinv.out)[:dinv.batch]
    tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
    res = oracle.forward(spec, weights, dinv.inv, tables=tables, want_pooled=False)
    c = oracle.check_output(got, res["out"], res["out_mag"], rtol)
    assert c["ok"], c
    return c


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_invoke_matches_oracle(pool, dtype):
    spec = spec_small(dtype)
    fn = prepare(pool, spec)
    try:
        w = workload.weights_arrays(spec)
        for B, seed in [(1, 1), (37, 2), (300, 3)]:
            d = DevInvocation(workload.make_invocation(spec, B, seed=seed))
            fn.invoke(*d.args())
            _check_inv(spec, w, d, RTOL[dtype])
        fn.check_errors()
    finally:
        fn.release()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_fused_batch_equals_isolated_bitwise(pool, dtype):
    torch = _torch()
    spec = spec_small(dtype, key="rt_fuse_" + dtype)
    fn = prepare(pool, spec)
    try:
        sizes = [5, 1, 130, 0, 77, 260]
        invs = [workload.make_invocation(spec, B, seed=100 + i) for i, B in enumerate(sizes)]
        fused = [DevInvocation(v) for v in invs]
        alone = [DevInvocation(v) for v in invs]
        fn.invoke_batch([d.args() for d in fused])
        for d in alone:
            fn.invoke(*d.args())
        torch.cuda.synchronize()
        w = workload.weights_arrays(spec)
        for a, b in zip(fused, alone):
            assert torch.equal(a.out[:a.batch], b.out[:b.batch])
            if a.batch:
                _check_inv(spec, w, a, RTOL[dtype])
    finally:
        fn.release()


def test_host_buffer_invocation_equals_device_invocation(pool):
    torch = _torch()
    spec = spec_small("bf16", key="rt_host")
    fn = prepare(pool, spec)
    try:
        invs = [workload.make_invocation(spec, B, seed=200 + i) for i, B in enumerate([3, 64, 17])]
        hosts = []
        outs = []
        for v in invs:
            o = np.full(v["batch"], np.nan, np.float32)
            outs.append(o)
            hosts.append((v["batch"], v["dense"].ctypes.data, v["indices"].ctypes.data, v["offsets"].ctypes.data,
                          v["indices"].size, o.ctypes.data))
        fn.invoke_batch_host(hosts)
        devs = [DevInvocation(v) for v in invs]
        fn.invoke_batch([d.args() for d in devs])
        torch.cuda.synchronize()
        for o, d in zip(outs, devs):
            assert np.array_equal(o, d.out[:d.batch].cpu().numpy())
    finally:
        fn.release()


def test_readonly_sharing_loads_once_and_refcounts_free(pool):
    spec = spec_small("f32", key="rt_share")
    s0 = pool.stats()
    f1 = prepare(pool, spec)
    f2 = prepare(pool, spec)
    f3 = prepare(pool, spec)
    f1.wait()
    s1 = pool.stats()
    wbytes = workload.weights_blob(spec).nbytes
    assert s1["h2d_bytes"] - s0["h2d_bytes"] == spec.table_bytes() + wbytes
    assert s1["hits"] - s0["hits"] == 2 and s1["misses"] - s0["misses"] == 1
    assert s1["functions"] == s0["functions"] + 1 and s1["refs"] == s0["refs"] + 3
    # all three handles see the same results
    d = [DevInvocation(workload.make_invocation(spec, 50, seed=9)) for _ in range(3)]
    for f, x in zip((f1, f2, f3), d):
        f.invoke(*x.args())
    _torch().cuda.synchronize()
    assert _torch().equal(d[0].out, d[1].out) and _torch().equal(d[0].out, d[2].out)
    f1.release()
    f2.release()
    assert pool.stats()["functions"] == s0["functions"] + 1
    f3.release()
    s2 = pool.stats()
    assert s2["functions"] == s0["functions"] and s2["resident_bytes"] == s0["resident_bytes"]
    assert s2["refs"] == s0["refs"]
    with pytest.raises(sage.SageError):
        f3.handle = ctypes.c_void_p(0)
        f3.release()


def test_reprepare_with_other_shape_is_invalid(pool):
    spec = spec_small("f32", key="rt_shape")
    f = prepare(pool, spec)
    other = spec_small("f32", key="rt_shape")
    other.rows = [r + 1 for r in other.rows]
    with pytest.raises(sage.SageError) as e:
        prepare(pool, other)
    assert e.value.status == -1
    f.release()


def test_budget_exhaustion_is_nomem():
    p = sage.Pool(device=0, budget_bytes=4 << 20)
    try:
        spec = spec_small("f32", key="rt_nomem")
        spec.rows = [200_000] * 4
        with pytest.raises(sage.SageError) as e:
            prepare(p, spec)
        assert e.value.status == -2
        assert p.stats()["functions"] == 0
    finally:
        p.destroy()


def test_staging_failure_is_sticky_and_releases_cleanly(pool):
    spec = spec_small("f32", key="rt_fail")
    f = prepare(pool, spec, fail_at_call=3)
    with pytest.raises(sage.SageError) as e:
        f.wait()
    assert e.value.status == -6
    d = DevInvocation(workload.make_invocation(spec, 4, seed=1))
    with pytest.raises(sage.SageError) as e:
        f.invoke(*d.args())
    assert e.value.status == -6
    n0 = pool.stats()["functions"]
    f.release()
    assert pool.stats()["functions"] == n0 - 1


def test_pool_destroy_is_busy_with_live_references():
    p = sage.Pool(device=0)
    spec = spec_small("f32", key="rt_busy")
    f = prepare(p, spec)
    with pytest.raises(sage.SageError) as e:
        p.destroy()
    assert e.value.status == -5
    f.release()
    p.destroy()


def test_invoke_waits_for_slow_staging(pool):
    """The pointer is handed out before the data is ready; the launch waits for it."""
    spec = spec_small("bf16", key="rt_slow")
    ctx, keep = workload.tables_ctx(spec)
    real = workload.lib().wl_fill_tables

    @workload.FILL_FN
    def slow_fill(dst, off, n, c):
        time.sleep(0.05)
        return real(dst, off, n, ctypes.addressof(ctx))

    args = workload.prepare_kwargs(spec)
    args["tables_fill"] = ctypes.cast(slow_fill, ctypes.c_void_p).value
    args["tables_ctx"] = None
    args["keep"] = (args["keep"], slow_fill, ctx, keep)
    t0 = time.time()
    f = pool.prepare(**args)
    assert time.time() - t0 < 0.5            # prepare does not wait for the data
    assert f.query() == sage.SAGE_PENDING
    d = DevInvocation(workload.make_invocation(spec, 40, seed=3))
    f.invoke(*d.args())
    _check_inv(spec, workload.weights_arrays(spec), d, RTOL["bf16"])
    assert f.query() == sage.SAGE_OK
    f.release()


def test_out_of_range_index_reported_by_check(pool):
    spec = spec_small("f32", key="rt_oob")
    f = prepare(pool, spec)
    inv = workload.make_invocation(spec, 8, seed=4)
    inv["indices"] = inv["indices"].copy()
    inv["indices"][0] = spec.rows[0] + 5
    d = DevInvocation(inv)
    f.invoke(*d.args())
    with pytest.raises(sage.SageError) as e:
        f.check_errors()
    assert e.value.status == -7
    f.check_errors()   # cleared
    f.release()


def test_concurrent_invocations_on_two_streams_and_threads(pool):
    torch = _torch()
    spec = spec_small("bf16", key="rt_conc")
    f = prepare(pool, spec, workspace_slots=3)
    try:
        invs = [workload.make_invocation(spec, 64 + 10 * i, seed=300 + i) for i in range(8)]
        ref = [DevInvocation(v) for v in invs]
        for d in ref:
            f.invoke(*d.args())
        torch.cuda.synchronize()
        got = [DevInvocation(v) for v in invs]
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]

        def work(k):
            for j in range(k, 8, 2):
                f.invoke(*got[j].args(), stream=streams[k])

        th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        for a, b in zip(ref, got):
            assert torch.equal(a.out, b.out)
    finally:
        f.release()


def test_workspace_grows_for_large_batches(pool):
    spec = spec_small("f32", key="rt_grow")
    f = prepare(pool, spec, max_batch=16)
    try:
        d = DevInvocation(workload.make_invocation(spec, 700, seed=5))
        f.invoke(*d.args())
        _check_inv(spec, workload.weights_arrays(spec), d, RTOL["f32"])
    finally:
        f.release()


@pytest.mark.parametrize("serial", [False, True])
def test_serial_and_parallel_setup_agree(serial):
    torch = _torch()
    p = sage.Pool(device=0, serial_setup=serial, torch_allocator=True)
    try:
        spec = spec_small("bf16", key="rt_setup")
        f = prepare(p, spec, tables_in_host_memory=True)
        d = DevInvocation(workload.make_invocation(spec, 33, seed=6))
        f.invoke(*d.args())
        _check_inv(spec, workload.weights_arrays(spec), d, RTOL["bf16"])
        st = p.stats()
        assert st["last_prepare_ms"] > 0 and st["ctx_ms"] > 0
        f.release()
    finally:
        p.destroy()


def test_autotune_keeps_results_bitwise_and_tuning_file_roundtrips(pool, tmp_path):
    torch = _torch()
    for dtype in ("f32", "bf16"):
        spec = spec_small(dtype, key="rt_tune_" + dtype)
        f = prepare(pool, spec)
        try:
            invs = [workload.make_invocation(spec, B, seed=400 + i) for i, B in enumerate([700, 900])]
            before = [DevInvocation(v) for v in invs]
            f.invoke_batch([d.args() for d in before])
            f.autotune(1600)
            after = [DevInvocation(v) for v in invs]
            f.invoke_batch([d.args() for d in after])
            torch.cuda.synchronize()
            for a, b in zip(before, after):
                assert torch.equal(a.out, b.out)
        finally:
            f.release()
    path = str(tmp_path / "tuning.txt")
    sage.tuning_save(path)
    lines = [l for l in open(path) if not l.startswith("#")]
    assert len(lines) >= 3
    sage.tuning_load(path)


def test_async_host_batches_overlap_and_match(pool):
    """Consecutive asynchronous host batches (alternating slots) give the device-path results."""
    torch = _torch()
    spec = spec_small("f32", key="rt_hasync")
    fn = prepare(pool, spec, workspace_slots=2)
    try:
        invs = [workload.make_invocation(spec, B, seed=500 + i) for i, B in enumerate([40, 300, 7, 128])]
        devs = [DevInvocation(v) for v in invs]
        fn.invoke_batch([d.args() for d in devs])
        outs = [[np.full(v["batch"], np.nan, np.float32) for v in invs] for _ in range(5)]
        stream = torch.cuda.Stream()
        for k in range(5):
            fn.invoke_batch_host_async([(v["batch"], v["dense"].ctypes.data, v["indices"].ctypes.data,
                                         v["offsets"].ctypes.data, v["indices"].size, o.ctypes.data)
                                        for v, o in zip(invs, outs[k])], stream=stream)
        stream.synchronize()
        for k in range(5):
            for o, d in zip(outs[k], devs):
                assert np.array_equal(o, d.out[:d.batch].cpu().numpy())
    finally:
        fn.release()


def test_host_allocator_buffers_serve_host_invocations(pool):
    """sage_host_alloc memory (page-locked, huge-page backed) as invocation buffers."""
    spec = spec_small("bf16", key="rt_hostalloc")
    fn = prepare(pool, spec)
    try:
        v = workload.make_invocation(spec, 200, seed=9)
        hv = {k: sage.host_copy(v[k]) for k in ("dense", "indices", "offsets")}
        assert all(np.array_equal(hv[k], v[k]) for k in hv)
        out = sage.host_empty(200, np.float32)
        fn.invoke_batch_host([(200, hv["dense"].ctypes.data, hv["indices"].ctypes.data, hv["offsets"].ctypes.data,
                               v["indices"].size, out.ctypes.data)])
        d = DevInvocation(v)
        fn.invoke(*d.args())
        _torch().cuda.synchronize()
        assert np.array_equal(out, d.out.cpu().numpy())
    finally:
        fn.release()


def _bad_offsets(v):
    """Malformed CSR variants of an invocation's offsets.  Each one keeps every bag
    inside [0, num_indices], so even an unchecked run would read only copied indices."""
    off = v["offsets"]
    n = v["indices"].size
    assert off[0] == 0 and off[-1] == n and n > 4
    start = off.copy()
    start[0] = 1                                    # does not start at 0
    short = off.copy()
    short[-1] = n - 1                               # does not end at num_indices
    dec = off.copy()
    j = int(np.argmax(off[1:-1] > 0)) + 1           # an inner offset above 0
    dec[j] = 0 if dec[j - 1] > 0 else dec[j]        # a step down
    if np.all(np.diff(dec) >= 0):
        dec[j + 1] = dec[j] - 1 if dec[j] > 0 else dec[j + 1]
    assert np.any(np.diff(dec) < 0)
    return {"start": start, "end": short, "decreasing": dec}


def test_host_offsets_are_checked_before_any_copy(pool):
    """Host-buffer batches and served requests with offsets that do not start at 0, step
    down, or do not end at num_indices are refused on the host (SAGE_ERR_INVALID), and a
    good invocation still runs afterwards."""
    spec = spec_small("bf16", key="rt_badcsr")
    fn = prepare(pool, spec)
    try:
        v = workload.make_invocation(spec, 64, seed=11)
        out = np.full(64, np.nan, np.float32)
        launches0 = sage.kernel_launches()
        for name, off in _bad_offsets(v).items():
            with pytest.raises(sage.SageError) as e:
                fn.invoke_batch_host([(64, v["dense"].ctypes.data, v["indices"].ctypes.data, off.ctypes.data,
                                       v["indices"].size, out.ctypes.data)])
            assert e.value.status == -1, name
            assert "offsets" in str(e.value), name
            with pytest.raises(sage.SageError) as e:
                sage.serve(pool, [workload.prepare_kwargs(spec)],
                           [(0, 0.0, 64, v["dense"].ctypes.data, v["indices"].ctypes.data, off.ctypes.data,
                             v["indices"].size, out.ctypes.data)])
            assert e.value.status == -1, name
        assert sage.kernel_launches() == launches0
        assert np.isnan(out).all()
        fn.invoke_batch_host([(64, v["dense"].ctypes.data, v["indices"].ctypes.data, v["offsets"].ctypes.data,
                               v["indices"].size, out.ctypes.data)])
        d = DevInvocation(v)
        fn.invoke(*d.args())
        _torch().cuda.synchronize()
        assert np.array_equal(out, d.out.cpu().numpy())
    finally:
        fn.release()


def test_multistage_exit_restages_from_the_host_cache():
    """Stage 2 of the multi-stage exit: released read-only data waits in host memory and a
    later prepare re-stages it from there without calling the producer."""
    torch = _torch()
    p = sage.Pool(device=0, host_cache_bytes=1 << 30)
    try:
        spec = spec_small("bf16", key="rt_stage2")
        inv = workload.make_invocation(spec, 120, seed=31)
        f = prepare(p, spec)
        d1 = DevInvocation(inv)
        f.invoke(*d1.args())
        torch.cuda.synchronize()
        f.release()
        st = p.stats()
        assert st["demotions"] == 1 and st["host_cache_entries"] == 1 and st["functions"] == 0
        assert st["host_cache_bytes"] == spec.table_bytes() + workload.weights_blob(spec).nbytes
        # a producer that fails on its first call proves the data came from the host cache
        f2 = prepare(p, spec, fail_at_call=1)
        f2.wait()
        d2 = DevInvocation(inv)
        f2.invoke(*d2.args())
        torch.cuda.synchronize()
        assert torch.equal(d1.out, d2.out)
        # and both against the oracle: the re-staged data is the function's data (Sec. 6.3)
        w = workload.weights_arrays(spec)
        _check_inv(spec, w, d1, RTOL["bf16"])
        _check_inv(spec, w, d2, RTOL["bf16"])
        st = p.stats()
        assert st["host_cache_hits"] == 1 and st["host_cache_entries"] == 0
        f2.release()
        st = p.stats()
        assert st["demotions"] == 2 and st["host_cache_entries"] == 1
    finally:
        p.destroy()


def test_host_cache_respects_its_budget():
    p = sage.Pool(device=0, host_cache_bytes=1 << 20)     # smaller than the function's data
    try:
        spec = spec_small("bf16", key="rt_stage2_small")
        f = prepare(p, spec)
        f.wait()
        f.release()
        st = p.stats()
        assert st["demotions"] == 0 and st["host_cache_entries"] == 0
    finally:
        p.destroy()


@pytest.mark.parametrize("tile", [(128, 3), (64, 4), (64, 2), (128, 103), (64, 104)])
def test_fp32_presplit_tile_configurations_bitwise(pool, tile):
    """Every configuration of the fp32 pre-split GEMM (incl. the persistent, double-buffered
    ones) gives the same bits as the default, and matches the oracle."""
    torch = _torch()
    spec = workload.spec_tiny(key="rt_pre_%d_%d" % tile, dtype="f32", n_tables=4, rows=3000, dim=64,
                              bot=(128, 64), top=(256, 128, 1), l_min=0, l_max=30)
    f = prepare(pool, spec, max_batch=3000)
    try:
        invs = [workload.make_invocation(spec, B, seed=600 + i) for i, B in enumerate([900, 1100, 13])]
        ref = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in ref])
        torch.cuda.synchronize()
        M = sum(v["batch"] for v in invs)
        for (K, N) in [(128, 64), (320, 256), (256, 128)]:
            if N % tile[0] == 0:
                sage.tuning_set(3, M, N, K, tile[0], tile[1])
        got = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in got])
        torch.cuda.synchronize()
        f.check_errors()
        for a, b in zip(ref, got):
            assert torch.equal(a.out, b.out)
        _check_inv(spec, workload.weights_arrays(spec), got[0], RTOL["f32"])
    finally:
        f.release()


@pytest.mark.parametrize("tile", [(128, 103), (64, 104)])
def test_fp32_head_fused_across_tiles_bitwise(pool, tile):
    """A last hidden layer wider than one tile (256 outputs, tiles of 128 or 64): each row's
    head is finished by whichever tile completes it (group sums + arrival counters), with the
    bits of the separate head kernel."""
    torch = _torch()
    spec = workload.spec_tiny(key="rt_hx_%d" % tile[0], dtype="f32", n_tables=3, rows=3000, dim=32,
                              bot=(64, 32), top=(128, 256, 1), l_min=0, l_max=30)
    f = prepare(pool, spec, max_batch=3000)
    try:
        invs = [workload.make_invocation(spec, B, seed=720 + i) for i, B in enumerate([1000, 7, 0, 1500])]
        M = sum(v["batch"] for v in invs)
        sage.tuning_set(3, M, 256, 128, 64, 4)          # non-persistent: separate head kernel
        ref = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in ref])
        torch.cuda.synchronize()
        sage.tuning_set(3, M, 256, 128, tile[0], tile[1])
        runs = []
        for _ in range(3):                              # counters carry over launches
            got = [DevInvocation(v) for v in invs]
            f.invoke_batch([d.args() for d in got])
            runs.append(got)
        torch.cuda.synchronize()
        f.check_errors()
        for got in runs:
            for a, b in zip(ref, got):
                assert torch.equal(a.out[:a.batch], b.out[:b.batch])
        _check_inv(spec, workload.weights_arrays(spec), runs[0][3], RTOL["f32"])
    finally:
        f.release()


@pytest.mark.parametrize("tile", [(128, 106), (64, 8), (128, 3)])
def test_bf16_head_fused_or_separate_bitwise(pool, tile):
    """The sigmoid head fused into the last hidden layer's epilogue (persistent tiles)
    gives the bits of the separate head kernel (other tiles), and matches the oracle."""
    torch = _torch()
    spec = workload.FunctionSpec(key="rt_head_%d_%d" % tile, dtype="bf16", rows=[4000, 3000, 5000], dim=64,
                                 bot_dims=[128, 64], top_dims=[256, 128, 1], alpha=1.1, l_min=0, l_max=40)
    f = prepare(pool, spec, max_batch=3000)
    try:
        invs = [workload.make_invocation(spec, B, seed=700 + i) for i, B in enumerate([900, 1100, 13, 0, 1])]
        M = sum(v["batch"] for v in invs)
        sage.tuning_set(1, M, 128, 256, 64, 8)          # separate head
        ref = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in ref])
        torch.cuda.synchronize()
        sage.tuning_set(1, M, 128, 256, tile[0], tile[1])
        got = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in got])
        # the arrival counters only grow: launches of other sizes in between (rows past
        # a smaller batch keep their counts) must not disturb the next full batch
        f.invoke_batch([d.args() for d in got[2:]])
        f.invoke_batch([d.args() for d in got[:1]])
        again = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in again])
        torch.cuda.synchronize()
        f.check_errors()
        for a, b, c in zip(ref, got, again):
            assert torch.equal(a.out[:a.batch], b.out[:b.batch])
            assert torch.equal(a.out[:a.batch], c.out[:c.batch])
        _check_inv(spec, workload.weights_arrays(spec), got[1], RTOL["bf16"])
    finally:
        f.release()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_cuda_graph_replay_equals_direct_launches(dtype):
    """Batches replayed through the captured CUDA graph (updated in place between batches
    of different sizes) give the same bits as direct launches."""
    torch = _torch()
    spec = spec_small(dtype, key="rt_graph_" + dtype)
    pd, pg = sage.Pool(device=0), sage.Pool(device=0, graphs=True)
    try:
        fd, fg = prepare(pd, spec), prepare(pg, spec)
        for round_ in range(3):
            sizes = [[300, 7, 55], [1], [128, 256, 1, 900]][round_]
            invs = [workload.make_invocation(spec, B, seed=700 + 10 * round_ + i) for i, B in enumerate(sizes)]
            a = [DevInvocation(v) for v in invs]
            b = [DevInvocation(v) for v in invs]
            fd.invoke_batch([d.args() for d in a])
            fg.invoke_batch([d.args() for d in b])
            c = DevInvocation(invs[0])
            fg.invoke(*c.args())
            torch.cuda.synchronize()
            for x, y in zip(a, b):
                assert torch.equal(x.out, y.out)
            assert torch.equal(a[0].out, c.out)
        fg.check_errors()
        fd.release()
        fg.release()
    finally:
        pd.destroy()
        pg.destroy()



def test_more_than_256_invocations_and_empty_members(pool):
    """A batch above the per-launch table size (256) runs as several fused launches;
    empty invocations are skipped; every member still equals its isolated invocation."""
    torch = _torch()
    spec = spec_small("f32", key="rt_many")
    f = prepare(pool, spec, max_batch=8192)
    try:
        sizes = [(i * 7) % 23 for i in range(300)]          # zeros every 23rd member
        invs = [workload.make_invocation(spec, B, seed=800 + i) for i, B in enumerate(sizes)]
        fused = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in fused])
        f.invoke_batch([])                                   # an empty batch is a no-op
        picks = [0, 1, 23, 100, 255, 256, 257, 299]          # both sides of the 256 boundary
        alone = [DevInvocation(invs[k]) for k in picks]
        for d in alone:
            f.invoke(*d.args())
        torch.cuda.synchronize()
        for k, d in zip(picks, alone):
            assert torch.equal(fused[k].out[:sizes[k]], d.out[:sizes[k]]), k
        _check_inv(spec, workload.weights_arrays(spec), fused[257], RTOL["f32"])
    finally:
        f.release()


@pytest.mark.parametrize("case", ["bf16_hidden_96", "row_96_bytes", "head_2_outputs"])
def test_invalid_descriptors_are_rejected(pool, case):
    if case == "bf16_hidden_96":    # a bf16 layer with K = 96 does not tile by 64
        spec = workload.FunctionSpec(key="rt_bad1", dtype="bf16", rows=[100] * 2, dim=64, bot_dims=[96, 64],
                                     top_dims=[128, 1], l_min=0, l_max=3)
    elif case == "row_96_bytes":    # rows must be a power-of-two number of bytes
        spec = workload.spec_tiny(key="rt_bad2", dtype="f32", dim=24, bot=(16, 24))
    else:                           # the head is one sigmoid output
        spec = workload.spec_tiny(key="rt_bad3", dtype="f32", top=(16, 2))
    before = pool.stats()["functions"]
    with pytest.raises(sage.SageError) as e:
        prepare(pool, spec)
    assert e.value.status == -1
    assert pool.stats()["functions"] == before


def test_bounded_wait_times_out_then_completes(pool):
    spec = spec_small("bf16", key="rt_timeout")
    ctx, keep = workload.tables_ctx(spec)
    real = workload.lib().wl_fill_tables

    @workload.FILL_FN
    def slow_fill(dst, off, n, c):
        time.sleep(0.2)
        return real(dst, off, n, ctypes.addressof(ctx))

    args = workload.prepare_kwargs(spec)
    args["tables_fill"] = ctypes.cast(slow_fill, ctypes.c_void_p).value
    args["tables_ctx"] = None
    args["keep"] = (args["keep"], slow_fill, ctx, keep)
    f = pool.prepare(**args)
    try:
        with pytest.raises(sage.SageError) as e:
            f.wait(timeout_us=1000)
        assert e.value.status == -4
        f.wait()
        assert f.query() == sage.SAGE_OK
    finally:
        f.release()


@pytest.mark.parametrize("tile", [(128, 103), (64, 104)])
def test_fp32_persistent_last_wave_split_bitwise(pool, tile):
    """A persistent fp32 layer whose last wave of tiles is short runs that wave as
    half-width items; the outputs keep the bits of the non-persistent kernel."""
    torch = _torch()
    spec = workload.spec_tiny(key="rt_split_%d" % tile[0], dtype="f32", n_tables=4, rows=5000, dim=64,
                              bot=(128, 64), top=(256, 128, 1), l_min=0, l_max=20)
    f = prepare(pool, spec, max_batch=4000)
    try:
        invs = [workload.make_invocation(spec, B, seed=1200 + i) for i, B in enumerate([3500, 3500, 3500])]
        M = 10500                                       # 83 row tiles: 166 or 332 column tiles
        for (K, N) in [(320, 256), (256, 128)]:
            sage.tuning_set(3, M, N, K, 64, 4)          # non-persistent reference
        ref = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in ref])
        torch.cuda.synchronize()
        sage.tuning_set(3, M, 256, 320, tile[0], tile[1])
        got = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in got])
        torch.cuda.synchronize()
        f.check_errors()
        for a, b in zip(ref, got):
            assert torch.equal(a.out, b.out)
        rows = np.arange(0, 3500, 251)
        ref_o, mag = oracle_rows(spec, workload.weights_arrays(spec), invs[2], rows)
        c = oracle.check_output(to_f64(got[2].out)[rows], ref_o, mag, RTOL["f32"])
        assert c["ok"], c
    finally:
        f.release()


@pytest.mark.parametrize("tile", [(256, 104), (128, 106)])
def test_bf16_persistent_last_wave_split_bitwise(pool, tile):
    """The persistent bf16 layer runs a short last wave as half-width items too; the
    outputs keep the bits of the non-persistent kernel."""
    torch = _torch()
    spec = workload.spec_tiny(key="rt_split16_%d" % tile[0], dtype="bf16", n_tables=4, rows=5000, dim=64,
                              bot=(128, 64), top=(256, 128, 1), l_min=0, l_max=20)
    f = prepare(pool, spec, max_batch=7000)
    try:
        invs = [workload.make_invocation(spec, 7000, seed=1300 + i) for i in range(3)]
        M = 21000                                       # 165 row tiles: 165 or 330 column tiles
        for (K, N) in [(320, 256), (256, 128)]:
            sage.tuning_set(1, M, N, K, 128, 6)         # non-persistent reference
        ref = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in ref])
        torch.cuda.synchronize()
        sage.tuning_set(1, M, 256, 320, tile[0], tile[1])
        got = [DevInvocation(v) for v in invs]
        f.invoke_batch([d.args() for d in got])
        torch.cuda.synchronize()
        f.check_errors()
        for a, b in zip(ref, got):
            assert torch.equal(a.out, b.out)
        rows = np.arange(0, 7000, 499)
        ref_o, mag = oracle_rows(spec, workload.weights_arrays(spec), invs[1], rows)
        c = oracle.check_output(to_f64(got[1].out)[rows], ref_o, mag, RTOL["bf16"])
        assert c["ok"], c
    finally:
        f.release()


@pytest.mark.parametrize("dtype,dim", [("f32", 32), ("bf16", 64), ("f32", 64), ("bf16", 128)])
def test_claimed_gather_work_resets_between_batches(pool, dtype, dim):
    """The runtime's gather claims its work from per-slot counters that the launch's
    last block resets: back-to-back fused batches of very different sizes on one
    handle (a batch with fewer bags than resident warps, a long one, the short one
    again) each equal the same invocations run alone."""
    torch = _torch()
    # 128-byte rows (one bag per warp, single bags or runs) and 256-byte rows (fp32:
    # lane groups, four bags per claim; bf16: runs of up to 8 bags)
    spec = workload.spec_tiny(key="rt_claims_%s_%d" % (dtype, dim), dtype=dtype, n_tables=4, rows=3000, dim=dim,
                              bot=(128, 64), top=(128, 64, 1), l_min=0, l_max=60)
    fn = prepare(pool, spec, max_batch=4000)
    try:
        plans = [[3, 1], [1500, 700, 0, 999], [3, 1], [2, 2, 2], [1500, 700, 0, 999]]
        for k, sizes in enumerate(plans):
            invs = [workload.make_invocation(spec, B, seed=1400 + 10 * k + i) for i, B in enumerate(sizes)]
            fused = [DevInvocation(v) for v in invs]
            alone = [DevInvocation(v) for v in invs]
            fn.invoke_batch([d.args() for d in fused])
            for d in alone:
                fn.invoke(*d.args())
            torch.cuda.synchronize()
            for a, b in zip(fused, alone):
                assert torch.equal(a.out[:a.batch], b.out[:b.batch]), (k, a.batch)
                assert not torch.isnan(a.out[:a.batch]).any()
        fn.check_errors()
        w = workload.weights_arrays(spec)
        _check_inv(spec, w, fused[0], RTOL[dtype])
    finally:
        fn.release()
