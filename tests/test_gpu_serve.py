"""The serving loop (sage_serve): continuous batching over several functions,
memory admission with eviction, linger release, cold vs warm accounting, and
each result equal alone and in the mix."""
import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, prepare

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


def _functions():
    a = workload.spec_tiny(key="sv_f32", dtype="f32", n_tables=3, rows=4000, dim=32, bot=(64, 32),
                           top=(64, 32, 1), l_min=1, l_max=20)
    b = workload.FunctionSpec(key="sv_bf16", dtype="bf16", rows=[5000, 3000, 8000, 2000], dim=64,
                              bot_dims=[128, 64], top_dims=[256, 64, 1], alpha=1.1, l_min=1, l_max=30)
    c = workload.FunctionSpec(key="sv_bf16b", dtype="bf16", rows=[20000] * 2, dim=128,
                              bot_dims=[128, 128], top_dims=[128, 64, 1], alpha=1.1, l_min=0, l_max=50)
    return [a, b, c]


class Trace:
    """Requests with host buffers (numpy; they outlive the replay)."""

    def __init__(self, specs, n, rate, seed, burst_fn=None):
        rng = np.random.default_rng(seed)
        self.specs = specs
        self.arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        self.fns = rng.integers(0, len(specs), size=n)
        if burst_fn is not None:
            self.arrivals[:20] = 0.0
            self.fns[:20] = burst_fn
        self.invs = []
        self.outs = []
        for k in range(n):
            B = int(rng.integers(1, 200))
            v = workload.make_invocation(specs[self.fns[k]], B, seed=seed * 1000 + k)
            self.invs.append(v)
            self.outs.append(np.full(B, np.nan, np.float32))

    def requests(self):
        return [(int(f), float(t), v["batch"], v["dense"].ctypes.data, v["indices"].ctypes.data,
                 v["offsets"].ctypes.data, v["indices"].size, o.ctypes.data)
                for f, t, v, o in zip(self.fns, self.arrivals, self.invs, self.outs)]


def test_serve_each_result_equals_its_isolated_invocation():
    """Served requests (fused host-buffer batches) equal, bit for bit, the same
    invocations run alone."""
    specs = _functions()
    tr = Trace(specs, 90, rate=400.0, seed=5, burst_fn=1)
    pool = sage.Pool(device=0)
    try:
        fkw = [workload.prepare_kwargs(s) for s in specs]
        res, st = sage.serve(pool, fkw, tr.requests(), lanes_per_fn=2)
        assert st["completed"] == 90 and all(r["status"] == 0 for r in res)
        assert st["batches"] < 90                      # requests were fused
        assert max(r["batch_invocations"] for r in res) > 1
        assert st["prepares"] == 3 and pool.stats()["functions"] == 0
        assert all(r["latency_ms"] >= r["queue_ms"] >= 0 for r in res)
        # isolated invocations of the same requests
        import torch
        fns = [prepare(pool, s) for s in specs]
        for k, (f, v, o) in enumerate(zip(tr.fns, tr.invs, tr.outs)):
            d = DevInvocation(v)
            fns[f].invoke(*d.args())
            torch.cuda.synchronize()
            alone = d.out[:v["batch"]].cpu().numpy()
            assert np.array_equal(alone, o), k          # bitwise: same per-row order alone and in the mix
        # and against the oracle for a few
        for k in range(0, 90, 15):
            s = specs[tr.fns[k]]
            ref = oracle.forward(s, workload.weights_arrays(s), tr.invs[k],
                                 row_source=lambda t, r, s=s: workload.table_rows(s, t, r), want_pooled=False)
            assert oracle.check_output(tr.outs[k], ref["out"], ref["out_mag"], RTOL[s.dtype])["ok"]
        for f in fns:
            f.release()
    finally:
        pool.destroy()


def test_serve_cold_then_warm_accounting():
    specs = _functions()[:2]
    tr = Trace(specs, 40, rate=100.0, seed=7)
    pool = sage.Pool(device=0)
    try:
        res, st = sage.serve(pool, [workload.prepare_kwargs(s) for s in specs], tr.requests())
        assert st["completed"] == 40
        assert 1 <= st["cold_requests"] < 40
        first = {f: min(k for k in range(40) if tr.fns[k] == f) for f in set(tr.fns.tolist())}
        for f, k in first.items():
            assert res[k]["cold"] == 1
        assert st["warm_p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    finally:
        pool.destroy()


def test_serve_admits_by_memory_and_evicts_idle_functions():
    specs = _functions()
    big = [workload.FunctionSpec(key="sv_big%d" % i, dtype="bf16", rows=[400_000] * 4, dim=128,
                                 bot_dims=[128, 128], top_dims=[128, 64, 1], alpha=1.1, l_min=1, l_max=10)
           for i in range(2)]
    one = big[0].table_bytes()
    # budget: one big function (plus workspaces) fits, two do not
    pool = sage.Pool(device=0, budget_bytes=int(one * 1.6))
    try:
        tr = Trace(big, 30, rate=1000.0, seed=9)
        tr.fns[:] = 0
        tr.fns[15:] = 1
        tr.arrivals[15:] += 0.3
        res, st = sage.serve(pool, [workload.prepare_kwargs(s) for s in big], tr.requests(), max_batch_rows=4096)
        assert st["completed"] == 30
        assert st["evictions"] >= 1 and st["prepares"] == 2
        for k in range(30):
            s = big[tr.fns[k]]
            if k % 7 == 0:
                ref = oracle.forward(s, workload.weights_arrays(s), tr.invs[k],
                                     row_source=lambda t, r, s=s: workload.table_rows(s, t, r), want_pooled=False)
                assert oracle.check_output(tr.outs[k], ref["out"], ref["out_mag"], RTOL["bf16"])["ok"]
    finally:
        pool.destroy()


def test_serve_linger_releases_idle_functions():
    specs = _functions()[:1]
    tr = Trace(specs, 10, rate=50.0, seed=11)
    tr.arrivals[5:] += 0.5                 # a gap longer than the linger
    pool = sage.Pool(device=0)
    try:
        res, st = sage.serve(pool, [workload.prepare_kwargs(s) for s in specs], tr.requests(), linger_s=0.1)
        assert st["completed"] == 10
        assert st["prepares"] == 2 and st["evictions"] >= 1
        assert res[5]["cold"] == 1
    finally:
        pool.destroy()
