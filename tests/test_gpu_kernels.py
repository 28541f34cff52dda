"""Parity of the sm_103a kernels (called one by one through the C-ABI) with the oracle."""
import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, bf16_dev, dev, tables_dev, to_f64

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")


def _torch():
    import torch
    return torch


def _run_gather(spec, inv, ldo=None, err=None):
    torch = _torch()
    T, D, B = spec.n_tables, spec.dim, inv["batch"]
    ldo = ldo or T * D
    tdt = torch.float32 if spec.dtype == "f32" else torch.bfloat16
    tabs = tables_dev(spec)
    out = torch.full((max(B, 1), ldo), 7.0, dtype=tdt, device="cuda")
    idx = dev(inv["indices"] if inv["indices"].size else np.zeros(1, np.int32))
    off = dev(inv["offsets"])
    sage.embedding_bag_sum(spec.dtype_code, tabs.data_ptr(), spec.rows, D, B, idx.data_ptr(), off.data_ptr(),
                           out.data_ptr(), ldo, err.data_ptr() if err is not None else None)
    torch.cuda.synchronize()
    return out


GATHER_CASES = [("f32", 4), ("f32", 8), ("f32", 16), ("f32", 32), ("f32", 64), ("f32", 128), ("f32", 256),
                ("bf16", 8), ("bf16", 16), ("bf16", 32), ("bf16", 64), ("bf16", 128), ("bf16", 256),
                ("bf16", 512)]


@pytest.mark.parametrize("dtype,dim", GATHER_CASES)
def test_gather_matches_oracle(dtype, dim):
    spec = workload.spec_tiny(key="g_%s_%d" % (dtype, dim), dtype=dtype, n_tables=5, rows=300, dim=dim,
                              l_min=0, l_max=70)
    inv = workload.make_invocation(spec, 37, seed=dim)
    tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
    ref, mag = oracle.bag_sum(tables, inv["indices"], inv["offsets"], 37)
    got = to_f64(_run_gather(spec, inv))
    c = oracle.check_close(got, ref, mag, RTOL[dtype])
    assert c["ok"], c


def test_gather_strided_output_leaves_other_columns():
    spec = workload.spec_tiny(key="g_strided", dtype="bf16", n_tables=3, rows=100, dim=64, l_min=1, l_max=9)
    inv = workload.make_invocation(spec, 20, seed=4)
    out = _run_gather(spec, inv, ldo=3 * 64 + 128)
    got = to_f64(out)
    tables = [workload.full_table(spec, t) for t in range(3)]
    ref, mag = oracle.bag_sum(tables, inv["indices"], inv["offsets"], 20)
    assert oracle.check_close(got[:, :192], ref, mag, RTOL["bf16"])["ok"]
    assert np.all(got[:, 192:] == 7.0)


def test_gather_long_bags_ragged_batch_and_empty_bags():
    spec = workload.spec_tiny(key="g_long", dtype="f32", n_tables=2, rows=5000, dim=64, l_min=0, l_max=300)
    inv = workload.make_invocation(spec, 2001, seed=5)
    L = np.diff(inv["offsets"])
    assert (L == 0).any() and L.max() > 64
    got = to_f64(_run_gather(spec, inv))
    tables = [workload.full_table(spec, t) for t in range(2)]
    ref, mag = oracle.bag_sum(tables, inv["indices"], inv["offsets"], 2001)
    c = oracle.check_close(got, ref, mag, RTOL["f32"])
    assert c["ok"], c
    empty = (L.reshape(2, 2001) == 0)
    for t in range(2):
        assert np.all(got[empty[t], t * 64:(t + 1) * 64] == 0.0)


def test_gather_single_sample_and_all_empty():
    spec = workload.spec_tiny(key="g_one", dtype="bf16", n_tables=4, rows=10, dim=128, l_min=0, l_max=0)
    inv = workload.make_invocation(spec, 1, seed=6)
    got = to_f64(_run_gather(spec, inv))
    assert np.all(got == 0.0)


def test_gather_is_deterministic_and_uniform_index_control():
    spec = workload.spec_tiny(key="g_det", dtype="bf16", n_tables=3, rows=4000, dim=128, l_min=1, l_max=100)
    inv = workload.make_invocation(spec, 300, seed=7, uniform_rows=True)
    a = _run_gather(spec, inv)
    b = _run_gather(spec, inv)
    assert _torch().equal(a, b)
    tables = [workload.full_table(spec, t) for t in range(3)]
    ref, mag = oracle.bag_sum(tables, inv["indices"], inv["offsets"], 300)
    assert oracle.check_close(to_f64(a), ref, mag, RTOL["bf16"])["ok"]


def test_gather_out_of_range_row_sets_error_and_is_skipped():
    torch = _torch()
    spec = workload.spec_tiny(key="g_oob", dtype="f32", n_tables=2, rows=50, dim=16, l_min=2, l_max=6)
    inv = workload.make_invocation(spec, 9, seed=8)
    bad = dict(inv)
    bad["indices"] = inv["indices"].copy()
    bad["indices"][3] = 50            # == rows: out of range
    bad["indices"][7] = -2
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = to_f64(_run_gather(spec, bad, err=err))
    assert int(err.item()) & 1
    # expected: the same bags with the two bad rows removed
    keep = np.ones(inv["indices"].size, bool)
    keep[[3, 7]] = False
    off = np.array([np.sum(keep[:o]) for o in inv["offsets"]], dtype=np.int64)
    tables = [workload.full_table(spec, t) for t in range(2)]
    ref, mag = oracle.bag_sum(tables, inv["indices"][keep], off, 9)
    assert oracle.check_close(got, ref, mag, RTOL["f32"])["ok"]


@pytest.mark.parametrize("dtype,dim", [("f32", 64), ("bf16", 128), ("bf16", 64), ("f32", 16)])
def test_gather_out_of_range_rows_in_full_and_tail_steps(dtype, dim):
    """Long bags (20..60 rows): bad rows inside a full step (the step's single range
    check fails and the step takes the per-row checked path), in a bag's tail, and in
    the fp32 lane-group kernel (256-byte rows): error bit set, only the bad rows skipped."""
    torch = _torch()
    spec = workload.spec_tiny(key="g_oob2_%s_%d" % (dtype, dim), dtype=dtype, n_tables=3, rows=400, dim=dim,
                              l_min=20, l_max=60)
    B = 23
    inv = workload.make_invocation(spec, B, seed=81)
    off = inv["offsets"]
    bad = dict(inv)
    bad["indices"] = inv["indices"].copy()
    pos = [int(off[0]) + 3, int(off[1]) - 1, int(off[B + 4]) + 17, int(off[2 * B + 7]) + 1]
    bad["indices"][pos[0]] = 400          # == rows
    bad["indices"][pos[1]] = 1 << 30
    bad["indices"][pos[2]] = -1
    bad["indices"][pos[3]] = 401
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = to_f64(_run_gather(spec, bad, err=err))
    assert int(err.item()) & 1
    keep = np.ones(inv["indices"].size, bool)
    keep[pos] = False
    off2 = np.array([np.sum(keep[:o]) for o in off], dtype=np.int64)
    tables = [workload.full_table(spec, t) for t in range(3)]
    ref, mag = oracle.bag_sum(tables, inv["indices"][keep], off2, B)
    c = oracle.check_close(got, ref, mag, RTOL[dtype])
    assert c["ok"], c
    # without bad rows: no error bit, and the bags that held them now include those rows
    err.zero_()
    good = to_f64(_run_gather(spec, inv, err=err))
    assert int(err.item()) == 0
    ref, mag = oracle.bag_sum(tables, inv["indices"], off, B)
    assert oracle.check_close(good, ref, mag, RTOL[dtype])["ok"]


# ------------------------------------------------------------------ dense layers

F32_SHAPES = [(1, 64, 16), (127, 512, 576), (300, 256, 512), (1000, 64, 256), (129, 12, 20), (513, 516, 260),
              (200, 128, 36), (4100, 192, 64)]


@pytest.mark.parametrize("M,N,K", F32_SHAPES)
@pytest.mark.parametrize("relu", [False, True])
def test_linear_f32_matches_oracle(M, N, K, relu):
    torch = _torch()
    rng = np.random.default_rng(M * 7 + N + K)
    x = rng.standard_normal((M, K)).astype(np.float32)
    W = (rng.standard_normal((N, K)) / np.sqrt(K)).astype(np.float32)
    b = rng.standard_normal(N).astype(np.float32)
    y = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    xd, Wd, bd = dev(x), dev(W), dev(b)
    sage.linear(sage.SAGE_F32, M, N, K, xd.data_ptr(), K, Wd.data_ptr(), bd.data_ptr(), relu, y.data_ptr(), N)
    torch.cuda.synchronize()
    ref, mag = oracle.linear(x, W, b, relu, xmag=np.abs(x))
    c = oracle.check_close(to_f64(y), ref, mag, RTOL["f32"])
    assert c["ok"], c
    if N % 64 == 0:
        # tensor-core path (three tf32 products): error below ~3 * 2^-22 of the magnitude bound
        assert c["max_scaled_err"] < 2e-6, c


BF16_SHAPES = [(1, 64, 64), (100, 128, 256), (128, 256, 512), (333, 1024, 3456), (1000, 512, 1024),
               (257, 64, 3392), (4096, 256, 512), (130, 192, 128)]


def _bf16_case(M, N, K, seed):
    rng = np.random.default_rng(seed)
    torch = _torch()
    rnd = lambda a: torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).float().numpy()
    x = rnd(np.abs(rng.standard_normal((M, K))) * 0.5)
    W = rnd(rng.uniform(-1, 1, (N, K)) * np.sqrt(6.0 / (K + N)))
    b = (rng.uniform(-1, 1, N) / np.sqrt(K)).astype(np.float32)
    return x, W, b


@pytest.mark.parametrize("M,N,K", BF16_SHAPES)
@pytest.mark.parametrize("relu", [False, True])
def test_linear_bf16_tcgen05_matches_oracle(M, N, K, relu):
    torch = _torch()
    x, W, b = _bf16_case(M, N, K, M + N + K)
    xd, Wd, bd = bf16_dev(x), bf16_dev(W), dev(b)
    y = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    sage.linear(sage.SAGE_BF16, M, N, K, xd.data_ptr(), K, Wd.data_ptr(), bd.data_ptr(), relu, y.data_ptr(), N,
                err.data_ptr())
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref, mag = oracle.linear(x, W, b, relu, xmag=np.abs(x))
    c = oracle.check_close(to_f64(y), ref, mag, RTOL["bf16"])
    assert c["ok"], c
    # fp32 accumulation + one bf16 rounding of the output: far inside the tolerance
    assert c["max_scaled_err"] < 5e-3, c


def test_linear_bf16_strided_output_slice():
    torch = _torch()
    M, N, K, ld, col = 200, 128, 256, 3456, 3328
    x, W, b = _bf16_case(M, N, K, 3)
    y = torch.full((M, ld), 3.0, dtype=torch.bfloat16, device="cuda")
    xd, Wd, bd = bf16_dev(x), bf16_dev(W), dev(b)
    sage.linear(sage.SAGE_BF16, M, N, K, xd.data_ptr(), K, Wd.data_ptr(), bd.data_ptr(), True,
                y[:, col:].data_ptr(), ld)
    torch.cuda.synchronize()
    ref, mag = oracle.linear(x, W, b, True, xmag=np.abs(x))
    got = to_f64(y)
    assert oracle.check_close(got[:, col:col + N], ref, mag, RTOL["bf16"])["ok"]
    assert np.all(got[:, :col] == 3.0)


def test_linear_bf16_rows_do_not_depend_on_batch():
    """A row's output is bitwise the same whether the batch has 300 or 1000 rows."""
    torch = _torch()
    N, K = 512, 1024
    x, W, b = _bf16_case(1000, N, K, 11)
    xd, Wd, bd = bf16_dev(x), bf16_dev(W), dev(b)
    y1 = torch.empty((1000, N), dtype=torch.bfloat16, device="cuda")
    y2 = torch.empty((300, N), dtype=torch.bfloat16, device="cuda")
    sage.linear(sage.SAGE_BF16, 1000, N, K, xd.data_ptr(), K, Wd.data_ptr(), bd.data_ptr(), True, y1.data_ptr(), N)
    sage.linear(sage.SAGE_BF16, 300, N, K, xd.data_ptr(), K, Wd.data_ptr(), bd.data_ptr(), True, y2.data_ptr(), N)
    torch.cuda.synchronize()
    assert torch.equal(y1[:300], y2)


def test_linear_rejects_unsupported_shapes():
    torch = _torch()
    x = torch.zeros((4, 100), dtype=torch.bfloat16, device="cuda")
    W = torch.zeros((64, 100), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(64, device="cuda")
    y = torch.zeros((4, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(sage.SageError):
        sage.linear(sage.SAGE_BF16, 4, 64, 100, x.data_ptr(), 100, W.data_ptr(), b.data_ptr(), False,
                    y.data_ptr(), 64)


BF16_TILES = [(256, 4), (128, 6), (64, 8), (256, 2), (128, 3), (64, 4), (256, 104), (128, 106)]
F32_TILES = [(128, 3), (64, 4), (64, 2)]


@pytest.mark.parametrize("tile", BF16_TILES)
def test_every_bf16_tile_configuration_matches_oracle(tile):
    torch = _torch()
    M, N, K = 700, 512, 1024
    x, W, b = _bf16_case(M, N, K, 17)
    xd, Wd, bd = bf16_dev(x), bf16_dev(W), dev(b)
    y = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda")
    sage.linear(sage.SAGE_BF16, M, N, K, xd.data_ptr(), K, Wd.data_ptr(), bd.data_ptr(), True, y.data_ptr(), N,
                tile=tile)
    ref_y = torch.empty_like(y)
    sage.linear(sage.SAGE_BF16, M, N, K, xd.data_ptr(), K, Wd.data_ptr(), bd.data_ptr(), True, ref_y.data_ptr(), N,
                tile=BF16_TILES[0])
    torch.cuda.synchronize()
    ref, mag = oracle.linear(x, W, b, True, xmag=np.abs(x))
    c = oracle.check_close(to_f64(y), ref, mag, RTOL["bf16"])
    assert c["ok"] and c["max_scaled_err"] < 5e-3, c
    assert torch.equal(y, ref_y)          # the tile shape does not change any output bit


@pytest.mark.parametrize("tile", F32_TILES)
def test_every_f32_tile_configuration_matches_oracle(tile):
    torch = _torch()
    M, N, K = 900, 256, 576
    rng = np.random.default_rng(23)
    x = rng.standard_normal((M, K)).astype(np.float32)
    W = (rng.standard_normal((N, K)) / np.sqrt(K)).astype(np.float32)
    b = rng.standard_normal(N).astype(np.float32)
    xd, Wd, bd = dev(x), dev(W), dev(b)
    y = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    sage.linear(sage.SAGE_F32, M, N, K, xd.data_ptr(), K, Wd.data_ptr(), bd.data_ptr(), False, y.data_ptr(), N,
                tile=tile)
    torch.cuda.synchronize()
    ref, mag = oracle.linear(x, W, b, False, xmag=np.abs(x))
    c = oracle.check_close(to_f64(y), ref, mag, RTOL["f32"])
    assert c["ok"] and c["max_scaled_err"] < 2e-6, c


def test_unknown_tile_configuration_is_rejected():
    torch = _torch()
    x = torch.zeros((4, 64), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(64, device="cuda")
    with pytest.raises(sage.SageError):
        sage.linear(sage.SAGE_BF16, 4, 64, 64, x.data_ptr(), 64, x.data_ptr(), b.data_ptr(), False, x.data_ptr(), 64,
                    tile=(96, 3))
