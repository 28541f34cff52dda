"""Pins of the CPU oracle to things other than itself (CPU only).

Each test checks the oracle against a closed form, a value computed by hand,
a brute-force formulation that differs from the oracle's loops, a library
routine, or a number the paper prints -- chosen so that a dropped term, a wrong
sign or index, a transposed operand or a wrong layer order fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_bags(rng, T, B, n_rows, max_len, allow_empty=True):
    lo = 0 if allow_empty else 1
    lengths = rng.integers(lo, max_len + 1, size=T * B)
    offsets = np.zeros(T * B + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    indices = np.empty(int(offsets[-1]), dtype=np.int32)
    for t in range(T):
        a, b = int(offsets[t * B]), int(offsets[(t + 1) * B])
        indices[a:b] = rng.integers(0, n_rows[t], size=b - a)
    return offsets, indices


# ------------------------------------------------------------ embedding-bag sum

def test_bag_sum_integer_bruteforce_count_matrix():
    """Integer tables: sums are exact in fp64; compare with a count-matrix product."""
    rng = np.random.default_rng(1)
    T, B, D = 3, 6, 4
    n_rows = [5, 4, 7]
    tables = [rng.integers(-9, 10, size=(n, D)).astype(np.float64) for n in n_rows]
    offsets, indices = _random_bags(rng, T, B, n_rows, 6)
    pooled, _ = oracle.bag_sum(tables, indices, offsets, B)
    for t in range(T):
        counts = np.zeros((B, n_rows[t]), dtype=np.int64)
        for b in range(B):
            for i in range(offsets[t * B + b], offsets[t * B + b + 1]):
                counts[b, indices[i]] += 1
        expect = counts @ tables[t].astype(np.int64)
        assert np.array_equal(pooled[:, t * D:(t + 1) * D], expect.astype(np.float64))


def test_bag_sum_all_ones_gives_bag_length():
    rng = np.random.default_rng(2)
    T, B, D = 2, 9, 5
    tables = [np.ones((11, D)), np.ones((3, D))]
    offsets, indices = _random_bags(rng, T, B, [11, 3], 7)
    pooled, mag = oracle.bag_sum(tables, indices, offsets, B)
    lengths = np.diff(offsets).reshape(T, B)
    for t in range(T):
        assert np.array_equal(pooled[:, t * D:(t + 1) * D], np.repeat(lengths[t][:, None], D, 1).astype(float))
    assert np.array_equal(mag, pooled)


def test_bag_sum_one_hot_rows_count_index_multiplicity():
    rng = np.random.default_rng(3)
    N = 6
    B = 5
    tables = [np.eye(N)]
    offsets, indices = _random_bags(rng, 1, B, [N], 9)
    pooled, _ = oracle.bag_sum(tables, indices, offsets, B)
    for b in range(B):
        bag = indices[offsets[b]:offsets[b + 1]]
        assert np.array_equal(pooled[b], np.bincount(bag, minlength=N).astype(float))


def test_bag_sum_matches_torch_embedding_bag_fp64():
    rng = np.random.default_rng(4)
    T, B, D = 4, 17, 8
    n_rows = [13, 29, 7, 50]
    tables = [rng.standard_normal((n, D)) for n in n_rows]
    offsets, indices = _random_bags(rng, T, B, n_rows, 12)
    pooled, mag = oracle.bag_sum(tables, indices, offsets, B)
    for t in range(T):
        base = offsets[t * B]
        idx = torch.from_numpy(indices[offsets[t * B]:offsets[(t + 1) * B]].astype(np.int64))
        off = torch.from_numpy(offsets[t * B:(t + 1) * B] - base)
        ref = torch.nn.functional.embedding_bag(idx, torch.from_numpy(tables[t]), off, mode="sum")
        np.testing.assert_allclose(pooled[:, t * D:(t + 1) * D], ref.numpy(), rtol=1e-13, atol=1e-13)
        refm = torch.nn.functional.embedding_bag(idx, torch.from_numpy(np.abs(tables[t])), off, mode="sum")
        np.testing.assert_allclose(mag[:, t * D:(t + 1) * D], refm.numpy(), rtol=1e-13, atol=1e-13)


def test_bag_sum_empty_bags_are_zero_and_duplicates_count():
    tables = [np.array([[1.5, -2.0], [0.25, 4.0]])]
    offsets = np.array([0, 0, 3, 3], dtype=np.int64)
    indices = np.array([1, 1, 0], dtype=np.int32)
    pooled, mag = oracle.bag_sum(tables, indices, offsets, 3)
    assert np.array_equal(pooled, np.array([[0, 0], [2.0, 6.0], [0, 0]]))
    assert np.array_equal(mag, np.array([[0, 0], [2.0, 10.0], [0, 0]]))


def test_bag_sum_rejects_out_of_range_rows():
    tables = [np.zeros((4, 2))]
    with pytest.raises(IndexError):
        oracle.bag_sum(tables, np.array([4], np.int32), np.array([0, 1], np.int64), 1)
    with pytest.raises(IndexError):
        oracle.bag_sum(tables, np.array([-1], np.int32), np.array([0, 1], np.int64), 1)


# ------------------------------------------------------------ linear / sigmoid

def test_linear_hand_worked_non_square():
    # x [1,2], W [3,2] (out=3, in=2), b [3]:  y_j = sum_k x_k W[j,k] + b_j
    x = np.array([[1.0, 2.0]])
    W = np.array([[1.0, -1.0], [2.0, 0.5], [0.0, 3.0]])
    b = np.array([0.5, -4.0, 1.0])
    y, _ = oracle.linear(x, W, b, relu=False)
    assert np.array_equal(y, np.array([[-0.5, -1.0, 7.0]]))
    y, _ = oracle.linear(x, W, b, relu=True)
    assert np.array_equal(y, np.array([[0.0, 0.0, 7.0]]))
    _, ym = oracle.linear(x, W, b, relu=True, xmag=np.abs(x))
    assert np.array_equal(ym, np.array([[3.5, 7.0, 7.0]]))


def test_linear_matches_torch_fp64():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((7, 19))
    W = rng.standard_normal((11, 19))
    b = rng.standard_normal(11)
    for relu in (False, True):
        y, _ = oracle.linear(x, W, b, relu)
        ref = torch.nn.functional.linear(torch.from_numpy(x), torch.from_numpy(W), torch.from_numpy(b))
        if relu:
            ref = torch.relu(ref)
        np.testing.assert_allclose(y, ref.numpy(), rtol=1e-13, atol=1e-13)


def test_sigmoid_closed_forms():
    assert oracle.sigmoid(0.0) == 0.5
    assert abs(oracle.sigmoid(math.log(3.0)) - 0.75) < 1e-15
    assert abs(oracle.sigmoid(-math.log(3.0)) - 0.25) < 1e-15
    for z in (-7.5, -1.0, 0.3, 12.0):
        assert abs(oracle.sigmoid(z) + oracle.sigmoid(-z) - 1.0) < 1e-15


# ------------------------------------------------------------ whole function

def _golden_function():
    with open(os.path.join(GOLDEN, "hand_worked_function.json")) as f:
        g = json.load(f)
    tables = [np.array(t, dtype=np.float32) for t in g["tables"]]
    spec = workload.FunctionSpec(key="hand", dtype="f32", rows=[len(t) for t in tables], dim=2,
                                 bot_dims=[len(l["b"]) for l in g["bottom"]],
                                 top_dims=[len(l["b"]) for l in g["top"]], n_dense=2)
    weights = [(np.array(l["W"], np.float32), np.array(l["b"], np.float32)) for l in g["bottom"] + g["top"]]
    inv = {"batch": len(g["dense"]), "dense": np.array(g["dense"], np.float32),
           "offsets": np.array(g["offsets"], np.int64), "indices": np.array(g["indices"], np.int32)}
    return g, spec, weights, tables, inv


def test_forward_hand_worked_example():
    g, spec, weights, tables, inv = _golden_function()
    res = oracle.forward(spec, weights, inv, tables=tables)
    assert np.array_equal(res["pooled"], np.array(g["expected_pooled"], dtype=np.float64))
    expect = [1.0 / (1.0 + math.exp(-z)) for z in g["expected_z"]]
    np.testing.assert_allclose(res["out"], expect, rtol=1e-15)


def test_forward_hand_worked_example_sample_subrange():
    g, spec, weights, tables, inv = _golden_function()
    res = oracle.forward(spec, weights, inv, tables=tables, b0=1, b1=3)
    assert np.array_equal(res["pooled"], np.array(g["expected_pooled"][1:], dtype=np.float64))
    expect = [1.0 / (1.0 + math.exp(-z)) for z in g["expected_z"][1:]]
    np.testing.assert_allclose(res["out"], expect, rtol=1e-15)


def _torch_function(spec, weights, tables, inv):
    """The function composed from torch fp64 library routines."""
    T, B = spec.n_tables, inv["batch"]
    nb = len(spec.bot_dims)
    Wt = [(torch.from_numpy(w.astype(np.float64)), torch.from_numpy(b.astype(np.float64))) for w, b in weights]
    h = torch.from_numpy(inv["dense"].astype(np.float64))
    for (w, b) in Wt[:nb]:
        h = torch.relu(torch.nn.functional.linear(h, w, b))
    pooled = []
    off = inv["offsets"]
    for t in range(T):
        base = off[t * B]
        idx = torch.from_numpy(inv["indices"][off[t * B]:off[(t + 1) * B]].astype(np.int64))
        o = torch.from_numpy(off[t * B:(t + 1) * B] - base)
        pooled.append(torch.nn.functional.embedding_bag(idx, torch.from_numpy(tables[t].astype(np.float64)), o,
                                                        mode="sum"))
    g = torch.cat(pooled + [h], dim=1)
    top = Wt[nb:]
    for i, (w, b) in enumerate(top):
        g = torch.nn.functional.linear(g, w, b)
        if i < len(top) - 1:
            g = torch.relu(g)
    return torch.sigmoid(g[:, 0]).numpy(), torch.cat(pooled, 1).numpy()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_forward_matches_torch_composition(dtype):
    spec = workload.spec_tiny(key="pin_fwd_" + dtype, dtype=dtype, n_tables=4, rows=40, dim=8,
                              bot=(16, 8), top=(16, 8, 1), l_min=0, l_max=6)
    weights = workload.weights_arrays(spec)
    tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
    inv = workload.make_invocation(spec, 23, seed=7)
    res = oracle.forward(spec, weights, inv, tables=tables, n_threads=3)
    ref_out, ref_pooled = _torch_function(spec, weights, tables, inv)
    np.testing.assert_allclose(res["pooled"], ref_pooled, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(res["out"], ref_out, rtol=1e-12, atol=1e-14)


def test_forward_row_source_equals_full_tables():
    spec = workload.spec_tiny(key="pin_rows", n_tables=3, rows=60, dim=4, l_min=1, l_max=9)
    weights = workload.weights_arrays(spec)
    tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
    inv = workload.make_invocation(spec, 12, seed=3)
    full = oracle.forward(spec, weights, inv, tables=tables)
    part = oracle.forward(spec, weights, inv, row_source=lambda t, r: workload.table_rows(spec, t, r), b0=4, b1=11)
    assert np.array_equal(full["out"][4:11], part["out"])
    assert np.array_equal(full["pooled"][4:11], part["pooled"])


def test_forward_magnitude_bounds_an_fp32_evaluation():
    """The magnitude bound m must dominate the error of an fp32 evaluation of the
    same function (torch fp32), scaled by a few units of fp32 roundoff per layer."""
    spec = workload.spec_tiny(key="pin_mag", n_tables=5, rows=30, dim=16, bot=(32, 16), top=(64, 32, 1),
                              l_min=0, l_max=30)
    weights = workload.weights_arrays(spec)
    tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
    inv = workload.make_invocation(spec, 40, seed=9)
    res = oracle.forward(spec, weights, inv, tables=tables)
    w32 = [(w.astype(np.float32), b.astype(np.float32)) for w, b in weights]
    with torch.no_grad():
        out32, pooled32 = _torch_function(spec, w32, tables, inv)
    # fp32 loses at most ~ n u per sum of n terms; 1e-5 covers these short sums
    c_p = oracle.check_close(pooled32, res["pooled"], res["pooled_mag"], 1e-5)
    c_o = oracle.check_close(out32, res["out"], res["out_mag"], 1e-5)
    assert c_p["ok"] and c_o["ok"], (c_p, c_o)
    # and a plausible 1% perturbation of one bag is caught by the same bound
    bad = pooled32.copy()
    bad[3, 5] += 0.01 * max(1e-3, abs(bad[3, 5]))
    assert not oracle.check_close(bad, res["pooled"], res["pooled_mag"], 1e-5)["ok"]


# ------------------------------------------------------------ batching

def test_pack_invocations_rebases_offsets_and_keeps_every_bag():
    spec = workload.spec_tiny(key="pin_pack", n_tables=3, rows=25, dim=4, l_min=0, l_max=7)
    sizes = [3, 1, 5, 2]
    invs = [workload.make_invocation(spec, B, seed=100 + i) for i, B in enumerate(sizes)]
    p = oracle.pack_invocations(invs, spec.n_tables)
    T, M = spec.n_tables, sum(sizes)
    assert p["batch"] == M
    assert list(p["row_base"]) == [0, 3, 4, 9, 11]
    assert p["offsets"][0] == 0 and p["offsets"][-1] == sum(v["indices"].size for v in invs)
    assert np.all(np.diff(p["offsets"]) >= 0)
    for i, v in enumerate(invs):
        B = v["batch"]
        for t in range(T):
            for b in range(B):
                g = t * M + p["row_base"][i] + b
                got = p["indices"][p["offsets"][g]:p["offsets"][g + 1]]
                want = v["indices"][v["offsets"][t * B + b]:v["offsets"][t * B + b + 1]]
                assert np.array_equal(got, want)
        assert np.array_equal(p["dense"][p["row_base"][i]:p["row_base"][i + 1]], v["dense"])


def test_shared_batch_equals_isolated_invocations():
    """N invocations fused into one batch give exactly the N isolated results."""
    spec = workload.spec_tiny(key="pin_share", n_tables=3, rows=25, dim=4, l_min=0, l_max=7)
    weights = workload.weights_arrays(spec)
    tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
    invs = [workload.make_invocation(spec, B, seed=200 + i) for i, B in enumerate([4, 1, 6])]
    p = oracle.pack_invocations(invs, spec.n_tables)
    fused = oracle.forward(spec, weights, p, tables=tables)
    for i, v in enumerate(invs):
        alone = oracle.forward(spec, weights, v, tables=tables)
        r0, r1 = p["row_base"][i], p["row_base"][i + 1]
        assert np.array_equal(fused["out"][r0:r1], alone["out"])
        assert np.array_equal(fused["pooled"][r0:r1], alone["pooled"])


# ------------------------------------------------------------ sharing model

def test_pool_model_loads_once_and_frees_at_zero():
    m = oracle.PoolModel(budget=100)
    assert m.prepare("f", 60) == "OK"
    assert m.prepare("f", 60) == "OK"
    assert m.refcount("f") == 2 and m.h2d_bytes == 60 and m.hits == 1 and m.misses == 1
    assert m.prepare("g", 50) == "NOMEM"
    assert m.prepare("f", 61) == "INVALID"
    assert m.release("f") == "OK" and m.refcount("f") == 1
    assert m.release("f") == "OK" and m.refcount("f") == 0 and m.used == 0
    assert m.prepare("g", 50) == "OK" and m.h2d_bytes == 110
    assert m.release("x") == "INVALID"


# ------------------------------------------------------------ setup-time model

def test_setup_latency_model_reproduces_table_tb_stage():
    with open(os.path.join(GOLDEN, "tb_stage_resnet50.json")) as f:
        g = json.load(f)
    for name, col in g["columns"].items():
        stages = {k: col[k] for k in ("cpu_ctx", "gpu_ctx", "cpu_data", "gpu_data", "compute", "return_data")}
        got = oracle.setup_latency_model(stages, parallel=col["parallel"])
        assert abs(got - col["end_to_end"]) < 0.051, (name, got, col["end_to_end"])
    # serial vs parallel on the cold column: the hidden data stages are the gain
    cold = g["columns"]["cold"]
    st = {k: cold[k] for k in ("cpu_ctx", "gpu_ctx", "cpu_data", "gpu_data", "compute", "return_data")}
    assert abs(oracle.setup_latency_model(st, parallel=False) - g["columns"]["baseline"]["end_to_end"]) < 0.051


def test_throughput_perf_definition():
    # Throughput_theo = T_period / T_comp; perf = app / theo
    assert oracle.throughput_perf(50.0, 10.0, 0.1) == 0.5


def test_check_output_applies_the_plain_relative_bound():
    """Final outputs must meet |got - ref| <= rtol |ref| as well as the magnitude-scaled
    bound: a 4% error under a loose bound (a deep network's magnitude sum) fails, fp32
    rounding noise passes, an exact result passes."""
    ref = np.array([0.5, 0.25, 0.9])
    mag = np.array([1e4, 1e4, 1e4])
    wrong = ref * 1.04
    assert oracle.check_close(wrong, ref, mag, 1e-5)["ok"]
    c = oracle.check_output(wrong, ref, mag, 1e-5)
    assert not c["ok"] and c["n_bad_plain"] == 3
    noisy = ref * (1 + 3e-7)
    assert oracle.check_output(noisy, ref, mag, 1e-5)["ok"]
    assert oracle.check_output(ref.copy(), ref, mag, 1e-5)["ok"]
    # the componentwise bound still applies on its own
    assert not oracle.check_output(ref + 1e-3, ref, np.full(3, 1.0), 1e-5)["ok"]
