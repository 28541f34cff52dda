"""The shared input generator: its random source and distributions (CPU only)."""
import math

import numpy as np
import pytest
import torch

import workload


def test_splitmix64_published_first_output():
    # SplitMix64 started at state 0: first output 0xE220A8397B1DCDAF
    assert workload.draw(0, 0) == 0xE220A8397B1DCDAF
    assert workload.lib().wl_draw(0, 0) == 0xE220A8397B1DCDAF


def test_c_and_python_splitmix_agree():
    rng = np.random.default_rng(0)
    for _ in range(200):
        s = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        e = int(rng.integers(0, 2 ** 40))
        assert workload.lib().wl_draw(s, e) == workload.draw(s, e)


def test_table_values_follow_the_stated_recipe():
    spec = workload.spec_tiny(key="wl_vals", dtype="f32", n_tables=2, rows=7, dim=3)
    seed = spec.table_seeds()[1]
    vals = workload.full_table(spec, 1).ravel()
    step = np.float32(np.float32(0.05) / np.float32(8388608.0))
    for e in range(vals.size):
        k = (workload.draw(seed, e) >> 40) - (1 << 23)
        assert vals[e] == np.float32(np.float32(k) * step)
    assert np.all(vals >= -0.05) and np.all(vals < 0.05)


def test_bf16_tables_are_round_to_nearest_even_of_fp32():
    f = workload.spec_tiny(key="wl_bf", dtype="f32", n_tables=1, rows=300, dim=16)
    b = workload.spec_tiny(key="wl_bf", dtype="bf16", n_tables=1, rows=300, dim=16)
    v32 = workload.full_table(f, 0)
    v16 = workload.full_table(b, 0)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(v16, ref)


def test_tables_blob_is_tables_concatenated():
    spec = workload.spec_tiny(key="wl_blob", dtype="bf16", n_tables=3, rows=11, dim=8)
    blob = workload.tables_blob(spec)
    bits = blob.view(np.uint16)
    got = workload.bf16_bits_to_f32(bits).reshape(-1, spec.dim)
    want = np.concatenate([workload.full_table(spec, t) for t in range(3)])
    assert np.array_equal(got, want)


def test_weights_are_xavier_uniform_and_biases_torch_default():
    spec = workload.spec_c1()
    ws = workload.weights_arrays(spec)
    for (W, b), (i, o) in zip(ws, spec.layer_dims()):
        bound = math.sqrt(6.0 / (i + o))
        assert W.shape == (o, i) and b.shape == (o,)
        assert np.abs(W).max() <= bound * (1 + 1e-6)
        assert np.abs(W).max() > 0.95 * bound or W.size < 200
        assert abs(W.mean()) < 4 * bound / math.sqrt(3 * W.size)
        assert np.abs(b).max() <= (1 / math.sqrt(i)) * (1 + 1e-6)


def test_weights_layout_is_256_byte_aligned():
    spec = workload.spec_c3()
    for wo, bo in workload.weights_layout(spec):
        assert wo % 256 == 0 and bo % 256 == 0


def test_affine_rank_map_is_a_bijection():
    for n in (1, 2, 7, 64, 1000, 1024):
        spec = workload.spec_tiny(key="wl_aff%d" % n, rows=n)
        a, c = workload.affine_map(spec, 0)
        rows = (a * np.arange(n) + c) % n
        assert np.array_equal(np.sort(rows), np.arange(n))


def test_zipf_top_rank_frequency_matches_closed_form():
    n, alpha, count = 1000, 1.05, 400_000
    rng = np.random.Generator(np.random.PCG64(11))
    ranks = workload.zipf_ranks(rng, n, alpha, count)
    h = sum(k ** -alpha for k in range(1, n + 1))
    for r in (0, 1, 9):
        p = (r + 1) ** -alpha / h
        f = np.mean(ranks == r)
        assert abs(f - p) < 5 * math.sqrt(p * (1 - p) / count), (r, f, p)
    assert ranks.min() >= 0 and ranks.max() <= n - 1


def test_invocation_csr_shapes_and_ranges():
    spec = workload.spec_c2()
    inv = workload.make_invocation(spec, 37, seed=5)
    T, B = spec.n_tables, 37
    off = inv["offsets"]
    assert off.shape == (T * B + 1,) and off[0] == 0 and off[-1] == inv["indices"].size
    L = np.diff(off)
    assert L.min() >= spec.l_min and L.max() <= spec.l_max
    for t in range(T):
        seg = inv["indices"][off[t * B]:off[(t + 1) * B]]
        assert seg.min() >= 0 and seg.max() < spec.rows[t]
    assert inv["dense"].shape == (B, 13) and inv["dense"].dtype == np.float32


def test_batch_size_distributions():
    u = workload.batch_sizes_uniform(5000, 1, 512, seed=1)
    assert u.min() >= 1 and u.max() <= 512 and abs(u.mean() - 256.5) < 8
    ln = workload.batch_sizes_lognormal(20000, seed=2)
    assert ln.min() >= 1 and ln.max() <= 4096
    assert abs(np.median(ln) - 256) < 12


def test_poisson_arrivals_rate():
    t = workload.poisson_arrivals(20000, 200.0, seed=3)
    assert np.all(np.diff(t) > 0)
    assert abs(20000 / t[-1] - 200.0) < 6
