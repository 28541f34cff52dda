"""Bottom layers 0 and 1 of a pre-split fp32 function fused into one kernel: layer 0
(13 dense features into the bottom MLP) is computed straight into
the A tiles of layer 1's tensor-core GEMM.  Every fused tile configuration gives the
bits of the two separate kernels (bottom0, then the pre-split GEMM), and the
function still matches the oracle."""
import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, DevInvocation, oracle_rows, prepare, to_f64

pytestmark = pytest.mark.gpu

sage = pytest.importorskip("paper_2404_14691_b300")

KIND_BOTTOM01 = 4
SEPARATE = (1, 1)
FUSED = [(256, 102), (128, 103), (64, 104), (256, 202)]   # (256, 202): layer 2 in the kernel too


@pytest.fixture(scope="module")
def pool():
    p = sage.Pool(device=0)
    yield p
    p.destroy()


def _spec(key, n_dense, bot, top=(128, 64, 1), dim=32):
    s = workload.spec_tiny(key=key, dtype="f32", n_tables=3, rows=4000, dim=dim, bot=bot, top=top,
                           l_min=0, l_max=30)
    s.n_dense = n_dense
    return s


# (n_dense, bottom dims): the batching workload's bottom MLP; two-layer bottoms whose
# layer 1 writes the concat buffer directly; the narrowest and widest layer 0
CASES = [
    ("b01_c2", 13, (512, 256, 64)),
    ("b01_two", 15, (64, 128)),
    ("b01_k1", 1, (32, 64, 64)),
    ("b01_n0max", 7, (512, 64)),
    # layer 2 in the kernel: 128 and 256 outputs (3 and 4 rounds of its k-blocks), and a
    # four-layer bottom whose layer 2 writes a workspace buffer instead of the concat
    ("b01_l2_128", 13, (256, 256, 128)),
    ("b01_l2_4", 9, (64, 256, 256, 64)),
]


def _same(a, b):
    import torch
    return torch.equal(a.out[:a.batch], b.out[:b.batch])


def _run(f, invs):
    import torch
    d = [DevInvocation(v) for v in invs]
    f.invoke_batch([x.args() for x in d])
    torch.cuda.synchronize()
    f.check_errors()
    return d


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fused_bottom_equals_separate_kernels_bitwise(pool, case):
    key, n_dense, bot = case
    spec = _spec(key, n_dense, bot)
    f = prepare(pool, spec, max_batch=4096)
    try:
        # ragged members (an empty one, a single row) so the last M tile is partial
        sizes = [700, 0, 1, 333, 129]
        invs = [workload.make_invocation(spec, B, seed=900 + i) for i, B in enumerate(sizes)]
        M = sum(sizes)
        N0, N1 = bot[0], bot[1]
        sage.tuning_set(KIND_BOTTOM01, M, N1, N0, *SEPARATE)
        ref = _run(f, invs)
        for tile in FUSED:
            if N1 % tile[0]:
                continue
            sage.tuning_set(KIND_BOTTOM01, M, N1, N0, *tile)
            got = _run(f, invs)
            for a, b in zip(ref, got):
                assert _same(a, b), (tile, a.batch)
        # one invocation alone (the kernel skips the invocation search) equals its batch row range
        one = _run(f, [invs[3]])
        assert _same(one[0], ref[3])
        tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
        w = workload.weights_arrays(spec)
        for d in (got[0], got[2], got[4]):
            res = oracle.forward(spec, w, d.inv, tables=tables, want_pooled=False)
            c = oracle.check_output(to_f64(d.out)[:d.batch], res["out"], res["out_mag"], RTOL["f32"])
            assert c["ok"], c
    finally:
        f.release()


def test_fused_bottom_is_the_default_and_counts_launches(pool):
    """Untuned, the batching workload's bottom MLP (13-512-256-64) runs as one kernel on a
    large batch (two launches fewer than with separate kernels pinned) and as separate
    kernels on a small one."""
    spec = _spec("b01_launches", 13, (512, 256, 64))
    f = prepare(pool, spec, max_batch=12000)
    try:
        small = [workload.make_invocation(spec, 300, seed=949)]
        _run(f, small)
        n0 = sage.kernel_launches()
        s_default = _run(f, small)
        n_small = sage.kernel_launches() - n0
        sage.tuning_set(KIND_BOTTOM01, 300, 256, 512, *SEPARATE)
        n0 = sage.kernel_launches()
        s_sep = _run(f, small)
        assert sage.kernel_launches() - n0 == n_small   # below 64 tiles: separate kernels by default
        assert _same(s_default[0], s_sep[0])
        invs = [workload.make_invocation(spec, B, seed=950 + i) for i, B in enumerate([6000, 3011])]
        M = 9011
        _run(f, invs)
        n0 = sage.kernel_launches()
        a = _run(f, invs)
        fused = sage.kernel_launches() - n0
        sage.tuning_set(KIND_BOTTOM01, M, 256, 512, *SEPARATE)
        n0 = sage.kernel_launches()
        b = _run(f, invs)
        separate = sage.kernel_launches() - n0
        assert separate == fused + 2
        for x, y in zip(a, b):
            assert _same(x, y)
    finally:
        f.release()


def test_autotune_chooses_a_bottom_form_and_keeps_bits(pool, tmp_path):
    spec = _spec("b01_tune", 13, (512, 256, 64))
    f = prepare(pool, spec, max_batch=4096)
    try:
        invs = [workload.make_invocation(spec, B, seed=970 + i) for i, B in enumerate([1500, 900])]
        before = _run(f, invs)
        f.autotune(2400)
        after = _run(f, invs)
        for x, y in zip(before, after):
            assert _same(x, y)
        path = str(tmp_path / "tune.txt")
        sage.tuning_save(path)
        rows = [l.split() for l in open(path) if not l.startswith("#")]
        b01 = [r for r in rows if r[1:5] == [str(KIND_BOTTOM01), "4096", "256", "512"]]
        assert len(b01) == 1
        assert (int(b01[0][5]), int(b01[0][6])) in FUSED + [SEPARATE]
    finally:
        f.release()


def test_unknown_bottom_tile_is_refused():
    with pytest.raises(sage.SageError):
        sage.tuning_set(KIND_BOTTOM01, 512, 256, 512, 128, 3)
    with pytest.raises(sage.SageError):
        sage.tuning_set(KIND_BOTTOM01, 512, 192, 512, 128, 103)   # 192 is not a multiple of 128


def test_fused_bottom_dense_rows_beyond_alignment(pool):
    """Dense rows of 13 floats start at every 4-byte offset; the fused kernel reads them
    element by element, so odd row starts are fine."""
    spec = _spec("b01_align", 13, (64, 64))
    f = prepare(pool, spec, max_batch=4096)
    try:
        invs = [workload.make_invocation(spec, B, seed=990 + i) for i, B in enumerate([3, 5, 7, 11])]
        M = 26
        sage.tuning_set(KIND_BOTTOM01, M, 64, 64, *SEPARATE)
        ref = _run(f, invs)
        sage.tuning_set(KIND_BOTTOM01, M, 64, 64, 64, 104)
        got = _run(f, invs)
        for a, b in zip(ref, got):
            assert _same(a, b)
        assert np.isfinite(to_f64(got[0].out)[:3]).all()
    finally:
        f.release()


def test_sixteen_dense_inputs_run_as_separate_kernels(pool):
    """Layer 0 with 16 inputs leaves no weight slot for the bias: the function runs
    bottom0 and the GEMM separately (same launch count as with separate kernels pinned)
    and still matches the oracle."""
    spec = _spec("b01_k16", 16, (64, 128))
    f = prepare(pool, spec, max_batch=4096)
    try:
        invs = [workload.make_invocation(spec, B, seed=1010 + i) for i, B in enumerate([200, 57])]
        _run(f, invs)
        n0 = sage.kernel_launches()
        got = _run(f, invs)
        default = sage.kernel_launches() - n0
        sage.tuning_set(KIND_BOTTOM01, 257, 128, 64, *SEPARATE)
        n0 = sage.kernel_launches()
        _run(f, invs)
        assert sage.kernel_launches() - n0 == default
        tables = [workload.full_table(spec, t) for t in range(spec.n_tables)]
        res = oracle.forward(spec, workload.weights_arrays(spec), got[1].inv, tables=tables, want_pooled=False)
        c = oracle.check_output(to_f64(got[1].out)[:got[1].batch], res["out"], res["out_mag"], RTOL["f32"])
        assert c["ok"], c
    finally:
        f.release()


def test_three_layer_form_falls_back_beyond_one_tile_per_sm(pool):
    """More 128-row tiles than SMs: the three-layer configuration runs as the two-layer
    kernel plus layer 2's GEMM, with the same bits."""
    import torch
    spec = _spec("b01_big", 13, (512, 256, 64))
    f = prepare(pool, spec, max_batch=20000)
    try:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        B = 128 * sms + 77                      # one tile more than SMs
        invs = [workload.make_invocation(spec, B, seed=1100)]
        sage.tuning_set(KIND_BOTTOM01, B, 256, 512, *SEPARATE)
        ref = _run(f, invs)
        sage.tuning_set(KIND_BOTTOM01, B, 256, 512, 256, 202)
        n0 = sage.kernel_launches()
        got = _run(f, invs)
        n_fused = sage.kernel_launches() - n0
        assert _same(ref[0], got[0])
        sage.tuning_set(KIND_BOTTOM01, B, 256, 512, *SEPARATE)
        n0 = sage.kernel_launches()
        _run(f, invs)
        assert sage.kernel_launches() - n0 == n_fused + 1   # bottom0 + GEMM instead of the fused kernel
        rows = np.arange(0, B, 997)
        out, mag = oracle_rows(spec, workload.weights_arrays(spec), got[0].inv, rows)
        c = oracle.check_output(to_f64(got[0].out)[rows], out, mag, RTOL["f32"])
        assert c["ok"], c
    finally:
        f.release()
