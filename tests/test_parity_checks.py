"""The element-wise checks of the full-size parity tests catch the mistakes they are
meant to catch (CPU only): a bag row dropped or counted twice, a whole bag missing,
a column shifted.  A plain model of the kernels' arithmetic (fp32 sums of the rows
in index order, one rounding to the output type) must pass; the same model with one
planted mistake must fail.  The oracle's bag sums are the plain definition (the
per-invocation result that read-only sharing must reproduce, Sec. 6.2)."""
import numpy as np
import pytest

import oracle
import workload
from helpers import RTOL, check_rounded_bag_sums, oracle_pooled


def _round_bf16(x32: np.ndarray) -> np.ndarray:
    """Round fp32 values to bf16 (nearest, ties to even), widened back to fp32."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _model_pooled(spec, inv, drop=None, dup=None, skip_bag=None):
    """fp32 bag sums in index order (the kernels' arithmetic up to the order of the
    adds), optionally with a planted mistake: drop / dup = (t, b) loses or repeats
    that bag's first row, skip_bag = (t, b) leaves that bag out."""
    B, T, D = inv["batch"], spec.n_tables, spec.dim
    out = np.zeros((B, T * D), np.float32)
    for t in range(T):
        for b in range(B):
            lo, hi = int(inv["offsets"][t * B + b]), int(inv["offsets"][t * B + b + 1])
            rows = list(inv["indices"][lo:hi])
            if (t, b) == drop:
                rows = rows[1:]
            if (t, b) == dup:
                rows = rows + rows[:1]
            if (t, b) == skip_bag:
                rows = []
            vals = workload.table_rows(spec, t, np.array(rows, dtype=np.int64)) if rows else np.zeros((0, D))
            s = np.zeros(D, np.float32)
            for v in vals:
                s = (s + v.astype(np.float32)).astype(np.float32)
            out[b, t * D:(t + 1) * D] = s
    return _round_bf16(out) if spec.dtype == "bf16" else out


@pytest.fixture(scope="module", params=["bf16", "f32"])
def case(request):
    dt = request.param
    dim = 128 if dt == "bf16" else 64
    spec = workload.FunctionSpec(key="pc_" + dt, dtype=dt, rows=[5000, 3000], dim=dim, bot_dims=[64, 64],
                                 top_dims=[64, 1], alpha=1.1, l_min=60, l_max=100)
    inv = workload.make_invocation(spec, 24, seed=5)
    ref, mag = oracle_pooled(spec, inv)
    return spec, inv, ref, mag


def _bits(spec):
    return 8 if spec.dtype == "bf16" else 24


def test_the_kernels_arithmetic_passes(case):
    spec, inv, ref, mag = case
    got = _model_pooled(spec, inv)
    c = check_rounded_bag_sums(got, ref, mag, _bits(spec))
    assert c["ok"], c
    assert oracle.check_close(got, ref, mag, RTOL[spec.dtype])["ok"]


@pytest.mark.parametrize("mistake", ["drop", "dup", "skip_bag"])
def test_a_planted_bag_mistake_fails(case, mistake):
    spec, inv, ref, mag = case
    got = _model_pooled(spec, inv, **{mistake: (1, 7)})
    c = check_rounded_bag_sums(got, ref, mag, _bits(spec))
    assert not c["ok"], (mistake, c)
    # the failures sit in bag (1, 7) alone
    bad = np.abs(got - ref) > 2.0 ** -_bits(spec) * np.abs(ref) + 2.0 ** -16 * mag
    rows, cols = np.nonzero(bad)
    assert set(rows.tolist()) == {7} and cols.min() >= spec.dim and cols.max() < 2 * spec.dim


def test_a_shifted_column_fails(case):
    spec, inv, ref, mag = case
    got = _model_pooled(spec, inv)
    got[:, 3], got[:, 4] = got[:, 4].copy(), got[:, 3].copy()
    assert not check_rounded_bag_sums(got, ref, mag, _bits(spec))["ok"]
