"""Shared helpers of the GPU tests: device buffers and invocation marshalling."""
import numpy as np

import oracle
import workload

RTOL = {"f32": 1e-5, "bf16": 2e-2}


def torch_mod():
    import torch
    return torch


def dev(a: np.ndarray):
    torch = torch_mod()
    assert a.dtype != np.float64, "device buffers of this library are never fp64"
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def tables_dev(spec):
    return dev(workload.tables_blob(spec))


def bf16_dev(values_f32: np.ndarray):
    """Device bf16 tensor holding exactly the given (bf16-representable) values."""
    torch = torch_mod()
    t = torch.from_numpy(np.ascontiguousarray(values_f32, dtype=np.float32))
    b = t.to(torch.bfloat16)
    assert torch.equal(b.float(), t), "values are not bf16-representable"
    return b.cuda()


def to_f64(t) -> np.ndarray:
    torch = torch_mod()
    return t.detach().to(torch.float64).cpu().numpy()


class DevInvocation:
    """One invocation's inputs on the device (+ an output buffer)."""

    def __init__(self, inv: dict):
        torch = torch_mod()
        self.inv = inv
        self.batch = int(inv["batch"])
        self.dense = dev(inv["dense"])
        self.offsets = dev(inv["offsets"])
        idx = inv["indices"] if inv["indices"].size else np.zeros(1, np.int32)
        self.indices = dev(idx)
        self.out = torch.full((max(1, self.batch),), float("nan"), dtype=torch.float32, device="cuda")

    def args(self):
        return (self.batch, self.dense.data_ptr(), self.indices.data_ptr(), self.offsets.data_ptr(),
                self.out.data_ptr())


def prepare(pool, spec, **kw):
    args = workload.prepare_kwargs(spec, fail_at_call=kw.pop("fail_at_call", 0),
                                   tables_in_host_memory=kw.pop("tables_in_host_memory", False))
    args.update(kw)
    return pool.prepare(**args)


def oracle_rows(spec, weights, inv, rows, n_threads=8):
    """Oracle outputs (out, out_mag) for the given sample rows of one invocation."""
    rows = np.asarray(rows)
    out = np.empty(rows.size)
    mag = np.empty(rows.size)
    src = lambda t, r: workload.table_rows(spec, t, r)
    # contiguous runs are computed together
    i = 0
    while i < rows.size:
        j = i
        while j + 1 < rows.size and rows[j + 1] == rows[j] + 1:
            j += 1
        res = oracle.forward(spec, weights, inv, row_source=src, b0=int(rows[i]), b1=int(rows[j]) + 1,
                             n_threads=n_threads, want_pooled=False)
        out[i:j + 1] = res["out"]
        mag[i:j + 1] = res["out_mag"]
        i = j + 1
    return out, mag


# ---------------------------------------------------------------- element-wise checks of intermediate buffers

def check_rounded_bag_sums(got, ref, mag, out_bits: int) -> dict:
    """Pooled bag sums against the oracle, with the bound that the arithmetic fixes.

    The kernels add a bag's rows in fp32 (any fixed order) and round the sum once to
    the output type: for bags of at most 128 rows the fp32 sum errs by at most
    127 * 2^-24 * mag <= 2^-17 * mag (mag = the sum of |terms|), and rounding to
    nearest with `out_bits` significand bits (bf16: 8, fp32: 24) adds at most
    2^-out_bits * |sum|.  So |got - ref| <= 2^-out_bits * |ref| + 2^-16 * mag.  For
    long bf16 bags this is far stricter than 2e-2 * mag, which most elements of a
    100-row bag with one row dropped would still meet."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mag = np.asarray(mag, dtype=np.float64)
    bound = 2.0 ** -out_bits * np.abs(ref) + 2.0 ** -16 * mag
    err = np.abs(got - ref)
    ok = err <= bound
    return {"ok": bool(ok.all()), "n": int(ok.size), "n_bad": int((~ok).sum()),
            "max_err_over_bound": float((err / np.where(bound > 0, bound, 1)).max()) if err.size else 0.0}


def oracle_pooled(spec, inv):
    """Oracle pooled bags [B, T*D] and magnitudes of one invocation (only referenced rows read)."""
    B = inv["batch"]
    tabs, idx, off = oracle.compact_tables(spec, inv, 0, B, lambda t, r: workload.table_rows(spec, t, r))
    return oracle.bag_sum(tabs, idx, off, B)


def oracle_bottom(spec, weights, dense):
    """Oracle bottom MLP output and magnitudes for dense rows [n, n_dense]."""
    h = np.asarray(dense, dtype=np.float64)
    m = np.abs(h)
    for l in range(len(spec.bot_dims)):
        W, b = weights[l]
        h, m = oracle.linear(h, W, b, relu=True, xmag=m)
    return h, m


def oracle_top0(spec, weights, concat, concat_mag, n_threads=8):
    """Oracle first top hidden layer ReLU(c V0^T + e0) and magnitudes, rows split over threads."""
    from concurrent.futures import ThreadPoolExecutor
    W, b = weights[len(spec.bot_dims)]
    n = concat.shape[0]
    cuts = np.linspace(0, n, n_threads + 1).astype(int)
    with ThreadPoolExecutor(n_threads) as ex:
        parts = list(ex.map(lambda k: oracle.linear(concat[cuts[k]:cuts[k + 1]], W, b, relu=True,
                                                    xmag=concat_mag[cuts[k]:cuts[k + 1]]), range(n_threads)))
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
