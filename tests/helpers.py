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
