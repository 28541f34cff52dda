"""Host side of cross-process sharing, no GPU: the attach request is sent before
any CUDA call (the function process may not have a context yet), and requests
that cannot be sent are refused with SAGE_ERR_INVALID."""
import os
import socket
import struct
import tempfile

import pytest

import workload

sage = pytest.importorskip("paper_2404_14691_b300")

# the first message: magic, type, status, nfd, 4 x u64, uuid[16], key[256], sig[4096]
MSG = struct.Struct("<Iiii4Q16s256s4096s")


def _spec():
    return workload.spec_tiny(key="share_host", dtype="f32", n_tables=3, rows=1000, dim=16, bot=(32, 16),
                              top=(32, 1))


def test_attach_begin_sends_the_request_without_a_gpu():
    path = os.path.join(tempfile.mkdtemp(), "owner.sock")
    srv = socket.socket(socket.AF_UNIX, socket.SOCK_SEQPACKET)
    srv.bind(path)
    srv.listen(1)
    try:
        spec = _spec()
        t = sage.attach_begin(path, **workload.prepare_kwargs(spec))
        conn, _ = srv.accept()
        data = conn.recv(MSG.size + 16)
        assert len(data) == MSG.size                     # one whole message
        magic, typ, status, nfd, tb, wb, tm, wm, uuid, key, sig = MSG.unpack(data)
        assert magic == 0x45474153 and typ == 1 and nfd == 0
        assert key.rstrip(b"\0").decode() == spec.key
        s = sig.rstrip(b"\0").decode()
        # the signature carries the shape and both item sizes
        assert s.endswith("|%d|%d" % (spec.table_bytes(), workload.prepare_kwargs(spec)["weights_bytes"]))
        assert ",".join(str(r) for r in spec.rows) in s
        conn.close()
        t.cancel()                                       # never completed (no GPU here)
    finally:
        srv.close()
        os.unlink(path)


def test_attach_begin_refusals():
    spec = _spec()
    kw = workload.prepare_kwargs(spec)
    missing = os.path.join(tempfile.mkdtemp(), "nobody.sock")
    with pytest.raises(sage.SageError) as e:
        sage.attach_begin(missing, **kw)                 # no owner listening
    assert e.value.status == -1
    with pytest.raises(sage.SageError) as e:
        sage.attach_begin("/tmp/" + "x" * 200, **kw)     # longer than a UNIX socket path
    assert e.value.status == -1
    bad = dict(kw)
    bad["top_dims"] = [32, 2]                            # the head must have one output
    with pytest.raises(sage.SageError) as e:
        sage.attach_begin(missing, **bad)
    assert e.value.status == -1
