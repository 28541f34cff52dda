"""The C-ABI library loads and exports every entry point include/sage.h declares (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sage.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sage_status|const char\*|int64_t|int)\s+(sage_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libsage():
    from paper_2404_14691_b300 import build
    build.build()
    from paper_2404_14691_b300 import _native
    return _native.lib()


# The boundary's calls: the paper's programming model (SageInit / SageRun /
# SageLoadToGPU, Sec. 4.2 and Sec. 5.2) and release (Sec. 6.3), plus the fused batch.
BOUNDARY = ("sage_pool_create", "sage_prepare", "sage_invoke", "sage_invoke_batch", "sage_wait",
            "sage_release", "sage_pool_destroy", "sage_pool_stats", "sage_last_error")


def _comment_before(name):
    """The comment block that precedes the declaration of `name` in the header."""
    src = open(HEADER).read()
    m = re.search(r"/\*((?:(?!\*/).)*)\*/\s*(?:sage_status|const char\*|int64_t|int)\s+%s\s*\(" % name, src,
                  flags=re.S)
    assert m, name
    return m.group(1)


def test_header_declares_the_boundary():
    names = _declared()
    for n in BOUNDARY + ("sage_embedding_bag_sum", "sage_linear", "sage_invoke_noalloc"):
        assert n in names, n


def test_every_boundary_call_cites_its_passage():
    """Each call of the boundary names the paper's section it implements, or says
    that the paper has no counterpart."""
    for n in BOUNDARY:
        c = _comment_before(n)
        assert re.search(r"Sec\. \d\.\d", c) or "no counterpart" in c, n


def test_library_exports_every_declared_symbol(libsage):
    for n in _declared():
        assert hasattr(libsage, n), n
        assert isinstance(getattr(libsage, n), ctypes._CFuncPtr)


def test_binding_declares_signatures_for_every_symbol(libsage):
    from paper_2404_14691_b300 import _native
    bound = {name for name, _, _ in _native.SIGNATURES}
    assert bound == set(_declared())


def test_exported_symbols_are_c_linkage(libsage):
    from paper_2404_14691_b300 import _native
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in _declared():
        assert n in syms, n


def test_ctypes_struct_sizes_match_the_header():
    """Compile a tiny C program against include/sage.h and compare sizeof/offsetof."""
    from paper_2404_14691_b300 import _native as N
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "sage.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(sage_pool_config), sizeof(sage_data_desc),
         sizeof(sage_fn_desc), sizeof(sage_invocation), sizeof(sage_host_invocation), sizeof(sage_pool_stats_t),
         offsetof(sage_fn_desc, weights), sizeof(sage_kernel_time), sizeof(sage_share_stats),
         offsetof(sage_pool_config, exportable), sizeof(sage_serve_config));
  return 0;
}
'''
    tmp = os.path.join("/tmp", "sage_abi_%d" % os.getpid())
    with open(tmp + ".c", "w") as f:
        f.write(prog)
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", tmp, tmp + ".c"])
    got = [int(x) for x in subprocess.check_output([tmp]).split()]
    want = [ctypes.sizeof(N.PoolConfig), ctypes.sizeof(N.DataDesc), ctypes.sizeof(N.FnDesc),
            ctypes.sizeof(N.Invocation), ctypes.sizeof(N.HostInvocation), ctypes.sizeof(N.PoolStats),
            N.FnDesc.weights.offset, ctypes.sizeof(N.KernelTime), ctypes.sizeof(N.ShareStats),
            N.PoolConfig.exportable.offset, ctypes.sizeof(N.ServeConfig)]
    assert got == want
    os.remove(tmp)
    os.remove(tmp + ".c")


def test_calls_without_gpu_fail_cleanly(libsage):
    """With no GPU visible, pool creation returns an error status (no crash)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    h = ctypes.c_void_p()
    st = libsage.sage_pool_create(None, ctypes.byref(h))
    assert st == -3
    assert libsage.sage_last_error()


def test_noalloc_refuses_misaligned_pointers_before_any_cuda_call(libsage):
    """With no GPU visible: the no-allocation entry point checks pointer alignment
    on the host before it makes any CUDA call, so a misaligned tables pointer is
    refused with SAGE_ERR_INVALID (not SAGE_ERR_CUDA)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible (the GPU test of the same refusal uses real buffers)")
    from paper_2404_14691_b300 import _native as N
    rows = (ctypes.c_int64 * 2)(100, 100)
    bot = (ctypes.c_int * 1)(16)
    top = (ctypes.c_int * 1)(1)
    empty = N.DataDesc(None, 0, 0, None, None, None)
    d = N.FnDesc(b"abi_na", 0, 2, rows, 16, 4, 1, bot, 1, top, 0, 0, empty, empty)
    inv = N.Invocation(4, 1 << 20, 1 << 20, 1 << 20, 1 << 20, 0)
    st = libsage.sage_invoke_noalloc(ctypes.byref(d), (1 << 20) + 16, 1 << 20, ctypes.byref(inv), None)
    assert st == -1
    assert b"aligned" in libsage.sage_last_error()
