"""The allocation-free stable merge, cr_stable_merge_noalloc.

Some callers cannot allocate device memory (a plug-in given only its input
and output buffers, a real-time loop that must not enter an allocator, code
running while its host framework owns every allocation).  For them the
library keeps the merge's tile table in a fixed array inside its device image
instead of a caller workspace.  These tests call that entry point through the
C ABI and check it bit for bit against the CPU oracle's stable merge (keys and
source tags) and against the workspace-based cr_stable_merge, on calls in a
row that reuse the array: a merge with more tiles than the small-merge
partition handles, then a small merge with a smaller tile right after it,
then 8-byte keys from offset views.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1303_4312_gb300 import _lib, build

MAX_TILES = (4 * 2**20 - 256) // 32


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


@pytest.mark.host_only
def test_noalloc_rejects_oversize_without_gpu(lib):
    """Beyond the array's capacity the call is refused before any launch.
    The sizes exceed the capacity under every tile shape the library offers
    (MAX_TILES times the largest TILE), so the refusal does not depend on
    which shape the call's geometry selects; sizes near 2^63, whose sum or
    tile count would overflow, are refused the same way."""
    nt, ipt, ilp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    largest = 0
    for s in range(lib.cr_tile_shape_count()):
        assert lib.cr_tile_shape_info(s, ctypes.byref(nt), ctypes.byref(ipt), ctypes.byref(ilp)) == 0
        largest = max(largest, nt.value * ipt.value * ilp.value)
    too_many = MAX_TILES * largest + 1
    i64max = 2**63 - 1
    for code, (m, n) in ((0, (too_many, 0)), (0, (too_many // 2, too_many // 2 + 1)),
                         (3, (too_many, 0)), (3, (1, too_many)), (0, (i64max - 1, 0)),
                         (0, (0, i64max)), (3, (2**62, 2**62)), (0, (i64max, i64max))):
        st = lib.cr_stable_merge_noalloc(code, ctypes.c_void_p(0x1_0000_0000), m,
                                         ctypes.c_void_p(0x10_0000_0000), n,
                                         ctypes.c_void_p(0x20_0000_0000), None, None)
        assert st == 1, (code, m, n)
        assert "scratch" in lib.cr_last_error().decode()
    # pointers need only their element alignment; a 2-byte offset of 4-byte
    # keys is refused
    assert lib.cr_stable_merge_noalloc(0, ctypes.c_void_p(0x1_0000_0002), 8,
                                       ctypes.c_void_p(0x10_0000_0000), 8,
                                       ctypes.c_void_p(0x20_0000_0000), None, None) == 3


def _merge_both(lib, A, B, code, tag):
    """Same merge through cr_stable_merge (with a workspace) and through
    cr_stable_merge_noalloc; returns both outputs (and tags)."""
    m, n = A.numel(), B.numel()
    dev = A.device
    s = torch.cuda.current_stream(dev).cuda_stream
    C1 = torch.empty(m + n, dtype=A.dtype, device=dev)
    C2 = torch.full((m + n,), -1, dtype=A.dtype, device=dev)
    T1 = torch.empty(m + n, dtype=torch.int32, device=dev) if tag else None
    T2 = torch.full((m + n,), -1, dtype=torch.int32, device=dev) if tag else None
    need = ctypes.c_size_t()
    _lib.check(lib.cr_merge_workspace_size(code, 0, m, n, ctypes.byref(need)))
    ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=dev)
    p = lambda t: None if t is None else t.data_ptr()
    _lib.check(lib.cr_stable_merge(code, A.data_ptr(), m, B.data_ptr(), n, C1.data_ptr(), p(T1),
                                   ws.data_ptr(), ws.numel(), s))
    _lib.check(lib.cr_stable_merge_noalloc(code, A.data_ptr(), m, B.data_ptr(), n,
                                           C2.data_ptr(), p(T2), s))
    torch.cuda.synchronize()
    return C1, C2, T1, T2


def _host(t, dt):
    return t.cpu().numpy().view(dt)


@pytest.mark.gpu
def test_noalloc_matches_oracle_on_calls_in_a_row(lib):
    g = torch.Generator(device="cuda").manual_seed(1234)
    # call 1: more tiles than the small-merge partition covers (> 4096 under
    # every tile shape), int32 keys, keys only
    m, n = 2**25 + 77, 2**25 - 5
    assert (m + n) // lib.cr_tile_size_for(0, 0, m, n) > 4096
    A = torch.sort(torch.randint(-2**31, 2**31 - 1, (m,), generator=g, device="cuda",
                                 dtype=torch.int32)).values
    B = torch.sort(torch.randint(-2**31, 2**31 - 1, (n,), generator=g, device="cuda",
                                 dtype=torch.int32)).values
    C1, C2, _, _ = _merge_both(lib, A, B, 0, tag=False)
    want, _ = oracle.merge(_host(A, np.int32), _host(B, np.int32))
    assert np.array_equal(_host(C2, np.int32), want)
    assert torch.equal(C1, C2)
    del A, B, C1, C2, want
    # call 2, right after: a small merge (m + n <= 2^23: the small geometry
    # class, with its own tile shape) with heavy duplicates and source tags,
    # so a stale table left by call 1 in the shared array would show up as
    # wrong output
    A = torch.sort(torch.randint(0, 1000, (3_000_001,), generator=g, device="cuda",
                                 dtype=torch.int32)).values
    B = torch.sort(torch.randint(0, 1000, (2_500_003,), generator=g, device="cuda",
                                 dtype=torch.int32)).values
    C1, C2, T1, T2 = _merge_both(lib, A, B, 0, tag=True)
    want, src = oracle.merge(_host(A, np.int32), _host(B, np.int32))
    assert np.array_equal(_host(C2, np.int32), want)
    assert np.array_equal(_host(T2, np.uint32).astype(np.int64), src)
    assert torch.equal(C1, C2) and torch.equal(T1, T2)
    # call 3: 8-byte signed keys from offset views (an array start that is
    # only 8-byte aligned), fewer tiles again
    A = torch.sort(torch.randint(-2**62, 2**62, (70_002,), generator=g, device="cuda",
                                 dtype=torch.int64)).values[1:]
    B = torch.sort(torch.randint(-2**62, 2**62, (123_458,), generator=g, device="cuda",
                                 dtype=torch.int64)).values[1:]
    assert A.data_ptr() % 16 == 8 and B.data_ptr() % 16 == 8
    C1, C2, _, _ = _merge_both(lib, A, B, 2, tag=False)
    want, _ = oracle.merge(_host(A, np.int64), _host(B, np.int64))
    assert np.array_equal(_host(C2, np.int64), want)
    assert torch.equal(C1, C2)
