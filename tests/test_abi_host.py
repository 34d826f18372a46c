"""Host-side checks of the C ABI that need no GPU: the library loads, every
symbol declared in include/corank.h is exported, and argument validation
rejects bad calls before anything is launched."""
import ctypes
import os
import re

import pytest

from paper_1303_4312_gb300 import _lib

pytestmark = pytest.mark.host_only

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "corank.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cr_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1303_4312_gb300 import build
    build.build()
    return _lib.load()


def test_every_declared_symbol_exported(lib):
    names = declared_symbols()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def _header_declarations():
    """name -> (return type, [parameter types]) for every cr_* function
    declared in include/corank.h."""
    src = open(os.path.join(ROOT, "include", "corank.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for ret, name, params in re.findall(
            r"((?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?)\s*\b(cr_[a-z_0-9]+)\s*\(([^)]*)\)\s*;",
            src):
        ps = [q.strip() for q in params.split(",") if q.strip() and q.strip() != "void"]
        types = [re.sub(r"\s*\b[A-Za-z_][A-Za-z_0-9]*$", "", q) if not q.endswith("*")
                 else q for q in ps]
        out[name] = (ret.strip(), types)
    return out


def _c_kind(t):
    t = t.replace("const ", "").strip()
    if "*" in t or t == "cr_stream":
        return "ptr"
    return {"int": "i32", "int64_t": "i64", "size_t": "u64", "uint64_t": "u64",
            "cr_status": "i32"}[t]


def _ctypes_kind(ct):
    if ct is None:
        return "void"
    if ct in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(ct, ctypes._Pointer):
        return "ptr"
    if ct is ctypes.c_int:
        return "i32"
    if ctypes.sizeof(ct) == 8:
        return "u64" if ct(-1).value > 0 else "i64"
    raise AssertionError(ct)


def test_binding_signatures_match_header():
    """Every declaration's parameter kinds (pointer, int, int64, uint64 or
    size_t) and return kind equal the ctypes signature the binding uses."""
    decls = _header_declarations()
    assert set(decls) == set(declared_symbols())
    for name, (ret, params) in decls.items():
        argtypes, restype = _lib.SIGNATURES[name]
        want = [_c_kind(p) for p in params]
        got = [_ctypes_kind(a) for a in argtypes]
        assert got == want, (name, params)
        assert _ctypes_kind(restype) == _c_kind(ret), (name, ret)


def test_status_strings(lib):
    for code, name in _lib.STATUS.items():
        assert lib.cr_status_string(code).decode() == name
    assert lib.cr_status_string(99).decode() == "CR_UNKNOWN"
    assert lib.cr_abi_version() == 200


def test_tile_sizes(lib):
    for kt in range(8):
        for vb in (0, 4, 8):
            t = lib.cr_tile_size(kt, vb)
            assert t > 0 and t % 4 == 0
    assert lib.cr_tile_size(8, 0) == 0
    assert lib.cr_tile_size(0, 3) == 0


def _err(lib):
    return lib.cr_last_error().decode()


def test_validation_without_gpu(lib):
    A = ctypes.c_void_p(0x10000)     # never dereferenced: validation fails first
    # null with nonzero size
    assert lib.cr_stable_merge(0, None, 5, None, 0, None, None, None, 0, None) == 1
    assert "NULL" in _err(lib)
    # bad key type
    assert lib.cr_stable_merge(9, A, 1, A, 1, A, None, A, 1 << 20, None) == 1
    # negative size
    assert lib.cr_stable_merge(0, A, -1, A, 1, A, None, A, 1 << 20, None) == 1
    # misaligned: not a multiple of the 4-byte key size (4-byte offsets are fine)
    assert lib.cr_stable_merge(0, ctypes.c_void_p(0x10002), 4, A, 4, ctypes.c_void_p(0x20000),
                               None, A, 1 << 20, None) == 3
    assert "aligned to 4" in _err(lib)
    # 8-byte keys need 8-byte alignment; a 4-byte aligned payload array is fine for
    # 4-byte payloads but not for 8-byte ones
    assert lib.cr_stable_merge(3, ctypes.c_void_p(0x10004), 4, A, 4, ctypes.c_void_p(0x20000),
                               None, A, 1 << 20, None) == 3
    assert lib.cr_stable_merge_kv(0, 8, A, ctypes.c_void_p(0x30004), 4, ctypes.c_void_p(0x40000),
                                  ctypes.c_void_p(0x50000), 4, ctypes.c_void_p(0x60000),
                                  ctypes.c_void_p(0x70000), None, ctypes.c_void_p(0x80000),
                                  1 << 20, None) == 3
    # the workspace itself must stay 16-byte aligned
    assert lib.cr_stable_merge(0, ctypes.c_void_p(0x10004), 4, A, 4, ctypes.c_void_p(0x20000),
                               None, ctypes.c_void_p(0x50008), 1 << 20, None) == 3
    assert "workspace" in _err(lib)
    # sizes whose products with an element width or whose sum would overflow
    assert lib.cr_stable_merge(0, A, 1 << 62, A, 1 << 62, A, None, A, 1 << 20, None) == 1
    assert lib.cr_merge_pass(0, 0, A, None, (1 << 63) - 1, 2, A, None, A, 1 << 20, None) == 1
    # output overlaps input
    assert lib.cr_stable_merge(0, ctypes.c_void_p(0x10000), 64, ctypes.c_void_p(0x30000), 64,
                               ctypes.c_void_p(0x10040), None, ctypes.c_void_p(0x50000), 1 << 20,
                               None) == 2
    # workspace too small
    assert lib.cr_stable_merge(0, ctypes.c_void_p(0x10000), 64, ctypes.c_void_p(0x30000), 64,
                               ctypes.c_void_p(0x40000), None, ctypes.c_void_p(0x50000), 16,
                               None) == 4
    # payload width
    assert lib.cr_stable_merge_kv(0, 3, A, A, 1, A, A, 1, A, A, None, A, 1 << 20, None) == 1
    # rank out of range (host-result and device-result forms)
    i, j = ctypes.c_int64(-5), ctypes.c_int64(-5)
    assert lib.cr_co_rank(0, A, 4, A, 4, 9, ctypes.byref(i), ctypes.byref(j), None) == 1
    assert lib.cr_co_rank(0, A, 4, A, 4, -1, ctypes.byref(i), ctypes.byref(j), None) == 1
    assert lib.cr_co_rank(0, A, 4, A, 4, 2, None, ctypes.byref(j), None) == 1
    assert lib.cr_co_rank_async(0, A, 4, A, 4, 9, A, None) == 1
    assert lib.cr_co_rank_async(0, A, 4, A, 4, 2, ctypes.c_void_p(0x10004), None) == 3
    # trivial ranks are answered on the host without a launch: rank 0, rank m + n,
    # and every rank of a merge with one empty side
    for m, n, k, want in ((4, 4, 0, (0, 0)), (4, 4, 8, (4, 4)), (0, 7, 5, (0, 5)),
                          (7, 0, 5, (5, 0))):
        assert lib.cr_co_rank(0, A, m, A, n, k, ctypes.byref(i), ctypes.byref(j), None) == 0
        assert (i.value, j.value) == want
    # tags need m + n <= 2^32
    big = 1 << 31
    assert lib.cr_stable_merge(0, ctypes.c_void_p(0x1_0000_0000), big,
                               ctypes.c_void_p(0x4_0000_0000), big + 1,
                               ctypes.c_void_p(0x8_0000_0000), ctypes.c_void_p(0x10_0000_0000),
                               ctypes.c_void_p(0x20_0000_0000), 1 << 40, None) == 1
    assert "2^32" in _err(lib)
    # merge pass width
    assert lib.cr_merge_pass(0, 0, A, None, 10, 0, A, None, A, 1 << 20, None) == 1
    # nothing to do is fine
    assert lib.cr_stable_merge(0, None, 0, None, 0, None, None, None, 0, None) == 0


def test_workspace_sizes(lib):
    out = ctypes.c_size_t()
    t = lib.cr_tile_size(0, 0)
    assert lib.cr_merge_workspace_size(0, 0, 5 * t, 3 * t + 1, ctypes.byref(out)) == 0
    assert out.value == 256 + 32 * 9
    assert lib.cr_batched_workspace_size(0, 4, 10, 1000, 2000, ctypes.byref(out)) == 0
    t4 = lib.cr_tile_size_class(0, 4, 3)          # the batched class
    assert out.value == 256 + 32 * ((3000 + t4 - 1) // t4 + 10) + 8 * 11
    assert lib.cr_merge_pass_workspace_size(3, 4, 1 << 20, 1024, ctypes.byref(out)) == 0
    t8 = lib.cr_tile_size_class(3, 4, 4)          # the pass class
    assert out.value == 256 + 32 * ((1 << 20) // 2048) * ((2048 + t8 - 1) // t8)


def test_tile_shapes(lib):
    """Shapes are listed, selectable per (key size, payload width), reflected
    in cr_tile_size, and refused where they do not fit shared memory."""
    n = lib.cr_tile_shape_count()
    assert n >= 2
    nt, ipt, ilp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    shapes = []
    for s in range(n):
        assert lib.cr_tile_shape_info(s, ctypes.byref(nt), ctypes.byref(ipt), ctypes.byref(ilp)) == 0
        assert nt.value % 32 == 0 and ipt.value % 2 == 1 and ilp.value >= 1
        shapes.append(nt.value * ipt.value * ilp.value)
    assert lib.cr_tile_shape_info(n, ctypes.byref(nt), ctypes.byref(ipt), None) == 1
    for kt in range(4):
        for vb in (0, 4, 8):
            before = [lib.cr_get_tile_shape_for(kt, vb, c) for c in range(5)]
            assert all(0 <= b < n for b in before)
            try:
                for s in range(n):
                    st = lib.cr_set_tile_shape(kt, vb, s)
                    assert st in (0, 7)
                    if st == 0:
                        assert lib.cr_get_tile_shape(kt, vb) == s
                        assert lib.cr_tile_size(kt, vb) == shapes[s]
            finally:
                for c, b in enumerate(before):
                    assert lib.cr_set_tile_shape_for(kt, vb, c, b) == 0
    # the largest tiles do not fit 8-byte keys with 8-byte payloads and tags
    assert lib.cr_set_tile_shape(3, 8, 0) == 7
    assert lib.cr_get_tile_shape(9, 0) == -1


def test_geometry_classes(lib):
    """Balanced, skewed and small merges can use different shapes;
    cr_tile_size_for and the workspace size follow the class of (m, n)."""
    kt = 3  # uint64
    b0, s0 = lib.cr_get_tile_shape_for(kt, 0, 0), lib.cr_get_tile_shape_for(kt, 0, 1)
    m0 = lib.cr_get_tile_shape_for(kt, 0, 2)
    try:
        assert lib.cr_set_tile_shape_for(kt, 0, 0, 2) == 0
        assert lib.cr_set_tile_shape_for(kt, 0, 1, 3) == 0
        nt, ipt, ilp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib.cr_tile_shape_info(2, ctypes.byref(nt), ctypes.byref(ipt), ctypes.byref(ilp))
        t2 = nt.value * ipt.value * ilp.value
        lib.cr_tile_shape_info(3, ctypes.byref(nt), ctypes.byref(ipt), ctypes.byref(ilp))
        t3 = nt.value * ipt.value * ilp.value
        big = 1 << 23                                             # small-class limit
        assert lib.cr_tile_size_for(kt, 0, big, big) == t2
        assert lib.cr_tile_size_for(kt, 0, big, 16 * big) == t2  # 16*min == max: balanced
        assert lib.cr_tile_size_for(kt, 0, big, 16 * big + 1) == t3   # skewed
        assert lib.cr_tile_size_for(kt, 0, 16 * big + 1, big) == t3
        assert lib.cr_tile_size(kt, 0) == t2
        out = ctypes.c_size_t()
        assert lib.cr_merge_workspace_size(kt, 0, 10, 100 * big, ctypes.byref(out)) == 0
        assert out.value == 256 + 32 * ((100 * big + 10 + t3 - 1) // t3)
        # small merges (m + n <= 2^23) use the third class, whatever their ratio
        assert lib.cr_set_tile_shape_for(kt, 0, 2, 0) == 0
        lib.cr_tile_shape_info(0, ctypes.byref(nt), ctypes.byref(ipt), ctypes.byref(ilp))
        t0 = nt.value * ipt.value * ilp.value
        assert lib.cr_get_tile_shape_for(kt, 0, 2) == 0
        for m, n in ((1000, 1000), (10, 100000), (big // 2, big // 2), (0, big)):
            assert lib.cr_tile_size_for(kt, 0, m, n) == t0, (m, n)
        assert lib.cr_tile_size_for(kt, 0, big // 2, big // 2 + 1) == t2
        assert lib.cr_merge_workspace_size(kt, 0, 10, 100000, ctypes.byref(out)) == 0
        assert out.value == 256 + 32 * ((100010 + t0 - 1) // t0)
        # classes other than 0 .. 4 are refused
        assert lib.cr_set_tile_shape_for(kt, 0, 5, 0) == 1
        assert lib.cr_set_tile_shape_for(kt, 0, -1, 0) == 1
        assert lib.cr_get_tile_shape_for(kt, 0, 5) == -1
        assert lib.cr_tile_size_class(kt, 0, 5) == 0
    finally:
        lib.cr_set_tile_shape_for(kt, 0, 0, b0)
        lib.cr_set_tile_shape_for(kt, 0, 1, s0)
        lib.cr_set_tile_shape_for(kt, 0, 2, m0)


def test_batched_and_pass_classes(lib):
    """Batched calls and merge passes take shapes of their own (classes 3 and
    4): their workspace sizes follow those shapes, not the single-merge ones;
    a pass-class shape with payloads is limited to tiles of 4096 elements."""
    nt, ipt, ilp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    tiles = []
    for s in range(lib.cr_tile_shape_count()):
        lib.cr_tile_shape_info(s, ctypes.byref(nt), ctypes.byref(ipt), ctypes.byref(ilp))
        tiles.append(nt.value * ipt.value * ilp.value)
    kt, vb = 0, 4
    saved = [lib.cr_get_tile_shape_for(kt, vb, c) for c in range(5)]
    saved0 = [lib.cr_get_tile_shape_for(kt, 0, c) for c in range(5)]
    out = ctypes.c_size_t()
    try:
        assert lib.cr_set_tile_shape_for(kt, vb, 0, 0) == 0
        assert lib.cr_set_tile_shape_for(kt, vb, 3, 2) == 0
        assert lib.cr_set_tile_shape_for(kt, vb, 4, 3) == 0
        assert lib.cr_tile_size_class(kt, vb, 3) == tiles[2]
        assert lib.cr_tile_size_class(kt, vb, 4) == tiles[3]
        assert lib.cr_tile_size(kt, vb) == tiles[0]
        assert lib.cr_batched_workspace_size(kt, vb, 3, 10000, 5000, ctypes.byref(out)) == 0
        assert out.value == 256 + 32 * ((15000 + tiles[2] - 1) // tiles[2] + 3) + 8 * 4
        assert lib.cr_merge_pass_workspace_size(kt, vb, 100000, 4096, ctypes.byref(out)) == 0
        tpp = (8192 + tiles[3] - 1) // tiles[3]
        npairs = (100000 + 8191) // 8192
        last = 100000 - 8192 * (npairs - 1)
        assert out.value == 256 + 32 * ((npairs - 1) * tpp + (last + tiles[3] - 1) // tiles[3])
        big = [s for s, t in enumerate(tiles) if t > 4096]
        for s in big:
            if lib.cr_set_tile_shape_for(kt, vb, 0, s) == 0:     # fits this combination
                assert lib.cr_set_tile_shape_for(kt, vb, 4, s) == 7
                assert b"4096" in lib.cr_last_error()
                # setting every class leaves the pass class as it was
                assert lib.cr_set_tile_shape(kt, vb, s) == 0
                assert lib.cr_get_tile_shape_for(kt, vb, 4) == 3
                assert lib.cr_get_tile_shape_for(kt, vb, 3) == s
            # keys-only passes are not recorded: any fitting shape is fine
            if lib.cr_set_tile_shape_for(kt, 0, 0, s) == 0:
                assert lib.cr_set_tile_shape_for(kt, 0, 4, s) == 0
    finally:
        for c, s in enumerate(saved):
            lib.cr_set_tile_shape_for(kt, vb, c, s)
        for c, s in enumerate(saved0):
            lib.cr_set_tile_shape_for(kt, 0, c, s)


def test_recorded_pass_sizes_and_validation(lib):
    """cr_merge_pass_record_size and the argument checks of the recorded pass
    (all fail before any launch)."""
    ws, fw = ctypes.c_size_t(), ctypes.c_size_t()
    for code, vb in ((0, 4), (1, 8), (2, 4), (3, 4), (3, 8)):
        t = lib.cr_tile_size_class(code, vb, 4)
        assert t % 128 == 0 and t <= 4096
        for N, w in ((1 << 20, 1024), (1 << 20, 3000), (12345, 100), (7, 1 << 40), (5000, 1)):
            assert lib.cr_merge_pass_record_size(code, vb, N, w, ctypes.byref(ws),
                                                 ctypes.byref(fw)) == 0
            we = min(w, N)
            npairs = (N + 2 * we - 1) // (2 * we)
            tpp = (2 * we + t - 1) // t
            last = N - 2 * we * (npairs - 1)
            ntiles = (npairs - 1) * tpp + (last + t - 1) // t
            assert ws.value == 256 + 32 * ntiles
            assert fw.value == ntiles * (t // 32)
    # keys-only payload width, bad width, NULL outputs
    assert lib.cr_merge_pass_record_size(0, 0, 100, 10, ctypes.byref(ws), ctypes.byref(fw)) == 1
    assert lib.cr_merge_pass_record_size(0, 4, 100, 0, ctypes.byref(ws), ctypes.byref(fw)) == 1
    assert lib.cr_merge_pass_record_size(0, 4, 100, 10, None, ctypes.byref(fw)) == 1

    N, w = 4096, 256
    assert lib.cr_merge_pass_record_size(0, 4, N, w, ctypes.byref(ws), ctypes.byref(fw)) == 0
    X, Xv = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000)
    Y, Yv = ctypes.c_void_p(0x300000), ctypes.c_void_p(0x400000)
    F, WS = ctypes.c_void_p(0x500000), ctypes.c_void_p(0x600000)
    rec = lambda *a: lib.cr_merge_pass_record(*a)
    # keys only is refused (the record serves a payload backward)
    assert rec(0, 0, X, None, N, w, Y, None, F, fw.value, WS, ws.value, None) == 1
    # too few flag words / too small workspace
    assert rec(0, 4, X, Xv, N, w, Y, Yv, F, fw.value - 1, WS, ws.value, None) == 4
    assert rec(0, 4, X, Xv, N, w, Y, Yv, F, fw.value, WS, ws.value - 1, None) == 4
    # flags overlapping the output keys, or misaligned
    assert rec(0, 4, X, Xv, N, w, Y, Yv, ctypes.c_void_p(0x300100), fw.value, WS, ws.value,
               None) == 2
    assert rec(0, 4, X, Xv, N, w, Y, Yv, ctypes.c_void_p(0x500004), fw.value, WS, ws.value,
               None) == 3
    # NULL flags with words to write
    assert rec(0, 4, X, Xv, N, w, Y, Yv, None, fw.value, WS, ws.value, None) == 1
    bwd = lambda *a: lib.cr_merge_pass_backward_recorded(*a)
    G, GX = ctypes.c_void_p(0x700000), ctypes.c_void_p(0x800000)
    assert bwd(0, 4, N, w, F, fw.value - 1, G, GX, WS, ws.value, None) == 4
    assert bwd(0, 4, N, w, F, fw.value, G, ctypes.c_void_p(0x700100), WS, ws.value, None) == 2
    assert bwd(0, 0, N, w, F, fw.value, G, GX, WS, ws.value, None) == 1
    assert bwd(0, 4, N, 0, F, fw.value, G, GX, WS, ws.value, None) == 1
    # nothing to do is fine
    assert bwd(0, 4, 0, w, None, 0, None, None, None, 0, None) == 0


def test_recorded_run_sort_validation(lib):
    X, Xv = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000)
    Y, Yv = ctypes.c_void_p(0x300000), ctypes.c_void_p(0x400000)
    P = ctypes.c_void_p(0x500000)
    N = 5000
    # keys-only payload width, NULL perm, misaligned or overlapping perm
    assert lib.cr_sort_runs_record(0, 0, X, None, N, Y, None, P, None) == 1
    assert lib.cr_sort_runs_record(0, 4, X, Xv, N, Y, Yv, None, None) == 1
    assert lib.cr_sort_runs_record(0, 4, X, Xv, N, Y, Yv, ctypes.c_void_p(0x500001), None) == 3
    assert lib.cr_sort_runs_record(0, 4, X, Xv, N, Y, Yv, ctypes.c_void_p(0x300010), None) == 2
    assert lib.cr_sort_runs_record(9, 4, X, Xv, N, Y, Yv, P, None) == 1
    G, GX = ctypes.c_void_p(0x600000), ctypes.c_void_p(0x700000)
    assert lib.cr_sort_runs_backward_recorded(0, N, P, G, GX, None) == 1
    assert lib.cr_sort_runs_backward_recorded(4, -1, P, G, GX, None) == 1
    assert lib.cr_sort_runs_backward_recorded(4, N, P, G, ctypes.c_void_p(0x600100), None) == 2
    assert lib.cr_sort_runs_backward_recorded(4, 0, None, None, None, None) == 0


def test_merge_runs_block_validation(lib):
    """Widths: powers of two from 1 (run formation) to half the chunk; bad
    payload widths, a permutation without payloads, misaligned or overlapping
    arrays are refused before any launch."""
    X, Xv = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000)
    Y, Yv = ctypes.c_void_p(0x300000), ctypes.c_void_p(0x400000)
    P = ctypes.c_void_p(0x500000)
    N = 5000
    R = lib.cr_merge_runs_block_length()
    assert R == 4096
    for bad in (0, -1, 3, 6, 12, R, 2 * R):
        assert lib.cr_merge_runs_block(0, 4, X, Xv, N, bad, Y, Yv, P, None) == 1, bad
        assert b"width" in lib.cr_last_error()
    assert lib.cr_merge_runs_block(0, 2, X, Xv, N, 1, Y, Yv, P, None) == 1
    assert lib.cr_merge_runs_block(0, 0, X, None, N, 1, Y, None, P, None) == 1
    assert lib.cr_merge_runs_block(99, 4, X, Xv, N, 1, Y, Yv, P, None) == 1
    assert lib.cr_merge_runs_block(0, 4, X, Xv, -1, 1, Y, Yv, P, None) == 1
    assert lib.cr_merge_runs_block(0, 4, X, Xv, N, 1, ctypes.c_void_p(0x300002), Yv, P,
                                   None) == 3
    assert lib.cr_merge_runs_block(0, 4, X, Xv, N, 1, ctypes.c_void_p(0x100010), Yv, P,
                                   None) == 2
    assert lib.cr_merge_runs_block(0, 4, X, Xv, N, 1, Y, Yv, ctypes.c_void_p(0x300100),
                                   None) == 2
    assert b"overlap" in lib.cr_last_error()
    assert lib.cr_merge_runs_block(0, 4, X, Xv, 0, 1, Y, Yv, P, None) == 0
    assert lib.cr_last_error() == b""
    G, GX = ctypes.c_void_p(0x600000), ctypes.c_void_p(0x700000)
    assert lib.cr_merge_runs_block_backward_recorded(0, N, P, G, GX, None) == 1
    assert lib.cr_merge_runs_block_backward_recorded(4, N, P, G, ctypes.c_void_p(0x600100),
                                                     None) == 2
    assert lib.cr_merge_runs_block_backward_recorded(4, N, ctypes.c_void_p(0x500001), G, GX,
                                                     None) == 3
    assert lib.cr_merge_runs_block_backward_recorded(4, 0, None, None, None, None) == 0


def test_key_type_encodings(lib):
    """Float and descending key types: sizes follow the storage width, and
    unknown codes or flags are refused."""
    F32, F64, DESC = 4, 5, 256
    for code, width in ((F32, 4), (F64, 8), (0 | DESC, 4), (3 | DESC, 8), (F32 | DESC, 4),
                        (F64 | DESC, 8)):
        t = lib.cr_tile_size(code, 0)
        assert t == lib.cr_tile_size(0 if width == 4 else 3, 0) and t > 0, code
    for code in (6, 7, 6 | DESC, 7 | DESC):          # 32-bit key pairs in 64-bit words
        assert lib.cr_tile_size(code, 0) == lib.cr_tile_size(3, 0)
    for bad in (8, 255, 512, 8 | DESC, -1, 0x10000 | 0):
        assert lib.cr_tile_size(bad, 0) == 0, bad
        assert lib.cr_stable_merge(bad, None, 0, None, 0, None, None, None, 0, None) == 1
    from paper_1303_4312_gb300 import _lib as L
    assert L.key_code("f32:desc") == F32 | DESC and L.key_code("u64") == 3
    with pytest.raises(ValueError):
        L.key_code("f16")


def test_selftest_argument_checks(lib):
    WS = ctypes.c_void_p(0x100000)
    assert lib.cr_selftest_bounded_wait(None, 256, 1000, None, None) == 1
    assert lib.cr_selftest_bounded_wait(WS, 8, 1000, None, None) == 1
    assert lib.cr_selftest_bounded_wait(ctypes.c_void_p(0x100004), 256, 1000, None, None) == 1
    assert lib.cr_selftest_bounded_wait(WS, 256, 0, None, None) == 1
    assert lib.cr_selftest_bounded_wait(WS, 256, 10**9, None, None) == 1
    assert b"limit_ns" in lib.cr_last_error()


def test_check_sorted_argument_checks(lib):
    A, O, WS = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000), ctypes.c_void_p(0x300000)
    assert lib.cr_check_sorted(99, A, 10, O, WS, 16, None) == 1
    assert lib.cr_check_sorted(0, A, -1, O, WS, 16, None) == 1
    assert lib.cr_check_sorted(0, None, 10, O, WS, 16, None) == 1
    assert lib.cr_check_sorted(0, A, 10, None, WS, 16, None) == 1
    assert lib.cr_check_sorted(0, A, 10, O, WS, 8, None) == 1
    assert lib.cr_check_sorted(0, ctypes.c_void_p(0x100002), 10, O, WS, 16, None) == 3
    assert b"aligned" in lib.cr_last_error()


def test_dist_co_rank_argument_checks(lib):
    """The block-distributed co-rank calls refuse bad arguments before any
    launch (fake device addresses are never dereferenced)."""
    P = ctypes.c_void_p
    S, R, X = P(0x100000), P(0x200000), P(0x300000)
    assert lib.cr_dist_co_rank_init(-1, 5, R, 4, S, None) == 1
    assert lib.cr_dist_co_rank_init(5, 5, None, 4, S, None) == 1
    assert lib.cr_dist_co_rank_init(5, 5, P(0x200004), 4, S, None) == 3
    assert lib.cr_dist_co_rank_init(5, 5, R, -1, S, None) == 1
    assert lib.cr_dist_co_rank_init(5, 5, None, 0, None, None) == 0      # nothing to do
    assert lib.cr_dist_co_rank_probes(5, 5, S, 4, None, X, None) == 1
    assert lib.cr_dist_co_rank_probes(5, 5, S, 4, X, P(0x400002), None) == 3
    assert lib.cr_dist_co_rank_answer(99, X, 0, 10, R, 4, S, None) == 1
    assert lib.cr_dist_co_rank_answer(0, X, 10, 5, R, 4, S, None) == 1      # hi < lo
    assert lib.cr_dist_co_rank_answer(0, None, 0, 10, R, 4, S, None) == 1
    assert lib.cr_dist_co_rank_answer(3, P(0x300004), 0, 10, R, 4, S, None) == 3
    assert lib.cr_dist_co_rank_answer(0, None, 7, 7, R, 0, S, None) == 0
    assert lib.cr_dist_co_rank_step(99, 5, 5, R, X, S, 4, None) == 1
    assert lib.cr_dist_co_rank_step(0, 5, 5, None, X, S, 4, None) == 1
    assert lib.cr_dist_co_rank_result(S, 4, R, X, None, None) == 1
    assert lib.cr_dist_co_rank_result(S, 4, R, X, P(0x500004), None) == 3
