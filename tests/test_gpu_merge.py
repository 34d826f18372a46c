"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element and bit for bit, on seeded inputs that span several tiles
with ragged tails, heavy ties, signed/unsigned orders and empty inputs."""
import numpy as np
import pytest
import torch

import oracle
import paper_1303_4312_gb300 as cr
from gpu_util import dev, host, key_type, restore_shapes, same_bits, save_shapes, sorted_keys

pytestmark = pytest.mark.gpu

KEY_DTYPES = [np.int32, np.uint32, np.int64, np.uint64]


def sizes_for(dt, vb=0):
    # the tile of the small single merges built here (geometry class "small")
    t = cr.tile_size(key_type(np.empty(0, dt)), vb, 1, 1)
    return [(0, 0), (1, 0), (0, 1), (1, 1), (3, 5), (17, 0), (0, 29), (t - 1, 1), (t, t),
            (2 * t + 3, t - 5), (5 * t + 11, 7), (7, 4 * t + 9), (1000, 3 * t + 777)]


@pytest.mark.parametrize("dt", KEY_DTYPES)
def test_merge_keys_and_tags(dt):
    rng = np.random.default_rng(100)
    for m, n in sizes_for(dt):
        for spread in (None, 3, 1000):
            A = sorted_keys(rng, m, dt, spread)
            B = sorted_keys(rng, n, dt, spread)
            C, T = cr.merge(dev(A), dev(B), key_type=key_type(A), tag=True)
            torch.cuda.synchronize()
            want, src = oracle.merge(A, B)
            assert same_bits(host(C, dt), want), (m, n, spread)
            assert np.array_equal(host(T, np.uint32).astype(np.int64), src), (m, n, spread)


@pytest.mark.parametrize("dt", KEY_DTYPES)
def test_special_orders(dt):
    """All keys equal; A entirely below B; B entirely below A."""
    t = cr.tile_size(key_type(np.empty(0, dt)), 0, 1, 1)
    m, n = 3 * t + 5, 2 * t + 9
    info = np.iinfo(dt)
    cases = [
        (np.full(m, 7, dt), np.full(n, 7, dt)),
        (np.arange(m).astype(dt), (np.arange(n) + m).astype(dt)),
        ((np.arange(m) + n).astype(dt), np.arange(n).astype(dt)),
        (np.full(m, info.max, dt), np.full(n, info.min, dt)),
    ]
    for A, B in cases:
        C, T = cr.merge(dev(A), dev(B), key_type=key_type(A), tag=True)
        torch.cuda.synchronize()
        want, src = oracle.merge(A, B)
        assert same_bits(host(C, dt), want)
        assert np.array_equal(host(T, np.uint32).astype(np.int64), src)


@pytest.mark.parametrize("dt", KEY_DTYPES)
@pytest.mark.parametrize("vdt", [np.float32, np.float64])
def test_merge_kv_and_backward(dt, vdt):
    rng = np.random.default_rng(101)
    vb = np.dtype(vdt).itemsize
    for m, n in sizes_for(dt, vb):
        A = sorted_keys(rng, m, dt, 50)
        B = sorted_keys(rng, n, dt, 50)
        Av = rng.standard_normal(m).astype(vdt)
        Bv = rng.standard_normal(n).astype(vdt)
        kt = key_type(A)
        Ck, Cv, T = cr.merge_kv(dev(A), dev(Av), dev(B), dev(Bv), key_type=kt, tag=True)
        gC = rng.standard_normal(m + n).astype(vdt)
        gA, gB = cr.merge_kv_backward(dev(A), dev(B), dev(gC), key_type=kt)
        torch.cuda.synchronize()
        wk, wv, src = oracle.merge_kv(A, Av, B, Bv)
        ga, gb = oracle.merge_grad(A, B, gC)
        assert same_bits(host(Ck, dt), wk), (m, n)
        assert same_bits(host(Cv, vdt), wv), (m, n)
        assert np.array_equal(host(T, np.uint32).astype(np.int64), src)
        assert same_bits(host(gA, vdt), ga), (m, n)
        assert same_bits(host(gB, vdt), gb), (m, n)


def test_payload_bits_nan_and_signed_zero():
    A = np.array([1, 2, 2, 5] * 1000, np.uint32)
    A.sort()
    B = np.array([0, 2, 9] * 1000, np.uint32)
    B.sort()
    rng = np.random.default_rng(7)
    Av = rng.integers(0, 2**32, len(A), dtype=np.uint32)
    Av[::3] = 0x7FC00001   # NaN payload
    Av[1::3] = 0x80000000  # -0.0
    Bv = rng.integers(0, 2**32, len(B), dtype=np.uint32)
    Ck, Cv = cr.merge_kv(dev(A), dev(Av.view(np.float32)), dev(B), dev(Bv.view(np.float32)),
                         key_type="u32")
    torch.cuda.synchronize()
    _, wv, _ = oracle.merge_kv(A, Av, B, Bv)
    assert same_bits(host(Cv, np.uint32), wv)


@pytest.mark.parametrize("dt", KEY_DTYPES)
def test_co_rank_every_rank(dt):
    """co_rank_many for every rank of several shapes equals Algorithm 1 on the host."""
    rng = np.random.default_rng(102)
    for m, n in [(0, 0), (0, 9), (9, 0), (1, 1), (37, 53), (1000, 3), (3000, 2500)]:
        for spread in (None, 2):
            A = sorted_keys(rng, m, dt, spread)
            B = sorted_keys(rng, n, dt, spread)
            ranks = np.arange(-2, m + n + 3, dtype=np.int64)
            oi, oj = cr.co_rank_many(dev(A), dev(B), torch.from_numpy(ranks).cuda(),
                                     key_type=key_type(A))
            wj, wk = oracle.co_rank_many(A, B, ranks)
            assert np.array_equal(oi.cpu().numpy(), wj)
            assert np.array_equal(oj.cpu().numpy(), wk)
            if m + n:
                r = int(rng.integers(0, m + n + 1))
                assert cr.co_rank(dev(A), dev(B), r, key_type=key_type(A)) == \
                    tuple(oracle.co_rank(r, A, B)[:2])


def test_co_rank_figure2_on_gpu():
    """The paper's Figure 2 example, through the C ABI."""
    from conftest import read_golden
    rows = {r[0]: r[1:] for r in read_golden("figure1.txt")}
    A = np.array([int(x) for x in rows["A"]], np.int32)
    B = np.array([int(x) for x in rows["B"]], np.int32)
    assert cr.co_rank(dev(A), dev(B), 22) == (12, 10)
    C = cr.merge(dev(A), dev(B))
    want = np.array([int(x) for x in rows["C"]], np.int32)
    assert np.array_equal(C.cpu().numpy(), want)


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
@pytest.mark.parametrize("vdt", [None, np.float32, np.float64])
def test_batched(dt, vdt):
    rng = np.random.default_rng(103)
    nseg = 300
    ms = np.floor(np.exp2(rng.random(nseg) * 13)).astype(np.int64)
    ns = np.floor(np.exp2(rng.random(nseg) * 13)).astype(np.int64)
    ms[::11] = 0
    ns[::7] = 0
    ms[5] = ns[5] = 0
    a_off = np.concatenate([[0], np.cumsum(ms)])
    b_off = np.concatenate([[0], np.cumsum(ns)])
    A = np.concatenate([sorted_keys(rng, x, dt, 40) for x in ms])
    B = np.concatenate([sorted_keys(rng, x, dt, 40) for x in ns])
    Av = rng.standard_normal(len(A)).astype(vdt or np.float32)
    Bv = rng.standard_normal(len(B)).astype(vdt or np.float32)
    kt = key_type(A)
    Ck, Cv = cr.batched_merge_kv(a_off, b_off, dev(A), dev(Av) if vdt else None, dev(B),
                                 dev(Bv) if vdt else None, key_type=kt)
    torch.cuda.synchronize()
    wk, wv = oracle.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
    assert same_bits(host(Ck, dt), wk)
    if vdt:
        assert same_bits(host(Cv, vdt), wv)
        gC = rng.standard_normal(len(A) + len(B)).astype(vdt)
        gA, gB = cr.batched_merge_kv_backward(a_off, b_off, dev(A), dev(B), dev(gC), key_type=kt)
        torch.cuda.synchronize()
        ga, gb = oracle.batched_merge_grad(a_off, b_off, A, B, gC)
        assert same_bits(host(gA, vdt), ga)
        assert same_bits(host(gB, vdt), gb)


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
def test_batched_segments_across_partition_blocks(dt):
    """Segments whose tiles span several blocks of the batched partition (a
    block owns 255 tiles and takes the end of its last tile from the next
    block's first co-rank), a lone segment, segments of exactly 255 tiles,
    and a table of empty segments only: keys, payloads and gradients equal
    the oracle's."""
    rng = np.random.default_rng(109)
    kt = key_type(np.empty(0, dt))
    t = cr.tile_size(kt, 4, cls="batched")  # batched calls use their own class
    cases = [
        ([255 * t // 2 + 7, 3, 600 * t // 2], [255 * t // 2 - 5, 0, 600 * t // 2 + 11]),
        ([5 * t + 1], [7 * t - 3]),
        ([0, 255 * t, 0, 1], [1, 0, 255 * t, 0]),
        ([0, 0, 0], [0, 0, 0]),
    ]
    for ms, ns in cases:
        ms, ns = np.array(ms, np.int64), np.array(ns, np.int64)
        a_off = np.concatenate([[0], np.cumsum(ms)])
        b_off = np.concatenate([[0], np.cumsum(ns)])
        A = np.concatenate([sorted_keys(rng, int(x), dt, 900) for x in ms])
        B = np.concatenate([sorted_keys(rng, int(x), dt, 900) for x in ns])
        Av = rng.standard_normal(len(A)).astype(np.float32)
        Bv = rng.standard_normal(len(B)).astype(np.float32)
        Ck, Cv = cr.batched_merge_kv(a_off, b_off, dev(A), dev(Av), dev(B), dev(Bv),
                                     key_type=kt)
        gC = rng.standard_normal(len(A) + len(B)).astype(np.float32)
        gA, gB = cr.batched_merge_kv_backward(a_off, b_off, dev(A), dev(B), dev(gC),
                                              key_type=kt)
        torch.cuda.synchronize()
        wk, wv = oracle.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
        ga, gb = oracle.batched_merge_grad(a_off, b_off, A, B, gC)
        assert same_bits(host(Ck, dt), wk), (list(ms), list(ns))
        assert same_bits(host(Cv, np.float32), wv), (list(ms), list(ns))
        assert same_bits(host(gA, np.float32), ga) and same_bits(host(gB, np.float32), gb)


def test_batched_bad_table_reports():
    A = np.arange(100, dtype=np.int32)
    B = np.arange(100, dtype=np.int32)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    for a_off in ([0, 50, 40, 100], [0, 50, 60, 101], [1, 50, 60, 100]):
        cr.batched_merge_kv(a_off, [0, 30, 60, 100], dev(A), None, dev(B), None, ws=ws)
        with pytest.raises(cr.CorankError) as e:
            cr.workspace_status(ws)
        assert e.value.name == "CR_EBADSEG"
    cr.batched_merge_kv([0, 50, 60, 100], [0, 30, 60, 100], dev(A), None, dev(B), None, ws=ws)
    cr.workspace_status(ws)


@pytest.mark.parametrize("N,w", [(1, 1), (10, 4), (5000, 16), (3 * 3840 + 5, 1024),
                                 (40000, 3000), (65536, 1024)])
def test_merge_pass_and_backward(N, w):
    rng = np.random.default_rng(104)
    X = rng.integers(0, 20, N).astype(np.uint64) * np.uint64(1 << 62)
    for a0 in range(0, N, w):
        X[a0:a0 + w].sort(kind="stable")
    Xv = rng.standard_normal(N).astype(np.float32)
    Y, Yv = cr.merge_pass(dev(X), dev(Xv), w, key_type="u64")
    gY = rng.standard_normal(N).astype(np.float32)
    gX = cr.merge_pass_backward(dev(X), dev(gY), w, key_type="u64")
    torch.cuda.synchronize()
    wy, wyv, src = oracle.merge_pass(X, Xv, w)
    assert same_bits(host(Y, np.uint64), wy)
    assert same_bits(host(Yv, np.float32), wyv)
    want = np.empty_like(gY)
    want[src] = gY
    assert same_bits(host(gX, np.float32), want)


def test_status_ok_after_calls():
    A = dev(np.arange(10000, dtype=np.int32))
    B = dev(np.arange(7000, dtype=np.int32))
    ws = torch.empty(cr.api.merge_workspace_bytes("i32", 0, 10000, 7000), dtype=torch.uint8,
                     device="cuda")
    cr.merge(A, B, ws=ws)
    cr.workspace_status(ws)


def test_argument_errors_on_device():
    A = torch.arange(64, dtype=torch.int32, device="cuda")
    B = torch.arange(64, dtype=torch.int32, device="cuda")
    # a 4-byte offset view is a valid array start for 4-byte keys ...
    C = cr.merge(A[1:], B)
    assert torch.equal(C, torch.sort(torch.cat([A[1:], B]), stable=True).values)
    # ... a start that is not a multiple of the key size is refused before
    # anything is launched (the raw pointer only reaches argument checks)
    from paper_1303_4312_gb300 import _lib
    lib = _lib.load()
    C = torch.empty(128, dtype=torch.int32, device="cuda")
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    st = lib.cr_stable_merge(0, A.data_ptr() + 2, 63, B.data_ptr(), 64, C.data_ptr(), None,
                             ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert _lib.STATUS[st] == "CR_EALIGN"
    buf = torch.zeros(256, dtype=torch.int32, device="cuda")
    with pytest.raises(cr.CorankError) as e:
        cr.merge(buf[:64], B, out=buf[:128])
    assert e.value.name == "CR_EALIAS"
    with pytest.raises(cr.CorankError) as e:
        cr.merge(A, B, ws=torch.empty(128, dtype=torch.uint8, device="cuda"))
    assert e.value.name == "CR_ENOSPACE"
    with pytest.raises(cr.CorankError) as e:
        cr.co_rank(A, B, 129)
    assert e.value.name == "CR_EINVAL"


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
@pytest.mark.parametrize("vdt", [None, np.float32])
def test_shared_corank_table_path(dt, vdt):
    """The two-step form (cr_merge_partition, then cr_merge_tiles and
    cr_merge_tiles_backward on the same tile table) against the oracle."""
    import ctypes
    from paper_1303_4312_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(105)
    vb = np.dtype(vdt).itemsize if vdt else 0
    kt = key_type(np.empty(0, dt))
    code = _lib.KEY_TYPES[kt]
    t = cr.tile_size(kt, vb, 1, 1)      # tile of these small merges
    for m, n in [(1, 0), (5 * t + 3, 2 * t - 1), (t, 7 * t), (123457, 98765)]:
        A = sorted_keys(rng, m, dt, 300)
        B = sorted_keys(rng, n, dt, 300)
        Ad, Bd = dev(A), dev(B)
        C = torch.empty(m + n, dtype=Ad.dtype, device="cuda")
        need = ctypes.c_size_t()
        _lib.check(lib.cr_merge_workspace_size(code, vb, m, n, ctypes.byref(need)))
        ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        _lib.check(lib.cr_merge_partition(code, vb, Ad.data_ptr(), m, Bd.data_ptr(), n,
                                          ws.data_ptr(), ws.numel(), s))
        if vdt is None:
            _lib.check(lib.cr_merge_tiles(code, 0, Ad.data_ptr(), None, m, Bd.data_ptr(), None, n,
                                          C.data_ptr(), None, None, ws.data_ptr(), ws.numel(), s))
            torch.cuda.synchronize()
            assert same_bits(host(C, dt), oracle.merge(A, B)[0])
            continue
        Av = rng.standard_normal(m).astype(vdt)
        Bv = rng.standard_normal(n).astype(vdt)
        Cv = torch.empty(m + n, dtype=torch.float32, device="cuda")
        Avd, Bvd = dev(Av), dev(Bv)   # keep the device copies alive until the kernel ran
        _lib.check(lib.cr_merge_tiles(code, vb, Ad.data_ptr(), Avd.data_ptr(), m,
                                      Bd.data_ptr(), Bvd.data_ptr(), n, C.data_ptr(),
                                      Cv.data_ptr(), None, ws.data_ptr(), ws.numel(), s))
        gC = rng.standard_normal(m + n).astype(vdt)
        gA = torch.empty(m, dtype=torch.float32, device="cuda")
        gB = torch.empty(n, dtype=torch.float32, device="cuda")
        gCd = dev(gC)
        _lib.check(lib.cr_merge_tiles_backward(code, vb, Ad.data_ptr(), m, Bd.data_ptr(), n,
                                               gCd.data_ptr(), gA.data_ptr() if m else None,
                                               gB.data_ptr() if n else None, ws.data_ptr(),
                                               ws.numel(), s))
        torch.cuda.synchronize()
        wk, wv, _ = oracle.merge_kv(A, Av, B, Bv)
        ga, gb = oracle.merge_grad(A, B, gC)
        assert same_bits(host(C, dt), wk)
        assert same_bits(host(Cv, np.float32), wv)
        assert same_bits(host(gA, np.float32), ga)
        assert same_bits(host(gB, np.float32), gb)
        cr.workspace_status(ws)


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
def test_geometry_class_boundary(dt):
    """Merges just inside and just outside the small-merge class (m + n =
    2^23 and 2^23 + 1), where the tile shape may switch: each uses the tile
    cr_tile_size_for reports (its workspace is sized for it) and equals the
    oracle's merge, keys and tags."""
    rng = np.random.default_rng(108)
    kt = key_type(np.empty(0, dt))
    limit = 1 << 23
    for m, n in ((limit // 2, limit // 2), (limit // 2, limit // 2 + 1), (7, limit - 7),
                 (7, limit), (limit // 16, limit - limit // 16 + 1)):
        A = sorted_keys(rng, m, dt, 5000)
        B = sorted_keys(rng, n, dt, 5000)
        t = cr.tile_size(kt, 0, m, n)
        assert t > 0
        need = cr.merge_workspace_bytes(kt, 0, m, n)
        assert need == 256 + 32 * ((m + n + t - 1) // t)
        C, T = cr.merge(dev(A), dev(B), key_type=kt, tag=True)
        torch.cuda.synchronize()
        want, src = oracle.merge(A, B)
        assert same_bits(host(C, dt), want), (m, n)
        assert np.array_equal(host(T, np.uint32).astype(np.int64), src), (m, n)


@pytest.mark.parametrize("dt", [np.int32, np.int64])
def test_streaming_merge_block_edges(dt):
    """Sizes around the streaming kernel's block and chunk boundaries: a few
    tiles per CTA, one tile per CTA, more CTAs than tiles, and inputs whose
    ends fall inside a 16-byte unit."""
    rng = np.random.default_rng(106)
    t = cr.tile_size(key_type(np.empty(0, dt)), 0, 1, 1)    # these merges are small
    for total in (t * 152 - 1, t * 304 + 5, t * 700 + 13, 3 * t + 1):
        assert cr.tile_size(key_type(np.empty(0, dt)), 0, total // 2, total - total // 2) == t
        for frac in (0.0, 0.01, 0.5, 0.97, 1.0):
            m = int(total * frac)
            n = total - m
            A = sorted_keys(rng, m, dt, None if frac == 0.5 else 7)
            B = sorted_keys(rng, n, dt, None if frac == 0.5 else 7)
            C, T = cr.merge(dev(A), dev(B), key_type=key_type(A), tag=True)
            torch.cuda.synchronize()
            want, src = oracle.merge(A, B)
            assert same_bits(host(C, dt), want), (total, frac)
            assert np.array_equal(host(T, np.uint32).astype(np.int64), src), (total, frac)


def test_every_tile_shape():
    """Every compiled tile shape gives the oracle's output (forward keys with
    tags, key-value forward and backward, batched), not only the default."""
    from paper_1303_4312_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(107)
    combos = [(np.int32, None), (np.int32, np.float32), (np.uint64, None), (np.uint64, np.float64),
              (np.int64, np.float32)]
    for dt, vdt in combos:
        kt = key_type(np.empty(0, dt))
        vb = np.dtype(vdt).itemsize if vdt else 0
        code = _lib.KEY_TYPES[kt]
        before = save_shapes(lib, code, vb)
        try:
            for shape in range(lib.cr_tile_shape_count()):
                if lib.cr_set_tile_shape(code, vb, shape) != 0:
                    continue
                t = cr.tile_size(kt, vb)
                m, n = 3 * t + 17, 2 * t - 3
                A = sorted_keys(rng, m, dt, 100)
                B = sorted_keys(rng, n, dt, 100)
                if vdt is None:
                    C, T = cr.merge(dev(A), dev(B), key_type=kt, tag=True)
                    torch.cuda.synchronize()
                    want, src = oracle.merge(A, B)
                    assert same_bits(host(C, dt), want), shape
                    assert np.array_equal(host(T, np.uint32).astype(np.int64), src), shape
                    continue
                Av = rng.standard_normal(m).astype(vdt)
                Bv = rng.standard_normal(n).astype(vdt)
                Ck, Cv = cr.merge_kv(dev(A), dev(Av), dev(B), dev(Bv), key_type=kt)
                gC = rng.standard_normal(m + n).astype(vdt)
                gA, gB = cr.merge_kv_backward(dev(A), dev(B), dev(gC), key_type=kt)
                a_off = np.array([0, m // 3, m // 3, m], np.int64)
                b_off = np.array([0, 5, n // 2, n], np.int64)
                Bk, Bkv = cr.batched_merge_kv(a_off, b_off, dev(A), dev(Av), dev(B), dev(Bv),
                                              key_type=kt)
                torch.cuda.synchronize()
                wk, wv, _ = oracle.merge_kv(A, Av, B, Bv)
                ga, gb = oracle.merge_grad(A, B, gC)
                bk, bv = oracle.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
                assert same_bits(host(Ck, dt), wk), shape
                assert same_bits(host(Cv, vdt), wv), shape
                assert same_bits(host(gA, vdt), ga), shape
                assert same_bits(host(gB, vdt), gb), shape
                assert same_bits(host(Bk, dt), bk), shape
                assert same_bits(host(Bkv, vdt), bv), shape
        finally:
            restore_shapes(lib, code, vb, before)


def test_table_for_another_shape_is_refused():
    """A tile table made under one shape and merged under another is refused
    on the device (status CR_EINTERNAL) instead of being misread."""
    import ctypes
    from paper_1303_4312_gb300 import _lib
    lib = _lib.load()
    code = _lib.KEY_TYPES["i32"]
    saved = save_shapes(lib, code, 0)
    before = saved[0]
    other = next(s for s in range(lib.cr_tile_shape_count())
                 if s != before and lib.cr_set_tile_shape(code, 0, s) == 0)
    try:
        A = torch.arange(0, 200000, 2, dtype=torch.int32, device="cuda")
        B = torch.arange(1, 200001, 2, dtype=torch.int32, device="cuda")
        C = torch.empty(200000, dtype=torch.int32, device="cuda")
        ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        _lib.check(lib.cr_set_tile_shape(code, 0, before))
        _lib.check(lib.cr_merge_partition(code, 0, A.data_ptr(), 100000, B.data_ptr(), 100000,
                                          ws.data_ptr(), ws.numel(), s))
        _lib.check(lib.cr_set_tile_shape(code, 0, other))
        _lib.check(lib.cr_merge_tiles(code, 0, A.data_ptr(), None, 100000, B.data_ptr(), None,
                                      100000, C.data_ptr(), None, None, ws.data_ptr(),
                                      ws.numel(), s))
        with pytest.raises(cr.CorankError) as e:
            cr.workspace_status(ws)
        assert e.value.name == "CR_EINTERNAL"
    finally:
        restore_shapes(lib, code, 0, saved)


def test_merge_many_overlapped_partitions():
    """MergeMany (partitions on a side stream, double-buffered tile tables)
    gives each pair's oracle merge, on three calls in a row."""
    rng = np.random.default_rng(108)
    pairs_h = [(sorted_keys(rng, 200003, np.int32, None), sorted_keys(rng, 150001, np.int32, None)),
               (sorted_keys(rng, 1000, np.uint64, None), sorted_keys(rng, 400000, np.uint64, None)),
               (sorted_keys(rng, 300000, np.int32, 16), sorted_keys(rng, 300000, np.int32, 16))]
    pairs = [(dev(a), dev(b)) for a, b in pairs_h]
    mm = cr.MergeMany(pairs, [key_type(a) for a, _ in pairs_h])
    for _ in range(3):
        outs = mm.run()
        mm.check()
        for (a, b), C in zip(pairs_h, outs):
            assert same_bits(host(C, a.dtype), oracle.merge(a, b)[0])


def test_host_merger_pipeline():
    """HostMerger: pinned host inputs -> device -> merge -> pinned host outputs,
    pipelined on three streams, equals the oracle on two runs in a row."""
    rng = np.random.default_rng(109)
    pairs = [(sorted_keys(rng, 300001, np.int32, None), sorted_keys(rng, 200003, np.int32, None)),
             (sorted_keys(rng, 5000, np.uint64, None), sorted_keys(rng, 700001, np.uint64, None))]
    hm = cr.HostMerger([(len(a), len(b), torch.int32 if a.dtype == np.int32 else torch.int64,
                         key_type(a)) for a, b in pairs])
    hosts = [(torch.from_numpy(a.view(np.int32 if a.dtype == np.int32 else np.int64)).pin_memory(),
              torch.from_numpy(b.view(np.int32 if b.dtype == np.int32 else np.int64)).pin_memory())
             for a, b in pairs]
    outs = [torch.empty(len(a) + len(b), dtype=hA.dtype).pin_memory()
            for (a, b), (hA, _) in zip(pairs, hosts)]
    for _ in range(2):
        for o in outs:
            o.fill_(0)
        hm.run(hosts, outs)
        hm.check()
        for (a, b), o in zip(pairs, outs):
            assert same_bits(o.numpy().view(a.dtype), oracle.merge(a, b)[0])


def test_host_merger_on_registered_buffers():
    """HostMerger with inputs and outputs in host_empty buffers (page-locked by
    cudaHostRegister): the buffers report pinned, have the asked shape and
    type, and two runs in a row equal the oracle; dropping them releases the
    registration after the device is idle, and new ones work again."""
    rng = np.random.default_rng(110)
    a = sorted_keys(rng, 400001, np.int32, None)
    b = sorted_keys(rng, 123457, np.int32, None)
    for _ in range(2):
        hA, hB = cr.host_empty(len(a), torch.int32), cr.host_empty(len(b), torch.int32)
        out = cr.host_empty(len(a) + len(b), torch.int32)
        assert hA.is_pinned() and hB.is_pinned() and out.is_pinned()
        assert hA.dtype == torch.int32 and out.shape == (len(a) + len(b),)
        hA.copy_(torch.from_numpy(a))
        hB.copy_(torch.from_numpy(b))
        hm = cr.HostMerger([(len(a), len(b), torch.int32, "i32")])
        for _ in range(2):
            out.fill_(0)
            hm.run([(hA, hB)], [out])
            hm.check()
            torch.cuda.synchronize()
            assert same_bits(out.numpy(), oracle.merge(a, b)[0])
        del hA, hB, out, hm


def test_sharded_merge_single_rank_nccl():
    """The sharded merge with the library's own co-rank and merge kernels, in
    a one-rank NCCL group on this GPU (plan, windows, gather)."""
    import os
    import socket
    import torch.distributed as dist
    from paper_1303_4312_gb300 import shard
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        rng = np.random.default_rng(112)
        A = sorted_keys(rng, 123457, np.int32, 500)
        B = sorted_keys(rng, 98765, np.int32, 500)
        C, p = shard.sharded_merge(dev(A), dev(B))
        assert (p.k0, p.k1) == (0, len(A) + len(B))
        assert same_bits(host(C, np.int32), oracle.merge(A, B)[0])
        # block-distributed form: remote-read co-ranks and window fetch over
        # NCCL (one rank), local merge by the library's kernels
        C, p = shard.distributed_merge(dev(A), dev(B), "i32")
        assert (p.i1, p.j1) == (len(A), len(B))
        assert same_bits(host(C, np.int32), oracle.merge(A, B)[0])
        Au = sorted_keys(rng, 5000, np.uint64)
        Bu = sorted_keys(rng, 7000, np.uint64)
        Av = rng.standard_normal(5000).astype(np.float32)
        Bv = rng.standard_normal(7000).astype(np.float32)
        C, Cv, p = shard.distributed_merge(dev(Au), dev(Bu), "u64", Av_blk=dev(Av),
                                           Bv_blk=dev(Bv))
        wk, wv, _ = oracle.merge_kv(Au, Av, Bu, Bv)
        assert same_bits(host(C, np.uint64), wk) and same_bits(host(Cv, np.float32), wv)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
def test_partition_alg2_table_matches(dt):
    """The sync-free partition (every tile co-ranks both ends with Algorithm 1)
    writes the same tile table as the shared partition: the merge is equal."""
    import ctypes
    from paper_1303_4312_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(113)
    kt = key_type(np.empty(0, dt))
    code = _lib.KEY_TYPES[kt]
    for m, n, spread in [(300001, 200003, None), (5, 400000, None), (250000, 250000, 4)]:
        A = sorted_keys(rng, m, dt, spread)
        B = sorted_keys(rng, n, dt, spread)
        Ad, Bd = dev(A), dev(B)
        need = ctypes.c_size_t()
        _lib.check(lib.cr_merge_workspace_size(code, 0, m, n, ctypes.byref(need)))
        s = torch.cuda.current_stream().cuda_stream
        tables = []
        for fn in (lib.cr_merge_partition, lib.cr_merge_partition_alg2):
            ws = torch.zeros(need.value, dtype=torch.uint8, device="cuda")
            _lib.check(fn(code, 0, Ad.data_ptr(), m, Bd.data_ptr(), n, ws.data_ptr(), ws.numel(), s))
            C = torch.empty(m + n, dtype=Ad.dtype, device="cuda")
            _lib.check(lib.cr_merge_tiles(code, 0, Ad.data_ptr(), None, m, Bd.data_ptr(), None, n,
                                          C.data_ptr(), None, None, ws.data_ptr(), ws.numel(), s))
            torch.cuda.synchronize()
            cr.workspace_status(ws)
            assert same_bits(host(C, dt), oracle.merge(A, B)[0])
            tables.append(ws.cpu())
        assert torch.equal(tables[0][8:], tables[1][8:])   # same records (header tile/ntiles too)


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
@pytest.mark.parametrize("vdt", [None, np.float32, np.float64])
def test_sort_runs_and_backward(dt, vdt):
    """Run formation: every run of sort_run_length() elements stably sorted
    (payloads follow; equal keys keep input order), and its backward."""
    rng = np.random.default_rng(114)
    R = cr.sort_run_length()
    kt = key_type(np.empty(0, dt))
    for N in (1, 5, R - 1, R, R + 1, 7 * R + 333):
        for spread in (None, 3):
            info = np.iinfo(dt)
            X = (rng.integers(info.min, info.max, N, dtype=dt, endpoint=True) if spread is None
                 else rng.integers(0, spread, N).astype(dt))
            Xv = rng.standard_normal(N).astype(vdt or np.float32)
            Y, Yv = cr.sort_runs(dev(X), dev(Xv) if vdt else None, key_type=kt)
            torch.cuda.synchronize()
            want = np.empty_like(X)
            wantv = np.empty_like(Xv)
            perm = np.empty(N, np.int64)
            for a0 in range(0, N, R):
                o = np.argsort(X[a0:a0 + R], kind="stable")
                want[a0:a0 + R] = X[a0:a0 + R][o]
                wantv[a0:a0 + R] = Xv[a0:a0 + R][o]
                perm[a0:a0 + R] = a0 + o
            assert same_bits(host(Y, dt), want), (N, spread)
            if vdt:
                assert same_bits(host(Yv, vdt), wantv), (N, spread)
                gY = rng.standard_normal(N).astype(vdt)
                gX = cr.sort_runs_backward(dev(X), dev(gY), key_type=kt)
                torch.cuda.synchronize()
                g = np.empty_like(gY)
                g[perm] = gY
                assert same_bits(host(gX, vdt), g), (N, spread)


def test_merge_sort_from_unsorted_input():
    """Full stable sort of unsorted input (run formation, then merge passes in
    CUDA graphs) and its payload gradient, against numpy's stable argsort."""
    rng = np.random.default_rng(115)
    for N in (1, 1000, 100003, 1 << 20):
        vals = rng.integers(0, 2**64, 4000, dtype=np.uint64)
        X = vals[rng.integers(0, len(vals), N)]
        Xv = rng.standard_normal(N).astype(np.float32)
        Xt = dev(X)
        Xvt = dev(Xv).requires_grad_(True)
        Y, Yv = cr.merge_sort(Xt, Xvt, key_type="u64")
        gY = rng.standard_normal(N).astype(np.float32)
        Yv.backward(dev(gY))
        torch.cuda.synchronize()
        o = np.argsort(X, kind="stable")
        assert same_bits(host(Y, np.uint64), X[o])
        assert same_bits(host(Yv.detach(), np.float32), Xv[o])
        g = np.empty_like(gY)
        g[o] = gY
        assert same_bits(host(Xvt.grad, np.float32), g)
