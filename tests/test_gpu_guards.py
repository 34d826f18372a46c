"""Structural checks of the GPU path:

* Proposition 2 on the device tile table: every tile carries exactly TILE
  outputs except the last, and the tiles' windows cover A, B and C exactly
  once, in order;
* guard canaries: every output of every row is written inside its own range
  only (sentinel bytes before and after each output array stay untouched),
  including the ragged 16-byte edges the plain stores handle;
* finite differences through autograd: the payload gradient of the
  key-value merge equals central differences of L = sum(w * Cv), exact for a
  permutation in float64 with h = 2^-4.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1303_4312_gb300 as cr
from paper_1303_4312_gb300 import _lib
from gpu_util import dev, host, same_bits, sorted_keys

pytestmark = pytest.mark.gpu


REC = np.dtype([("ga", "<i8"), ("gb", "<i8"), ("gc", "<i8"), ("alen", "<i4"), ("blen", "<i4")])


def read_table(raw):
    """(status, tile, ntiles, ga, gb, gc, alen, blen) of a workspace's bytes:
    a 256-byte header {int32 status, int32 tile, int64 ntiles} and 32-byte
    records {int64 ga, gb, gc; int32 alen, blen}."""
    raw = np.ascontiguousarray(raw)
    status, tile = raw[:8].view(np.int32)
    ntiles = int(raw[8:16].view(np.int64)[0])
    rec = raw[256:256 + 32 * ntiles].view(REC)
    return (int(status), int(tile), ntiles, rec["ga"].copy(), rec["gb"].copy(),
            rec["gc"].copy(), rec["alen"].astype(np.int64), rec["blen"].astype(np.int64))


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
def test_tile_table_is_balanced_and_exact(dt):
    """Proposition 2: tile t holds exactly TILE outputs (the last one the
    remainder), and consecutive tiles continue each other's A, B and C
    windows, so every element belongs to exactly one tile; the co-ranks at
    the tile ends are Algorithm 1's (oracle)."""
    rng = np.random.default_rng(600)
    lib = _lib.load()
    kt = "i32" if dt == np.int32 else "u64"
    for m, n in [(100000, 77777), (5, 300000), (1 << 20, 1 << 20), (7, 0), (123456, 1),
                 (1 << 23, (1 << 23) + 5)]:
        A = sorted_keys(rng, m, dt, 1000)
        B = sorted_keys(rng, n, dt, 1000)
        ws = torch.zeros(cr.api.merge_workspace_bytes(kt, 0, m, n), dtype=torch.uint8,
                         device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        a, b = dev(A), dev(B)          # held until the kernel has run
        _lib.check(lib.cr_merge_partition(_lib.key_code(kt), 0, a.data_ptr(), m,
                                          b.data_ptr(), n, ws.data_ptr(), ws.numel(), s))
        torch.cuda.synchronize()
        status, tile, nt, ga, gb, gc, alen, blen = read_table(ws.cpu().numpy())
        assert status == 0 and tile == lib.cr_tile_size_for(_lib.key_code(kt), 0, m, n)
        assert nt == (m + n + tile - 1) // tile
        ln = alen + blen
        assert np.all(ln[:-1] == tile) and 0 < ln[-1] <= tile
        assert np.array_equal(gc, np.arange(nt) * tile)
        assert ga[0] == 0 and gb[0] == 0
        assert np.array_equal(ga[1:], ga[:-1] + alen[:-1]) and ga[-1] + alen[-1] == m
        assert np.array_equal(gb[1:], gb[:-1] + blen[:-1]) and gb[-1] + blen[-1] == n
        j, _ = oracle.co_rank_many(A, B, gc)
        assert np.array_equal(ga, j)


GUARD = 4096     # sentinel bytes on each side of every output (multiple of 16)


def guarded(n, dtype):
    """A device array of n elements with GUARD sentinel bytes before and
    after it; returns (whole buffer, the view)."""
    es = torch.empty(0, dtype=dtype).element_size()
    buf = torch.full((2 * GUARD + n * es,), 0xA5, dtype=torch.uint8, device="cuda")
    view = buf[GUARD:GUARD + n * es].view(dtype)
    return buf, view


def untouched(buf):
    b = buf.cpu().numpy()
    return bool(np.all(b[:GUARD] == 0xA5) and np.all(b[-GUARD:] == 0xA5))


def test_outputs_stay_inside_their_ranges():
    rng = np.random.default_rng(601)
    for m, n in [(1, 0), (3, 5), (1000, 1), (12345, 54321), (3 * 3840 + 7, 11)]:
        A = sorted_keys(rng, m, np.int32, 50)
        B = sorted_keys(rng, n, np.int32, 50)
        Av = rng.standard_normal(m).astype(np.float32)
        Bv = rng.standard_normal(n).astype(np.float32)
        # keys + tags
        bc, C = guarded(m + n, torch.int32)
        bt, T = guarded(m + n, torch.int32)
        cr.merge(dev(A), dev(B), tag=True, out=C, out_tag=T)
        torch.cuda.synchronize()
        assert untouched(bc) and untouched(bt), (m, n)
        want, src = oracle.merge(A, B)
        assert same_bits(host(C, np.int32), want)
        # key-value forward and backward
        bk, Ck = guarded(m + n, torch.int32)
        bv, Cv = guarded(m + n, torch.float32)
        lib = _lib.load()
        ws = torch.zeros(cr.api.merge_workspace_bytes("i32", 4, m, n), dtype=torch.uint8,
                         device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        a, av, b, bvv = dev(A), dev(Av), dev(B), dev(Bv)
        _lib.check(lib.cr_stable_merge_kv(0, 4, a.data_ptr(), av.data_ptr(), m, b.data_ptr(),
                                          bvv.data_ptr(), n, Ck.data_ptr(), Cv.data_ptr(), None,
                                          ws.data_ptr(), ws.numel(), s))
        gC = dev(rng.standard_normal(m + n).astype(np.float32))
        bga, gA = guarded(m, torch.float32)
        bgb, gB = guarded(n, torch.float32)
        _lib.check(lib.cr_stable_merge_kv_backward(0, 4, a.data_ptr(), m, b.data_ptr(), n,
                                                   gC.data_ptr(), gA.data_ptr(), gB.data_ptr(),
                                                   ws.data_ptr(), ws.numel(), s))
        torch.cuda.synchronize()
        assert untouched(bk) and untouched(bv) and untouched(bga) and untouched(bgb), (m, n)
        ga, gb = oracle.merge_grad(A, B, host(gC, np.float32))
        assert same_bits(host(gA, np.float32), ga) and same_bits(host(gB, np.float32), gb)


def test_pass_outputs_stay_inside_their_ranges():
    rng = np.random.default_rng(602)
    for N, w in [(1, 1), (9, 4), (50001, 1000), (3 * 1792 + 5, 1792)]:
        X = rng.integers(0, 30, N).astype(np.uint64)
        for a0 in range(0, N, w):
            X[a0:a0 + w].sort(kind="stable")
        Xv = rng.standard_normal(N).astype(np.float32)
        by, Y = guarded(N, torch.int64)
        byv, Yv = guarded(N, torch.float32)
        _, _, rec = cr.merge_pass_record(dev(X), dev(Xv), w, key_type="u64", out=(Y, Yv))
        bgx, gX = guarded(N, torch.float32)
        cr.merge_pass_backward_recorded(rec, dev(rng.standard_normal(N).astype(np.float32)),
                                        out=gX)
        torch.cuda.synchronize()
        assert untouched(by) and untouched(byv) and untouched(bgx), (N, w)
        wy, _, _ = oracle.merge_pass(X, Xv, w)
        assert same_bits(host(Y, np.uint64), wy)


def test_batched_outputs_stay_inside_their_ranges():
    import ctypes
    rng = np.random.default_rng(603)
    nseg = 40
    ms = rng.integers(0, 500, nseg)
    ns = rng.integers(0, 500, nseg)
    a_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    A = np.concatenate([np.sort(rng.integers(0, 9, x)) for x in ms]).astype(np.int32)
    B = np.concatenate([np.sort(rng.integers(0, 9, x)) for x in ns]).astype(np.int32)
    Av = rng.standard_normal(len(A)).astype(np.float32)
    Bv = rng.standard_normal(len(B)).astype(np.float32)
    at, bt = len(A), len(B)
    N = at + bt
    bk, Ck = guarded(N, torch.int32)
    bv, Cv = guarded(N, torch.float32)
    bga, gA = guarded(at, torch.float32)
    bgb, gB = guarded(bt, torch.float32)
    lib = _lib.load()
    need = ctypes.c_size_t()
    _lib.check(lib.cr_batched_workspace_size(0, 4, nseg, at, bt, ctypes.byref(need)))
    ws = torch.zeros(max(need.value, 256), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    ao, bo = torch.from_numpy(a_off).cuda(), torch.from_numpy(b_off).cuda()
    a, av, b, bvv = dev(A), dev(Av), dev(B), dev(Bv)
    gC = dev(rng.standard_normal(N).astype(np.float32))
    _lib.check(lib.cr_batched_merge_kv(0, 4, nseg, ao.data_ptr(), bo.data_ptr(), a.data_ptr(),
                                       av.data_ptr(), at, b.data_ptr(), bvv.data_ptr(), bt,
                                       Ck.data_ptr(), Cv.data_ptr(), ws.data_ptr(), ws.numel(), s))
    _lib.check(lib.cr_batched_merge_kv_backward(0, 4, nseg, ao.data_ptr(), bo.data_ptr(),
                                                a.data_ptr(), at, b.data_ptr(), bt, gC.data_ptr(),
                                                gA.data_ptr(), gB.data_ptr(), ws.data_ptr(),
                                                ws.numel(), s))
    torch.cuda.synchronize()
    cr.workspace_status(ws)
    assert untouched(bk) and untouched(bv) and untouched(bga) and untouched(bgb)
    wk, wv = oracle.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
    assert same_bits(host(Ck, np.int32), wk) and same_bits(host(Cv, np.float32), wv)
    ga, gb = oracle.batched_merge_grad(a_off, b_off, A, B, host(gC, np.float32))
    assert same_bits(host(gA, np.float32), ga) and same_bits(host(gB, np.float32), gb)


def test_kv_autograd_finite_differences():
    """dL/dAv and dL/dBv of L = sum(w * Cv) through MergeKV, against central
    differences with h = 2^-4 in float64 (exact: C is a permutation)."""
    rng = np.random.default_rng(604)
    m, n = 300, 200
    A = sorted_keys(rng, m, np.int32, 20)
    B = sorted_keys(rng, n, np.int32, 20)
    Av = torch.tensor(rng.standard_normal(m), dtype=torch.float64, device="cuda",
                      requires_grad=True)
    Bv = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda",
                      requires_grad=True)
    w = torch.tensor(rng.standard_normal(m + n), dtype=torch.float64, device="cuda")
    Ak, Bk = dev(A), dev(B)
    _, Cv = cr.MergeKV.apply(Ak, Av, Bk, Bv, "i32")
    (Cv * w).sum().backward()
    h = 2.0 ** -4
    # the two sums differ in one term only, so the central difference equals
    # that term's weight up to the rounding of the float64 sums
    for i in rng.integers(0, m, 12):
        ap = Av.detach().clone()
        am = Av.detach().clone()
        ap[i] += h
        am[i] -= h
        lp = (cr.merge_kv(Ak, ap, Bk, Bv.detach(), key_type="i32")[1] * w).sum()
        lm = (cr.merge_kv(Ak, am, Bk, Bv.detach(), key_type="i32")[1] * w).sum()
        fd = float((lp - lm) / (2 * h))
        assert abs(fd - float(Av.grad[i])) <= 1e-9, (i, fd, float(Av.grad[i]))
    for i in rng.integers(0, n, 12):
        bp = Bv.detach().clone()
        bm = Bv.detach().clone()
        bp[i] += h
        bm[i] -= h
        lp = (cr.merge_kv(Ak, Av.detach(), Bk, bp, key_type="i32")[1] * w).sum()
        lm = (cr.merge_kv(Ak, Av.detach(), Bk, bm, key_type="i32")[1] * w).sum()
        assert abs(float((lp - lm) / (2 * h)) - float(Bv.grad[i])) <= 1e-9


def test_batched_many_segments_scan_carry():
    """More segments than one pass of the segment scan covers (8192 per
    pass): the carried prefix across passes, empty segments included."""
    rng = np.random.default_rng(605)
    nseg = 20011
    ms = rng.integers(0, 40, nseg)
    ns = rng.integers(0, 40, nseg)
    ms[::7] = 0
    ns[::11] = 0
    a_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    A = np.concatenate([np.sort(rng.integers(0, 5, x)) for x in ms]).astype(np.int32)
    B = np.concatenate([np.sort(rng.integers(0, 5, x)) for x in ns]).astype(np.int32)
    Av = rng.standard_normal(len(A)).astype(np.float32)
    Bv = rng.standard_normal(len(B)).astype(np.float32)
    Ck, Cv = cr.batched_merge_kv(torch.from_numpy(a_off).cuda(), torch.from_numpy(b_off).cuda(),
                                 dev(A), dev(Av), dev(B), dev(Bv))
    torch.cuda.synchronize()
    wk, wv = oracle.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
    assert same_bits(host(Ck, np.int32), wk) and same_bits(host(Cv, np.float32), wv)
