"""GPU parity for key orders other than the storage type's own: float keys in
IEEE-754 totalOrder (CR_KEY_F32/F64) and descending orders (CR_KEY_DESC),
against the oracle's order map (merge_in_order: the plain merge of the
order keys).  Every row of the path runs in each order: single merge with
tags, key-value forward and backward, co-ranks, batched merge, recorded merge
pass and its backward, and the full sort from unsorted input."""
import numpy as np
import pytest
import torch

import oracle
import paper_1303_4312_gb300 as cr
from gpu_util import dev, host, same_bits

pytestmark = pytest.mark.gpu

ORDERS = ["f32", "f64", "f32:desc", "f64:desc", "i32:desc", "u32:desc", "i64:desc", "u64:desc",
          "pair_u32", "pair_i32", "pair_i32:desc"]
DT = {"f32": np.float32, "f64": np.float64, "i32": np.int32, "u32": np.uint32,
      "i64": np.int64, "u64": np.uint64, "pair_u32": np.uint64, "pair_i32": np.uint64}


def draw(rng, size, kt, distinct=None):
    """Keys of `kt`'s storage type: floats mixing NaNs of both signs and kinds,
    signed zeros, infinities, subnormals and ordinary values; integers over
    the full range (or from `distinct` values)."""
    base = kt.split(":")[0]
    dt = DT[base]
    if base[0] == "f":
        ut = np.uint32 if dt == np.float32 else np.uint64
        bits = rng.integers(0, np.iinfo(ut).max, size, dtype=ut, endpoint=True)
        x = bits.view(dt).copy()
        normal = (rng.standard_normal(size) * 10.0 ** rng.integers(-5, 5, size)).astype(dt)
        pick = rng.random(size) < 0.6
        x[pick] = normal[pick]
        specials = np.array([0.0, -0.0, np.inf, -np.inf], dtype=dt)
        sp = rng.random(size) < 0.05
        x[sp] = specials[rng.integers(0, 4, int(sp.sum()))]
    elif base.startswith("pair"):
        # few distinct major keys, so the minor key decides often
        major = rng.integers(0, 2**32, max(1, size // 50 + 1), dtype=np.uint64)
        x = (major[rng.integers(0, len(major), size)] << np.uint64(32)) | \
            rng.integers(0, 2**32, size, dtype=np.uint64)
    else:
        info = np.iinfo(dt)
        x = rng.integers(info.min, info.max, size, dtype=dt, endpoint=True)
    if distinct is not None and size:
        x = x[rng.integers(0, distinct, size) % max(1, size)]
    return x


def in_order(x, kt):
    return x[np.argsort(oracle.order_key(x, kt), kind="stable")]


@pytest.mark.parametrize("kt", ORDERS)
def test_merge_with_tags_and_co_ranks(kt):
    rng = np.random.default_rng(400)
    t = cr.tile_size(kt, 0, 1, 1)       # tile of these small merges
    for m, n in [(0, 5), (7, 0), (3 * t + 5, 2 * t - 1), (100, 9 * t), (20000, 20000)]:
        for distinct in (None, 9):
            A = in_order(draw(rng, m, kt, distinct), kt)
            B = in_order(draw(rng, n, kt, distinct), kt)
            C, T = cr.merge(dev(A), dev(B), key_type=kt, tag=True)
            torch.cuda.synchronize()
            want, src = oracle.merge_in_order(A, B, kt)
            assert same_bits(host(C, A.dtype), want), (kt, m, n)
            assert np.array_equal(host(T, np.uint32).astype(np.int64), src), (kt, m, n)
            ranks = np.unique(np.concatenate([rng.integers(0, m + n + 1, 50), [0, m + n]]))
            ci, cj = cr.co_rank_many(dev(A), dev(B), torch.from_numpy(ranks).cuda(), key_type=kt)
            ka, kb = oracle.order_key(A, kt), oracle.order_key(B, kt)
            oj, ok = oracle.co_rank_many(ka, kb, ranks)
            assert np.array_equal(ci.cpu().numpy(), oj) and np.array_equal(cj.cpu().numpy(), ok)


@pytest.mark.parametrize("kt", ["f32", "f64:desc", "i32:desc", "u64:desc"])
def test_kv_forward_backward(kt):
    rng = np.random.default_rng(401)
    m, n = 50001, 77777
    A = in_order(draw(rng, m, kt, 1000), kt)
    B = in_order(draw(rng, n, kt, 1000), kt)
    Av = rng.standard_normal(m).astype(np.float32)
    Bv = rng.standard_normal(n).astype(np.float32)
    Ck, Cv = cr.merge_kv(dev(A), dev(Av), dev(B), dev(Bv), key_type=kt)
    gC = rng.standard_normal(m + n).astype(np.float32)
    gA, gB = cr.merge_kv_backward(dev(A), dev(B), dev(gC), key_type=kt)
    torch.cuda.synchronize()
    want, src = oracle.merge_in_order(A, B, kt)
    assert same_bits(host(Ck, A.dtype), want)
    assert same_bits(host(Cv, np.float32), np.concatenate([Av, Bv])[src])
    g = np.empty(m + n, dtype=np.float32)
    g[src] = gC
    assert same_bits(host(gA, np.float32), g[:m]) and same_bits(host(gB, np.float32), g[m:])


@pytest.mark.parametrize("kt", ["f32", "i64:desc"])
def test_batched_in_order(kt):
    rng = np.random.default_rng(402)
    nseg = 300
    ms = rng.integers(0, 3000, nseg)
    ns = rng.integers(0, 3000, nseg)
    a_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    A = np.concatenate([in_order(draw(rng, int(x), kt, 50), kt) for x in ms])
    B = np.concatenate([in_order(draw(rng, int(x), kt, 50), kt) for x in ns])
    Av = rng.standard_normal(len(A)).astype(np.float32)
    Bv = rng.standard_normal(len(B)).astype(np.float32)
    Ck, Cv = cr.batched_merge_kv(torch.from_numpy(a_off).cuda(), torch.from_numpy(b_off).cuda(),
                                 dev(A), dev(Av), dev(B), dev(Bv), key_type=kt)
    torch.cuda.synchronize()
    wk, wv = [], []
    for s in range(nseg):
        a, b = A[a_off[s]:a_off[s + 1]], B[b_off[s]:b_off[s + 1]]
        c, src = oracle.merge_in_order(a, b, kt)
        wk.append(c)
        wv.append(np.concatenate([Av[a_off[s]:a_off[s + 1]], Bv[b_off[s]:b_off[s + 1]]])[src])
    assert same_bits(host(Ck, A.dtype), np.concatenate(wk))
    assert same_bits(host(Cv, np.float32), np.concatenate(wv))


@pytest.mark.parametrize("kt", ["f64", "u32:desc", "f32:desc"])
def test_recorded_pass_in_order(kt):
    rng = np.random.default_rng(403)
    N, w = 100003, 1000
    X = draw(rng, N, kt, 500)
    for a0 in range(0, N, w):
        X[a0:a0 + w] = in_order(X[a0:a0 + w], kt)
    Xv = rng.standard_normal(N).astype(np.float32)
    Y, Yv, rec = cr.merge_pass_record(dev(X), dev(Xv), w, key_type=kt)
    gY = rng.standard_normal(N).astype(np.float32)
    gX = cr.merge_pass_backward_recorded(rec, dev(gY))
    torch.cuda.synchronize()
    cr.workspace_status(rec.ws)
    # expected pass: every pair merged in order
    src = np.empty(N, dtype=np.int64)
    for a0 in range(0, N, 2 * w):
        m = min(w, N - a0)
        n = min(w, N - a0 - m)
        _, s = oracle.merge_in_order(X[a0:a0 + m], X[a0 + m:a0 + m + n], kt)
        src[a0:a0 + m + n] = a0 + s
    assert same_bits(host(Y, X.dtype), X[src]) and same_bits(host(Yv, np.float32), Xv[src])
    g = np.empty_like(gY)
    g[src] = gY
    assert same_bits(host(gX, np.float32), g)


@pytest.mark.parametrize("kt", ["f32", "f64:desc", "i32:desc", "u64:desc", "pair_i32"])
@pytest.mark.parametrize("record", [True, False])
def test_sort_from_unsorted_in_order(kt, record):
    rng = np.random.default_rng(404)
    for N in (1, 5000, 300001):
        X = draw(rng, N, kt, 4000)
        Xv = rng.standard_normal(N).astype(np.float32)
        Xt = dev(X)
        Xvt = dev(Xv).requires_grad_(True)
        Y, Yv = cr.merge_sort(Xt, Xvt, key_type=kt, record=record)
        gY = rng.standard_normal(N).astype(np.float32)
        Yv.backward(dev(gY))
        torch.cuda.synchronize()
        o = np.argsort(oracle.order_key(X, kt), kind="stable")
        assert same_bits(host(Y, X.dtype), X[o]), N
        assert same_bits(host(Yv.detach(), np.float32), Xv[o]), N
        g = np.empty_like(gY)
        g[o] = gY
        assert same_bits(host(Xvt.grad, np.float32), g), N


@pytest.mark.parametrize("kt", ["i32", "u32", "i64", "u64"] + ORDERS)
def test_check_sorted(kt):
    """cr_check_sorted: -1 on sorted input; else the first position whose key
    comes before its predecessor in kt's order (numpy on the oracle's order
    keys)."""
    rng = np.random.default_rng(405)
    for N in (0, 1, 2, 1000, 300001):
        X = in_order(draw(rng, N, kt, 5000), kt)
        assert cr.check_sorted(dev(X), key_type=kt) == -1, N
        if N < 2:
            continue
        for _ in range(3):
            Y = X.copy()
            p, q = sorted(rng.integers(0, N, 2))
            Y[p], Y[q] = Y[q], Y[p]
            k = oracle.order_key(Y, kt)
            bad = np.nonzero(k[1:] < k[:-1])[0]
            want = int(bad[0]) + 1 if len(bad) else -1
            assert cr.check_sorted(dev(Y), key_type=kt) == want, (N, p, q)


@pytest.mark.parametrize("kt", ["i32:desc", "u64:desc", "f32", "f64:desc"])
def test_large_orders_keys_payloads_backward(kt):
    """Large merges through the compile-time order kernels (descending
    integer orders compare with the operands swapped; float totalOrder keys
    use the fixed float map): 2^24 + 2^24 keys (2^23 + 2^23 for 8-byte keys;
    inputs with their payloads above the 129 MB L2, thousands of tiles) with
    float32 payloads, forward and payload backward, against the oracle bit
    for bit."""
    import ctypes
    from paper_1303_4312_gb300 import _lib
    rng = np.random.default_rng(sum(map(ord, kt)))
    base = kt.split(":")[0]
    half = 1 << (23 if DT[base]().itemsize == 8 else 24)
    A = in_order(draw(rng, half, kt, distinct=None if base[0] == "f" else 1 << 20), kt)
    B = in_order(draw(rng, half - 12345, kt, distinct=None if base[0] == "f" else 1 << 20), kt)
    Av = rng.standard_normal(len(A)).astype(np.float32)
    Bv = rng.standard_normal(len(B)).astype(np.float32)
    gC = rng.standard_normal(len(A) + len(B)).astype(np.float32)
    Ck, Cv = cr.merge_kv(dev(A), dev(Av), dev(B), dev(Bv), key_type=kt)
    gA, gB = cr.merge_kv_backward(dev(A), dev(B), dev(gC), key_type=kt)
    torch.cuda.synchronize()
    want, src = oracle.merge_in_order(A, B, kt)
    assert same_bits(host(Ck, A.dtype), want)
    m = len(A)
    wv = np.where(src < m, Av[np.minimum(src, m - 1)], Bv[np.maximum(src - m, 0)])
    assert same_bits(host(Cv, np.float32), wv.astype(np.float32))
    ga = np.empty(m, np.float32)
    gb = np.empty(len(B), np.float32)
    ga[src[src < m]] = gC[src < m]
    gb[src[src >= m] - m] = gC[src >= m]
    assert same_bits(host(gA, np.float32), ga)
    assert same_bits(host(gB, np.float32), gb)
