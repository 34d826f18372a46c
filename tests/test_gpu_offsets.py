"""GPU parity for arrays that start anywhere their element size allows.

Algorithm 2 (Section 3) hands each processing element the windows
A[j_r, j_{r+1}) and B[k_r, k_{r+1}) of the inputs; passing such a window is
passing a pointer into the middle of an array.  The library accepts every
array start aligned to its element size (16-byte boundaries are needed only by
its own workspace and flag buffers), so these tests merge offset views --
keys, payloads, tags, gradients and outputs each at every element offset
inside a 16-byte chunk -- and compare them bit for bit with the CPU oracle.
The last tests run the sharded merge's default path (co-ranks and the block
merge through this library) for every rank of world sizes 2 and 3 on one
GPU, one rank after another, against the oracle's blocks.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1303_4312_gb300 as cr
from gpu_util import dev, host, key_type, same_bits, sorted_keys
from paper_1303_4312_gb300 import shard

pytestmark = pytest.mark.gpu


def _view(a: np.ndarray, off: int) -> torch.Tensor:
    """Device copy of `a` starting `off` elements after a 256-byte aligned
    allocation (so the view's start is off * itemsize bytes past a 16-byte
    boundary)."""
    buf = dev(np.concatenate([np.zeros(off, a.dtype), a]))
    v = buf[off:]
    if len(a):
        assert v.data_ptr() % 16 == (off * a.itemsize) % 16
    return v


def _empty_view(n: int, dtype: torch.dtype, off: int, fill: int = -7) -> torch.Tensor:
    buf = torch.full((n + off + 4,), fill, dtype=dtype, device="cuda")
    return buf[off:off + n]


def _offsets(dt):
    return range(16 // np.dtype(dt).itemsize)


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
def test_offset_views_keys_and_tags(dt):
    rng = np.random.default_rng(301)
    kt = key_type(np.empty(0, dt))
    t = cr.tile_size(kt, 0, 1, 1)
    E = 16 // np.dtype(dt).itemsize
    for m, n in [(1, 2), (3, 0), (t + 5, 2 * t - 3), (3 * t + 7, t + 1)]:
        A = sorted_keys(rng, m, dt, 500)
        B = sorted_keys(rng, n, dt, 500)
        want, src = oracle.merge(A, B)
        for s in range(E):
            for u in range(E):
                Ad, Bd = _view(A, s), _view(B, (s + u) % E)
                C = _empty_view(m + n, Ad.dtype, u)
                T = _empty_view(m + n, torch.int32, (3 * s + u) % 4)
                cr.merge(Ad, Bd, key_type=kt, tag=True, out=C, out_tag=T)
                torch.cuda.synchronize()
                assert same_bits(host(C, dt), want), (m, n, s, u)
                assert np.array_equal(host(T, np.uint32).astype(np.int64), src), (m, n, s, u)


@pytest.mark.parametrize("dt", [np.uint32, np.int64])
@pytest.mark.parametrize("vdt", [np.float32, np.float64])
def test_offset_views_kv_and_backward(dt, vdt):
    rng = np.random.default_rng(302)
    kt = key_type(np.empty(0, dt))
    vb = np.dtype(vdt).itemsize
    t = cr.tile_size(kt, vb, 1, 1)
    EK, EV = 16 // np.dtype(dt).itemsize, 16 // vb
    for m, n in [(2, 1), (2 * t + 3, t - 1), (t - 2, 4 * t + 5)]:
        A = sorted_keys(rng, m, dt, 200)
        B = sorted_keys(rng, n, dt, 200)
        Av = rng.standard_normal(m).astype(vdt)
        Bv = rng.standard_normal(n).astype(vdt)
        gC = rng.standard_normal(m + n).astype(vdt)
        wk, wv, _ = oracle.merge_kv(A, Av, B, Bv)
        ga, gb = oracle.merge_grad(A, B, gC)
        for s in range(max(EK, EV)):
            Ad, Bd = _view(A, s % EK), _view(B, (s + 1) % EK)
            Avd, Bvd = _view(Av, (s + 2) % EV), _view(Bv, (s + 3) % EV)
            Ck, Cv = cr.merge_kv(Ad, Avd, Bd, Bvd, key_type=kt)
            torch.cuda.synchronize()
            assert same_bits(host(Ck, dt), wk), (m, n, s)
            assert host(Cv, vdt).tobytes() == wv.tobytes(), (m, n, s)
            gA, gB = cr.merge_kv_backward(Ad, Bd, _view(gC, (s + 1) % EV), key_type=kt)
            torch.cuda.synchronize()
            assert host(gA, vdt).tobytes() == ga.tobytes(), (m, n, s)
            assert host(gB, vdt).tobytes() == gb.tobytes(), (m, n, s)


def test_offset_views_output_payloads_and_gradients():
    """Outputs written through offset views (the storer's bulk interior and
    its ragged edges both move), through the two-step form."""
    import ctypes
    from paper_1303_4312_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(303)
    t = cr.tile_size("i32", 4, 1, 1)
    m, n = 3 * t + 11, 2 * t - 7
    A = sorted_keys(rng, m, np.int32, 100)
    B = sorted_keys(rng, n, np.int32, 100)
    Av = rng.standard_normal(m).astype(np.float32)
    Bv = rng.standard_normal(n).astype(np.float32)
    gC = rng.standard_normal(m + n).astype(np.float32)
    wk, wv, _ = oracle.merge_kv(A, Av, B, Bv)
    ga, gb = oracle.merge_grad(A, B, gC)
    Ad, Bd, Avd, Bvd, gCd = dev(A), dev(B), dev(Av), dev(Bv), dev(gC)
    need = ctypes.c_size_t()
    _lib.check(lib.cr_merge_workspace_size(0, 4, m, n, ctypes.byref(need)))
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for u in range(4):
        Ck = _empty_view(m + n, torch.int32, u)
        Cv = _empty_view(m + n, torch.float32, 3 - u)
        gA = _empty_view(m, torch.float32, (u + 1) % 4)
        gB = _empty_view(n, torch.float32, (u + 2) % 4)
        _lib.check(lib.cr_merge_partition(0, 4, Ad.data_ptr(), m, Bd.data_ptr(), n,
                                          ws.data_ptr(), ws.numel(), s))
        _lib.check(lib.cr_merge_tiles(0, 4, Ad.data_ptr(), Avd.data_ptr(), m, Bd.data_ptr(),
                                      Bvd.data_ptr(), n, Ck.data_ptr(), Cv.data_ptr(), None,
                                      ws.data_ptr(), ws.numel(), s))
        _lib.check(lib.cr_merge_tiles_backward(0, 4, Ad.data_ptr(), m, Bd.data_ptr(), n,
                                               gCd.data_ptr(), gA.data_ptr(), gB.data_ptr(),
                                               ws.data_ptr(), ws.numel(), s))
        torch.cuda.synchronize()
        cr.workspace_status(ws)
        assert same_bits(host(Ck, np.int32), wk), u
        assert host(Cv, np.float32).tobytes() == wv.tobytes(), u
        assert host(gA, np.float32).tobytes() == ga.tobytes(), u
        assert host(gB, np.float32).tobytes() == gb.tobytes(), u
        # the views' neighbours are untouched
        base = Ck._base if Ck._base is not None else None
        if base is not None:
            assert int(base[:u].ne(-7).sum()) == 0 and int(base[u + m + n:].ne(-7).sum()) == 0


def test_offset_views_batched_and_pass():
    """The batched merge and a merge pass over offset views."""
    rng = np.random.default_rng(304)
    sizes_a = [0, 5, 3000, 1, 777]
    sizes_b = [4, 0, 2500, 9000, 1]
    a_off = np.concatenate([[0], np.cumsum(sizes_a)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(sizes_b)]).astype(np.int64)
    A = np.concatenate([np.sort(rng.integers(0, 50, s).astype(np.int32)) for s in sizes_a])
    B = np.concatenate([np.sort(rng.integers(0, 50, s).astype(np.int32)) for s in sizes_b])
    Av = rng.standard_normal(len(A)).astype(np.float32)
    Bv = rng.standard_normal(len(B)).astype(np.float32)
    wk, wv = oracle.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
    for s in range(4):
        Ck, Cv = cr.batched_merge_kv(a_off, b_off, _view(A, s), _view(Av, 3 - s),
                                     _view(B, (s + 1) % 4), _view(Bv, (s + 2) % 4))
        torch.cuda.synchronize()
        assert same_bits(host(Ck, np.int32), wk), s
        assert host(Cv, np.float32).tobytes() == wv.tobytes(), s
    # one merge pass (runs of 1000) and its recorded form
    X = np.concatenate([np.sort(rng.integers(0, 2**40, 1000, dtype=np.uint64))
                        for _ in range(9)])[:8500]
    Xv = rng.standard_normal(len(X)).astype(np.float32)
    wy, wyv, _ = oracle.merge_pass(X, Xv, 1000)
    Y, Yv = cr.merge_pass(_view(X, 1), _view(Xv, 3), 1000, key_type="u64")
    torch.cuda.synchronize()
    assert same_bits(host(Y, np.uint64), wy)
    assert host(Yv, np.float32).tobytes() == wyv.tobytes()


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
def test_host_result_co_rank(dt):
    """cr_co_rank (result on the host) against Algorithm 1 in the oracle,
    on offset views, at every rank of a small case and sampled ranks of a
    larger one."""
    rng = np.random.default_rng(305)
    kt = key_type(np.empty(0, dt))
    for m, n, ranks in [(7, 5, range(13)), (40000, 70001, None)]:
        A = sorted_keys(rng, m, dt, 30)
        B = sorted_keys(rng, n, dt, 30)
        Ad, Bd = _view(A, 1), _view(B, 0)
        if ranks is None:
            ranks = [0, 1, m, n, m + n - 1, m + n] + list(rng.integers(0, m + n, 40))
        for k in ranks:
            j, kk, _ = oracle.co_rank(int(k), A, B)
            assert cr.co_rank(Ad, Bd, int(k), key_type=kt) == (j, kk), k
        out = cr.api.co_rank_async(Ad, Bd, m, key_type=kt)
        torch.cuda.synchronize()
        j, kk, _ = oracle.co_rank(m, A, B)
        assert out.tolist() == [j, kk]


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("dt", [np.int32, np.uint64])
def test_sharded_merge_default_path_every_rank(world, dt):
    """shard.plan + shard.merge_block with this library's co_rank and merge
    (the default path of sharded_merge), for every rank of the group, run one
    after another on this GPU: the windows A[i0:i1], B[j0:j1] start at
    arbitrary elements.  Each block equals the oracle's output block, and the
    blocks concatenate to the whole merge."""
    rng = np.random.default_rng(306 + world)
    kt = key_type(np.empty(0, dt))
    for m, n in [(100003, 77777), (5, 123457), (1, 0)]:
        A = sorted_keys(rng, m, dt, 1000)
        B = sorted_keys(rng, n, dt, 1000)
        want, _ = oracle.merge(A, B)
        Ad, Bd = dev(A), dev(B)
        blocks = []
        for r in range(world):
            p = shard.plan(m, n, world, r, lambda k: cr.co_rank(Ad, Bd, k, key_type=kt))
            blk = shard.merge_block(Ad, Bd, p, lambda a, b: cr.merge(a, b, key_type=kt))
            torch.cuda.synchronize()
            lo, hi = shard.block_bounds(m + n, world, r)
            assert same_bits(host(blk, dt), want[lo:hi]), (m, n, r)
            blocks.append(host(blk, dt))
        assert same_bits(np.concatenate(blocks), want)
