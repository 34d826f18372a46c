"""The sharded merge plan on CPU ranks (gloo): every rank co-ranks the
ends of its equal output block, merges its windows, and the gathered blocks
equal the whole stable merge.  On these CPU ranks the local merges come
from the CPU oracle and the co-rank iterations of the block-distributed form
from HostSearch below (test-only injections: the library's kernels need a
GPU, where tests/test_gpu_dist.py runs them); the oracle checks every
result."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1303_4312_gb300 import shard


def _as_key(v: int, key_type: str) -> int:
    """A key read back from an int64 carrier (the stored key's bits, sign-
    or zero-extended from its width), as a Python int whose integer order is
    the key type's order: unsigned types are masked to their width; float
    bits (IEEE-754 totalOrder) keep positives and flip the magnitude of
    negatives; pairs of signed halves flip both sign bits; ':desc' negates."""
    base, _, mod = key_type.partition(":")
    bits = 32 if base in ("i32", "u32", "f32") else 64
    if base.startswith("pair"):
        v &= (1 << 64) - 1
        if base == "pair_i32":
            v ^= (1 << 63) | (1 << 31)
        return -v if mod == "desc" else v
    if base[0] == "u":
        v &= (1 << bits) - 1
    else:
        v = ((v + (1 << (bits - 1))) & ((1 << bits) - 1)) - (1 << (bits - 1))
        if base[0] == "f" and v < 0:
            v ^= (1 << (bits - 1)) - 1
    return -v if mod == "desc" else v


class HostSearch:
    """Test double of the library's block-distributed co-rank
    (api.DistCoRank) on CPU tensors: the same state (rank k, co-ranks i, j,
    their low bounds, finished flag), probes and Algorithm-1 iteration,
    written out in Python; keys compared through _as_key."""

    def __init__(self, m, n, ranks, key_type, device):
        self.m, self.n, self.kt = m, n, key_type
        self.st = [[k, min(k, m), k - min(k, m), max(0, k - n), max(0, k - m), False]
                   for k in ranks]

    def iterations(self):
        return int(min(self.m, self.n)).bit_length() + 1

    def probes(self):
        pa, pb = [], []
        for _, i, j, _, _, done in self.st:
            c1 = not done and i > 0 and j < self.n
            c2 = not done and j > 0 and i < self.m
            pa += [i - 1 if c1 else -1, i if c2 else -1]
            pb += [j - 1 if c2 else -1, j if c1 else -1]
        return torch.tensor(pa, dtype=torch.int64), torch.tensor(pb, dtype=torch.int64)

    def answer(self, blk, lo, idx):
        out = torch.zeros(idx.numel(), dtype=torch.int64)
        mine = (idx >= lo) & (idx < lo + blk.numel())
        if bool(mine.any()):
            out[mine] = blk[idx[mine] - lo].to(torch.int64)
        return out

    def step(self, va, vb):
        va, vb, key = va.tolist(), vb.tolist(), lambda v: _as_key(v, self.kt)
        for q, s in enumerate(self.st):
            _, i, j, il, jl, done = s
            if done:
                continue
            if i > 0 and j < self.n and key(vb[2 * q + 1]) < key(va[2 * q]):
                d = (i - il + 1) // 2
                s[4], s[1], s[2] = j, i - d, j + d
            elif j > 0 and i < self.m and not key(vb[2 * q]) < key(va[2 * q + 1]):
                d = (j - jl + 1) // 2
                s[3], s[1], s[2] = i, i + d, j - d
            else:
                s[5] = True

    def result(self):
        return [(s[1], s[2]) for s in self.st], sum(not s[5] for s in self.st)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cases, out_q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for A, B in cases:
            a, b = A.numpy(), B.numpy()
            co = lambda k: oracle.co_rank(k, a, b)[:2]
            merge = lambda x, y: torch.from_numpy(oracle.merge(x.numpy(), y.numpy())[0])
            C, p = shard.sharded_merge(A, B, co_rank=co, merge=merge)
            out_q.put((rank, p.size, C.numpy().tobytes()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_merge_two_cpu_ranks(world):
    import oracle
    rng = np.random.default_rng(110)
    cases = []
    for m, n, spread in [(1000, 777, 50), (0, 5, 3), (7, 0, 3), (1, 1, 2), (5001, 12, 1000)]:
        A = np.sort(rng.integers(0, spread, m)).astype(np.int64)
        B = np.sort(rng.integers(0, spread, n)).astype(np.int64)
        cases.append((torch.from_numpy(A), torch.from_numpy(B)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world * len(cases))]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for ci, (A, B) in enumerate(cases):
        want = oracle.merge(A.numpy(), B.numpy())[0].tobytes()
        got = [r for r in results if r[2] == want]
        assert len(got) >= world, f"case {ci}: gathered output differs from the stable merge"


def test_plan_blocks_are_balanced():
    """Proposition 2 for the rank blocks: sizes differ by at most one and the
    co-ranked windows tile A and B exactly."""
    import oracle
    rng = np.random.default_rng(111)
    a = np.sort(rng.integers(0, 9, 1234))
    b = np.sort(rng.integers(0, 9, 777))
    for world in (1, 2, 3, 7, 64):
        plans = [shard.plan(len(a), len(b), world, r, lambda k: oracle.co_rank(k, a, b)[:2])
                 for r in range(world)]
        sizes = [p.size for p in plans]
        assert max(sizes) - min(sizes) <= 1 and sum(sizes) == len(a) + len(b)
        assert plans[0].i0 == 0 and plans[-1].i1 == len(a)
        for p, q in zip(plans, plans[1:]):
            assert (p.k1, p.i1, p.j1) == (q.k0, q.i0, q.j0)
        blocks = [oracle.merge(a[p.i0:p.i1], b[p.j0:p.j1])[0] for p in plans]
        assert np.array_equal(np.concatenate(blocks), oracle.merge(a, b)[0])
    with pytest.raises(ValueError):
        shard.block_bounds(10, 2, 2)


def _dist_worker(rank, world, port, cases, out_q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for ci, (A, Av, B, Bv, a_cuts, b_cuts, kt) in enumerate(cases):
            a_blk = torch.from_numpy(A[a_cuts[rank]:a_cuts[rank + 1]].copy())
            b_blk = torch.from_numpy(B[b_cuts[rank]:b_cuts[rank + 1]].copy())
            dt = A.dtype

            def merge(x, y):
                return torch.from_numpy(oracle.merge(x.numpy().view(dt), y.numpy().view(dt))[0]
                                        .view(x.numpy().dtype))

            def merge_kv(x, xv, y, yv):
                c, cv, _ = oracle.merge_kv(x.numpy().view(dt), xv.numpy(), y.numpy().view(dt),
                                           yv.numpy())
                return torch.from_numpy(c.view(x.numpy().dtype)), torch.from_numpy(cv)

            a_t = torch.from_numpy(a_blk.numpy().view(np.int64 if dt.itemsize == 8 else np.int32))
            b_t = torch.from_numpy(b_blk.numpy().view(np.int64 if dt.itemsize == 8 else np.int32))
            if Av is None:
                C, p = shard.distributed_merge(a_t, b_t, kt, merge=merge, search=HostSearch)
                Cv = None
            else:
                av = torch.from_numpy(Av[a_cuts[rank]:a_cuts[rank + 1]].copy())
                bv = torch.from_numpy(Bv[b_cuts[rank]:b_cuts[rank + 1]].copy())
                C, Cv, p = shard.distributed_merge(a_t, b_t, kt, Av_blk=av, Bv_blk=bv,
                                                   merge=merge_kv, search=HostSearch)
            out_q.put((ci, rank, (p.k0, p.k1, p.i0, p.i1, p.j0, p.j1), C.numpy().tobytes(),
                       None if Cv is None else Cv.numpy().tobytes()))
    finally:
        dist.destroy_process_group()


def _cuts(rng, total, world):
    """Random block boundaries 0 = c0 <= c1 <= ... <= c_world = total (some
    blocks empty)."""
    inner = np.sort(rng.integers(0, total + 1, world - 1))
    if world > 2:
        inner[0] = inner[1]          # one empty block
    return [0, *inner.tolist(), total]


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_merge_block_inputs(world):
    """Block-distributed A and B: Algorithm 1 with remote point reads finds
    every rank's block co-ranks, the windows are fetched from their owners,
    and each rank's merged block equals that slice of the stable merge
    (keys and payloads), for signed and unsigned orders."""
    import oracle
    rng = np.random.default_rng(112 + world)
    cases = []
    for m, n, spread, dt, kv in [(1000, 777, 50, np.int32, False), (0, 9, 3, np.int32, False),
                                 (7, 0, 3, np.int64, True), (1, 1, 2, np.int32, False),
                                 (5001, 12, 1000, np.uint64, True), (300, 4000, 7, np.uint32, True),
                                 (2048, 2048, None, np.uint64, False)]:
        info = np.iinfo(dt)
        if spread is None:
            A = np.sort(rng.integers(info.min, info.max, m, dtype=dt, endpoint=True))
            B = np.sort(rng.integers(info.min, info.max, n, dtype=dt, endpoint=True))
        else:
            top = dt(info.max - spread) if info.min == 0 else dt(0)
            A = np.sort(rng.integers(0, spread, m).astype(dt) + top)
            B = np.sort(rng.integers(0, spread, n).astype(dt) + top)
        Av = rng.standard_normal(m).astype(np.float32) if kv else None
        Bv = rng.standard_normal(n).astype(np.float32) if kv else None
        kt = {np.int32: "i32", np.uint32: "u32", np.int64: "i64", np.uint64: "u64"}[dt]
        cases.append((A, Av, B, Bv, _cuts(rng, m, world), _cuts(rng, n, world), kt))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dist_worker, args=(r, world, port, cases, q))
             for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=180) for _ in range(world * len(cases))]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for ci, (A, Av, B, Bv, _, _, _) in enumerate(cases):
        if Av is None:
            want, _ = oracle.merge(A, B)
            wantv = None
        else:
            want, wantv, _ = oracle.merge_kv(A, Av, B, Bv)
        got = sorted((r for r in results if r[0] == ci), key=lambda r: r[1])
        assert len(got) == world
        for rank, (_, _, (k0, k1, i0, i1, j0, j1), cb, cvb) in enumerate(got):
            assert (k0, k1) == shard.block_bounds(len(A) + len(B), world, rank)
            assert (i0, j0) == tuple(oracle.co_rank(k0, A, B)[:2])
            assert (i1, j1) == tuple(oracle.co_rank(k1, A, B)[:2])
            assert cb == want[k0:k1].tobytes(), (ci, rank)
            if wantv is not None:
                assert cvb == wantv[k0:k1].tobytes(), (ci, rank)


@pytest.mark.parametrize("kt", ["i32", "u32", "i64", "u64", "f32", "f64", "pair_u32", "pair_i32",
                                "i32:desc", "f64:desc", "pair_i32:desc"])
def test_remote_key_order_matches_oracle(kt):
    """The CPU test double compares keys read back through int64 carriers
    (_as_key): their order must be the oracle's order for every key type,
    including floats (totalOrder), pairs and descending orders."""
    import oracle
    rng = np.random.default_rng(113)
    base = kt.split(":")[0]
    width = 32 if base in ("i32", "u32", "f32") else 64
    ut = np.uint32 if width == 32 else np.uint64
    bits = rng.integers(0, np.iinfo(ut).max, 3000, dtype=ut, endpoint=True)
    bits[:30] = bits[30:60]
    st = {32: np.int32, 64: np.int64}[width]
    carriers = bits.view(st).astype(np.int64)        # what the ranks all-reduce
    keys = [_as_key(int(v), kt) for v in carriers]
    ref = np.argsort(oracle.order_key(bits, kt if base[0] != "f" else kt), kind="stable")
    got = sorted(range(len(keys)), key=lambda i: keys[i])
    assert np.array_equal(got, ref)


def _dist_order_worker(rank, world, port, cases, out_q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for ci, (A, B, a_cuts, b_cuts, kt) in enumerate(cases):
            dt = A.dtype
            carrier = np.int64 if dt.itemsize == 8 else np.int32

            def merge(x, y):
                c, _ = oracle.merge_in_order(x.numpy().view(dt), y.numpy().view(dt), kt)
                return torch.from_numpy(c.view(carrier))

            a_t = torch.from_numpy(A[a_cuts[rank]:a_cuts[rank + 1]].copy().view(carrier))
            b_t = torch.from_numpy(B[b_cuts[rank]:b_cuts[rank + 1]].copy().view(carrier))
            C, p = shard.distributed_merge(a_t, b_t, kt, merge=merge, search=HostSearch)
            out_q.put((ci, rank, (p.k0, p.k1, p.i0, p.i1, p.j0, p.j1), C.numpy().tobytes()))
    finally:
        dist.destroy_process_group()


def _in_order(x, kt):
    import oracle
    return x[np.argsort(oracle.order_key(x, kt), kind="stable")]


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_merge_in_key_orders(world):
    """Block-distributed A and B in other key orders (IEEE totalOrder floats
    with NaNs of both signs, signed zeros and infinities; descending; signed
    32-bit pairs): the remote co-ranks equal the oracle's co-ranks of the
    order keys, and every rank's block equals that slice of the oracle's
    merge in that order."""
    import oracle
    rng = np.random.default_rng(140 + world)
    specials32 = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan], np.float32)
    cases = []
    for kt, m, n in [("f32", 700, 555), ("f64:desc", 300, 901), ("i64:desc", 64, 0),
                     ("pair_i32", 1000, 777), ("f32:desc", 0, 33)]:
        base = kt.split(":")[0]
        if base == "f32":
            A = rng.standard_normal(m).astype(np.float32)
            B = rng.standard_normal(n).astype(np.float32)
            A[: min(m, 6)] = specials32[: min(m, 6)]
            B[: min(n, 6)] = specials32[: min(n, 6)]
        elif base == "f64":
            A = np.round(rng.standard_normal(m), 1)
            B = np.round(rng.standard_normal(n), 1)
        elif base == "i64":
            A = rng.integers(-5, 5, m).astype(np.int64)
            B = rng.integers(-5, 5, n).astype(np.int64)
        else:
            major = rng.integers(0, 4, m + n).astype(np.uint64) * np.uint64(0x7FFFFFFF)
            minor = rng.integers(0, 2**32, m + n, dtype=np.uint64)
            w = (major << np.uint64(32)) | minor
            A, B = w[:m].copy(), w[m:].copy()
        A, B = _in_order(A, kt), _in_order(B, kt)
        cases.append((A, B, _cuts(rng, m, world), _cuts(rng, n, world), kt))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dist_order_worker, args=(r, world, port, cases, q))
             for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=180) for _ in range(world * len(cases))]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for ci, (A, B, _, _, kt) in enumerate(cases):
        want, _ = oracle.merge_in_order(A, B, kt)
        ka, kb = oracle.order_key(A, kt), oracle.order_key(B, kt)
        got = sorted((r for r in results if r[0] == ci), key=lambda r: r[1])
        assert len(got) == world
        for rank, (_, _, (k0, k1, i0, i1, j0, j1), cb) in enumerate(got):
            assert (k0, k1) == shard.block_bounds(len(A) + len(B), world, rank)
            assert (i0, j0) == tuple(oracle.co_rank(k0, ka, kb)[:2]), (kt, rank)
            assert (i1, j1) == tuple(oracle.co_rank(k1, ka, kb)[:2]), (kt, rank)
            assert cb == want[k0:k1].tobytes(), (kt, rank)
