"""GPU parity of the block-distributed co-rank (cr_dist_co_rank_*: Algorithm
1 with remote point reads, the distributed reading of Algorithm 2 in
Section 3).  The ranks of a process group are emulated one after another on
this GPU: every emulated rank answers the probes that fall in its own blocks
with the library's answer kernel, the answers are summed on the device (what
the all-reduce does between real ranks), and the library's step kernel runs
the iteration.  The co-ranks of every block boundary equal the CPU oracle's
Algorithm 1, in every key order, within the iteration bound."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import dev
from paper_1303_4312_gb300 import api, shard

pytestmark = pytest.mark.gpu


def _cuts(rng, total, world):
    inner = np.sort(rng.integers(0, total + 1, world - 1))
    if world > 2:
        inner[0] = inner[1]              # one empty block
    return [0, *inner.tolist(), total]


def _emulated_co_ranks(A, B, a_cuts, b_cuts, ks, kt):
    world = len(a_cuts) - 1
    a_blk = [dev(A[a_cuts[r]:a_cuts[r + 1]]) for r in range(world)]
    b_blk = [dev(B[b_cuts[r]:b_cuts[r + 1]]) for r in range(world)]
    s = api.DistCoRank(len(A), len(B), ks, kt, "cuda")
    for _ in range(s.iterations()):
        pa, pb = s.probes()
        va = sum(s.answer(a_blk[r], a_cuts[r], pa) for r in range(world))
        vb = sum(s.answer(b_blk[r], b_cuts[r], pb) for r in range(world))
        s.step(va, vb)
    return s.result()


def _in_order(x, kt):
    return x[np.argsort(oracle.order_key(x, kt), kind="stable")]


@pytest.mark.parametrize("world", [2, 3, 8])
def test_block_distributed_co_rank_matches_oracle(world):
    rng = np.random.default_rng(700 + world)
    for m, n, dt, spread in [(100003, 77777, np.int32, 50), (0, 999, np.int32, 3),
                             (5, 123457, np.uint64, None), (40000, 40000, np.uint32, 7),
                             (1, 1, np.int64, 2), (3000, 2, np.int64, None)]:
        info = np.iinfo(dt)
        if spread is None:
            A = np.sort(rng.integers(info.min, info.max, m, dtype=dt, endpoint=True))
            B = np.sort(rng.integers(info.min, info.max, n, dtype=dt, endpoint=True))
        else:
            A = np.sort(rng.integers(0, spread, m).astype(dt))
            B = np.sort(rng.integers(0, spread, n).astype(dt))
        kt = {np.int32: "i32", np.uint32: "u32", np.int64: "i64", np.uint64: "u64"}[dt]
        ks = [shard.block_bounds(m + n, world, g)[0] for g in range(world)] + [m + n]
        res, live = _emulated_co_ranks(A, B, _cuts(rng, m, world), _cuts(rng, n, world), ks, kt)
        assert live == 0
        for k, (i, j) in zip(ks, res):
            assert (i, j) == tuple(oracle.co_rank(k, A, B)[:2]), (m, n, kt, k)


def test_block_distributed_co_rank_every_rank_and_key_order():
    """Every output rank of small cases (the searches need not be block
    boundaries), in IEEE totalOrder floats with signed zeros, infinities and
    NaNs, descending orders and lexicographic pairs, against Algorithm 1 on
    the oracle's order keys; a rank outside [0, m + n] comes back as (-1, -1)."""
    rng = np.random.default_rng(710)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan], np.float32)
    for kt, m, n in [("f32", 300, 211), ("f64:desc", 97, 160), ("i32:desc", 50, 50),
                     ("pair_i32", 128, 255), ("u64:desc", 0, 31)]:
        base = kt.split(":")[0]
        if base == "f32":
            A = rng.standard_normal(m).astype(np.float32)
            B = rng.standard_normal(n).astype(np.float32)
            A[:6], B[:6] = specials, specials
        elif base == "f64":
            A = np.round(rng.standard_normal(m), 1)
            B = np.round(rng.standard_normal(n), 1)
        elif base == "pair_i32":
            major = rng.integers(0, 3, m + n).astype(np.uint64) * np.uint64(0x7FFFFFFF)
            w = (major << np.uint64(32)) | rng.integers(0, 2**32, m + n, dtype=np.uint64)
            A, B = w[:m].copy(), w[m:].copy()
        elif base == "u64":
            A = rng.integers(0, 2**64, m, dtype=np.uint64)
            B = rng.integers(0, 2**64, n, dtype=np.uint64)
        else:
            A = rng.integers(-4, 4, m).astype(np.int32)
            B = rng.integers(-4, 4, n).astype(np.int32)
        A, B = _in_order(A, kt), _in_order(B, kt)
        ks = list(range(m + n + 1)) + [m + n + 1, -1]
        res, live = _emulated_co_ranks(A, B, _cuts(rng, m, 3), _cuts(rng, n, 3), ks, kt)
        assert live == 0
        ka, kb = oracle.order_key(A, kt), oracle.order_key(B, kt)
        for k, (i, j) in zip(ks[:-2], res):
            assert (i, j) == tuple(oracle.co_rank(k, ka, kb)[:2]), (kt, k)
        assert res[-2:] == [(-1, -1), (-1, -1)]
