"""The sharded merge plan on two CPU ranks (gloo): every rank co-ranks the
ends of its equal output block, merges its windows, and the gathered blocks
equal the whole stable merge.  Co-rank and local merge come from the CPU
oracle here (test-only injection); on GPUs they are the library's kernels."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1303_4312_gb300 import shard


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
