"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times: every output element compared with the CPU oracle (keys,
payloads, tags and gradients bit for bit).

Workloads (seeded; device-generated with torch, then copied to the host for
the oracle):
  single_i32_tag   m=2^20, n=3*2^19 int32 in [0, 2^16) + uint32 source tags
  large_i32        m=n=2^28 int32 over the full range
  skewed_u64       m=2^20, n=2^29 uint64 over the full range
  dup16_i32        m=n=2^28 int32 from 16 distinct values
  kv_u32_f32       m=n=2^27 uint32 keys in [0, 2^20), float32 payloads, + backward
  batched_i32_f32  8192 log-uniform segment pairs (~3.4e8 elements), + backward
  sort_u64_f32     2^27 uint64 keys (2^20 distinct) from runs of 1024, + backward
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1303_4312_gb300 as cr
from paper_1303_4312_gb300 import workloads as W
from gpu_util import host, same_bits

pytestmark = pytest.mark.gpu


def _free():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_single_i32_tag_full():
    A, B = W.single_i32_tag(seed=1)
    C, T = cr.merge(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), tag=True)
    torch.cuda.synchronize()
    want, src = oracle.merge(A, B)
    assert np.array_equal(C.cpu().numpy(), want)
    assert np.array_equal(host(T, np.uint32).astype(np.int64), src)
    # stability witness: among equal keys, tags strictly increase
    tags = host(T, np.uint32).astype(np.int64)
    eq = want[1:] == want[:-1]
    assert np.all(tags[1:][eq] > tags[:-1][eq])


@pytest.mark.parametrize("name", ["large_i32", "skewed_u64", "dup16_i32"])
def test_large_single_merge_full(name):
    gen = {"large_i32": W.t_large_i32, "skewed_u64": W.t_skewed_u64,
           "dup16_i32": W.t_dup16_i32}[name]
    A, B = gen()
    kt = "u64" if name == "skewed_u64" else "i32"
    hdt = np.uint64 if kt == "u64" else np.int32
    C = cr.merge(A, B, key_type=kt)
    torch.cuda.synchronize()
    a, b = host(A, hdt), host(B, hdt)
    del A, B
    c = host(C, hdt)
    del C
    _free()
    want, _ = oracle.merge(a, b)
    assert np.array_equal(c, want)


def test_kv_u32_f32_full_forward_backward():
    Ak, Av, Bk, Bv = W.t_kv_u32_f32()
    Ck, Cv = cr.merge_kv(Ak, Av, Bk, Bv, key_type="u32")
    g = torch.Generator(device="cuda").manual_seed(55)
    gC = torch.randn(Ck.numel(), generator=g, device="cuda")
    gA, gB = cr.merge_kv_backward(Ak, Bk, gC, key_type="u32")
    torch.cuda.synchronize()
    a, av, b, bv = host(Ak, np.uint32), host(Av, np.float32), host(Bk, np.uint32), host(Bv, np.float32)
    wk, wv, _ = oracle.merge_kv(a, av, b, bv)
    assert np.array_equal(host(Ck, np.uint32), wk)
    assert same_bits(host(Cv, np.float32), wv)
    del wk, wv
    ga, gb = oracle.merge_grad(a, b, host(gC, np.float32))
    assert same_bits(host(gA, np.float32), ga)
    assert same_bits(host(gB, np.float32), gb)


def test_kv_autograd_small():
    """torch.autograd.Function: backward routes grad(Cv) by recomputed co-ranks."""
    Ak, Av, Bk, Bv = W.t_kv_u32_f32(shift=10)
    Av.requires_grad_(True)
    Bv.requires_grad_(True)
    Ck, Cv = cr.MergeKV.apply(Ak, Av, Bk, Bv, "u32")
    w = torch.randn(Cv.numel(), device="cuda")
    (Cv * w).sum().backward()
    a, b = host(Ak, np.uint32), host(Bk, np.uint32)
    ga, gb = oracle.merge_grad(a, b, host(w, np.float32))
    assert same_bits(host(Av.grad, np.float32), ga)
    assert same_bits(host(Bv.grad, np.float32), gb)


def test_batched_full_forward_backward():
    a_off, b_off, A, Av, B, Bv = W.t_batched_i32_f32()
    Ck, Cv = cr.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
    gC = torch.randn(Ck.numel(), generator=torch.Generator(device="cuda").manual_seed(56),
                     device="cuda")
    gA, gB = cr.batched_merge_kv_backward(a_off, b_off, A, B, gC)
    torch.cuda.synchronize()
    a, av, b, bv = host(A, np.int32), host(Av, np.float32), host(B, np.int32), host(Bv, np.float32)
    wk, wv = oracle.batched_merge_kv(a_off, b_off, a, av, b, bv)
    assert np.array_equal(host(Ck, np.int32), wk)
    assert same_bits(host(Cv, np.float32), wv)
    del wk, wv
    ga, gb = oracle.batched_merge_grad(a_off, b_off, a, b, host(gC, np.float32))
    assert same_bits(host(gA, np.float32), ga)
    assert same_bits(host(gB, np.float32), gb)


def test_batched_graph_capture_replays():
    """The batched forward and backward captured into CUDA graphs
    (BatchedMergeGraph) and replayed on two sets of inputs for one segment
    table (log-uniform sizes as in the batched workload, with empty
    segments), against the oracle bit for bit."""
    rng = np.random.default_rng(57)
    ms, ns = W.log_uniform_sizes(58, 300, max_log2=14)
    ms[5] = 0
    ns[7] = 0
    a_off, b_off = W.offsets(ms), W.offsets(ns)
    g = cr.BatchedMergeGraph(a_off, b_off, torch.int32, torch.float32, "cuda")
    for rep in range(2):
        A = np.concatenate([np.sort(rng.integers(0, 1 << 24, m)) for m in ms]).astype(np.int32)
        B = np.concatenate([np.sort(rng.integers(0, 1 << 24, n)) for n in ns]).astype(np.int32)
        Av = rng.standard_normal(len(A)).astype(np.float32)
        Bv = rng.standard_normal(len(B)).astype(np.float32)
        gC = rng.standard_normal(len(A) + len(B)).astype(np.float32)
        Ck, Cv = g.forward(torch.from_numpy(A).cuda(), torch.from_numpy(Av).cuda(),
                           torch.from_numpy(B).cuda(), torch.from_numpy(Bv).cuda())
        torch.cuda.synchronize()
        wk, wv = oracle.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
        assert np.array_equal(host(Ck, np.int32), wk), rep
        assert same_bits(host(Cv, np.float32), wv), rep
        gA, gB = g.backward(torch.from_numpy(gC).cuda())
        torch.cuda.synchronize()
        g.check()
        ga, gb = oracle.batched_merge_grad(a_off, b_off, A, B, gC)
        assert same_bits(host(gA, np.float32), ga), rep
        assert same_bits(host(gB, np.float32), gb), rep


def test_merge_sort_full_graph_forward_backward():
    X, Xv = W.t_sort_u64_f32()
    Xv.requires_grad_(True)
    Y, Yv = cr.merge_sort(X, Xv, run=1024, key_type="u64", graph=True)
    gY = torch.randn(Yv.numel(), generator=torch.Generator(device="cuda").manual_seed(57),
                     device="cuda")
    Yv.backward(gY)
    torch.cuda.synchronize()
    x, xv = host(X, np.uint64), host(Xv.detach(), np.float32)
    o = np.argsort(x, kind="stable")          # independent of the oracle and of the GPU path
    assert np.array_equal(host(Y, np.uint64), x[o])
    assert same_bits(host(Yv.detach(), np.float32), xv[o])
    want = np.empty_like(xv)
    want[o] = host(gY, np.float32)
    assert same_bits(host(Xv.grad, np.float32), want)
    # and the oracle's own merge chain agrees
    wy, wyv, perm = oracle.merge_sort(x, xv, 1024)
    assert np.array_equal(perm, o)


def test_merge_beyond_2_31_elements_sampled():
    """64-bit indexing: a merge of m + n = 2^31 + 3000 int32 keys (8.6 GB in,
    8.6 GB out).  Checked at sampled output ranks one by one against the
    oracle's Algorithm 1 (the element at rank r is A[i] or B[j] of the
    oracle's co-rank of r), plus order and multiset properties on the device."""
    m, n = (1 << 30) + 1000, (1 << 30) + 2000
    g = torch.Generator(device="cuda").manual_seed(99)
    A = torch.sort(torch.randint(-(1 << 31), 1 << 31, (m,), generator=g, device="cuda",
                                 dtype=torch.int64).to(torch.int32)).values
    B = torch.sort(torch.randint(-(1 << 31), 1 << 31, (n,), generator=g, device="cuda",
                                 dtype=torch.int64).to(torch.int32)).values
    C = cr.merge(A, B)
    torch.cuda.synchronize()
    assert bool((C[1:] >= C[:-1]).all())
    assert int(C.to(torch.int64).sum()) == int(A.to(torch.int64).sum()) + int(B.to(torch.int64).sum())
    a, b = A.cpu().numpy(), B.cpu().numpy()
    rng = np.random.default_rng(9)
    ranks = np.unique(np.concatenate([rng.integers(0, m + n, 200),
                                      [0, m + n - 1, (1 << 31) - 1, 1 << 31, (1 << 31) + 1]]))
    j, k = oracle.co_rank_many(a, b, ranks)
    c = C[torch.from_numpy(ranks).cuda()].cpu().numpy()
    for r, jj, kk, got in zip(ranks, j, k, c):
        take_b = kk < n and (jj >= m or b[kk] < a[jj])
        assert got == (b[kk] if take_b else a[jj]), r
    # the device co-rank at the same ranks agrees with the oracle
    oi, oj = cr.co_rank_many(A, B, torch.from_numpy(ranks).cuda())
    assert np.array_equal(oi.cpu().numpy(), j) and np.array_equal(oj.cpu().numpy(), k)


def test_merge_sort_beyond_2_31_elements_properties():
    """64-bit indexing through the whole sort chain (run formation in the
    shared-memory stage, then 20 recorded passes) on 2^31 + 4097 unsorted
    int32 keys with many ties.  The payload of element x is its index x (as
    uint32 bits), so the result is checked exactly by properties that fix a
    stable sort at any size: the keys come out ordered, the payloads form a
    permutation that reproduces them (Y[t] = X[idx[t]]), equal keys keep
    increasing indices (stability), and the payload gradient is routed
    through that same permutation (gX[idx[t]] = gY[t]).  The checks run in
    chunks and are reduced to plain booleans before any assert, so a failure
    never formats a 2^31-element tensor."""
    _free()
    N = (1 << 31) + 4097
    g = torch.Generator(device="cuda").manual_seed(131)
    X = torch.randint(0, 1 << 20, (N,), generator=g, device="cuda", dtype=torch.int32)
    Xv = torch.arange(N, device="cuda", dtype=torch.int64).to(torch.int32)
    Xv = Xv.view(torch.float32).clone().requires_grad_(True)     # index bits as payload
    Y, Yv = cr.merge_sort(X, Xv, key_type="i32")
    gY = torch.arange(N, device="cuda", dtype=torch.int64).mul_(7).remainder_(1 << 23)
    gY = gY.to(torch.int32).view(torch.float32)                  # exact, distinct bit patterns
    Yv.backward(gY)
    torch.cuda.synchronize()
    ok = {"sorted": True, "gather": True, "stable": True, "grad": True}
    seen = torch.zeros(N, dtype=torch.int8, device="cuda")
    gX, gy, pv = Xv.grad.view(torch.int32), gY.view(torch.int32), Yv.detach().view(torch.int32)
    C = 1 << 28
    for c0 in range(0, N, C):
        c1 = min(N, c0 + C)
        p = pv[c0:c1].to(torch.int64) & 0xFFFFFFFF              # idx[t], read as uint32
        y = Y[c0:c1]
        ok["sorted"] &= bool((y[1:] >= y[:-1]).all())
        ok["stable"] &= bool(((p[1:] > p[:-1]) | (y[1:] != y[:-1])).all())
        if c0 > 0:                                               # across the chunk seam
            yp, y0 = int(Y[c0 - 1]), int(y[0])
            pp, p0 = int(pv[c0 - 1]) & 0xFFFFFFFF, int(p[0])
            ok["sorted"] &= yp <= y0
            ok["stable"] &= yp != y0 or pp < p0
        ok["gather"] &= bool((X[p] == y).all())
        ok["grad"] &= bool((gX[p] == gy[c0:c1]).all())
        seen[p] = 1
        del p, y
    ok["permutation"] = bool(seen.all())
    # release the ~115 GB before asserting: a failing test's frame would
    # otherwise keep it alive for the rest of the session
    del seen, gX, gy, pv, X, Xv, Y, Yv, gY
    _free()
    assert all(ok.values()), ok
