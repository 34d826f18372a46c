"""The synthetic input recipes (paper_1303_4312_gb300/workloads.py) produce
what the design states: sizes, value ranges, distinct-value counts, sorted
inputs, seeded determinism, and the same segment tables on the host and the
device generators.  All on the CPU, at reduced sizes where the recipe takes
a size shift."""
import numpy as np
import pytest
import torch

from paper_1303_4312_gb300 import workloads as W


def is_sorted(x):
    return bool(np.all(x[1:] >= x[:-1]))


def test_batched_segment_table():
    """8192 pairs, each size log-uniform in [1, 2^18], drawn independently for
    A and B: seeded total 334,605,537 elements; the x3 variant of 24,576
    pairs totals 1,026,276,529 (about 2^30)."""
    ms, ns = W.log_uniform_sizes(6, 8192)
    assert len(ms) == len(ns) == 8192
    assert ms.min() >= 1 and ns.min() >= 1 and ms.max() <= 1 << 18 and ns.max() <= 1 << 18
    assert int(ms.sum() + ns.sum()) == 334_605_537
    assert not np.array_equal(ms, ns)
    ms3, ns3 = W.log_uniform_sizes(6, 24576)
    assert int(ms3.sum() + ns3.sum()) == 1_026_276_529
    # log-uniform: about as many sizes in each octave
    octaves = np.bincount(np.floor(np.log2(np.concatenate([ms, ns]))).astype(int), minlength=19)
    assert octaves[:18].min() > 0.5 * octaves[:18].mean()


def test_single_i32_tag():
    A, B = W.single_i32_tag(seed=1)
    assert (A.dtype, B.dtype) == (np.int32, np.int32)
    assert (len(A), len(B)) == (1 << 20, 3 << 19)
    assert is_sorted(A) and is_sorted(B)
    assert A.min() >= 0 and max(A.max(), B.max()) < 1 << 16


@pytest.mark.parametrize("gen,m,n,dt", [("large_i32", 1 << 22, 1 << 22, np.int32),
                                        ("skewed_u64", 1 << 14, 1 << 23, np.uint64),
                                        ("dup16_i32", 1 << 22, 1 << 22, np.int32)])
def test_large_merges_at_one_64th(gen, m, n, dt):
    A, B = getattr(W, gen)(shift=6)
    assert (A.dtype, B.dtype, len(A), len(B)) == (dt, dt, m, n)
    assert is_sorted(A) and is_sorted(B)
    if gen == "dup16_i32":
        assert len(np.unique(np.concatenate([A, B]))) == 16
    elif dt == np.int32:
        assert A.min() < -(1 << 30) and A.max() > 1 << 30        # full signed range
    else:
        assert B.max() > np.uint64(1 << 63)                       # full unsigned range


def test_kv_and_sort_inputs():
    Ak, Av, Bk, Bv = W.kv_u32_f32(shift=6)
    assert Ak.dtype == np.uint32 and Av.dtype == np.float32 and len(Ak) == 1 << 21
    assert is_sorted(Ak) and is_sorted(Bk) and max(Ak.max(), Bk.max()) < 1 << 20
    X, Xv = W.sort_u64_f32(shift=9)
    assert X.dtype == np.uint64 and Xv.dtype == np.float32 and len(X) == 1 << 18
    assert all(is_sorted(X[a:a + 1024]) for a in range(0, len(X), 1024))
    assert len(np.unique(X)) <= 1 << 20
    Xu, _ = W.sort_u64_f32(shift=9, run=None)
    assert not all(is_sorted(Xu[a:a + 1024]) for a in range(0, len(Xu), 1024))


def test_seeded_determinism():
    a1, b1 = W.single_i32_tag(seed=1, shift=4)
    a2, b2 = W.single_i32_tag(seed=1, shift=4)
    a3, _ = W.single_i32_tag(seed=2, shift=4)
    assert a1.tobytes() == a2.tobytes() and b1.tobytes() == b2.tobytes()
    assert a1.tobytes() != a3.tobytes()


def test_device_generators_match_the_recipes():
    """The torch generators (run here on the CPU device) give the same shapes
    and properties, and the batched one the same segment table as the host
    generator."""
    dev = torch.device("cpu")
    A, B = W.t_large_i32(device=dev, shift=6)
    assert A.dtype == torch.int32 and A.numel() == B.numel() == 1 << 22
    assert bool((A[1:] >= A[:-1]).all()) and bool((B[1:] >= B[:-1]).all())
    a_off, b_off, Ak, _, Bk, _ = W.t_batched_i32_f32(nseg=64, device=dev)
    ha, hb, *_ = W.batched_i32_f32(nseg=64)
    assert np.array_equal(a_off.cpu().numpy() if torch.is_tensor(a_off) else a_off, ha)
    assert np.array_equal(b_off.cpu().numpy() if torch.is_tensor(b_off) else b_off, hb)
    a = Ak.numpy()
    offs = ha
    assert all(is_sorted(a[offs[q]:offs[q + 1]]) for q in range(64))
    X, Xv = W.t_sort_u64_f32(device=dev, shift=10)
    x = X.numpy().view(np.uint64)
    assert all(is_sorted(x[a:a + 1024]) for a in range(0, len(x), 1024))
