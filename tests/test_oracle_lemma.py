"""Pins of the CPU oracle's co-rank and merge to Lemma 1, Propositions 1-2,
brute force and closed forms -- all independent of the oracle's own code."""
import itertools
import math

import numpy as np
import pytest

import oracle

DTYPES = [np.int32, np.uint32, np.int64, np.uint64]


def brute_merge(A, B):
    """Stable sort of the origin-tagged concatenation A || B with Python's
    (stable) sorted: equal keys keep A-before-B and their order inside each
    array, which is exactly the stable merge of Section 2."""
    tagged = [(int(x), t) for t, x in enumerate(list(A) + list(B))]
    out = sorted(tagged, key=lambda e: e[0])
    return [e[0] for e in out], [e[1] for e in out]


def lemma1(A, B, i, j):
    """Both conditions of Lemma 1 for the split j + k = i (int compare)."""
    m, n = len(A), len(B)
    k = i - j
    if not (0 <= j <= m and 0 <= k <= n):
        return False
    c1 = j == 0 or k == n or int(A[j - 1]) <= int(B[k])
    c2 = k == 0 or j == m or int(B[k - 1]) < int(A[j])
    return c1 and c2


def small_cases(seed, count, max_len=12):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        m = int(rng.integers(0, max_len + 1))
        n = int(rng.integers(0, max_len + 1))
        spread = int(rng.choice([1, 2, 3, 50]))
        A = np.sort(rng.integers(0, spread, m)).astype(np.int32)
        B = np.sort(rng.integers(0, spread, n)).astype(np.int32)
        yield A, B


def test_lemma1_every_rank_and_unique():
    """For every rank i of small cases: the returned (j, k) satisfies both
    Lemma 1 conditions, and it is the only split that does (enumeration)."""
    for A, B in small_cases(11, 1500):
        m, n = len(A), len(B)
        for i in range(m + n + 1):
            j, k, _ = oracle.co_rank(i, A, B)
            assert j + k == i
            assert lemma1(A, B, i, j)
            ok = [jj for jj in range(max(0, i - n), min(i, m) + 1) if lemma1(A, B, i, jj)]
            assert ok == [j]


def test_prefix_property_vs_brute_force():
    """Lemma 1's prefix property: j = number of A elements among the first i
    outputs of the stable merge, taken from brute force."""
    for A, B in small_cases(12, 800):
        m = len(A)
        keys, tags = brute_merge(A, B)
        for i in range(len(keys) + 1):
            j, k, _ = oracle.co_rank(i, A, B)
            assert j == sum(1 for t in tags[:i] if t < m)


@pytest.mark.parametrize("dt", DTYPES)
def test_merge_vs_brute_force(dt):
    """The sequential merge equals the stable sort of the tagged concatenation
    (keys and source positions), for every key type."""
    for A, B in small_cases(13, 600):
        A = A.astype(dt)
        B = B.astype(dt)
        C, src = oracle.merge(A, B)
        keys, tags = brute_merge(A, B)
        assert [int(x) for x in C] == keys
        assert list(src) == tags


def test_key_order_signed_and_unsigned():
    """int32/int64 compare signed, uint32/uint64 unsigned: the same bit
    patterns merge into different orders."""
    rng = np.random.default_rng(5)
    for dt in DTYPES:
        info = np.iinfo(dt)
        for _ in range(50):
            A = np.sort(rng.integers(info.min, info.max, 20, dtype=dt, endpoint=True))
            B = np.sort(rng.integers(info.min, info.max, 17, dtype=dt, endpoint=True))
            C, src = oracle.merge(A, B)
            keys, tags = brute_merge(A, B)
            assert [int(x) for x in C] == keys
            assert list(src) == tags


def test_all_ranks_exhaustive_tiny():
    """Every pair of sorted sequences over {0,1,2} with m, n <= 4, every rank."""
    seqs = [()]
    for L in range(1, 5):
        seqs += list(itertools.combinations_with_replacement(range(3), L))
    for a in seqs:
        for b in seqs:
            A = np.array(a, dtype=np.int64)
            B = np.array(b, dtype=np.int64)
            _, tags = brute_merge(A, B)
            for i in range(len(a) + len(b) + 1):
                j, k, _ = oracle.co_rank(i, A, B)
                assert j == sum(1 for t in tags[:i] if t < len(a))


def test_closed_forms():
    """Special cases with a closed-form answer."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        m = int(rng.integers(0, 40))
        n = int(rng.integers(0, 40))
        A = np.sort(rng.integers(0, 100, m)).astype(np.int64)
        B = np.sort(rng.integers(0, 100, n)).astype(np.int64)
        for i in range(m + n + 1):
            # i = 0 and i = m + n
            if i == 0:
                assert oracle.co_rank(i, A, B)[:2] == (0, 0)
            if i == m + n:
                assert oracle.co_rank(i, A, B)[:2] == (m, n)
        # m = 0 / n = 0: the merge is a copy
        E = np.empty(0, dtype=np.int64)
        np.testing.assert_array_equal(oracle.merge(A, E)[0], A)
        np.testing.assert_array_equal(oracle.merge(E, B)[0], B)
        # all keys equal: every A element first, so j = min(i, m)
        Aq = np.full(m, 7, dtype=np.int64)
        Bq = np.full(n, 7, dtype=np.int64)
        # max A < min B: j = min(i, m);  max B < min A: j = max(0, i - n)
        Alo = np.arange(m, dtype=np.int64)
        Bhi = np.arange(n, dtype=np.int64) + 1000
        Ahi = np.arange(m, dtype=np.int64) + 1000
        Blo = np.arange(n, dtype=np.int64)
        for i in range(m + n + 1):
            assert oracle.co_rank(i, Aq, Bq)[0] == min(i, m)
            assert oracle.co_rank(i, Alo, Bhi)[0] == min(i, m)
            assert oracle.co_rank(i, Ahi, Blo)[0] == max(0, i - n)


def test_out_of_range_rank():
    A = np.arange(5, dtype=np.int32)
    B = np.arange(3, dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.co_rank(-1, A, B)
    with pytest.raises(ValueError):
        oracle.co_rank(9, A, B)
    j, k = oracle.co_rank_many(A, B, np.array([-1, 0, 8, 9]))
    assert list(j) == [-1, 0, 5, -1] and list(k) == [-1, 0, 3, -1]


def test_iteration_bound_and_k_low():
    """Proposition 1: the number of moving iterations is logarithmic.  The
    printed bound ceil(log2 min(m, n, i, m+n-i)) is off by one (A = [19],
    B = [5, 15, 28, 38, 41], i = 2 needs one move with min = 1); the bound
    ceil(log2(min + 1)) holds.  The oracle also reports (-2) if the second
    condition ever fired before k_low was set, which the paper rules out."""
    j, k, moves = oracle.co_rank(2, np.array([19], np.int64),
                                 np.array([5, 15, 28, 38, 41], np.int64))
    assert (j, k, moves) == (0, 2, 1)
    for A, B in small_cases(14, 1500, max_len=40):
        m, n = len(A), len(B)
        for i in range(m + n + 1):
            _, _, moves, states = oracle.co_rank(i, A, B, trace=True)
            mn = min(m, n, i, m + n - i)
            assert moves <= math.ceil(math.log2(mn + 1))
            if moves:
                assert states[1][4] == 1   # first move is always on condition 1


def test_co_rank_large_random_vs_searchsorted():
    """Larger arrays: j equals the number of A elements whose position in the
    stable merge is below i.  That position has the closed form
    j' + #{B < A[j']} (all smaller B keys precede A[j'], equal ones follow),
    counted here with numpy's searchsorted, independently of Algorithm 1."""
    rng = np.random.default_rng(21)
    for _ in range(30):
        m = int(rng.integers(0, 3000))
        n = int(rng.integers(0, 3000))
        A = np.sort(rng.integers(0, 500, m)).astype(np.int32)
        B = np.sort(rng.integers(0, 500, n)).astype(np.int32)
        ranks = rng.integers(0, m + n + 1, 200)
        j, k = oracle.co_rank_many(A, B, ranks)
        # Position of A[j'] in C is j' + #{B < A[j']}; A-count of C[:i] is
        # the number of j' with that position < i.
        posA = np.arange(m) + np.searchsorted(B, A, side="left")
        for r, jj in zip(ranks, j):
            assert jj == int(np.count_nonzero(posA < r))


def test_alg2_partition_independence_and_balance():
    """Proposition 2: Algorithm 2 gives the same output for every p, and every
    processing element merges floor or ceil of (m+n)/p elements."""
    rng = np.random.default_rng(8)
    for _ in range(40):
        m = int(rng.integers(0, 5000))
        n = int(rng.integers(0, 5000))
        A = np.sort(rng.integers(0, 64, m)).astype(np.int32)
        B = np.sort(rng.integers(0, 64, n)).astype(np.int32)
        C, _ = oracle.merge(A, B)
        for p in (1, 2, 3, 7, 16, 33):
            got, counts = oracle.parallel_merge(A, B, p)
            np.testing.assert_array_equal(got, C)
            tot = m + n
            assert counts.sum() == tot
            assert counts.max() <= -(-tot // p)
            assert counts.min() >= tot // p


def test_co_rank_cross_checked_with_merge_sources():
    """The oracle's two independent statements agree: Algorithm 1's co-rank j
    of every rank i equals the number of A elements among the first i
    outputs of the two-pointer merge (j = #{t < i : src[t] < m})."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        m, n = rng.integers(0, 400, 2)
        spread = int(rng.choice([2, 10, 1000]))
        A = np.sort(rng.integers(0, spread, m)).astype(np.int64)
        B = np.sort(rng.integers(0, spread, n)).astype(np.int64)
        _, src = oracle.merge(A, B)
        from_a = np.concatenate([[0], np.cumsum(src < m)])
        ranks = np.arange(m + n + 1)
        j, k = oracle.co_rank_many(A, B, ranks)
        assert np.array_equal(j, from_a) and np.array_equal(k, ranks - from_a)
