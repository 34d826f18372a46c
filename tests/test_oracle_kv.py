"""Pins of the oracle's key-value merge, gradient, batched merge and merge sort
against brute force, closed forms, finite differences and numpy's stable
argsort -- none of which share code with the oracle."""
import numpy as np
import pytest

import oracle
from paper_1303_4312_gb300 import workloads


def _case(rng, m, n, spread, kdt=np.int32, vdt=np.float32):
    A = np.sort(rng.integers(0, spread, m)).astype(kdt)
    B = np.sort(rng.integers(0, spread, n)).astype(kdt)
    Av = rng.standard_normal(m).astype(vdt)
    Bv = rng.standard_normal(n).astype(vdt)
    return A, Av, B, Bv


@pytest.mark.parametrize("vdt", [np.float32, np.float64, np.int32, np.int64])
def test_merge_kv_vs_stable_argsort(vdt):
    """Key-value merge = numpy stable argsort of the concatenation A || B
    applied to keys and payloads (A precedes B, so the stable sort is the
    stable merge)."""
    rng = np.random.default_rng(31)
    for _ in range(100):
        m, n = int(rng.integers(0, 300)), int(rng.integers(0, 300))
        A, Av, B, Bv = _case(rng, m, n, int(rng.choice([2, 16, 1000])), vdt=vdt)
        C, Cv, src = oracle.merge_kv(A, Av, B, Bv)
        o = np.argsort(np.concatenate([A, B]), kind="stable")
        np.testing.assert_array_equal(C, np.concatenate([A, B])[o])
        assert Cv.tobytes() == np.concatenate([Av, Bv])[o].tobytes()
        np.testing.assert_array_equal(src, o)


def test_payload_bits_preserved():
    """Payloads are copied as bits: NaN payloads, -0.0 and denormals survive."""
    A = np.array([1, 2, 2, 5], np.uint32)
    B = np.array([0, 2, 9], np.uint32)
    bits = np.array([0x7FC00001, 0x80000000, 0x00000001, 0xFF800000], np.uint32)
    Av = bits.view(np.float32)
    Bv = np.array([0x7F800001, 0x80000001, 0x3F800000], np.uint32).view(np.float32)
    _, Cv, _ = oracle.merge_kv(A, Av, B, Bv)
    want = np.array([0x7F800001, 0x7FC00001, 0x80000000, 0x00000001, 0x80000001,
                     0xFF800000, 0x3F800000], np.uint32)
    np.testing.assert_array_equal(Cv.view(np.uint32), want)


def test_grad_closed_form():
    """Gradient closed form: A[j] lands at j + #{B < A[j]}, B[k] at
    k + #{A <= B[k]} (searchsorted), so gA[j] = gC[j + #{B < A[j]}] and
    gB[k] = gC[k + #{A <= B[k]}]."""
    rng = np.random.default_rng(32)
    for _ in range(100):
        m, n = int(rng.integers(0, 500)), int(rng.integers(0, 500))
        A, _, B, _ = _case(rng, m, n, int(rng.choice([2, 16, 1000])))
        gC = rng.standard_normal(m + n).astype(np.float32)
        gA, gB = oracle.merge_grad(A, B, gC)
        posA = np.arange(m) + np.searchsorted(B, A, side="left")
        posB = np.arange(n) + np.searchsorted(A, B, side="right")
        np.testing.assert_array_equal(gA, gC[posA])
        np.testing.assert_array_equal(gB, gC[posB])
        # the two position maps tile the output exactly once
        assert sorted(np.concatenate([posA, posB]).tolist()) == list(range(m + n))


def test_grad_finite_differences():
    """L = sum(w * C_v) is linear in the payloads; central differences with
    h = 2^-4 in float64 give dL/dAv[j] exactly, and it must equal the
    oracle gradient for gC = w."""
    rng = np.random.default_rng(33)
    m, n = 40, 57
    A, Av, B, Bv = _case(rng, m, n, 10, vdt=np.float64)
    w = rng.standard_normal(m + n)
    gA, gB = oracle.merge_grad(A, B, w)
    h = 2.0 ** -4

    def L(av, bv):
        return float(np.sum(w * oracle.merge_kv(A, av, B, bv)[1]))

    for j in range(m):
        e = np.zeros(m)
        e[j] = h
        d = (L(Av + e, Bv) - L(Av - e, Bv)) / (2 * h)
        assert d == pytest.approx(gA[j], rel=1e-12, abs=1e-12)
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        d = (L(Av, Bv + e) - L(Av, Bv - e)) / (2 * h)
        assert d == pytest.approx(gB[k], rel=1e-12, abs=1e-12)


def test_batched_vs_per_segment_argsort():
    """Batched merge: every segment equals the stable argsort of its own
    concatenation; empty segments (m_s = 0 or n_s = 0) included."""
    rng = np.random.default_rng(34)
    ms = rng.integers(0, 50, 64)
    ns = rng.integers(0, 50, 64)
    ms[::7] = 0
    ns[::5] = 0
    a_off, b_off = workloads.offsets(ms), workloads.offsets(ns)
    A = np.concatenate([np.sort(rng.integers(0, 9, x)) for x in ms]).astype(np.int32)
    B = np.concatenate([np.sort(rng.integers(0, 9, x)) for x in ns]).astype(np.int32)
    Av = rng.standard_normal(len(A)).astype(np.float32)
    Bv = rng.standard_normal(len(B)).astype(np.float32)
    C, Cv = oracle.batched_merge_kv(a_off, b_off, A, Av, B, Bv)
    gC = rng.standard_normal(len(C)).astype(np.float32)
    gA, gB = oracle.batched_merge_grad(a_off, b_off, A, B, gC)
    for q in range(64):
        a, b = slice(a_off[q], a_off[q + 1]), slice(b_off[q], b_off[q + 1])
        c = slice(a_off[q] + b_off[q], a_off[q + 1] + b_off[q + 1])
        keys = np.concatenate([A[a], B[b]])
        o = np.argsort(keys, kind="stable")
        np.testing.assert_array_equal(C[c], keys[o])
        np.testing.assert_array_equal(Cv[c], np.concatenate([Av[a], Bv[b]])[o])
        g = np.empty(len(keys), np.float32)
        g[o] = gC[c]
        np.testing.assert_array_equal(gA[a], g[:ms[q]])
        np.testing.assert_array_equal(gB[b], g[ms[q]:])


@pytest.mark.parametrize("N,run", [(1 << 12, 16), (5000, 64), (4096 + 17, 1024), (1, 4), (0, 8),
                                   (3001, 1)])
def test_merge_sort_vs_stable_argsort(N, run):
    """Bottom-up merge sort from sorted runs = numpy stable argsort (unsigned
    64-bit keys from few distinct values, so ties are common), and its payload
    gradient gX[perm[t]] = gY[t] matches the argsort permutation."""
    rng = np.random.default_rng(35)
    vals = workloads.distinct_values(rng, 50, np.uint64)
    X = vals[rng.integers(0, 50, N)] if N else np.empty(0, np.uint64)
    for a0 in range(0, N, run):
        X[a0:a0 + run] = np.sort(X[a0:a0 + run], kind="stable")
    Xv = rng.standard_normal(N).astype(np.float32)
    Y, Yv, perm = oracle.merge_sort(X, Xv, run)
    o = np.argsort(X, kind="stable")
    np.testing.assert_array_equal(Y, X[o])
    np.testing.assert_array_equal(Yv, Xv[o])
    np.testing.assert_array_equal(perm, o)


def test_merge_pass_tail_pairs():
    """A pass whose last pair has a short B run, or no B run at all."""
    rng = np.random.default_rng(36)
    for N in (10, 16, 23, 31, 33):
        w = 8
        X = rng.integers(0, 5, N).astype(np.int64)
        for a0 in range(0, N, w):
            X[a0:a0 + w].sort()
        Y, _, src = oracle.merge_pass(X, None, w)
        for a0 in range(0, N, 2 * w):
            seg = X[a0:a0 + 2 * w]
            o = np.argsort(seg, kind="stable")
            np.testing.assert_array_equal(Y[a0:a0 + 2 * w], seg[o])
            np.testing.assert_array_equal(src[a0:a0 + 2 * w], a0 + o)
