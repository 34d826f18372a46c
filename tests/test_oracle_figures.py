"""Pins of the CPU oracle to the values the paper prints (Figures 1-3)."""
import numpy as np
import pytest

import oracle
from conftest import read_golden


def _fig1():
    rows = {r[0]: r[1:] for r in read_golden("figure1.txt")}
    A = np.array([int(x) for x in rows["A"]], dtype=np.int32)
    B = np.array([int(x) for x in rows["B"]], dtype=np.int32)
    C = np.array([int(x) for x in rows["C"]], dtype=np.int32)
    alpha = (int(rows["alpha"][1]), int(rows["alpha"][3]))
    beta = (int(rows["beta"][1]), int(rows["beta"][3]))
    return A, B, C, alpha, beta


@pytest.mark.parametrize("dt", [np.int32, np.uint32, np.int64, np.uint64])
def test_figure1_merge(dt):
    """Figure 1: merging the printed A and B gives the printed C, with alpha =
    A[8] at C[13] and beta = B[5] at C[14] (stability: A before B on ties)."""
    A, B, C, (aj, ai), (bk, bi) = _fig1()
    assert len(A) == 18 and len(B) == 24 and len(C) == 42
    got, src = oracle.merge(A.astype(dt), B.astype(dt))
    np.testing.assert_array_equal(got, C.astype(dt))
    assert src[ai] == aj
    assert src[bi] == len(A) + bk
    assert A[aj] == B[bk]


def test_figure2_co_rank():
    """Figure 2: co_rank(22) on the Figure 1 arrays is (j, k) = (12, 10)."""
    A, B, C, _, _ = _fig1()
    (i, j, k), = [[int(x) for x in r] for r in read_golden("figure2.txt")]
    gj, gk, moves = oracle.co_rank(i, A, B)
    assert (gj, gk) == (j, k)
    # Lemma 1's prefix property: the first i outputs merge A[:j] and B[:k].
    head, _ = oracle.merge(A[:j], B[:k])
    np.testing.assert_array_equal(head, C[:i])


def test_figure3_trace():
    """Figure 3: the states of Algorithm 1 printed for i = 22 -- start, one
    step on the first Lemma condition, one step on the second."""
    A, B, _, _, _ = _fig1()
    rows = read_golden("figure3.txt")
    i = int(rows[0][1])
    want = [tuple(int(x) for x in r[1:]) for r in rows[1:]]
    j, k, moves, states = oracle.co_rank(i, A, B, trace=True)
    assert states[:len(want)] == want
    # the run ends on Figure 2's answer, within Proposition 1's printed bound
    assert (j, k) == (12, 10)
    assert moves <= int(np.ceil(np.log2(min(len(A), len(B), i, len(A) + len(B) - i))))


def test_figure1_alg2_every_p():
    """Algorithm 2 on the Figure 1 arrays gives the printed C for every p."""
    A, B, C, _, _ = _fig1()
    for p in range(1, 43 + 3):
        got, counts = oracle.parallel_merge(A, B, p)
        np.testing.assert_array_equal(got, C)
        assert counts.sum() == 42
        assert counts.max() - counts.min() <= 1
