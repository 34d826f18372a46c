"""GPU parity of run formation (cr_sort_runs, cr_sort_runs_backward and
cr_merge_runs_block from width 1): every run of sort_run_length()
consecutive elements comes out as numpy's stable argsort of that run in the
key order (oracle.order_key), payloads and the recorded chunk permutation
following, and the backward routes gradients through the same permutation.
Key patterns: all keys equal (every comparison a tie), only the lowest byte
varying, only the top byte (the sign bit of signed and float storage among
it), two values differing in one middle byte, the sign bit and the lowest
bit, and full-range keys, in every key order; lengths leave a ragged last
run."""
import numpy as np
import pytest
import torch

import oracle
import paper_1303_4312_gb300 as cr
from gpu_util import dev, host, same_bits

pytestmark = pytest.mark.gpu

STORAGE = {"i32": np.int32, "u32": np.uint32, "i64": np.int64, "u64": np.uint64,
           "f32": np.float32, "f64": np.float64, "pair_i32": np.uint64, "pair_u32": np.uint64}


def bit_patterns(rng, n, bits):
    ut = np.uint32 if bits == 32 else np.uint64
    one = ut(1)
    full = rng.integers(0, np.iinfo(ut).max, n, dtype=ut, endpoint=True)
    base = rng.integers(0, np.iinfo(ut).max, dtype=ut, endpoint=True)
    low = ut(0xff)
    top = ut(0xff) << ut(bits - 8)
    mid = ut(bits // 2)
    yield "full", full
    yield "equal", np.full(n, base, ut)
    yield "low byte", (base & ~low) | (full & low)
    yield "top byte", (base & ~top) | (full & top)
    yield "middle byte", base ^ (rng.integers(0, 2, n).astype(ut) << mid)
    yield "sign bit", base ^ (rng.integers(0, 2, n).astype(ut) << ut(bits - 1)) ^ (full & one)


def per_run_order(keys, R):
    o = np.empty(len(keys), np.int64)
    for a0 in range(0, len(keys), R):
        o[a0:a0 + R] = a0 + np.argsort(keys[a0:a0 + R], kind="stable")
    return o


@pytest.mark.parametrize("kt", ["i32", "u32", "i64", "u64", "f32", "f64", "f32:desc",
                                "i64:desc", "u32:desc", "pair_i32", "pair_u32:desc"])
def test_run_formation_digit_patterns(kt):
    rng = np.random.default_rng(900 + sum(map(ord, kt)))
    R = cr.sort_run_length()
    dt = STORAGE[kt.split(":")[0]]
    bits = 8 * np.dtype(dt).itemsize
    N = 3 * R + 777
    for name, b in bit_patterns(rng, N, bits):
        X = b.view(dt)
        Xv = rng.standard_normal(N).astype(np.float32)
        o = per_run_order(oracle.order_key(X, kt), R)
        Y, Yv = cr.sort_runs(dev(X), dev(Xv), key_type=kt)
        gY = rng.standard_normal(N).astype(np.float32)
        gX = cr.sort_runs_backward(dev(X), dev(gY), key_type=kt)
        Y2, Yv2, perm = cr.merge_runs_block(dev(X), dev(Xv), 1, key_type=kt, record=True)
        torch.cuda.synchronize()
        assert same_bits(host(Y, dt), X[o]), name
        assert same_bits(host(Yv, np.float32), Xv[o]), name
        g = np.empty_like(gY)
        g[o] = gY
        assert same_bits(host(gX, np.float32), g), name
        assert same_bits(host(Y2, dt), X[o]) and same_bits(host(Yv2, np.float32), Xv[o]), name
        base = (np.arange(N) // R) * R
        assert np.array_equal(host(perm, np.uint16).astype(np.int64) + base, o), name


@pytest.mark.parametrize("vb", [0, 8])
def test_run_formation_lengths_and_payload_widths(vb):
    """Keys only and 8-byte payloads, lengths from one element to several runs
    with a ragged tail, keys drawn from few values (long runs of ties)."""
    rng = np.random.default_rng(950 + vb)
    R = cr.sort_run_length()
    for N in (1, 2, 31, 32, 33, 255, 257, R - 1, R, R + 1, 2 * R + 4095):
        X = rng.integers(-3, 3, N).astype(np.int64)
        Xv = rng.standard_normal(N) if vb else None
        o = per_run_order(X, R)
        Y, Yv = cr.sort_runs(dev(X), dev(Xv) if vb else None, key_type="i64")
        torch.cuda.synchronize()
        assert same_bits(host(Y, np.int64), X[o]), N
        if vb:
            assert same_bits(host(Yv, np.float64), Xv[o]), N
