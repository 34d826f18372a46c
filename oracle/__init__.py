"""CPU oracle for the co-rank / stable-merge path (test infrastructure only).

This package is the plain, sequential, obviously-correct statement of what the
GPU path computes (Siebert & Traeff, "Perfectly load-balanced, optimal, stable,
parallel merge").  It is used by ``tests/``, by ``__graft_entry__.smoke()`` and
by the CPU-baseline leg of ``bench.py`` -- nothing else.  It never imports the
product package and shares no code with it; the product package never imports
this one.

All merge arithmetic lives in ``oracle.c`` (compiled with gcc into
``oracle/_build/liboracle.so``); this module marshals numpy arrays and holds
one numpy bit map, ``order_key``, which turns keys of any supported order
(floats in IEEE-754 totalOrder, descending orders) into unsigned integers
merged in their natural order.

Notation is the paper's: output rank ``i``, co-ranks ``j`` (into A) and ``k``
(into B), ``j + k == i``.  (The product C-ABI names the same triple
``(k; i, j)``.)

Every function here is pinned in ``tests/test_oracle_*.py`` against values the
paper prints (Figures 1-3), Lemma 1 checked for every rank of small cases,
brute force with Python's stable ``sorted``, closed forms, and numpy's stable
argsort.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_SUFFIX = {
    np.dtype(np.int32): "i32",
    np.dtype(np.uint32): "u32",
    np.dtype(np.int64): "i64",
    np.dtype(np.uint64): "u64",
}

_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain -O2, portable: no -march flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                        "-Wall", "-Wno-unused-function", _SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            for suf in _SUFFIX.values():
                f = getattr(lib, f"orc_co_rank_{suf}")
                f.argtypes = [_P, _I64, _P, _I64, _I64, _P, _P, _P, _I64]
                f.restype = _I64
                f = getattr(lib, f"orc_co_rank_many_{suf}")
                f.argtypes = [_P, _I64, _P, _I64, _P, _I64, _P, _P]
                f.restype = None
                f = getattr(lib, f"orc_merge_{suf}")
                f.argtypes = [_P, _I64, _P, _I64, _P, _P]
                f.restype = None
                f = getattr(lib, f"orc_merge_kv_{suf}")
                f.argtypes = [_P, _P, _I64, _P, _P, _I64, _I64, _P, _P, _P]
                f.restype = ctypes.c_int
                f = getattr(lib, f"orc_merge_grad_{suf}")
                f.argtypes = [_P, _I64, _P, _I64, _P, _I64, _P, _P]
                f.restype = ctypes.c_int
                f = getattr(lib, f"orc_batched_merge_kv_{suf}")
                f.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _I64, _P, _P]
                f.restype = ctypes.c_int
                f = getattr(lib, f"orc_batched_merge_grad_{suf}")
                f.argtypes = [_I64, _P, _P, _P, _P, _P, _I64, _P, _P]
                f.restype = ctypes.c_int
                f = getattr(lib, f"orc_merge_pass_{suf}")
                f.argtypes = [_P, _P, _I64, _I64, _I64, _P, _P, _P]
                f.restype = ctypes.c_int
                f = getattr(lib, f"orc_parallel_merge_{suf}")
                f.argtypes = [_P, _I64, _P, _I64, _P, _I64, _P]
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _keys(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype not in _SUFFIX:
        raise TypeError(f"oracle keys must be int32/uint32/int64/uint64, got {a.dtype}")
    return a


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _fn(name: str, dtype) -> ctypes._CFuncPtr:
    return getattr(_load(), f"{name}_{_SUFFIX[np.dtype(dtype)]}")


def _check_same(A, B):
    if A.dtype != B.dtype:
        raise TypeError("A and B must have the same key dtype")


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
def co_rank(i: int, A: np.ndarray, B: np.ndarray, trace: bool = False):
    """Algorithm 1: the co-ranks (j, k) of output rank i, 0 <= i <= m+n.

    Returns ``(j, k, moves)`` where ``moves`` counts the iterations that moved
    (j, k); with ``trace=True`` also a list of states
    ``(j, k, j_low, k_low, branch)`` (k_low = -1 while unset; branch 0 =
    start, 1 = first Lemma condition violated, 2 = second).
    """
    A = _keys(A)
    B = _keys(B)
    _check_same(A, B)
    j = ctypes.c_int64()
    k = ctypes.c_int64()
    cap = 256
    tr = np.zeros(5 * cap, dtype=np.int64) if trace else None
    moves = _fn("orc_co_rank", A.dtype)(_ptr(A), len(A), _ptr(B), len(B), int(i),
                                        ctypes.byref(j), ctypes.byref(k), _ptr(tr), cap)
    if moves == -1:
        raise ValueError(f"rank {i} outside [0, {len(A) + len(B)}]")
    if moves == -2:
        raise AssertionError("Algorithm 1 read k_low before setting it")
    if trace:
        states = [tuple(int(x) for x in tr[5 * s:5 * s + 5]) for s in range(min(moves + 1, cap))]
        return j.value, k.value, moves, states
    return j.value, k.value, moves


def co_rank_many(A: np.ndarray, B: np.ndarray, ranks: np.ndarray):
    """Algorithm 1 for every rank in ``ranks``; (-1, -1) for ranks outside [0, m+n]."""
    A = _keys(A)
    B = _keys(B)
    _check_same(A, B)
    ranks = np.ascontiguousarray(ranks, dtype=np.int64)
    j = np.empty(len(ranks), dtype=np.int64)
    k = np.empty(len(ranks), dtype=np.int64)
    _fn("orc_co_rank_many", A.dtype)(_ptr(A), len(A), _ptr(B), len(B), _ptr(ranks),
                                     len(ranks), _ptr(j), _ptr(k))
    return j, k


# --------------------------------------------------------------------------
# Sequential stable merge and its key-value / gradient forms
# --------------------------------------------------------------------------
def merge(A: np.ndarray, B: np.ndarray):
    """Sequential stable merge. Returns (C, src) with src[i] = j (A[j]) or m+k (B[k])."""
    A = _keys(A)
    B = _keys(B)
    _check_same(A, B)
    C = np.empty(len(A) + len(B), dtype=A.dtype)
    src = np.empty(len(A) + len(B), dtype=np.int64)
    _fn("orc_merge", A.dtype)(_ptr(A), len(A), _ptr(B), len(B), _ptr(C), _ptr(src))
    return C, src


def _vals(v: np.ndarray, n: int) -> np.ndarray:
    v = np.ascontiguousarray(v)
    if len(v) != n:
        raise ValueError("payload length differs from key length")
    if v.dtype.itemsize not in (4, 8):
        raise TypeError("payloads must be 4 or 8 bytes wide")
    return v


def merge_kv(A, Av, B, Bv):
    """Key-value stable merge (payload bits follow their key). Returns (C, Cv, src)."""
    A = _keys(A)
    B = _keys(B)
    _check_same(A, B)
    Av = _vals(Av, len(A))
    Bv = _vals(Bv, len(B))
    if Av.dtype != Bv.dtype:
        raise TypeError("payload dtypes differ")
    vb = Av.dtype.itemsize
    C = np.empty(len(A) + len(B), dtype=A.dtype)
    Cv = np.empty(len(A) + len(B), dtype=Av.dtype)
    src = np.empty(len(A) + len(B), dtype=np.int64)
    rc = _fn("orc_merge_kv", A.dtype)(_ptr(A), _ptr(Av), len(A), _ptr(B), _ptr(Bv), len(B),
                                      vb, _ptr(C), _ptr(Cv), _ptr(src))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return C, Cv, src


def merge_grad(A, B, gC):
    """Payload gradient of the key-value merge: returns (gA, gB) (bit copies of gC)."""
    A = _keys(A)
    B = _keys(B)
    _check_same(A, B)
    gC = _vals(gC, len(A) + len(B))
    gA = np.empty(len(A), dtype=gC.dtype)
    gB = np.empty(len(B), dtype=gC.dtype)
    rc = _fn("orc_merge_grad", A.dtype)(_ptr(A), len(A), _ptr(B), len(B), _ptr(gC),
                                        gC.dtype.itemsize, _ptr(gA), _ptr(gB))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return gA, gB


# --------------------------------------------------------------------------
# Batched (segmented) merge
# --------------------------------------------------------------------------
def batched_merge_kv(a_off, b_off, A, Av, B, Bv):
    """Segment q: A[a_off[q]:a_off[q+1]] merged with B[b_off[q]:b_off[q+1]] into
    C[a_off[q]+b_off[q] : ...]. Returns (C, Cv)."""
    A = _keys(A)
    B = _keys(B)
    _check_same(A, B)
    Av = _vals(Av, len(A))
    Bv = _vals(Bv, len(B))
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    nseg = len(a_off) - 1
    C = np.empty(len(A) + len(B), dtype=A.dtype)
    Cv = np.empty(len(A) + len(B), dtype=Av.dtype)
    rc = _fn("orc_batched_merge_kv", A.dtype)(nseg, _ptr(a_off), _ptr(b_off), _ptr(A), _ptr(Av),
                                              _ptr(B), _ptr(Bv), Av.dtype.itemsize,
                                              _ptr(C), _ptr(Cv))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return C, Cv


def batched_merge_grad(a_off, b_off, A, B, gC):
    A = _keys(A)
    B = _keys(B)
    _check_same(A, B)
    gC = _vals(gC, len(A) + len(B))
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    b_off = np.ascontiguousarray(b_off, dtype=np.int64)
    gA = np.empty(len(A), dtype=gC.dtype)
    gB = np.empty(len(B), dtype=gC.dtype)
    rc = _fn("orc_batched_merge_grad", A.dtype)(len(a_off) - 1, _ptr(a_off), _ptr(b_off),
                                                _ptr(A), _ptr(B), _ptr(gC), gC.dtype.itemsize,
                                                _ptr(gA), _ptr(gB))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return gA, gB


# --------------------------------------------------------------------------
# Bottom-up merge sort as a chain of merge passes
# --------------------------------------------------------------------------
def merge_pass(X, Xv, w: int):
    """One bottom-up pass: adjacent runs of width w merged pairwise. Returns (Y, Yv, src)."""
    X = _keys(X)
    N = len(X)
    vb = 0
    if Xv is not None:
        Xv = _vals(Xv, N)
        vb = Xv.dtype.itemsize
    Y = np.empty(N, dtype=X.dtype)
    Yv = np.empty(N, dtype=Xv.dtype) if Xv is not None else None
    src = np.empty(N, dtype=np.int64)
    rc = _fn("orc_merge_pass", X.dtype)(_ptr(X), _ptr(Xv), N, int(w), vb, _ptr(Y), _ptr(Yv),
                                        _ptr(src))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return Y, Yv, src


def merge_sort(X, Xv, run: int):
    """Bottom-up stable merge sort of X whose runs of width ``run`` are already
    sorted: passes of width run, 2 run, 4 run, ... until one run remains.

    Returns (Y, Yv, perm) with Y[t] = X[perm[t]]; the payload gradient of the
    sort is gX[perm[t]] = gY[t].
    """
    X = _keys(X)
    Y, Yv = X.copy(), (None if Xv is None else np.ascontiguousarray(Xv).copy())
    perm = np.arange(len(X), dtype=np.int64)
    w = int(run)
    while w < len(X):
        Y, Yv, src = merge_pass(Y, Yv, w)
        perm = perm[src]
        w *= 2
    return Y, Yv, perm


# --------------------------------------------------------------------------
# Algorithm 2
# --------------------------------------------------------------------------
def parallel_merge(A, B, p: int):
    """Algorithm 2 on p POSIX threads. Returns (C, counts) with counts[r] the
    number of output elements processing element r merged."""
    A = _keys(A)
    B = _keys(B)
    _check_same(A, B)
    C = np.empty(len(A) + len(B), dtype=A.dtype)
    counts = np.empty(int(p), dtype=np.int64)
    rc = _fn("orc_parallel_merge", A.dtype)(_ptr(A), len(A), _ptr(B), len(B), _ptr(C), int(p),
                                            _ptr(counts))
    if rc != 0:
        raise RuntimeError("oracle could not start its threads")
    return C, counts


# ---------------------------------------------------------------------------
# Key orders (the paper's merge is stated for any total order, Section 2).
# ---------------------------------------------------------------------------
_ORDER_BITS = {"i32": 32, "u32": 32, "f32": 32, "i64": 64, "u64": 64, "f64": 64,
               "pair_u32": 64, "pair_i32": 64}


def order_key(a: np.ndarray, key_type: str) -> np.ndarray:
    """Unsigned integers whose natural order is `key_type`'s order on the
    bit patterns of `a`:

      u32, u64  the value itself;
      i32, i64  two's complement with the sign bit flipped (offset binary);
      f32, f64  IEEE 754-2008 totalOrder (Section 5.10): a negative value
                (sign bit set) has every bit complemented, a non-negative one
                has its sign bit set, so -NaN < -inf < ... < -0 < +0 < ... <
                +inf < +NaN with NaN payloads ordered as the standard says;
      pair_u32  a 64-bit word holding (major, minor) uint32 keys, major in
                the high half: lexicographic order is the word's own order;
      pair_i32  the same with int32 halves: each half offset binary;
      ":desc"   appended to any of these: the complement of the above.
    """
    base, _, mod = key_type.partition(":")
    bits = _ORDER_BITS[base]
    ut = np.uint32 if bits == 32 else np.uint64
    u = np.ascontiguousarray(a).view(ut).copy()
    sign = ut(1) << ut(bits - 1)
    if base == "pair_i32":
        u ^= ut((1 << 63) | (1 << 31))
    elif base == "pair_u32":
        pass
    elif base[0] == "i":
        u ^= sign
    elif base[0] == "f":
        neg = (u & sign) != 0
        u = np.where(neg, ~u, u | sign).astype(ut)
    if mod == "desc":
        u = ~u
    return u


def merge_in_order(A: np.ndarray, B: np.ndarray, key_type: str):
    """Stable merge of A and B sorted in `key_type`'s order: the plain merge
    of their order keys, applied to the original elements.  Returns (C, src)
    with C = concat(A, B)[src]."""
    _, src = merge(order_key(A, key_type), order_key(B, key_type))
    return np.concatenate([A, B])[src], src
