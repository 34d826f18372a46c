"""Seeded synthetic inputs shaped like the stable-merge workloads.

This module only draws random numbers and sorts them into valid inputs
(ascending arrays, segment tables, pre-sorted runs).  It holds none of the
merge or co-rank arithmetic; both the GPU path and the CPU oracle consume what
it returns.

Two backends:

* ``numpy`` (host, exact across machines) for the small and medium cases the
  oracle checks element by element;
* ``torch`` (device, ``torch.Generator`` on CUDA) for the full-size cases,
  where host sorting of 2^28-element arrays would dominate run time.

Unsigned 64-bit keys are produced by sorting signed 64-bit draws and then
flipping the sign bit, which maps signed order onto unsigned order; they are
returned in an int64 container whose bits are the uint64 keys.

Workloads (sizes at ``shift=0``; ``shift=s`` divides every size by 2^s):

* ``single_i32_tag``   A m=2^20, B n=3*2^19, int32 uniform in [0, 2^16).
* ``large_i32``        m=n=2^28 int32 uniform over the whole int32 range.
* ``skewed_u64``       m=2^20, n=2^29 uint64 uniform over the whole range.
* ``dup16_i32``        m=n=2^28 int32 drawn from 16 distinct values.
* ``kv_u32_f32``       m=n=2^27 uint32 keys in [0, 2^20), float32 N(0,1)
                       payloads (the keys fit in 31 bits, so the int32
                       container holds them unchanged).
* ``batched_i32_f32``  8192 segment pairs, m_s and n_s independently
                       floor(2^(18u)) clamped to [1, 2^18], u ~ U[0,1);
                       int32 keys uniform in [0, 2^24) sorted per segment,
                       float32 payloads, int64 offsets.
* ``sort_u64_f32``     2^27 uint64 keys drawn from 2^20 distinct values,
                       float32 payloads, pre-sorted (stably) in runs of 1024.
"""
from __future__ import annotations

import numpy as np

SIGN64 = np.uint64(1 << 63)


# --------------------------------------------------------------------------
# numpy (host) generators
# --------------------------------------------------------------------------
def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def sorted_ints(rng: np.random.Generator, size: int, lo: int, hi: int, dtype) -> np.ndarray:
    """`size` uniform integers in [lo, hi) of `dtype`, sorted ascending."""
    a = rng.integers(lo, hi, size=size, dtype=np.int64 if hi <= 2**63 else np.uint64)
    a = np.sort(a.astype(dtype, copy=False), kind="stable")
    return a


def sorted_full_range(rng: np.random.Generator, size: int, dtype) -> np.ndarray:
    """`size` keys uniform over the whole range of `dtype`, sorted ascending."""
    info = np.iinfo(dtype)
    a = rng.integers(info.min, info.max, size=size, dtype=dtype, endpoint=True)
    return np.sort(a, kind="stable")


def sorted_from_values(rng: np.random.Generator, size: int, values: np.ndarray) -> np.ndarray:
    pick = rng.integers(0, len(values), size=size)
    return np.sort(values[pick], kind="stable")


def distinct_values(rng: np.random.Generator, count: int, dtype) -> np.ndarray:
    info = np.iinfo(dtype)
    out = np.unique(rng.integers(info.min, info.max, size=count, dtype=dtype, endpoint=True))
    while len(out) < count:
        extra = rng.integers(info.min, info.max, size=count - len(out), dtype=dtype, endpoint=True)
        out = np.unique(np.concatenate([out, extra]))
    return rng.permutation(out)


def single_i32_tag(seed: int = 1, shift: int = 0):
    r = _rng(seed)
    m, n = (1 << 20) >> shift, (3 << 19) >> shift
    A = sorted_ints(r, m, 0, 1 << 16, np.int32)
    B = sorted_ints(r, n, 0, 1 << 16, np.int32)
    return A, B


def large_i32(seed: int = 2, shift: int = 0):
    r = _rng(seed)
    m = n = (1 << 28) >> shift
    return sorted_full_range(r, m, np.int32), sorted_full_range(r, n, np.int32)


def skewed_u64(seed: int = 3, shift: int = 0):
    r = _rng(seed)
    m, n = (1 << 20) >> shift, (1 << 29) >> shift
    return sorted_full_range(r, m, np.uint64), sorted_full_range(r, n, np.uint64)


def dup16_i32(seed: int = 4, shift: int = 0):
    r = _rng(seed)
    vals = distinct_values(r, 16, np.int32)
    m = n = (1 << 28) >> shift
    return sorted_from_values(r, m, vals), sorted_from_values(r, n, vals)


def kv_u32_f32(seed: int = 5, shift: int = 0):
    """Keys as uint32 (values < 2^20), payloads float32 N(0,1)."""
    r = _rng(seed)
    m = n = (1 << 27) >> shift
    A = sorted_ints(r, m, 0, 1 << 20, np.uint32)
    B = sorted_ints(r, n, 0, 1 << 20, np.uint32)
    Av = r.standard_normal(m, dtype=np.float32)
    Bv = r.standard_normal(n, dtype=np.float32)
    return A, Av, B, Bv


def log_uniform_sizes(seed: int, nseg: int, max_log2: int = 18) -> tuple[np.ndarray, np.ndarray]:
    """m_s, n_s = clamp(floor(2^(max_log2 * u)), 1, 2^max_log2), u ~ U[0,1)."""
    r = _rng(seed)
    u = r.random((2, nseg))
    s = np.floor(np.exp2(max_log2 * u)).astype(np.int64)
    s = np.clip(s, 1, 1 << max_log2)
    return s[0], s[1]


def offsets(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def batched_i32_f32(seed: int = 6, nseg: int = 8192, max_log2: int = 18):
    """Segment tables and per-segment-sorted keys (host)."""
    ms, ns = log_uniform_sizes(seed, nseg, max_log2)
    a_off, b_off = offsets(ms), offsets(ns)
    r = _rng(seed + 1000)
    A = r.integers(0, 1 << 24, size=int(a_off[-1]), dtype=np.int32)
    B = r.integers(0, 1 << 24, size=int(b_off[-1]), dtype=np.int32)
    for q in range(nseg):
        A[a_off[q]:a_off[q + 1]].sort(kind="stable")
        B[b_off[q]:b_off[q + 1]].sort(kind="stable")
    Av = r.standard_normal(len(A), dtype=np.float32)
    Bv = r.standard_normal(len(B), dtype=np.float32)
    return a_off, b_off, A, Av, B, Bv


def sort_u64_f32(seed: int = 7, shift: int = 0, run: int | None = 1024,
                 distinct: int = 1 << 20):
    """uint64 keys from `distinct` values, runs of `run` sorted stably (payload
    follows; run=None: left unsorted)."""
    r = _rng(seed)
    N = (1 << 27) >> shift
    vals = distinct_values(r, distinct, np.uint64)
    X = vals[r.integers(0, len(vals), size=N)]
    Xv = r.standard_normal(N, dtype=np.float32)
    if run is None:
        return X, Xv
    for a0 in range(0, N, run):
        o = np.argsort(X[a0:a0 + run], kind="stable")
        X[a0:a0 + run] = X[a0:a0 + run][o]
        Xv[a0:a0 + run] = Xv[a0:a0 + run][o]
    return X, Xv


# --------------------------------------------------------------------------
# torch (device) generators for the full-size cases
# --------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _gen(seed: int, device):
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def t_sorted_i32(g, size: int, lo: int, hi: int, device):
    torch = _torch()
    a = torch.randint(lo, hi, (size,), generator=g, device=device, dtype=torch.int64)
    return torch.sort(a.to(torch.int32)).values


def t_sorted_full_i32(g, size: int, device):
    return t_sorted_i32(g, size, -(1 << 31), 1 << 31, device)


def t_sorted_full_u64(g, size: int, device):
    """uint64 keys uniform over the whole range, ascending, in an int64 container."""
    torch = _torch()
    s = torch.randint(-(1 << 63), (1 << 63) - 1, (size,), generator=g, device=device,
                      dtype=torch.int64)
    s = torch.sort(s).values
    return s ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=device)


def t_large_i32(seed: int = 2, device="cuda", shift: int = 0):
    g = _gen(seed, device)
    m = n = (1 << 28) >> shift
    return t_sorted_full_i32(g, m, device), t_sorted_full_i32(g, n, device)


def t_skewed_u64(seed: int = 3, device="cuda", shift: int = 0):
    g = _gen(seed, device)
    m, n = (1 << 20) >> shift, (1 << 29) >> shift
    return t_sorted_full_u64(g, m, device), t_sorted_full_u64(g, n, device)


def t_dup16_i32(seed: int = 4, device="cuda", shift: int = 0):
    torch = _torch()
    vals = torch.from_numpy(distinct_values(_rng(seed), 16, np.int32)).to(device)
    g = _gen(seed, device)
    m = n = (1 << 28) >> shift
    A = torch.sort(vals[torch.randint(0, 16, (m,), generator=g, device=device)]).values
    B = torch.sort(vals[torch.randint(0, 16, (n,), generator=g, device=device)]).values
    return A, B


def t_kv_u32_f32(seed: int = 5, device="cuda", shift: int = 0):
    torch = _torch()
    g = _gen(seed, device)
    m = n = (1 << 27) >> shift
    A = t_sorted_i32(g, m, 0, 1 << 20, device)
    B = t_sorted_i32(g, n, 0, 1 << 20, device)
    Av = torch.randn(m, generator=g, device=device, dtype=torch.float32)
    Bv = torch.randn(n, generator=g, device=device, dtype=torch.float32)
    return A, Av, B, Bv


def t_batched_i32_f32(seed: int = 6, nseg: int = 8192, max_log2: int = 18, device="cuda"):
    """Same segment table as the numpy generator; keys drawn on the device and
    sorted per segment with one global sort of (segment << 32 | key)."""
    torch = _torch()
    ms, ns = log_uniform_sizes(seed, nseg, max_log2)
    a_off, b_off = offsets(ms), offsets(ns)
    g = _gen(seed + 1000, device)

    def seg_sorted(off):
        total = int(off[-1])
        seg = torch.repeat_interleave(torch.arange(len(off) - 1, device=device),
                                      torch.from_numpy(np.diff(off)).to(device))
        key = torch.randint(0, 1 << 24, (total,), generator=g, device=device, dtype=torch.int64)
        comp = torch.sort((seg << 32) | key).values
        return (comp & 0xFFFFFFFF).to(torch.int32)

    A = seg_sorted(a_off)
    B = seg_sorted(b_off)
    Av = torch.randn(len(A), generator=g, device=device, dtype=torch.float32)
    Bv = torch.randn(len(B), generator=g, device=device, dtype=torch.float32)
    return a_off, b_off, A, Av, B, Bv


def t_sort_u64_f32(seed: int = 7, device="cuda", shift: int = 0, run: int | None = 1024,
                   distinct: int = 1 << 20):
    """uint64 keys (int64 container) from `distinct` values, runs stably
    pre-sorted (run=None: left unsorted)."""
    torch = _torch()
    N = (1 << 27) >> shift
    vals = distinct_values(_rng(seed), distinct, np.uint64).view(np.int64)
    vals = torch.from_numpy(vals).to(device)
    g = _gen(seed, device)
    X = vals[torch.randint(0, len(vals), (N,), generator=g, device=device)]
    Xv = torch.randn(N, generator=g, device=device, dtype=torch.float32)
    if run is None:
        return X, Xv
    flip = torch.tensor(-(1 << 63), dtype=torch.int64, device=device)
    rows = (X ^ flip).view(-1, run)        # signed order of the flipped bits == unsigned order
    srt = torch.sort(rows, dim=1, stable=True)
    X = (srt.values ^ flip).reshape(-1)
    Xv = torch.gather(Xv.view(-1, run), 1, srt.indices).reshape(-1)
    return X, Xv
