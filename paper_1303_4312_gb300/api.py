"""PyTorch-facing API over libcorank.so.

PyTorch supplies device memory, the current stream and autograd; every
co-rank and merge step runs in the library's CUDA kernels.  Tensors must be
contiguous CUDA tensors; offset views (``A[i0:i1]``) are accepted as they
are (arrays need only be aligned to their element size).

Key types: int32 -> "i32", int64 -> "i64", uint32 -> "u32", uint64 -> "u64".
Unsigned keys can also travel in signed containers of the same width when
``key_type="u32"`` / ``"u64"`` is passed explicitly.  Payloads and gradients
are any 4- or 8-byte dtype; their bits are copied, never computed on.

Notation: the paper's (rank i; co-ranks j, k) is this API's (k; i, j).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib

_DTYPE_KEY = {torch.int32: "i32", torch.int64: "i64", torch.float32: "f32",
              torch.float64: "f64"}
for _name, _kt in (("uint32", "u32"), ("uint64", "u64")):
    if hasattr(torch, _name):
        _DTYPE_KEY[getattr(torch, _name)] = _kt


def _key_code(t: torch.Tensor, key_type: str | None) -> int:
    """Key type code for tensor t: from key_type ("i32", "u32", "i64", "u64",
    "f32", "f64", "pair_u32", "pair_i32", optionally ":desc"), else from t's
    dtype (ascending)."""
    if key_type is None:
        if t.dtype not in _DTYPE_KEY:
            raise TypeError(f"key dtype {t.dtype} is not int32/int64/uint32/uint64/float32/"
                            "float64")
        key_type = _DTYPE_KEY[t.dtype]
    code = _lib.key_code(key_type)
    if t.element_size() != _lib.key_bytes(code):
        raise TypeError(f"{key_type} keys need {_lib.key_bytes(code)}-byte elements")
    return code


def _dev(*ts: torch.Tensor) -> torch.device:
    dev = None
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensors must be CUDA tensors")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError("tensors are on different devices")
    return dev


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(dev) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def _ws(nbytes: int, dev) -> torch.Tensor:
    # 256-byte granularity keeps the allocation 16-byte aligned.
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)


def _size(fn, *args) -> int:
    out = ctypes.c_size_t()
    _lib.check(fn(*args, ctypes.byref(out)))
    return out.value


TILE_CLASSES = {"balanced": 0, "skewed": 1, "small": 2, "batched": 3, "pass": 4}


def tile_size(key_type: str, val_bytes: int = 0, m: int | None = None,
              n: int | None = None, cls: str | int | None = None) -> int:
    """Output elements per tile used for this key type and payload width: by
    a single merge of m and n elements when given (its geometry class), by
    class `cls` when given ("balanced", "skewed", "small", "batched" for
    batched calls, "pass" for merge passes), else by large balanced merges."""
    lib = _lib.load()
    code = _lib.key_code(key_type)
    if cls is not None:
        c = TILE_CLASSES[cls] if isinstance(cls, str) else int(cls)
        return int(lib.cr_tile_size_class(code, int(val_bytes), c))
    if m is None and n is None:
        return int(lib.cr_tile_size(code, int(val_bytes)))
    return int(lib.cr_tile_size_for(code, int(val_bytes), int(m or 0), int(n or 0)))


# ---------------------------------------------------------------------------
# co_rank (Algorithm 1)
# ---------------------------------------------------------------------------
def co_rank(A: torch.Tensor, B: torch.Tensor, k: int, key_type: str | None = None):
    """(i, j) with i + j == k: the first k outputs of the stable merge are
    A[:i] merged with B[:j] (Lemma 1).  Synchronises the current stream."""
    lib = _lib.load()
    dev = _dev(A, B)
    kt = _key_code(A, key_type)
    if B.dtype != A.dtype:
        raise TypeError("A and B dtypes differ")
    i, j = ctypes.c_int64(), ctypes.c_int64()
    with torch.cuda.device(dev):
        _lib.check(lib.cr_co_rank(kt, _ptr(A), A.numel(), _ptr(B), B.numel(), int(k),
                                  ctypes.byref(i), ctypes.byref(j), _stream(dev)))
    return i.value, j.value


def co_rank_async(A: torch.Tensor, B: torch.Tensor, k: int, out: torch.Tensor | None = None,
                  key_type: str | None = None) -> torch.Tensor:
    """(i, j) of rank k written to a 2-element int64 device tensor on the
    current stream, without waiting (usable inside CUDA-graph capture)."""
    lib = _lib.load()
    dev = _dev(A, B, out)
    kt = _key_code(A, key_type)
    if B.dtype != A.dtype:
        raise TypeError("A and B dtypes differ")
    if out is None:
        out = torch.empty(2, dtype=torch.int64, device=dev)
    elif out.dtype != torch.int64 or out.numel() < 2:
        raise ValueError("out must hold two int64 values")
    _lib.check(lib.cr_co_rank_async(kt, _ptr(A), A.numel(), _ptr(B), B.numel(), int(k),
                                    _ptr(out), _stream(dev)))
    return out


def co_rank_many(A: torch.Tensor, B: torch.Tensor, ks: torch.Tensor, key_type: str | None = None):
    """Co-ranks of every rank in ks (int64, device). Returns (i, j) tensors;
    -1 for ranks outside [0, m+n]."""
    lib = _lib.load()
    ks = ks.to(torch.int64).contiguous()
    dev = _dev(A, B, ks)
    kt = _key_code(A, key_type)
    oi = torch.empty_like(ks)
    oj = torch.empty_like(ks)
    _lib.check(lib.cr_co_rank_many(kt, _ptr(A), A.numel(), _ptr(B), B.numel(), _ptr(ks),
                                   ks.numel(), _ptr(oi), _ptr(oj), _stream(dev)))
    return oi, oj


class DistCoRank:
    """Algorithm 1 for block-distributed A and B (the library's
    cr_dist_co_rank_* calls): `cnt` searches whose state lives on `device`.
    One iteration is probes() -> answer() on every rank's blocks -> a sum of
    the answers over the ranks -> step().  m, n: global lengths."""

    def __init__(self, m: int, n: int, ranks, key_type: str, device):
        self.lib = _lib.load()
        self.m, self.n = int(m), int(n)
        self.code = _lib.key_code(key_type)
        self.dev = torch.device(device)
        r = torch.as_tensor(list(ranks) if not torch.is_tensor(ranks) else ranks,
                            dtype=torch.int64).to(self.dev).contiguous()
        self.cnt = r.numel()
        self.state = torch.empty(6 * self.cnt, dtype=torch.int64, device=self.dev)
        self._pa = torch.empty(2 * self.cnt, dtype=torch.int64, device=self.dev)
        self._pb = torch.empty(2 * self.cnt, dtype=torch.int64, device=self.dev)
        self._live = torch.empty(1, dtype=torch.int64, device=self.dev)
        _lib.check(self.lib.cr_dist_co_rank_init(self.m, self.n, _ptr(r), self.cnt,
                                                 _ptr(self.state), _stream(self.dev)))
        self._ranks = r

    def iterations(self) -> int:
        """Iterations after which every search has finished: the corrected
        bound of Proposition 1, ceil(log2(min(m, n) + 1)), plus the final
        check."""
        return int(min(self.m, self.n)).bit_length() + 1

    def probes(self):
        """(pa, pb): the A and B positions the next iteration reads (-1: none)."""
        _lib.check(self.lib.cr_dist_co_rank_probes(self.m, self.n, _ptr(self.state), self.cnt,
                                                   _ptr(self._pa), _ptr(self._pb),
                                                   _stream(self.dev)))
        return self._pa, self._pb

    def answer(self, blk: torch.Tensor, lo: int, idx: torch.Tensor) -> torch.Tensor:
        """Keys (int64 bits) of the positions in idx that fall in this rank's
        block blk = X[lo, lo + len(blk)), 0 for the others."""
        out = torch.empty(idx.numel(), dtype=torch.int64, device=self.dev)
        if blk.numel():
            _dev(blk, idx)
        _lib.check(self.lib.cr_dist_co_rank_answer(self.code, _ptr(blk) if blk.numel() else None,
                                                   int(lo), int(lo) + blk.numel(), _ptr(idx),
                                                   idx.numel(), _ptr(out), _stream(self.dev)))
        return out

    def step(self, va: torch.Tensor, vb: torch.Tensor) -> None:
        """One iteration of Algorithm 1 with the summed answers to probes()."""
        va, vb = va.contiguous(), vb.contiguous()
        _lib.check(self.lib.cr_dist_co_rank_step(self.code, self.m, self.n, _ptr(va), _ptr(vb),
                                                 _ptr(self.state), self.cnt, _stream(self.dev)))

    def result(self):
        """([(i, j) per search], number of unfinished searches); synchronises."""
        oi = torch.empty(self.cnt, dtype=torch.int64, device=self.dev)
        oj = torch.empty(self.cnt, dtype=torch.int64, device=self.dev)
        _lib.check(self.lib.cr_dist_co_rank_result(_ptr(self.state), self.cnt, _ptr(oi),
                                                   _ptr(oj), _ptr(self._live), _stream(self.dev)))
        return list(zip(oi.tolist(), oj.tolist())), int(self._live.item())


# ---------------------------------------------------------------------------
# stable merge (Algorithm 2, equal tiles)
# ---------------------------------------------------------------------------
def merge_workspace_bytes(key_type: str, val_bytes: int, m: int, n: int) -> int:
    lib = _lib.load()
    return _size(lib.cr_merge_workspace_size, _lib.key_code(key_type), int(val_bytes), int(m),
                 int(n))


def merge(A: torch.Tensor, B: torch.Tensor, key_type: str | None = None, tag: bool = False,
          out: torch.Tensor | None = None, out_tag: torch.Tensor | None = None,
          ws: torch.Tensor | None = None):
    """Stable merge of A and B, both sorted in key_type's order (ties: A
    first).

    With ``tag=True`` also returns the uint32 source tags (as int32 bits):
    i for A[i], m + j for B[j]."""
    lib = _lib.load()
    dev = _dev(A, B)
    kt = _key_code(A, key_type)
    if B.dtype != A.dtype:
        raise TypeError("A and B dtypes differ")
    m, n = A.numel(), B.numel()
    C = out if out is not None else torch.empty(m + n, dtype=A.dtype, device=dev)
    T = None
    if tag:
        T = out_tag if out_tag is not None else torch.empty(m + n, dtype=torch.int32, device=dev)
    need = _size(lib.cr_merge_workspace_size, kt, 0, m, n)
    if ws is None:
        ws = _ws(need, dev)
    _lib.check(lib.cr_stable_merge(kt, _ptr(A), m, _ptr(B), n, _ptr(C), _ptr(T), _ptr(ws),
                                   ws.numel(), _stream(dev)))
    return (C, T) if tag else C


class MergeMany:
    """Stable merges of several independent (A, B) pairs, with each pair's
    grid-level co-rank pass (cr_merge_partition) issued on a side stream
    ahead of the tile merges, which run in order on the caller's stream.

    The partition is latency-bound and co-resides with a running tile-merge
    kernel on the same SMs, so all but the first pair's partition overlap a
    previous merge.  Tile tables are double-buffered per pair, so calling
    ``run`` again (e.g. every step of a loop) lets the side stream run one
    call ahead.  Results are bit-identical to ``merge`` on each pair.
    """

    def __init__(self, pairs, key_types=None, device=None):
        self.pairs = list(pairs)
        self.key_types = list(key_types) if key_types else [None] * len(self.pairs)
        dev = device or self.pairs[0][0].device
        self.dev = torch.device(dev)
        lib = _lib.load()
        self.codes = []
        self.outs = []
        self.ws = []
        for (A, B), kt in zip(self.pairs, self.key_types):
            _dev(A, B)
            code = _key_code(A, kt)
            m, n = A.numel(), B.numel()
            need = _size(lib.cr_merge_workspace_size, code, 0, m, n)
            self.codes.append(code)
            self.outs.append(torch.empty(m + n, dtype=A.dtype, device=self.dev))
            self.ws.append([torch.zeros(max(need, 256), dtype=torch.uint8, device=self.dev)
                            for _ in range(2)])
        self.side = torch.cuda.Stream(self.dev)
        self.part_done = [None] * len(self.pairs)
        self.tile_done = [[None, None] for _ in self.pairs]
        self.calls = 0

    def run(self, events=None):
        """Issue every merge once; returns the outputs (valid in stream order
        on the current stream).  `events`, if given, is a list receiving
        (start, end) CUDA events around each tile merge."""
        lib = _lib.load()
        main = torch.cuda.current_stream(self.dev)
        buf = self.calls & 1
        sp, mp = self.side.cuda_stream, main.cuda_stream
        for q, ((A, B), code) in enumerate(zip(self.pairs, self.codes)):
            ws = self.ws[q][buf]
            if self.tile_done[q][buf] is not None:
                self.side.wait_event(self.tile_done[q][buf])   # table buffer is free again
            _lib.check(lib.cr_merge_partition(code, 0, _ptr(A), A.numel(), _ptr(B), B.numel(),
                                              _ptr(ws), ws.numel(), sp))
            ev = torch.cuda.Event()
            ev.record(self.side)
            self.part_done[q] = ev
        for q, ((A, B), code) in enumerate(zip(self.pairs, self.codes)):
            ws = self.ws[q][buf]
            main.wait_event(self.part_done[q])
            e0 = e1 = None
            if events is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(main)
            _lib.check(lib.cr_merge_tiles(code, 0, _ptr(A), None, A.numel(), _ptr(B), None,
                                          B.numel(), _ptr(self.outs[q]), None, None, _ptr(ws),
                                          ws.numel(), mp))
            done = torch.cuda.Event(enable_timing=events is not None)
            done.record(main)
            self.tile_done[q][buf] = done
            if events is not None:
                events.append((e0, done))
        self.calls += 1
        return self.outs

    def check(self):
        """Synchronise and raise if any device-side status was recorded."""
        torch.cuda.synchronize(self.dev)
        for pair in self.ws:
            for ws in pair:
                _lib.check(_lib.load().cr_workspace_status(_ptr(ws), _stream(self.dev)))


class _HostRegistration:
    """An anonymous host mapping page-locked with cudaHostRegister for as long
    as this object lives; the device is synchronised before the pages are
    released, so no copy can still be reading or writing them."""

    def __init__(self, nbytes: int):
        import mmap
        self.mm = mmap.mmap(-1, max(int(nbytes), 1))
        self.base = torch.frombuffer(self.mm, dtype=torch.uint8)
        self.ptr = self.base.data_ptr()
        rc = torch.cuda.cudart().cudaHostRegister(self.ptr, len(self.mm), 0)
        if int(rc) != 0:
            raise _lib.CorankError(f"cudaHostRegister of {len(self.mm)} bytes failed ({int(rc)})")

    def __del__(self):
        try:
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaHostUnregister(self.ptr)
        except Exception:
            pass


def host_empty(numel: int, dtype=torch.float32) -> torch.Tensor:
    """A page-locked host tensor for fast, asynchronous copies to and from the
    GPU (`HostMerger`'s inputs and outputs), on freshly mapped anonymous
    memory registered with cudaHostRegister.  On a GB300 whose host memory
    other processes had used heavily, such buffers copied device-to-host at
    193 GB/s and both ways at once at 299 GB/s where ``pin_memory=True``
    (cudaHostAlloc) buffers reached 123 and 117 GB/s (8 GiB each way); the
    copy speed in that state also depends on which host memory a buffer
    lands on, so this is not a guarantee.  The registration lasts as long as
    the returned tensor object; a view that outlives it still reads and
    writes the memory, as unpinned memory."""
    es = torch.empty(0, dtype=dtype).element_size()
    reg = _HostRegistration(int(numel) * es)
    t = reg.base[:int(numel) * es].view(dtype)
    t._corank_host_registration = reg
    return t


class HostMerger:
    """Stable merges of (A, B) pairs that live in pinned host memory (for
    example from `host_empty`).

    Each pair is copied to the device on an input-copy stream, merged on a
    compute stream and copied back on an output-copy stream; events order
    the three per pair, so the output copy of one pair overlaps the input
    copy of the next (the two copy directions run concurrently) and both
    overlap the merges.  Device buffers and workspaces are allocated once and
    reused by every ``run``; events order each buffer's reuse across calls,
    so the input copies of one call overlap the output copies of the
    previous one.  The caller's current stream waits at the end of ``run``
    for every output copy, so events recorded on it around a series of
    ``run`` calls time the whole pipeline and a synchronisation of it makes
    the outputs readable.  The input copies do not wait for the caller's
    earlier work: host inputs are read asynchronously, so the caller must not
    overwrite them before its stream has passed the end of the ``run`` that
    reads them.
    """

    def __init__(self, shapes, device="cuda"):
        """shapes: list of (m, n, torch dtype, key_type or None)."""
        lib = _lib.load()
        self.dev = torch.device(device)
        self.items = []
        for m, n, dtype, kt in shapes:
            A = torch.empty(m, dtype=dtype, device=self.dev)
            code = _key_code(A, kt)
            need = _size(lib.cr_merge_workspace_size, code, 0, m, n)
            self.items.append({
                "m": m, "n": n, "code": code, "A": A,
                "B": torch.empty(n, dtype=dtype, device=self.dev),
                "C": torch.empty(m + n, dtype=dtype, device=self.dev),
                "ws": torch.zeros(max(need, 256), dtype=torch.uint8, device=self.dev),
                "in_free": None, "out_free": None})
        self.s_in = torch.cuda.Stream(self.dev)
        self.s_comp = torch.cuda.Stream(self.dev)
        self.s_out = torch.cuda.Stream(self.dev)

    def run(self, host_pairs, host_outs):
        """host_pairs[i] = (A, B) pinned CPU tensors; host_outs[i] receives C."""
        lib = _lib.load()
        caller = torch.cuda.current_stream(self.dev)
        done = []
        for it, (hA, hB), hC in zip(self.items, host_pairs, host_outs):
            if hA.numel() != it["m"] or hB.numel() != it["n"] or hC.numel() != it["m"] + it["n"]:
                raise ValueError("host buffers do not match the planned sizes")
            if it["in_free"] is not None:
                self.s_in.wait_event(it["in_free"])     # previous merge read the inputs
            with torch.cuda.stream(self.s_in):
                it["A"].copy_(hA, non_blocking=True)
                it["B"].copy_(hB, non_blocking=True)
            loaded = torch.cuda.Event()
            loaded.record(self.s_in)
            self.s_comp.wait_event(loaded)
            if it["out_free"] is not None:
                self.s_comp.wait_event(it["out_free"])  # previous output copy finished
            _lib.check(lib.cr_stable_merge(it["code"], _ptr(it["A"]), it["m"], _ptr(it["B"]),
                                           it["n"], _ptr(it["C"]), None, _ptr(it["ws"]),
                                           it["ws"].numel(), self.s_comp.cuda_stream))
            merged = torch.cuda.Event()
            merged.record(self.s_comp)
            it["in_free"] = merged
            self.s_out.wait_event(merged)
            with torch.cuda.stream(self.s_out):
                hC.copy_(it["C"], non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(self.s_out)
            it["out_free"] = copied
            done.append(copied)
        for ev in done:
            caller.wait_event(ev)
        return host_outs

    def check(self):
        torch.cuda.synchronize(self.dev)
        for it in self.items:
            _lib.check(_lib.load().cr_workspace_status(_ptr(it["ws"]), _stream(self.dev)))


def merge_many(pairs, key_types=None):
    """Stable merges of independent (A, B) pairs with overlapped partitions
    (see MergeMany).  Returns the list of outputs."""
    return MergeMany(pairs, key_types).run()


def merge_kv(Ak, Av, Bk, Bv, key_type: str | None = None, tag: bool = False, ws=None):
    """Key-value stable merge; payload bits follow their keys.
    Returns (Ck, Cv) or (Ck, Cv, tags)."""
    lib = _lib.load()
    dev = _dev(Ak, Av, Bk, Bv)
    kt = _key_code(Ak, key_type)
    if Bk.dtype != Ak.dtype or Bv.dtype != Av.dtype:
        raise TypeError("A and B dtypes differ")
    vb = Av.element_size()
    m, n = Ak.numel(), Bk.numel()
    if Av.numel() != m or Bv.numel() != n:
        raise ValueError("payload and key lengths differ")
    Ck = torch.empty(m + n, dtype=Ak.dtype, device=dev)
    Cv = torch.empty(m + n, dtype=Av.dtype, device=dev)
    T = torch.empty(m + n, dtype=torch.int32, device=dev) if tag else None
    need = _size(lib.cr_merge_workspace_size, kt, vb, m, n)
    if ws is None:
        ws = _ws(need, dev)
    _lib.check(lib.cr_stable_merge_kv(kt, vb, _ptr(Ak), _ptr(Av), m, _ptr(Bk), _ptr(Bv), n,
                                      _ptr(Ck), _ptr(Cv), _ptr(T), _ptr(ws), ws.numel(),
                                      _stream(dev)))
    return (Ck, Cv, T) if tag else (Ck, Cv)


def merge_kv_backward(Ak, Bk, gC, key_type: str | None = None, ws=None):
    """Payload gradient of merge_kv: (gA, gB), bit-routed from gC by
    recomputed co-ranks (no stored permutation)."""
    lib = _lib.load()
    gC = gC.contiguous()
    dev = _dev(Ak, Bk, gC)
    kt = _key_code(Ak, key_type)
    vb = gC.element_size()
    m, n = Ak.numel(), Bk.numel()
    if gC.numel() != m + n:
        raise ValueError("gradient length differs from m + n")
    gA = torch.empty(m, dtype=gC.dtype, device=dev)
    gB = torch.empty(n, dtype=gC.dtype, device=dev)
    need = _size(lib.cr_merge_workspace_size, kt, vb, m, n)
    if ws is None:
        ws = _ws(need, dev)
    _lib.check(lib.cr_stable_merge_kv_backward(kt, vb, _ptr(Ak), m, _ptr(Bk), n, _ptr(gC),
                                               _ptr(gA), _ptr(gB), _ptr(ws), ws.numel(),
                                               _stream(dev)))
    return gA, gB


class MergeKV(torch.autograd.Function):
    """(Ck, Cv) = stable merge of (Ak, Av) and (Bk, Bv), differentiable in the
    payloads.  Only the keys are saved; backward recomputes the tile co-ranks
    and routes grad(Cv) to grad(Av), grad(Bv)."""

    @staticmethod
    def forward(ctx, Ak, Av, Bk, Bv, key_type=None):
        Ck, Cv = merge_kv(Ak, Av, Bk, Bv, key_type=key_type)
        ctx.save_for_backward(Ak, Bk)
        ctx.key_type = key_type
        ctx.mark_non_differentiable(Ck)
        return Ck, Cv

    @staticmethod
    def backward(ctx, gCk, gCv):
        Ak, Bk = ctx.saved_tensors
        if gCv is None:
            return None, None, None, None, None
        gA, gB = merge_kv_backward(Ak, Bk, gCv, key_type=ctx.key_type)
        return None, gA, None, gB, None


def merge_kv_autograd(Ak, Av, Bk, Bv, key_type: str | None = None):
    return MergeKV.apply(Ak, Av, Bk, Bv, key_type)


# ---------------------------------------------------------------------------
# batched (segmented) merge
# ---------------------------------------------------------------------------
def _offsets(off, dev) -> torch.Tensor:
    if not torch.is_tensor(off):
        off = torch.as_tensor(off, dtype=torch.int64)
    return off.to(device=dev, dtype=torch.int64).contiguous()


def batched_merge_kv(a_off, b_off, Ak, Av, Bk, Bv, key_type: str | None = None, ws=None,
                     out=None):
    """nseg merges in one persistent launch: segment s merges
    Ak[a_off[s]:a_off[s+1]] with Bk[b_off[s]:b_off[s+1]] into
    Ck[a_off[s]+b_off[s] : a_off[s+1]+b_off[s+1]].  Av/Bv may be None."""
    lib = _lib.load()
    dev = _dev(Ak, Av, Bk, Bv)
    kt = _key_code(Ak, key_type)
    ao, bo = _offsets(a_off, dev), _offsets(b_off, dev)
    nseg = ao.numel() - 1
    vb = Av.element_size() if Av is not None else 0
    at, bt = Ak.numel(), Bk.numel()
    if out is None:
        Ck = torch.empty(at + bt, dtype=Ak.dtype, device=dev)
        Cv = torch.empty(at + bt, dtype=Av.dtype, device=dev) if vb else None
    else:
        Ck, Cv = out
    need = _size(lib.cr_batched_workspace_size, kt, vb, nseg, at, bt)
    if ws is None:
        ws = _ws(need, dev)
    _lib.check(lib.cr_batched_merge_kv(kt, vb, nseg, _ptr(ao), _ptr(bo), _ptr(Ak), _ptr(Av), at,
                                       _ptr(Bk), _ptr(Bv), bt, _ptr(Ck), _ptr(Cv), _ptr(ws),
                                       ws.numel(), _stream(dev)))
    return Ck, Cv


def batched_merge_kv_backward(a_off, b_off, Ak, Bk, gC, key_type: str | None = None, ws=None,
                              out=None):
    lib = _lib.load()
    gC = gC.contiguous()
    dev = _dev(Ak, Bk, gC)
    kt = _key_code(Ak, key_type)
    ao, bo = _offsets(a_off, dev), _offsets(b_off, dev)
    nseg = ao.numel() - 1
    vb = gC.element_size()
    at, bt = Ak.numel(), Bk.numel()
    if out is None:
        gA = torch.empty(at, dtype=gC.dtype, device=dev)
        gB = torch.empty(bt, dtype=gC.dtype, device=dev)
    else:
        gA, gB = out
    need = _size(lib.cr_batched_workspace_size, kt, vb, nseg, at, bt)
    if ws is None:
        ws = _ws(need, dev)
    _lib.check(lib.cr_batched_merge_kv_backward(kt, vb, nseg, _ptr(ao), _ptr(bo), _ptr(Ak), at,
                                                _ptr(Bk), bt, _ptr(gC), _ptr(gA), _ptr(gB),
                                                _ptr(ws), ws.numel(), _stream(dev)))
    return gA, gB


class BatchedMergeGraph:
    """Batched merges of a fixed segment table, forward and payload
    backward, each captured once into a CUDA graph and then replayed: one
    replay runs the segment scan, the batched partition and the persistent
    tile merge (cr_batched_merge_kv, or its backward) on static buffers.

    a_off, b_off: the segment tables (nseg + 1 int64 entries each, host or
    device); key_dtype / val_dtype: torch dtypes of keys and payloads.
    forward(Ak, Av, Bk, Bv) copies the inputs into the static buffers (unless
    they are those buffers: `inputs()`), replays and returns (Ck, Cv);
    backward(gC) does the same for the gradient and returns (gA, gB).  The
    returned tensors are the static outputs, overwritten by the next replay.
    """

    def __init__(self, a_off, b_off, key_dtype, val_dtype, device="cuda",
                 key_type: str | None = None):
        self.dev = torch.device(device)
        self.ao = _offsets(a_off, self.dev)
        self.bo = _offsets(b_off, self.dev)
        at, bt = int(self.ao[-1].item()), int(self.bo[-1].item())
        self.Ak = torch.zeros(at, dtype=key_dtype, device=self.dev)
        self.Bk = torch.zeros(bt, dtype=key_dtype, device=self.dev)
        self.Av = torch.zeros(at, dtype=val_dtype, device=self.dev)
        self.Bv = torch.zeros(bt, dtype=val_dtype, device=self.dev)
        self.Ck = torch.empty(at + bt, dtype=key_dtype, device=self.dev)
        self.Cv = torch.empty(at + bt, dtype=val_dtype, device=self.dev)
        self.gC = torch.zeros(at + bt, dtype=val_dtype, device=self.dev)
        self.gA = torch.empty(at, dtype=val_dtype, device=self.dev)
        self.gB = torch.empty(bt, dtype=val_dtype, device=self.dev)
        self.key_type = key_type
        lib = _lib.load()
        kt = _key_code(self.Ak, key_type)
        vb = self.Av.element_size()
        need = _size(lib.cr_batched_workspace_size, kt, vb, self.ao.numel() - 1, at, bt)
        self.ws = _ws(need, self.dev)
        self._gf = self._capture(self._fwd)
        self._gb = self._capture(self._bwd)

    def _fwd(self):
        batched_merge_kv(self.ao, self.bo, self.Ak, self.Av, self.Bk, self.Bv,
                         key_type=self.key_type, ws=self.ws, out=(self.Ck, self.Cv))

    def _bwd(self):
        batched_merge_kv_backward(self.ao, self.bo, self.Ak, self.Bk, self.gC,
                                  key_type=self.key_type, ws=self.ws, out=(self.gA, self.gB))

    def _capture(self, body):
        # one eager run first (kernel attributes are set on first use), then capture
        s = torch.cuda.Stream(self.dev)
        s.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(s):
            body()
        torch.cuda.current_stream(self.dev).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            body()
        return g

    def inputs(self):
        """The static input buffers (Ak, Av, Bk, Bv) and gradient buffer gC."""
        return self.Ak, self.Av, self.Bk, self.Bv, self.gC

    def forward(self, Ak=None, Av=None, Bk=None, Bv=None):
        for dst, src in ((self.Ak, Ak), (self.Av, Av), (self.Bk, Bk), (self.Bv, Bv)):
            if src is not None and src is not dst:
                dst.copy_(src)
        self._gf.replay()
        return self.Ck, self.Cv

    def backward(self, gC=None):
        if gC is not None and gC is not self.gC:
            self.gC.copy_(gC)
        self._gb.replay()
        return self.gA, self.gB

    def check(self):
        """Device status of the last replay (raises CorankError on a device error)."""
        workspace_status(self.ws)


# ---------------------------------------------------------------------------
# merge-sort passes
# ---------------------------------------------------------------------------
def merge_pass_workspace_bytes(key_type: str, val_bytes: int, N: int, width: int) -> int:
    lib = _lib.load()
    return _size(lib.cr_merge_pass_workspace_size, _lib.key_code(key_type), int(val_bytes),
                 int(N), int(width))


def merge_pass(X, Xv, width: int, key_type: str | None = None, out=None, ws=None):
    """One bottom-up pass: runs of `width` in X merged pairwise. Returns (Y, Yv)."""
    lib = _lib.load()
    dev = _dev(X, Xv)
    kt = _key_code(X, key_type)
    vb = Xv.element_size() if Xv is not None else 0
    N = X.numel()
    if out is None:
        Y = torch.empty_like(X)
        Yv = torch.empty_like(Xv) if Xv is not None else None
    else:
        Y, Yv = out
    if ws is None:
        ws = _ws(_size(lib.cr_merge_pass_workspace_size, kt, vb, N, int(width)), dev)
    _lib.check(lib.cr_merge_pass(kt, vb, _ptr(X), _ptr(Xv), N, int(width), _ptr(Y), _ptr(Yv),
                                 _ptr(ws), ws.numel(), _stream(dev)))
    return Y, Yv


def merge_pass_backward(X, gY, width: int, key_type: str | None = None, out=None, ws=None):
    """Payload gradient of merge_pass; X are the pass's input keys."""
    lib = _lib.load()
    dev = _dev(X, gY)
    kt = _key_code(X, key_type)
    vb = gY.element_size()
    N = X.numel()
    gX = out if out is not None else torch.empty_like(gY)
    if ws is None:
        ws = _ws(_size(lib.cr_merge_pass_workspace_size, kt, vb, N, int(width)), dev)
    _lib.check(lib.cr_merge_pass_backward(kt, vb, _ptr(X), N, int(width), _ptr(gY), _ptr(gX),
                                          _ptr(ws), ws.numel(), _stream(dev)))
    return gX


@dataclass
class PassRecord:
    """What a recorded merge pass leaves for its backward: the pass's tile
    table (ws) and one source bit per output (flags), for N elements merged
    with run width `width`."""
    ws: torch.Tensor
    flags: torch.Tensor
    N: int
    width: int
    key_code: int
    val_bytes: int


def merge_pass_record_bytes(key_type: str, val_bytes: int, N: int, width: int):
    """(workspace bytes, flag words) of a recorded pass under the current tile shape."""
    lib = _lib.load()
    wsb, fw = ctypes.c_size_t(), ctypes.c_size_t()
    _lib.check(lib.cr_merge_pass_record_size(_lib.key_code(key_type), int(val_bytes), int(N),
                                             int(width), ctypes.byref(wsb), ctypes.byref(fw)))
    return wsb.value, fw.value


def new_pass_record(key_type: str, val_bytes: int, N: int, width: int, device) -> PassRecord:
    wsb, fw = merge_pass_record_bytes(key_type, val_bytes, N, width)
    dev = torch.device(device)
    return PassRecord(_ws(wsb, dev),
                      torch.empty(max(fw, 4), dtype=torch.int32, device=dev),
                      int(N), int(width), _lib.key_code(key_type), int(val_bytes))


def merge_pass_record(X, Xv, width: int, key_type: str | None = None, out=None,
                      record: PassRecord | None = None):
    """merge_pass that also records the merge decisions for
    merge_pass_backward_recorded.  Returns (Y, Yv, record)."""
    lib = _lib.load()
    dev = _dev(X, Xv)
    kt = _key_code(X, key_type)
    vb = Xv.element_size()
    N = X.numel()
    Y, Yv = out if out is not None else (torch.empty_like(X), torch.empty_like(Xv))
    if record is None:
        record = new_pass_record(kt, vb, N, width, dev)
    _lib.check(lib.cr_merge_pass_record(kt, vb, _ptr(X), _ptr(Xv), N, int(width), _ptr(Y),
                                        _ptr(Yv), _ptr(record.flags), record.flags.numel(),
                                        _ptr(record.ws), record.ws.numel(), _stream(dev)))
    record.N, record.width, record.key_code, record.val_bytes = N, int(width), kt, vb
    return Y, Yv, record


def merge_pass_backward_recorded(record: PassRecord, gY, out=None):
    """Payload gradient of a recorded merge pass, routed from its record
    (no keys are read)."""
    lib = _lib.load()
    dev = _dev(gY)
    gX = out if out is not None else torch.empty_like(gY)
    _lib.check(lib.cr_merge_pass_backward_recorded(
        record.key_code, gY.element_size(), record.N, record.width, _ptr(record.flags),
        record.flags.numel(), _ptr(gY), _ptr(gX), _ptr(record.ws), record.ws.numel(),
        _stream(dev)))
    return gX


def check_sorted(A: torch.Tensor, key_type: str | None = None) -> int:
    """-1 if A is sorted in key_type's order, else the first position p with
    A[p] before A[p-1] (a debug check of the merge's precondition)."""
    lib = _lib.load()
    dev = _dev(A)
    kt = _key_code(A, key_type)
    out = torch.empty(1, dtype=torch.int64, device=dev)
    ws = _ws(16, dev)
    _lib.check(lib.cr_check_sorted(kt, _ptr(A), A.numel(), _ptr(out), _ptr(ws), ws.numel(),
                                   _stream(dev)))
    return int(out.item())


def workspace_status(ws: torch.Tensor) -> None:
    """Synchronise the current stream and raise if the last call that used
    `ws` recorded a device-side error."""
    lib = _lib.load()
    _lib.check(lib.cr_workspace_status(_ptr(ws), _stream(ws.device)))


# ---------------------------------------------------------------------------
# bottom-up stable merge sort: a chain of merge passes, optionally replayed
# from CUDA graphs
# ---------------------------------------------------------------------------
def sort_run_length() -> int:
    """Length of the runs cr_sort_runs sorts (the merge sort's first width)."""
    return int(_lib.load().cr_sort_run_length())


def sort_runs(X, Xv=None, key_type: str | None = None, out=None):
    """Stably sort every run of sort_run_length() elements of X (payload Xv
    follows).  Returns (Y, Yv)."""
    lib = _lib.load()
    dev = _dev(X, Xv)
    kt = _key_code(X, key_type)
    vb = Xv.element_size() if Xv is not None else 0
    if out is None:
        Y = torch.empty_like(X)
        Yv = torch.empty_like(Xv) if Xv is not None else None
    else:
        Y, Yv = out
    _lib.check(lib.cr_sort_runs(kt, vb, _ptr(X), _ptr(Xv), X.numel(), _ptr(Y), _ptr(Yv),
                                _stream(dev)))
    return Y, Yv


def sort_runs_backward(X, gY, key_type: str | None = None, out=None):
    """Payload gradient of sort_runs; X are its input keys."""
    lib = _lib.load()
    dev = _dev(X, gY)
    kt = _key_code(X, key_type)
    gX = out if out is not None else torch.empty_like(gY)
    _lib.check(lib.cr_sort_runs_backward(kt, gY.element_size(), _ptr(X), X.numel(), _ptr(gY),
                                         _ptr(gX), _stream(dev)))
    return gX


def sort_runs_record(X, Xv, key_type: str | None = None, out=None, perm=None):
    """sort_runs that also writes each run's permutation (int16 container of
    uint16 in-run indices) for sort_runs_backward_recorded.  Returns
    (Y, Yv, perm)."""
    lib = _lib.load()
    dev = _dev(X, Xv)
    kt = _key_code(X, key_type)
    Y, Yv = out if out is not None else (torch.empty_like(X), torch.empty_like(Xv))
    if perm is None:
        perm = torch.empty(X.numel(), dtype=torch.int16, device=dev)
    _lib.check(lib.cr_sort_runs_record(kt, Xv.element_size(), _ptr(X), _ptr(Xv), X.numel(),
                                       _ptr(Y), _ptr(Yv), _ptr(perm), _stream(dev)))
    return Y, Yv, perm


def sort_runs_backward_recorded(perm, gY, out=None):
    """Payload gradient of sort_runs_record from its permutation (no keys)."""
    lib = _lib.load()
    dev = _dev(perm, gY)
    gX = out if out is not None else torch.empty_like(gY)
    _lib.check(lib.cr_sort_runs_backward_recorded(gY.element_size(), gY.numel(), _ptr(perm),
                                                  _ptr(gY), _ptr(gX), _stream(dev)))
    return gX


def merge_runs_block_length() -> int:
    """Chunk length of merge_runs_block (the width its runs reach)."""
    return int(_lib.load().cr_merge_runs_block_length())


def merge_runs_block(X, Xv, width: int, key_type: str | None = None, out=None, perm=None,
                     record: bool = False):
    """The merge passes width, 2 width, ... up to merge_runs_block_length()
    done inside shared memory, one chunk per CTA (width a power of two; width
    1 sorts every chunk of any input stably).  Returns (Y, Yv, perm); perm
    (the chunk permutation, int16 container of uint16 indices) only with
    record=True or a perm buffer given."""
    lib = _lib.load()
    dev = _dev(X, Xv)
    kt = _key_code(X, key_type)
    vb = Xv.element_size() if Xv is not None else 0
    if out is None:
        Y = torch.empty_like(X)
        Yv = torch.empty_like(Xv) if Xv is not None else None
    else:
        Y, Yv = out
    if perm is None and record:
        perm = torch.empty(X.numel(), dtype=torch.int16, device=dev)
    _lib.check(lib.cr_merge_runs_block(kt, vb, _ptr(X), _ptr(Xv), X.numel(), int(width),
                                       _ptr(Y), _ptr(Yv), _ptr(perm), _stream(dev)))
    return Y, Yv, perm


def merge_runs_block_backward_recorded(perm, gY, out=None):
    """Payload gradient of a recorded merge_runs_block (no keys read)."""
    lib = _lib.load()
    dev = _dev(perm, gY)
    gX = out if out is not None else torch.empty_like(gY)
    _lib.check(lib.cr_merge_runs_block_backward_recorded(gY.element_size(), gY.numel(),
                                                         _ptr(perm), _ptr(gY), _ptr(gX),
                                                         _stream(dev)))
    return gX


class MergeSortPlan:
    """Buffers and (optionally) CUDA graphs for a stable merge sort of N keys
    with payloads.

    With ``run`` given, the input's runs of ``run`` elements must already be
    sorted; with ``run=None`` any input is accepted (runs of one element).
    The runs are merged pairwise, width run, 2 run, 4 run, ..., in stages:
    with ``record=True`` and a power-of-two ``run`` up to half of
    merge_runs_block_length(), the widths below that length are merged in
    one shared-memory stage (merge_runs_block; from unsorted input it sorts
    every chunk of that length), the rest by merge passes over HBM
    (cr_merge_pass*).  With ``record=False`` unsorted input is first sorted
    into runs of sort_run_length() (run formation, cr_sort_runs), whose
    backward replays that sort.

    The backward needs every stage's merge decisions.  With ``record=True``
    (default) each forward stage records them (a merge pass: its tile table
    plus one bit per element; the shared-memory stage: its chunk
    permutation, two bytes per element) and the backward routes
    gradients from those records without reading keys; keys then ping-pong
    between two buffers.  With ``record=False`` the input keys of every pass
    are kept ((passes + 1) * N key slots) and the backward re-merges them
    (cr_merge_pass_backward).  Payloads and gradients ping-pong between two
    buffers; with run formation the unsorted input keys are kept too.
    Forward and backward are each captured once into a CUDA graph
    (``graph=True``) and replayed.  The tile shape must not change between
    a recorded forward and its backward.
    """

    def __init__(self, N: int, run: int | None, key_dtype, val_dtype, device="cuda",
                 key_type: str | None = None, graph: bool = True, record: bool = True):
        self.N = int(N)
        self.record = bool(record)
        # run formation by cr_sort_runs (recompute form only): its own step
        self.form_runs = run is None and not self.record
        if run is None:
            self.run = sort_run_length() if self.form_runs else 1
        else:
            self.run = int(run)
        self.device = torch.device(device)
        self.key_type = key_type
        R = merge_runs_block_length()
        w = self.run
        self.stages = []            # ("block", width) or ("pass", width)
        if (self.record and w < self.N and w >= 1 and w <= R // 2
                and (w & (w - 1)) == 0):
            self.stages.append(("block", w))
            w = R
        while w < self.N:
            self.stages.append(("pass", w))
            w *= 2
        self.widths = [w for kind, w in self.stages if kind == "pass"]
        S = len(self.stages)
        nkeys = 2 if self.record else S + 1
        self.keys = [torch.empty(self.N, dtype=key_dtype, device=self.device)
                     for _ in range(nkeys)]
        self.vals = [torch.empty(self.N, dtype=val_dtype, device=self.device) for _ in range(2)]
        self.grads = [torch.empty(self.N, dtype=val_dtype, device=self.device) for _ in range(2)]
        self.input_keys = (torch.empty(self.N, dtype=key_dtype, device=self.device)
                           if self.form_runs else None)
        kt = key_type or _DTYPE_KEY[key_dtype]
        vb = torch.empty(0, dtype=val_dtype).element_size()
        self.records = [None] * S       # per stage: PassRecord or block permutation
        self.ws = None
        if self.record:
            for i, (kind, w) in enumerate(self.stages):
                self.records[i] = (new_pass_record(kt, vb, self.N, w, self.device)
                                   if kind == "pass" else
                                   torch.empty(self.N, dtype=torch.int16, device=self.device))
        else:
            need = max([merge_pass_workspace_bytes(kt, vb, self.N, w) for w in self.widths]
                       + [256])
            self.ws = _ws(need, self.device)
        self.use_graph = graph
        self._gf = None
        self._gb = None

    @property
    def passes(self) -> int:
        """Number of merge stages (shared-memory stage and HBM passes)."""
        return len(self.stages)

    def _key_buf(self, i: int) -> torch.Tensor:
        """Input keys of stage i (i == passes: the sorted output)."""
        return self.keys[i & 1] if self.record else self.keys[i]

    def _load(self, X, Xv):
        if self.form_runs:
            self.input_keys.copy_(X)
            self.vals[1].copy_(Xv)
        else:
            self.keys[0].copy_(X)
            self.vals[0].copy_(Xv)

    def run_formation(self):
        """Recompute form with unsorted input: sort runs of sort_run_length()
        (the recorded form forms runs in its shared-memory stage)."""
        if self.form_runs:
            sort_runs(self.input_keys, self.vals[1], key_type=self.key_type,
                      out=(self.keys[0], self.vals[0]))

    def run_stage(self, i: int):
        """Forward of stage i: keys/payloads of parity i -> parity i + 1."""
        kind, w = self.stages[i]
        src = (self._key_buf(i), self.vals[i & 1])
        out = (self._key_buf(i + 1), self.vals[(i + 1) & 1])
        if kind == "block":
            merge_runs_block(*src, w, key_type=self.key_type, out=out, perm=self.records[i])
        elif self.record:
            merge_pass_record(*src, w, key_type=self.key_type, out=out, record=self.records[i])
        else:
            merge_pass(*src, w, key_type=self.key_type, out=out, ws=self.ws)

    def run_stage_backward(self, i: int):
        """Backward of stage i: gradients of parity i + 1 -> parity i."""
        kind, w = self.stages[i]
        src, dst = self.grads[(i + 1) & 1], self.grads[i & 1]
        if kind == "block":
            merge_runs_block_backward_recorded(self.records[i], src, out=dst)
        elif self.record:
            merge_pass_backward_recorded(self.records[i], src, out=dst)
        else:
            merge_pass_backward(self.keys[i], src, w, key_type=self.key_type, out=dst,
                                ws=self.ws)

    def run_formation_backward(self):
        if self.form_runs:
            sort_runs_backward(self.input_keys, self.grads[0], key_type=self.key_type,
                               out=self.grads[1])

    def _forward_body(self):
        self.run_formation()
        for i in range(len(self.stages)):
            self.run_stage(i)

    def _backward_body(self):
        for i in reversed(range(len(self.stages))):
            self.run_stage_backward(i)
        self.run_formation_backward()

    def _grad_out(self):
        return self.grads[1] if self.form_runs else self.grads[0]

    def _capture(self, body):
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            body()                       # warm-up outside the capture
        torch.cuda.current_stream(self.device).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            body()
        return g

    def forward(self, X: torch.Tensor, Xv: torch.Tensor):
        """Sort; returns views of the plan's output buffers (keys, payloads)."""
        self._load(X, Xv)
        if self.use_graph and (self.passes or self.form_runs):
            if self._gf is None:
                self._gf = self._capture(self._forward_body)
                self._load(X, Xv)
            self._gf.replay()
        else:
            self._forward_body()
        return self._key_buf(self.passes), self.vals[self.passes & 1]

    def backward(self, gY: torch.Tensor) -> torch.Tensor:
        """Payload gradient of the sort: gX[perm[t]] = gY[t]."""
        self.grads[self.passes & 1].copy_(gY)
        if self.use_graph and (self.passes or self.form_runs):
            if self._gb is None:
                self._gb = self._capture(self._backward_body)
                self.grads[self.passes & 1].copy_(gY)
            self._gb.replay()
        else:
            self._backward_body()
        return self._grad_out()


class _MergeSortFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Xv, plan):
        Y, Yv = plan.forward(X, Xv)
        ctx.plan = plan
        ctx.mark_non_differentiable(Y)
        return Y.clone(), Yv.clone()

    @staticmethod
    def backward(ctx, gY, gYv):
        if gYv is None:
            return None, None, None
        return None, ctx.plan.backward(gYv.contiguous()).clone(), None


def merge_sort(X: torch.Tensor, Xv: torch.Tensor, run: int | None = None,
               key_type: str | None = None, graph: bool = True,
               plan: MergeSortPlan | None = None, record: bool = True):
    """Stable merge sort of X carrying payloads Xv; differentiable in Xv.
    run=None sorts any input (runs are formed on the GPU first); an integer
    run declares that X's runs of that width are already sorted.  Returns
    (keys, payloads)."""
    _dev(X, Xv)
    if plan is None:
        plan = MergeSortPlan(X.numel(), run, X.dtype, Xv.dtype, X.device, key_type, graph,
                             record)
    return _MergeSortFn.apply(X, Xv, plan)
