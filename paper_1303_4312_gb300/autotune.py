"""Autotuner for the tile shape of the merge kernels.

For every (key size, payload width) combination and each class it times the
calls of that class under each tile shape the library offers for the
combination, keeps the fastest, and writes a JSON table keyed by GPU name and
compute capability:

* balanced: one merge of m = n (2^log2_size elements in all);
* skewed: one merge with an input 512 times longer than the other;
* small: m = n with 2^21 elements in all (below the small-merge limit);
* batched: one batched call over segment pairs whose sizes are drawn
  log-uniformly in [1, 2^18] (m and n independent, keys uniform in
  [0, 2^24) sorted per segment), as many pairs as fill 2^log2_size
  elements on average;
* pass: merge-sort passes over 2^log2_size elements at run widths 4096 and
  2^(log2_size-1) (recorded forward and recorded backward with payloads,
  the plain pass for keys only).

Forward and, with payloads, backward times are summed.  ``apply()`` loads
the table for the current GPU (if one exists and was made for the library's
list of shapes) and selects those shapes through ``cr_set_tile_shape_for``;
the package does this on first use.

Usage on a GPU:  python -m paper_1303_4312_gb300.autotune [--log2-size 26]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import re

from . import _lib

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_DIR = os.path.join(HERE, "tuning")

# (key type name, payload bytes) combinations; uint keys share the kernels'
# shapes with the int keys of the same width.
COMBOS = [("i32", 0), ("i32", 4), ("i32", 8), ("i64", 0), ("i64", 4), ("i64", 8)]
CLASSES = (("balanced", 0), ("skewed", 1), ("small", 2), ("batched", 3), ("pass", 4))


def shape_list(lib) -> list:
    """[nt, ipt, ilp] of every tile shape the library offers, by index."""
    out = []
    nt, ipt, ilp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    for sh in range(lib.cr_tile_shape_count()):
        _lib.check(lib.cr_tile_shape_info(sh, ctypes.byref(nt), ctypes.byref(ipt),
                                          ctypes.byref(ilp)))
        out.append([nt.value, ipt.value, ilp.value])
    return out


def _slug(name: str) -> str:
    return re.sub(r"[^A-Za-z0-9]+", "_", name).strip("_").lower()


def table_path(gpu_name: str) -> str:
    return os.path.join(TABLE_DIR, f"{_slug(gpu_name)}.json")


def apply(lib=None, gpu_name: str | None = None, cc: str | None = None,
          path: str | None = None) -> dict | None:
    """Select the tuned shapes for this GPU (or from the table at `path`).
    Returns the table used, or None when there is none for this GPU or it
    was made for another list of shapes or compute capability."""
    lib = lib or _lib.load()
    if path is not None:
        gpu_name = gpu_name or ""
    elif gpu_name is None:
        try:
            import torch
            if not torch.cuda.is_available():
                return None
            gpu_name = torch.cuda.get_device_name()
            cc = "%d.%d" % torch.cuda.get_device_capability()
        except Exception:
            return None
    path = path or table_path(gpu_name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    # a table names shapes by index: it is valid for the same list of shapes
    if table.get("shape_list") != shape_list(lib) or (cc and table.get("cc") != cc):
        return None
    for key, entry in table.get("shapes", {}).items():
        kt, vb = key.split(":")
        for cls, index in CLASSES:
            if cls in entry:
                _lib.check(lib.cr_set_tile_shape_for(_lib.KEY_TYPES[kt], int(vb), index,
                                                     int(entry[cls]["shape"])))
    return table


def _inputs_batched(kt: str, vb: int, log2_size: int, g, dev):
    """Segment tables and per-segment sorted keys of a batched tuning case."""
    import numpy as np
    import torch
    from . import workloads
    nseg = max(16, (1 << log2_size) // 42000)
    ms, ns = workloads.log_uniform_sizes(4321, nseg)
    a_off = torch.from_numpy(workloads.offsets(ms)).to(dev)
    b_off = torch.from_numpy(workloads.offsets(ns)).to(dev)
    kdt = torch.int32 if kt == "i32" else torch.int64

    def seg_sorted(sizes):
        total = int(sizes.sum())
        seg = torch.repeat_interleave(torch.arange(nseg, device=dev),
                                      torch.from_numpy(np.asarray(sizes)).to(dev))
        key = torch.randint(0, 1 << 24, (total,), generator=g, device=dev, dtype=torch.int64)
        return (torch.sort(seg * (1 << 24) + key).values & ((1 << 24) - 1)).to(kdt)
    A, B = seg_sorted(ms), seg_sorted(ns)
    return nseg, a_off, b_off, A, B


def _time(fns, reps):
    import torch
    row = {}
    for name, fn in fns:
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        row[name] = e0.elapsed_time(e1) / reps
    return row


def _time_batched(lib, kt: str, vb: int, log2_size: int, reps: int):
    import torch
    code = _lib.KEY_TYPES[kt]
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(4321)
    nseg, ao, bo, A, B = _inputs_batched(kt, vb, log2_size, g, dev)
    at, bt = A.numel(), B.numel()
    vdt = {4: torch.float32, 8: torch.float64}.get(vb)
    Av = torch.randn(at, generator=g, device=dev, dtype=vdt) if vb else None
    Bv = torch.randn(bt, generator=g, device=dev, dtype=vdt) if vb else None
    C = torch.empty(at + bt, dtype=A.dtype, device=dev)
    Cv = torch.empty(at + bt, device=dev, dtype=vdt) if vb else None
    gC = torch.randn(at + bt, generator=g, device=dev, dtype=vdt) if vb else None
    gA = torch.empty(at, device=dev, dtype=vdt) if vb else None
    gB = torch.empty(bt, device=dev, dtype=vdt) if vb else None
    p = lambda t: None if t is None else t.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    results = {}
    for shape in range(lib.cr_tile_shape_count()):
        if lib.cr_set_tile_shape_for(code, vb, 3, shape) != 0:
            continue
        need = ctypes.c_size_t()
        _lib.check(lib.cr_batched_workspace_size(code, vb, nseg, at, bt, ctypes.byref(need)))
        ws = torch.empty(need.value, dtype=torch.uint8, device=dev)

        def fwd():
            _lib.check(lib.cr_batched_merge_kv(code, vb, nseg, p(ao), p(bo), p(A), p(Av), at,
                                               p(B), p(Bv), bt, p(C), p(Cv), p(ws), ws.numel(),
                                               s))

        def bwd():
            _lib.check(lib.cr_batched_merge_kv_backward(code, vb, nseg, p(ao), p(bo), p(A), at,
                                                        p(B), bt, p(gC), p(gA), p(gB), p(ws),
                                                        ws.numel(), s))
        results[shape] = _time((("fwd", fwd), ("bwd", bwd)) if vb else (("fwd", fwd),), reps)
        _lib.check(lib.cr_workspace_status(p(ws), s))
    return results


def _time_pass(lib, kt: str, vb: int, log2_size: int, reps: int):
    import torch
    code = _lib.KEY_TYPES[kt]
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(8765)
    N = 1 << log2_size
    kdt = torch.int32 if kt == "i32" else torch.int64
    lo, hi = (-(1 << 31), 1 << 31) if kt == "i32" else (-(1 << 62), 1 << 62)
    raw = torch.randint(lo, hi, (N,), generator=g, device=dev, dtype=torch.int64).to(kdt)
    vdt = {4: torch.float32, 8: torch.float64}.get(vb)
    Xv = torch.randn(N, generator=g, device=dev, dtype=vdt) if vb else None
    Y = torch.empty_like(raw)
    Yv = torch.empty_like(Xv) if vb else None
    gY = torch.randn(N, generator=g, device=dev, dtype=vdt) if vb else None
    gX = torch.empty_like(gY) if vb else None
    p = lambda t: None if t is None else t.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    widths = (4096, N // 2)
    Xs = [torch.sort(raw.view(-1, w)).values.reshape(-1) for w in widths]
    results = {}
    for shape in range(lib.cr_tile_shape_count()):
        if lib.cr_set_tile_shape_for(code, vb, 4, shape) != 0:
            continue
        fns = []
        for X, w in zip(Xs, widths):
            wsb, fw = ctypes.c_size_t(), ctypes.c_size_t()
            if vb:
                _lib.check(lib.cr_merge_pass_record_size(code, vb, N, w, ctypes.byref(wsb),
                                                         ctypes.byref(fw)))
            else:
                _lib.check(lib.cr_merge_pass_workspace_size(code, vb, N, w, ctypes.byref(wsb)))
            ws = torch.empty(max(wsb.value, 256), dtype=torch.uint8, device=dev)
            fl = torch.empty(max(fw.value, 4), dtype=torch.int32, device=dev)

            def fwd(X=X, w=w, ws=ws, fl=fl, nfw=fw.value):
                if vb:
                    _lib.check(lib.cr_merge_pass_record(code, vb, p(X), p(Xv), N, w, p(Y), p(Yv),
                                                        p(fl), nfw, p(ws), ws.numel(), s))
                else:
                    _lib.check(lib.cr_merge_pass(code, 0, p(X), None, N, w, p(Y), None, p(ws),
                                                 ws.numel(), s))

            def bwd(w=w, ws=ws, fl=fl, nfw=fw.value):
                _lib.check(lib.cr_merge_pass_backward_recorded(code, vb, N, w, p(fl), nfw, p(gY),
                                                               p(gX), p(ws), ws.numel(), s))
            fns.append((f"fwd_w{w}", fwd))
            if vb:
                fns.append((f"bwd_w{w}", bwd))
        # forward first (the backward routes through the record it leaves)
        fwd_fns = [f for f in fns if f[0].startswith("fwd")]
        row = _time(fwd_fns, reps)
        if vb:
            for (name, fn), (_, f) in zip([f for f in fns if f[0].startswith("bwd")], fwd_fns):
                f()
                row.update(_time(((name, fn),), reps))
        results[shape] = row
    return results


def _time_combo(lib, kt: str, vb: int, log2_size: int, reps: int, cls: int):
    import torch
    code = _lib.KEY_TYPES[kt]
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(1234)
    total = 1 << (min(log2_size, 21) if cls == 2 else log2_size)
    m = total // 513 if cls == 1 else total // 2
    n = total - m
    kdt = torch.int32 if kt == "i32" else torch.int64
    lo, hi = (-(1 << 31), 1 << 31) if kt == "i32" else (-(1 << 62), 1 << 62)
    A = torch.sort(torch.randint(lo, hi, (m,), generator=g, device=dev, dtype=torch.int64)
                   .to(kdt)).values
    B = torch.sort(torch.randint(lo, hi, (n,), generator=g, device=dev, dtype=torch.int64)
                   .to(kdt)).values
    vdt = {4: torch.float32, 8: torch.float64}.get(vb)
    Av = torch.randn(m, generator=g, device=dev, dtype=vdt) if vb else None
    Bv = torch.randn(n, generator=g, device=dev, dtype=vdt) if vb else None
    C = torch.empty(m + n, dtype=kdt, device=dev)
    Cv = torch.empty(m + n, dtype=vdt, device=dev) if vb else None
    gC = torch.randn(m + n, device=dev, dtype=vdt) if vb else None
    gA = torch.empty(m, device=dev, dtype=vdt) if vb else None
    gB = torch.empty(n, device=dev, dtype=vdt) if vb else None
    p = lambda t: None if t is None else t.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    results = {}
    for shape in range(lib.cr_tile_shape_count()):
        if lib.cr_set_tile_shape_for(code, vb, cls, shape) != 0:
            continue
        need = ctypes.c_size_t()
        _lib.check(lib.cr_merge_workspace_size(code, vb, m, n, ctypes.byref(need)))
        ws = torch.empty(need.value, dtype=torch.uint8, device=dev)

        def fwd():
            _lib.check(lib.cr_stable_merge_kv(code, vb, p(A), p(Av), m, p(B), p(Bv), n, p(C),
                                              p(Cv), None, p(ws), ws.numel(), s))

        def bwd():
            _lib.check(lib.cr_stable_merge_kv_backward(code, vb, p(A), m, p(B), n, p(gC), p(gA),
                                                       p(gB), p(ws), ws.numel(), s))

        row = {}
        for name, fn in (("fwd", fwd), ("bwd", bwd)) if vb else (("fwd", fwd),):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            row[name] = e0.elapsed_time(e1) / reps
        _lib.check(lib.cr_workspace_status(p(ws), s))
        results[shape] = row
    return results


def tune(log2_size: int = 26, reps: int = 10, write: bool = True,
         out: str | None = None) -> dict:
    import torch
    lib = _lib.load()
    name = torch.cuda.get_device_name()
    cc = "%d.%d" % torch.cuda.get_device_capability()
    table = {"gpu": name, "cc": cc, "abi": lib.cr_abi_version(), "log2_size": log2_size,
             "shape_list": shape_list(lib), "shapes": {}}
    for kt, vb in COMBOS:
        code = _lib.KEY_TYPES[kt]
        entry = {}
        for cls, index in CLASSES:
            before = lib.cr_get_tile_shape_for(code, vb, index)
            if cls == "batched":
                res = _time_batched(lib, kt, vb, log2_size, reps)
            elif cls == "pass":
                res = _time_pass(lib, kt, vb, log2_size, reps)
            else:
                res = _time_combo(lib, kt, vb, log2_size, reps, index)
            best = min(res, key=lambda s: sum(res[s].values()))
            nt, ipt, ilp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            _lib.check(lib.cr_tile_shape_info(best, ctypes.byref(nt), ctypes.byref(ipt),
                                              ctypes.byref(ilp)))
            entry[cls] = {
                "shape": best, "nt": nt.value, "ipt": ipt.value, "ilp": ilp.value,
                "ms": {str(s): {k: round(v, 4) for k, v in r.items()} for s, r in res.items()}}
            _lib.check(lib.cr_set_tile_shape_for(code, vb, index, before))
        table["shapes"][f"{kt}:{vb}"] = entry
    if write:
        path = out or table_path(name)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
    return table


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--log2-size", type=int, default=26)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--no-write", action="store_true")
    ap.add_argument("--out", default=None, help="table path (default: tuning/<gpu>.json)")
    a = ap.parse_args()
    print(json.dumps(tune(a.log2_size, a.reps, not a.no_write, a.out), indent=1))
