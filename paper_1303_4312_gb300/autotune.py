"""Autotuner for the tile shape of the merge kernels.

For every (key size, payload width) combination and each geometry class
(balanced: m = n; skewed: one input 512 times longer than the other; small:
m = n with 2^21 elements in all, below the library's small-merge limit) it times
the forward merge (and, with payloads, the backward) of a seeded random
problem under each tile shape the library offers for that combination, keeps
the fastest, and writes a JSON table keyed by GPU name and compute
capability.  ``apply()`` loads the
table for the current GPU (if one exists) and selects those shapes through
``cr_set_tile_shape``; the package does this on first use.

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
CLASSES = (("balanced", 0), ("skewed", 1), ("small", 2))


def _slug(name: str) -> str:
    return re.sub(r"[^A-Za-z0-9]+", "_", name).strip("_").lower()


def table_path(gpu_name: str) -> str:
    return os.path.join(TABLE_DIR, f"{_slug(gpu_name)}.json")


def apply(lib=None, gpu_name: str | None = None, cc: str | None = None) -> dict | None:
    """Select the tuned shapes for this GPU.  Returns the table used, or None."""
    lib = lib or _lib.load()
    if gpu_name is None:
        try:
            import torch
            if not torch.cuda.is_available():
                return None
            gpu_name = torch.cuda.get_device_name()
            cc = "%d.%d" % torch.cuda.get_device_capability()
        except Exception:
            return None
    path = table_path(gpu_name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    if table.get("abi") != lib.cr_abi_version() or (cc and table.get("cc") != cc):
        return None
    for key, entry in table.get("shapes", {}).items():
        kt, vb = key.split(":")
        for cls, index in CLASSES:
            if cls in entry:
                _lib.check(lib.cr_set_tile_shape_for(_lib.KEY_TYPES[kt], int(vb), index,
                                                     int(entry[cls]["shape"])))
    return table


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
             "shapes": {}}
    for kt, vb in COMBOS:
        code = _lib.KEY_TYPES[kt]
        entry = {}
        for cls, index in CLASSES:
            before = lib.cr_get_tile_shape_for(code, vb, index)
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
