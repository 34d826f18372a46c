"""Benchmark of the stable-merge hot path on GB300.

One step = the three large single merges, each through the C ABI as the
two launches of cr_stable_merge (the grid-level co-rank partition writing one
record per equal output tile, then the persistent tile merge), back to
back on one stream:

  large_i32   m = n = 2^28 int32 keys uniform over the full int32 range
  skewed_u64  m = 2^20, n = 2^29 uint64 keys uniform over the full range
  dup16_i32   m = n = 2^28 int32 keys drawn from 16 distinct values

Inputs are seeded synthetic arrays (device-generated, sorted), far larger
than L2 (129 MB), so no flush is needed between steps.

  value     merged elements/s over the whole job, inputs resident in HBM,
            CUDA events around exactly K steps (max over ranks)
  e2e       the same metric with the inputs copied from pinned host memory
            and the merged outputs copied back inside every timed step
  roofline  the tile-merge kernel: algorithmic bytes (each input element read
            once, each output written once) / its CUDA-event time, against the
            measured HBM copy bandwidth
  cpu_baseline  the CPU oracle (Algorithm 2 on POSIX threads over all host
            cores) on full steps of the same inputs
  rows      the task's other configurations, forward and backward, each timed
            on its own inputs with CUDA events after the headline (N=1 only):
            single_i32_tag (keys + tags, L2 flushed), kv_u32_f32 (forward
            merge, backward with recomputed co-ranks), batched_i32_f32 (8192
            segment pairs, one call per direction) and sort_u64_f32 (recorded
            merge-sort chain, one CUDA graph per direction), with a clock
            record of their own

`--impl reference` times the CPU oracle as the reference arm.
Launch: python bench.py [--gpus N] [--steps K] [--warmup W]; N>1 via
torchrun, one process per GPU, each merging its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "merged elements/s and achieved HBM GB/s (% of GB300 peak), fwd and bwd, bit-exact"
UNIT = "elements/s"
WORKLOAD = "large_single_merges"
FALLBACK_HBM_GBS = 6800.0

MERGES = [
    # name, generator, key type, key bytes
    ("large_i32", "t_large_i32", "i32", 4),
    ("skewed_u64", "t_skewed_u64", "u64", 8),
    ("dup16_i32", "t_dup16_i32", "i32", 4),
]


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=None,
                   help="steps of the end-to-end measurement (default: --steps)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-rows", action="store_true",
                   help="skip the other configurations' forward/backward rows of the default "
                        "line")
    p.add_argument("--shift", type=int, default=0,
                   help="divide every workload size by 2^shift (for quick runs)")
    p.add_argument("--workload", default=WORKLOAD,
                   choices=[WORKLOAD, "single_tag", "kv", "batched", "merge_sort",
                            "partition_variants", "orders"],
                   help="the default is the headline workload; the others measure the "
                        "remaining rows of the path (one JSON line each)")
    p.add_argument("--batched-pairs", type=int, default=8192,
                   help="segment pairs of the batched workload (8192 as specified; 24576 "
                        "reaches about 2^30 elements)")
    p.add_argument("--tile-shape", type=int, default=None,
                   help="force tile shape S (cr_tile_shape_info) for every key type and "
                        "payload width it fits, instead of the tuned table")
    return p.parse_args()


def force_tile_shape(lib, shape):
    """--tile-shape: select `shape` wherever it fits (others keep theirs)."""
    if shape is None:
        return
    for code in range(4):
        for vb in (0, 4, 8):
            lib.cr_set_tile_shape(code, vb, shape)


def tile_shapes(lib, combos):
    """NTxIPTxILP of the balanced, skewed and small-merge shape for each
    (label, key code, vb)."""
    import ctypes
    out = {}
    for label, code, vb in combos:
        row = []
        for cls in (0, 1, 2):
            s = lib.cr_get_tile_shape_for(code, vb, cls)
            nt, ipt, ilp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            lib.cr_tile_shape_info(s, ctypes.byref(nt), ctypes.byref(ipt), ctypes.byref(ilp))
            row.append(f"{nt.value}x{ipt.value}x{ilp.value}")
        out[label] = row if len(set(row)) > 1 else row[0]
    return out


# ---------------------------------------------------------------------------
# distributed plumbing (timing only; the data path has no collective)
# ---------------------------------------------------------------------------
def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist.init_process_group("gloo")
    return rank, world, local, dist


def reduce_max(x: float, dist, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_inputs(device, shift: int):
    from paper_1303_4312_gb300 import workloads as W
    out = []
    for name, gen, kt, kb in MERGES:
        A, B = getattr(W, gen)(device=device, shift=shift)
        out.append({"name": name, "A": A, "B": B, "kt": kt, "kb": kb,
                    "m": A.numel(), "n": B.numel()})
    return out


def algorithmic_bytes(mg) -> int:
    """Each input key read once, each output key written once."""
    return 2 * (mg["m"] + mg["n"]) * mg["kb"]


# nominal HBM3e bandwidth of one GB300 (the measured copy peak is the
# roofline denominator; the nominal figure is reported beside it)
NOMINAL_HBM_GBS = 7900.0


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# sources that define the tile-merge and partition kernels the headline step
# runs and their launch configuration (other kernels do not change them)
DIGEST_SOURCES = ("cr_device.cuh", "cr_merge.cuh", "cr_partition.cuh", "cr_launch.cuh",
                  "cr_keyops_impl.cuh", "cr_keys_i32_fwd.cu", "cr_keys_u64_fwd.cu",
                  "cr_keys_i32.cu", "cr_keys_u64.cu")


def kernel_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1303_4312_gb300", "csrc")
    for f in DIGEST_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(shift: int):
    """DRAM bytes per tile-merge launch from the committed ncu summary, if it
    was taken on the current kernel sources and this workload size."""
    path = os.path.join(ROOT, "profiles", "merge_tiles_large_single_merges.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_digest:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"workload_shift:\s*(\d+)", text)
    if not (m and t and s) or m.group(1) != kernel_digest() or int(s.group(1)) != shift:
        return None
    return float(t.group(1))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local, dist):
    import torch
    from paper_1303_4312_gb300 import _lib, build
    from paper_1303_4312_gb300 import api

    build.build()
    lib = _lib.load()
    force_tile_shape(lib, args.tile_shape)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    merges = make_inputs(dev, args.shift)
    for mg in merges:
        mg["C"] = torch.empty(mg["m"] + mg["n"], dtype=mg["A"].dtype, device=dev)
        need = api.merge_workspace_bytes(mg["kt"], 0, mg["m"], mg["n"])
        mg["ws"] = torch.empty(need, dtype=torch.uint8, device=dev)
        mg["code"] = _lib.KEY_TYPES[mg["kt"]]
    torch.cuda.synchronize()

    def launch(mg, ev=None):
        # cr_stable_merge's two launches, issued as its two steps so that
        # each kernel can be timed on its own
        A, B, C, ws = mg["A"], mg["B"], mg["C"], mg["ws"]
        if ev is not None:
            ev[0].record(stream)
        _lib.check(lib.cr_merge_partition(mg["code"], 0, A.data_ptr(), mg["m"], B.data_ptr(),
                                          mg["n"], ws.data_ptr(), ws.numel(), sp))
        if ev is not None:
            ev[1].record(stream)
        _lib.check(lib.cr_merge_tiles(mg["code"], 0, A.data_ptr(), None, mg["m"], B.data_ptr(),
                                      None, mg["n"], C.data_ptr(), None, None, ws.data_ptr(),
                                      ws.numel(), sp))
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        for mg in merges:
            launch(mg)
    torch.cuda.synchronize()
    for mg in merges:
        api.workspace_status(mg["ws"])

    K = args.steps
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in merges]
           for _ in range(K)]
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    barrier(dist)
    torch.cuda.synchronize()
    for k in range(K):
        for mg, ev in zip(merges, evs[k]):
            launch(mg, ev)
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop() if clocks else None
    for mg in merges:
        api.workspace_status(mg["ws"])

    total_ms = evs[0][0][0].elapsed_time(evs[K - 1][-1][2])
    step_spans = sorted(evs[k][0][0].elapsed_time(evs[k][-1][2]) for k in range(K))
    part_ms = {mg["name"]: sum(evs[k][q][0].elapsed_time(evs[k][q][1]) for k in range(K)) / K
               for q, mg in enumerate(merges)}
    tile_ms = {mg["name"]: sum(evs[k][q][1].elapsed_time(evs[k][q][2]) for k in range(K))
               for q, mg in enumerate(merges)}
    total_ms = reduce_max(total_ms, dist, dev)
    elems = sum(mg["m"] + mg["n"] for mg in merges)
    ms_per_step = total_ms / K
    value = world * elems * K / (total_ms / 1e3)

    peak, peak_kind = measured_peak()
    alg_bytes = sum(algorithmic_bytes(mg) for mg in merges)
    achieved = alg_bytes * K / (sum(tile_ms.values()) / 1e3) / 1e9
    step_gbs = alg_bytes / (ms_per_step / 1e3) / 1e9

    # end to end: pinned host inputs -> device -> merge -> pinned host outputs
    e2e = run_e2e(args, merges, lib, dev, stream, dist, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_from(merges)

    # the other configurations (forward and backward), one GPU only
    rows = None
    if world == 1 and not args.no_rows:
        for mg in merges:
            del mg["A"], mg["B"], mg["C"], mg["ws"]
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        rows = run_rows(args, lib, dev, stream, peak)

    if rank != 0:
        return None
    per_merge = {mg["name"]: {
        "elements": mg["m"] + mg["n"],
        "partition_ms": round(part_ms[mg["name"]], 4),
        "tile_kernel_ms": round(tile_ms[mg["name"]] / K, 4),
        "tile_kernel_gbs": round(algorithmic_bytes(mg) / (tile_ms[mg["name"]] / K / 1e3) / 1e9, 1),
    } for mg in merges}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+uint64 keys",
        "data": "synthetic (seeded, sorted; device-generated)",
        "config": {"workload": WORKLOAD, "merges": [f"{m[0]}" for m in MERGES],
                   "elements_per_step": elems, "l2": "inputs larger than L2 (no flush)",
                   "size_shift": args.shift, "parallelism": f"replicas x{world}"},
        "tile_shapes": tile_shapes(lib, [("int32", 0, 0), ("uint64", 3, 0)]),
        "hbm_gbs_step": round(step_gbs, 1),
        "frac_of_peak_step": round(step_gbs / peak, 4),
        "per_merge": per_merge,
        "partition_ms_per_step": round(sum(part_ms.values()), 4),
        "step_ms": {"median": round(step_spans[K // 2], 4), "best": round(step_spans[0], 4),
                    "worst": round(step_spans[-1], 4)},

        "roofline": {"kernel": "merge_tiles_kernel", "bound": "hbm",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "frac_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "traffic": recorded_traffic(args.shift),
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_launch": alg_bytes / len(merges)},
        "e2e": e2e,
        "rows": rows,
        "gpu_launches": 2 * len(merges) * K,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    return line


def run_e2e(args, merges, lib, dev, stream, dist, world):
    """The step through HostMerger: inputs from pinned host memory, outputs
    back to pinned host memory, copies and merges pipelined on three streams."""
    import torch
    from paper_1303_4312_gb300 import api
    K = args.e2e_steps or args.steps
    hosts, outs = [], []
    for mg in merges:
        hA = api.host_empty(mg["m"], mg["A"].dtype)
        hB = api.host_empty(mg["n"], mg["A"].dtype)
        hA.copy_(mg["A"])
        hB.copy_(mg["B"])
        hosts.append((hA, hB))
        outs.append(api.host_empty(mg["m"] + mg["n"], mg["A"].dtype))
    hm = api.HostMerger([(mg["m"], mg["n"], mg["A"].dtype, mg["kt"]) for mg in merges], dev)
    torch.cuda.synchronize()
    h2d = sum((mg["m"] + mg["n"]) * mg["kb"] for mg in merges)
    d2h = h2d
    for _ in range(max(1, min(args.warmup, 3))):
        hm.run(hosts, outs)
    hm.check()
    barrier(dist)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        hm.run(hosts, outs)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    hm.check()
    ms = reduce_max(e0.elapsed_time(e1), dist, dev)
    # the merged outputs really came back: equal to the device-resident result
    for mg, hC in zip(merges, outs):
        assert torch.equal(hC[: 1 << 20], mg["C"][: 1 << 20].cpu())
    elems = sum(mg["m"] + mg["n"] for mg in merges)
    return {"value": world * elems * K / (ms / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": K,
            "ms_per_step": ms / K, "api": "HostMerger (registered host buffers from host_empty, 3 streams)"}


# ---------------------------------------------------------------------------
# the other configurations, forward and backward, in the default line
# ---------------------------------------------------------------------------
def _gbs(nbytes, ms):
    return nbytes / (ms / 1e3) / 1e9


def _dir_row(N, ms, alg_bytes, peak, kernel_ms=None, kernel_bytes=None, launches=None):
    """One direction of a row: its whole time (every kernel of the call)
    and, when given, its merge kernel's own time, each as algorithmic GB/s
    and fractions of the measured and the nominal HBM bandwidth."""
    g = _gbs(alg_bytes, ms)
    out = {"ms": round(ms, 4), "elements_per_s": N / (ms / 1e3), "gbs": round(g, 1),
           "frac": round(g / peak, 4), "frac_nominal": round(g / NOMINAL_HBM_GBS, 4),
           "alg_bytes": int(alg_bytes)}
    if kernel_ms is not None:
        gk = _gbs(kernel_bytes if kernel_bytes is not None else alg_bytes, kernel_ms)
        out["merge_kernel"] = {"ms": round(kernel_ms, 4), "gbs": round(gk, 1),
                               "frac": round(gk / peak, 4),
                               "frac_nominal": round(gk / NOMINAL_HBM_GBS, 4)}
    if launches is not None:
        out["launches_per_step"] = launches
    return out


def _timed(stream, K, W, body, labels):
    """Run body(mark) W + K times; `mark(label)` records an event after a
    launch (label None opens a step).  Returns per-label mean ms over the K
    timed steps."""
    import torch
    tot = {lb: 0.0 for lb in labels}
    marks = []
    for k in range(W + K):
        cur = []

        def mark(label=None):
            if k >= W:
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                cur.append((label, ev))
        body(mark)
        if k >= W:
            marks.append(cur)
    torch.cuda.synchronize()
    for cur in marks:
        for (_, a), (label, b) in zip(cur, cur[1:]):
            if label is not None:
                tot[label] += a.elapsed_time(b)
    return {lb: v / K for lb, v in tot.items()}


def row_single_tag(lib, dev, stream, K, W, peak, shift):
    """single_i32_tag: keys and source tags, L2 flushed before every step."""
    import torch
    from paper_1303_4312_gb300 import _lib, api
    from paper_1303_4312_gb300 import workloads as Wk
    A, B = Wk.single_i32_tag(seed=1, shift=shift)
    A, B = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    m, n = A.numel(), B.numel()
    C = torch.empty(m + n, dtype=torch.int32, device=dev)
    T = torch.empty(m + n, dtype=torch.int32, device=dev)
    ws = torch.empty(api.merge_workspace_bytes("i32", 0, m, n), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sp = stream.cuda_stream
    p = lambda t: t.data_ptr()

    def body(mark):
        flush.fill_(1)
        mark()
        _lib.check(lib.cr_merge_partition(0, 0, p(A), m, p(B), n, p(ws), ws.numel(), sp))
        mark("partition")
        _lib.check(lib.cr_merge_tiles(0, 0, p(A), None, m, p(B), None, n, p(C), None, p(T),
                                      p(ws), ws.numel(), sp))
        mark("tiles")
    t = _timed(stream, K, W, body, ["partition", "tiles"])
    api.workspace_status(ws)
    N = m + n
    return {"workload": "single_i32_tag", "elements": N, "l2": "flushed before every step",
            "fwd": _dir_row(N, t["partition"] + t["tiles"], 12 * N, peak, t["tiles"],
                            launches=2),
            "note": "2.6M elements: launch- and latency-bound, not an HBM-roofline case"}


def row_kv(lib, dev, stream, K, W, peak, shift):
    """kv_u32_f32: forward key-value merge, backward payload routing with
    the co-ranks recomputed from the keys (a partition launch of its own)."""
    import torch
    from paper_1303_4312_gb300 import _lib, api
    from paper_1303_4312_gb300 import workloads as Wk
    Ak, Av, Bk, Bv = Wk.t_kv_u32_f32(device=dev, shift=shift)
    m, n = Ak.numel(), Bk.numel()
    N = m + n
    Ck = torch.empty(N, dtype=torch.int32, device=dev)
    Cv = torch.empty(N, dtype=torch.float32, device=dev)
    gC = torch.randn(N, device=dev, generator=torch.Generator(device=dev).manual_seed(15))
    gA = torch.empty(m, device=dev)
    gB = torch.empty(n, device=dev)
    ws = torch.empty(api.merge_workspace_bytes("u32", 4, m, n), dtype=torch.uint8, device=dev)
    sp = stream.cuda_stream
    p = lambda t: t.data_ptr()

    def body(mark):
        mark()
        _lib.check(lib.cr_merge_partition(1, 4, p(Ak), m, p(Bk), n, p(ws), ws.numel(), sp))
        mark("fwd_partition")
        _lib.check(lib.cr_merge_tiles(1, 4, p(Ak), p(Av), m, p(Bk), p(Bv), n, p(Ck), p(Cv), None,
                                      p(ws), ws.numel(), sp))
        mark("fwd_tiles")
        _lib.check(lib.cr_merge_partition(1, 4, p(Ak), m, p(Bk), n, p(ws), ws.numel(), sp))
        mark("bwd_partition")
        _lib.check(lib.cr_merge_tiles_backward(1, 4, p(Ak), m, p(Bk), n, p(gC), p(gA), p(gB),
                                               p(ws), ws.numel(), sp))
        mark("bwd_tiles")
    t = _timed(stream, K, W, body, ["fwd_partition", "fwd_tiles", "bwd_partition", "bwd_tiles"])
    api.workspace_status(ws)
    return {"workload": "kv_u32_f32", "elements": N,
            "fwd": _dir_row(N, t["fwd_partition"] + t["fwd_tiles"], 16 * N, peak, t["fwd_tiles"],
                            launches=2),
            "bwd": _dir_row(N, t["bwd_partition"] + t["bwd_tiles"], 12 * N, peak, t["bwd_tiles"],
                            launches=2),
            "l2": "inputs larger than L2 (no flush)"}


def row_batched(lib, dev, stream, K, W, peak, pairs=8192):
    """batched_i32_f32: one cr_batched_merge_kv call (segment scan,
    partition, persistent tile merge) and its backward."""
    import ctypes
    import torch
    from paper_1303_4312_gb300 import _lib, api
    from paper_1303_4312_gb300 import workloads as Wk
    a_off, b_off, A, Av, B, Bv = Wk.t_batched_i32_f32(device=dev, nseg=pairs)
    ao = torch.from_numpy(a_off).to(dev)
    bo = torch.from_numpy(b_off).to(dev)
    at, bt = A.numel(), B.numel()
    nseg = len(a_off) - 1
    N = at + bt
    Ck = torch.empty(N, dtype=torch.int32, device=dev)
    Cv = torch.empty(N, dtype=torch.float32, device=dev)
    gC = torch.randn(N, device=dev, generator=torch.Generator(device=dev).manual_seed(16))
    gA = torch.empty(at, device=dev)
    gB = torch.empty(bt, device=dev)
    need = ctypes.c_size_t()
    _lib.check(lib.cr_batched_workspace_size(0, 4, nseg, at, bt, ctypes.byref(need)))
    ws = torch.empty(need.value, dtype=torch.uint8, device=dev)
    sp = stream.cuda_stream
    p = lambda t: t.data_ptr()

    def body(mark):
        mark()
        _lib.check(lib.cr_batched_merge_kv(0, 4, nseg, p(ao), p(bo), p(A), p(Av), at, p(B), p(Bv),
                                           bt, p(Ck), p(Cv), p(ws), ws.numel(), sp))
        mark("fwd")
        _lib.check(lib.cr_batched_merge_kv_backward(0, 4, nseg, p(ao), p(bo), p(A), at, p(B), bt,
                                                    p(gC), p(gA), p(gB), p(ws), ws.numel(), sp))
        mark("bwd")
    t = _timed(stream, K, W, body, ["fwd", "bwd"])
    api.workspace_status(ws)
    del Ck, Cv, gA, gB, ws
    # the same two calls captured into CUDA graphs (BatchedMergeGraph) and
    # replayed on its static buffers, filled once with these inputs
    g = api.BatchedMergeGraph(ao, bo, torch.int32, torch.float32, dev)
    for dst, src in zip(g.inputs(), (A, Av, B, Bv, gC)):
        dst.copy_(src)
    del A, Av, B, Bv, gC

    def gbody(mark):
        mark()
        g.forward()
        mark("fwd")
        g.backward()
        mark("bwd")
    tg = _timed(stream, K, W, gbody, ["fwd", "bwd"])
    g.check()
    del g
    nt, ipt, ilp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    shape = lib.cr_get_tile_shape_for(0, 4, 0)
    lib.cr_tile_shape_info(shape, ctypes.byref(nt), ctypes.byref(ipt), ctypes.byref(ilp))
    return {"workload": "batched_i32_f32", "elements": N, "segments": nseg,
            "tile_shape": f"{nt.value}x{ipt.value}x{ilp.value}",
            "fwd": _dir_row(N, t["fwd"], 16 * N, peak, launches=3),
            "bwd": _dir_row(N, t["bwd"], 12 * N, peak, launches=3),
            "fwd_graph": _dir_row(N, tg["fwd"], 16 * N, peak, launches=3),
            "bwd_graph": _dir_row(N, tg["bwd"], 12 * N, peak, launches=3),
            "note": "each direction is one call (segment scan + partition + tile merge); "
                    "*_graph: the same call captured in a CUDA graph and replayed"}


def row_sort(lib, dev, stream, K, W, peak, shift):
    """sort_u64_f32: the recorded merge-sort chain from runs of 1024, each
    direction one CUDA-graph replay (shared-memory stage for the widths below
    4096, then HBM passes)."""
    import torch
    from paper_1303_4312_gb300 import api
    from paper_1303_4312_gb300 import workloads as Wk
    X, Xv = Wk.t_sort_u64_f32(device=dev, shift=shift)
    N = X.numel()
    gY = torch.randn(N, device=dev, generator=torch.Generator(device=dev).manual_seed(17))
    plan = api.MergeSortPlan(N, 1024, X.dtype, Xv.dtype, dev, key_type="u64", graph=True,
                             record=True)
    plan.forward(X, Xv)
    plan.backward(gY)
    fwd_b = sum(26.0 if kd == "block" else 24 + 1 / 8 for kd, _ in plan.stages) * N
    bwd_b = sum(10.0 if kd == "block" else 8 + 1 / 8 for kd, _ in plan.stages) * N

    def body(mark):
        plan.keys[0].copy_(X)
        plan.vals[0].copy_(Xv)
        plan.grads[plan.passes & 1].copy_(gY)
        mark()
        plan._gf.replay()
        mark("fwd")
        plan._gb.replay()
        mark("bwd")
    t = _timed(stream, K, W, body, ["fwd", "bwd"])
    launches = len(plan.stages)
    stages = [f"{kd}:{w}" for kd, w in plan.stages]
    del plan
    return {"workload": "sort_u64_f32", "elements": N, "stages": stages,
            "fwd": _dir_row(N, t["fwd"], fwd_b, peak),
            "bwd": _dir_row(N, t["bwd"], bwd_b, peak),
            "note": "bytes summed over stages (keys + payloads in and out, plus the recorded "
                    "flag bit or chunk permutation; backward gY in, gX out plus the record); "
                    f"{launches} stages, each one or two kernel launches, in one graph per "
                    "direction"}


def run_rows(args, lib, dev, stream, peak):
    """The task's other configurations, forward and backward, each on its
    own inputs (created, timed and freed in turn), inside one clock-sampling
    window."""
    import torch
    K, W = args.steps, max(3, args.warmup)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    rows = {}
    for name, fn in (("single_i32_tag", lambda: row_single_tag(lib, dev, stream, K, W, peak,
                                                                args.shift)),
                     ("kv_u32_f32", lambda: row_kv(lib, dev, stream, K, W, peak, args.shift)),
                     ("batched_i32_f32", lambda: row_batched(lib, dev, stream, K, W, peak,
                                                             args.batched_pairs)),
                     ("sort_u64_f32", lambda: row_sort(lib, dev, stream, K, W, peak,
                                                       args.shift))):
        rows[name] = fn()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    rows["clocks"] = clocks.stop()
    rows["steps"], rows["warmup"] = K, W
    return rows


# ---------------------------------------------------------------------------
# the other rows of the path, one measured line each
# ---------------------------------------------------------------------------
class KernelTimer:
    """CUDA events around each launch of a step; sums per label."""

    def __init__(self, stream):
        import torch
        self.torch = torch
        self.stream = stream
        self.marks = []

    def mark(self, label=None):
        ev = self.torch.cuda.Event(enable_timing=True)
        ev.record(self.stream)
        self.marks.append((label, ev))

    def totals(self):
        out = {}
        for (_, a), (label, b) in zip(self.marks, self.marks[1:]):
            if label is not None:
                out[label] = out.get(label, 0.0) + a.elapsed_time(b)
        return out


def _l2_flush_buffer(dev):
    import torch
    return torch.empty(256 << 20, dtype=torch.uint8, device=dev)


def run_row(args):
    import torch
    from paper_1303_4312_gb300 import _lib, api, build
    from paper_1303_4312_gb300 import workloads as W
    build.build()
    lib = _lib.load()
    force_tile_shape(lib, args.tile_shape)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    peak, peak_kind = measured_peak()
    K, Wm = args.steps, args.warmup
    ptr = lambda t: None if t is None else t.data_ptr()
    res = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": Wm,
           "higher_is_better": True, "data": "synthetic (seeded)", "peak_gbs": peak,
           "peak_source": peak_kind}

    def finish(timer_totals, alg, name, elems, extra=None, combos=()):
        step_ms = sum(timer_totals.values()) / K
        res.update({"value": elems / (step_ms / 1e3), "ms_per_step": step_ms,
                    "config": {"workload": name, "elements_per_step": elems,
                               "size_shift": args.shift,
                               "tile_shapes": tile_shapes(lib, combos)}})
        kern = {}
        for label, ms in timer_totals.items():
            b = alg.get(label)
            kern[label] = {"ms": round(ms / K, 4)}
            if b:
                gbs = b / (ms / K / 1e3) / 1e9
                kern[label].update({"gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                                    "frac_nominal": round(gbs / NOMINAL_HBM_GBS, 4),
                                    "alg_bytes": b})
        res["kernels"] = kern
        if extra:
            res.update(extra)
        return res

    if args.workload == "single_tag":
        A, B = W.single_i32_tag(seed=1, shift=args.shift)
        A, B = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
        m, n = A.numel(), B.numel()
        C = torch.empty(m + n, dtype=torch.int32, device=dev)
        T = torch.empty(m + n, dtype=torch.int32, device=dev)
        ws = torch.empty(api.merge_workspace_bytes("i32", 0, m, n), dtype=torch.uint8, device=dev)
        flush = _l2_flush_buffer(dev)
        timer = KernelTimer(stream)
        for k in range(Wm + K):
            flush.fill_(k & 0xFF)      # L2 flush between steps (outside the timed marks)
            if k >= Wm:
                timer.mark()
            _lib.check(lib.cr_merge_partition(0, 0, ptr(A), m, ptr(B), n, ptr(ws), ws.numel(), sp))
            if k >= Wm:
                timer.mark("partition")
            _lib.check(lib.cr_merge_tiles(0, 0, ptr(A), None, m, ptr(B), None, n, ptr(C), None,
                                          ptr(T), ptr(ws), ws.numel(), sp))
            if k >= Wm:
                timer.mark("tiles_keys_tags")
            if k >= Wm:
                timer.marks.append((None, timer.marks[-1][1]))
        torch.cuda.synchronize()
        api.workspace_status(ws)
        tot = {k: v for k, v in timer.totals().items()}
        # warm: the same two launches back to back, inputs left in L2 (the
        # whole problem is 31 MB); and the one-call form in a CUDA graph
        warm = KernelTimer(stream)
        for k in range(Wm + K):
            if k >= Wm:
                warm.mark()
            _lib.check(lib.cr_merge_partition(0, 0, ptr(A), m, ptr(B), n, ptr(ws), ws.numel(), sp))
            if k >= Wm:
                warm.mark("partition")
            _lib.check(lib.cr_merge_tiles(0, 0, ptr(A), None, m, ptr(B), None, n, ptr(C), None,
                                          ptr(T), ptr(ws), ws.numel(), sp))
            if k >= Wm:
                warm.mark("tiles_keys_tags")
                warm.marks.append((None, warm.marks[-1][1]))
        torch.cuda.synchronize()
        wt = warm.totals()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            api.merge(A, B, key_type="i32", tag=True, out=C, out_tag=T, ws=ws)
        stream.wait_stream(side)
        with torch.cuda.graph(g):
            api.merge(A, B, key_type="i32", tag=True, out=C, out_tag=T, ws=ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(Wm):
            g.replay()
        e0.record(stream)
        for _ in range(K):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        api.workspace_status(ws)
        graph_ms = e0.elapsed_time(e1) / K
        return finish(tot, {"tiles_keys_tags": 12 * (m + n)}, "single_i32_tag", m + n,
                      {"l2": "flushed between steps (256 MB write)",
                       "warm": {"partition_ms": round(wt["partition"] / K, 4),
                                "tiles_ms": round(wt["tiles_keys_tags"] / K, 4),
                                "graph_ms_per_merge": round(graph_ms, 4),
                                "note": "inputs resident in L2; graph: one cr_stable_merge "
                                        "call (both launches) replayed back to back"}},
                      combos=[("int32", 0, 0)])

    if args.workload == "partition_variants":
        # the paper's two forms of the block co-ranks: shared (computed once
        # per boundary, cr_merge_partition) and sync-free (every tile co-ranks
        # both of its ends, cr_merge_partition_alg2); same tile merge after
        merges = make_inputs(dev, args.shift)
        out = {}
        tot_shared = tot_free = 0.0
        for mg in merges:
            code = _lib.KEY_TYPES[mg["kt"]]
            m, n = mg["m"], mg["n"]
            A, B = mg["A"], mg["B"]
            C = torch.empty(m + n, dtype=A.dtype, device=dev)
            ws = torch.empty(api.merge_workspace_bytes(mg["kt"], 0, m, n), dtype=torch.uint8,
                             device=dev)
            res = {}
            for name, fn in (("shared", lib.cr_merge_partition), ("alg2", lib.cr_merge_partition_alg2)):
                timer = KernelTimer(stream)
                for k in range(Wm + K):
                    t = k >= Wm
                    if t:
                        timer.mark()
                    _lib.check(fn(code, 0, ptr(A), m, ptr(B), n, ptr(ws), ws.numel(), sp))
                    if t:
                        timer.mark("partition")
                    _lib.check(lib.cr_merge_tiles(code, 0, ptr(A), None, m, ptr(B), None, n, ptr(C),
                                                  None, None, ptr(ws), ws.numel(), sp))
                    if t:
                        timer.mark("tiles")
                torch.cuda.synchronize()
                api.workspace_status(ws)
                tt = timer.totals()
                res[name] = {"partition_ms": round(tt["partition"] / K, 4),
                             "tiles_ms": round(tt["tiles"] / K, 4)}
            tot_shared += res["shared"]["partition_ms"] + res["shared"]["tiles_ms"]
            tot_free += res["alg2"]["partition_ms"] + res["alg2"]["tiles_ms"]
            out[mg["name"]] = res
        elems = sum(mg["m"] + mg["n"] for mg in merges)
        r = {"metric": METRIC, "unit": UNIT, "value": elems / (tot_shared / 1e3),
             "ms_per_step": tot_shared, "ms_per_step_alg2": tot_free,
             "config": {"workload": "partition_variants", "elements_per_step": elems,
                        "size_shift": args.shift},
             "per_merge": out, "steps": K, "warmup": Wm}
        return r

    if args.workload == "orders":
        # the same keys-only merge in several key orders: the storage type's
        # own (int32), IEEE-754 totalOrder floats, descending; the orders
        # other than the native one map the staged keys in shared memory
        torch_gen = torch.Generator(device=dev).manual_seed(8)
        rows = {}
        for kt, dt in (("i32", torch.int32), ("i32:desc", torch.int32), ("f32", torch.float32),
                       ("f32:desc", torch.float32), ("f64", torch.float64)):
            m = n = ((1 << 28) >> args.shift) if dt != torch.float64 else ((1 << 27) >> args.shift)
            vals = torch.randn(m + n, generator=torch_gen, device=dev)
            if dt == torch.int32:
                vals = (vals * (1 << 28)).to(torch.int32)
            else:
                vals = vals.to(dt)
            desc = kt.endswith(":desc")
            A = torch.sort(vals[:m], descending=desc, stable=True).values
            B = torch.sort(vals[m:], descending=desc, stable=True).values
            del vals
            code = _lib.key_code(kt)
            C = torch.empty(m + n, dtype=dt, device=dev)
            ws = torch.empty(api.merge_workspace_bytes(kt, 0, m, n), dtype=torch.uint8, device=dev)
            timer = KernelTimer(stream)
            for k in range(Wm + K):
                t = k >= Wm
                if t:
                    timer.mark()
                _lib.check(lib.cr_merge_partition(code, 0, ptr(A), m, ptr(B), n, ptr(ws),
                                                  ws.numel(), sp))
                if t:
                    timer.mark("partition")
                _lib.check(lib.cr_merge_tiles(code, 0, ptr(A), None, m, ptr(B), None, n, ptr(C),
                                              None, None, ptr(ws), ws.numel(), sp))
                if t:
                    timer.mark("tiles")
            torch.cuda.synchronize()
            api.workspace_status(ws)
            tt = timer.totals()
            b = 2 * (m + n) * A.element_size()
            gbs = b / (tt["tiles"] / K / 1e3) / 1e9
            rows[kt] = {"elements": m + n, "partition_ms": round(tt["partition"] / K, 4),
                        "tiles_ms": round(tt["tiles"] / K, 4), "tiles_gbs": round(gbs, 1),
                        "tiles_frac": round(gbs / peak, 4)}
            del A, B, C, ws
            torch.cuda.empty_cache()
        tot = sum(r["partition_ms"] + r["tiles_ms"] for r in rows.values())
        elems = sum(r["elements"] for r in rows.values())
        return {"metric": METRIC, "unit": UNIT, "value": elems / (tot / 1e3), "ms_per_step": tot,
                "config": {"workload": "orders", "size_shift": args.shift,
                           "orders": list(rows)}, "per_order": rows, "steps": K, "warmup": Wm,
                "peak_gbs": peak, "peak_source": peak_kind}

    if args.workload == "kv":
        Ak, Av, Bk, Bv = W.t_kv_u32_f32(device=dev, shift=args.shift)
        m, n = Ak.numel(), Bk.numel()
        Ck = torch.empty(m + n, dtype=torch.int32, device=dev)
        Cv = torch.empty(m + n, dtype=torch.float32, device=dev)
        gC = torch.randn(m + n, device=dev)
        gA = torch.empty(m, device=dev)
        gB = torch.empty(n, device=dev)
        ws = torch.empty(api.merge_workspace_bytes("u32", 4, m, n), dtype=torch.uint8, device=dev)
        timer = KernelTimer(stream)
        for k in range(Wm + K):
            t = k >= Wm
            if t:
                timer.mark()
            _lib.check(lib.cr_merge_partition(1, 4, ptr(Ak), m, ptr(Bk), n, ptr(ws), ws.numel(), sp))
            if t:
                timer.mark("fwd_partition")
            _lib.check(lib.cr_merge_tiles(1, 4, ptr(Ak), ptr(Av), m, ptr(Bk), ptr(Bv), n, ptr(Ck),
                                          ptr(Cv), None, ptr(ws), ws.numel(), sp))
            if t:
                timer.mark("fwd_tiles")
            # backward recomputes the partition from the keys (nothing stored)
            _lib.check(lib.cr_merge_partition(1, 4, ptr(Ak), m, ptr(Bk), n, ptr(ws), ws.numel(), sp))
            if t:
                timer.mark("bwd_partition")
            _lib.check(lib.cr_merge_tiles_backward(1, 4, ptr(Ak), m, ptr(Bk), n, ptr(gC), ptr(gA),
                                                   ptr(gB), ptr(ws), ws.numel(), sp))
            if t:
                timer.mark("bwd_tiles")
                timer.marks.append((None, timer.marks[-1][1]))
        torch.cuda.synchronize()
        api.workspace_status(ws)
        tot = timer.totals()
        N = m + n
        fwd_ms = (tot["fwd_partition"] + tot["fwd_tiles"]) / K
        bwd_ms = (tot["bwd_partition"] + tot["bwd_tiles"]) / K
        return finish(tot, {"fwd_tiles": 16 * N, "bwd_tiles": 12 * N}, "kv_u32_f32", N,
                      {"fwd": {"ms": round(fwd_ms, 4), "elements_per_s": N / (fwd_ms / 1e3),
                               "gbs": round(16 * N / (fwd_ms / 1e3) / 1e9, 1)},
                       "bwd": {"ms": round(bwd_ms, 4), "elements_per_s": N / (bwd_ms / 1e3),
                               "gbs": round(12 * N / (bwd_ms / 1e3) / 1e9, 1)}},
                      combos=[("uint32+f32", 1, 4)])

    if args.workload == "batched":
        a_off, b_off, A, Av, B, Bv = W.t_batched_i32_f32(device=dev, nseg=args.batched_pairs)
        ao = torch.from_numpy(a_off).to(dev)
        bo = torch.from_numpy(b_off).to(dev)
        at, bt = A.numel(), B.numel()
        nseg = len(a_off) - 1
        Ck = torch.empty(at + bt, dtype=torch.int32, device=dev)
        Cv = torch.empty(at + bt, dtype=torch.float32, device=dev)
        gC = torch.randn(at + bt, device=dev)
        gA = torch.empty(at, device=dev)
        gB = torch.empty(bt, device=dev)
        need = ctypes.c_size_t()
        _lib.check(lib.cr_batched_workspace_size(0, 4, nseg, at, bt, ctypes.byref(need)))
        ws = torch.empty(need.value, dtype=torch.uint8, device=dev)
        timer = KernelTimer(stream)
        for k in range(Wm + K):
            t = k >= Wm
            if t:
                timer.mark()
            _lib.check(lib.cr_batched_merge_kv(0, 4, nseg, ptr(ao), ptr(bo), ptr(A), ptr(Av), at,
                                               ptr(B), ptr(Bv), bt, ptr(Ck), ptr(Cv), ptr(ws),
                                               ws.numel(), sp))
            if t:
                timer.mark("fwd")
            _lib.check(lib.cr_batched_merge_kv_backward(0, 4, nseg, ptr(ao), ptr(bo), ptr(A), at,
                                                        ptr(B), bt, ptr(gC), ptr(gA), ptr(gB),
                                                        ptr(ws), ws.numel(), sp))
            if t:
                timer.mark("bwd")
                timer.marks.append((None, timer.marks[-1][1]))
        torch.cuda.synchronize()
        api.workspace_status(ws)
        tot = timer.totals()
        N = at + bt
        name = "batched_i32_f32" if nseg == 8192 else f"batched_i32_f32_{nseg}_pairs"
        return finish(tot, {"fwd": 16 * N, "bwd": 12 * N}, name, N,
                      {"segments": nseg, "note": "fwd/bwd include the segment scan and "
                       "partition launches (3 kernels each)"},
                      combos=[("int32+f32", 0, 4)])

    if args.workload == "merge_sort":
        # Both backward forms of the merge-sort chain: "record" (each forward
        # pass records its merge decisions, one bit per element, and the
        # backward routes gradients from them) and "recompute" (the backward
        # re-merges every pass's saved input keys).
        X, Xv = W.t_sort_u64_f32(device=dev, shift=args.shift)
        N = X.numel()
        gY = torch.randn(N, device=dev)
        # algorithmic bytes per element and stage: forward keys + payloads in
        # and out (+ one flag bit recorded by a pass, + the 2-byte chunk
        # permutation recorded by the shared-memory stage); backward gY in,
        # gX out (+ the flag bit or the permutation, or the pass's input keys
        # re-read)
        def stage_bytes(mode, kind):
            if kind == "block":
                return 26.0, 10.0
            return (24 + 1 / 8, 8 + 1 / 8) if mode == "record" else (24.0, 16.0)
        rows, per_pass, alg = {}, {}, {}
        for mode in ("record", "recompute"):
            plan = api.MergeSortPlan(N, 1024, X.dtype, Xv.dtype, dev, key_type="u64",
                                     graph=True, record=mode == "record")
            plan.forward(X, Xv)       # captures the forward graph
            plan.backward(gY)         # captures the backward graph
            timer = KernelTimer(stream)
            for k in range(Wm + K):
                t = k >= Wm
                plan.keys[0].copy_(X)
                plan.vals[0].copy_(Xv)
                plan.grads[plan.passes & 1].copy_(gY)
                if t:
                    timer.mark()
                plan._gf.replay()
                if t:
                    timer.mark("fwd_graph")
                plan._gb.replay()
                if t:
                    timer.mark("bwd_graph")
                    timer.marks.append((None, timer.marks[-1][1]))
            torch.cuda.synchronize()
            rows[mode] = timer.totals()
            alg[mode] = (sum(stage_bytes(mode, kd)[0] for kd, _ in plan.stages) * N,
                         sum(stage_bytes(mode, kd)[1] for kd, _ in plan.stages) * N)
            # per-stage breakdown: the same chain stage by stage outside the
            # graphs (partition + tile kernel, shared-memory stage, or routing)
            P = plan.passes
            plan.keys[0].copy_(X)
            plan.vals[0].copy_(Xv)
            plan.grads[P & 1].copy_(gY)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * P + 2)]
            for i in range(P):
                ev[i].record(stream)
                plan.run_stage(i)
            ev[P].record(stream)
            for i in reversed(range(P)):
                plan.run_stage_backward(i)
                ev[2 * P - i].record(stream)
            torch.cuda.synchronize()
            pp = []
            for i, (kind, w) in enumerate(plan.stages):
                f = ev[i].elapsed_time(ev[i + 1])
                b = ev[2 * P - i - 1].elapsed_time(ev[2 * P - i])
                fb, bb = stage_bytes(mode, kind)
                pp.append({"stage": kind, "width": w, "fwd_ms": round(f, 4), "bwd_ms": round(b, 4),
                           "fwd_gbs": round(fb * N / (f / 1e3) / 1e9, 1),
                           "bwd_gbs": round(bb * N / (b / 1e3) / 1e9, 1)})
            per_pass[mode] = pp
            del plan
            torch.cuda.empty_cache()
        # unsorted input: the recorded chain from runs of one element (its
        # shared-memory stage sorts every chunk of 4096, then HBM passes)
        Xu, Xuv = W.t_sort_u64_f32(device=dev, shift=args.shift, run=None)
        plan = api.MergeSortPlan(N, None, Xu.dtype, Xuv.dtype, dev, key_type="u64", graph=True)
        plan.forward(Xu, Xuv)
        plan.backward(gY)
        timer = KernelTimer(stream)
        for k in range(Wm + K):
            t = k >= Wm
            plan._load(Xu, Xuv)
            plan.grads[plan.passes & 1].copy_(gY)
            if t:
                timer.mark()
            plan._gf.replay()
            if t:
                timer.mark("fwd_graph")
            plan._gb.replay()
            if t:
                timer.mark("bwd_graph")
                timer.marks.append((None, timer.marks[-1][1]))
        torch.cuda.synchronize()
        un = {lb: round(ms / K, 4) for lb, ms in timer.totals().items()}
        stages_un = [f"{kd}:{w}" for kd, w in plan.stages]
        del plan
        torch.cuda.empty_cache()
        # the same from unsorted input in the recompute form: runs of 4096
        # formed by cr_sort_runs, backward by replaying it and re-merging
        plan = api.MergeSortPlan(N, None, Xu.dtype, Xuv.dtype, dev, key_type="u64", graph=True,
                                 record=False)
        plan.forward(Xu, Xuv)
        plan.backward(gY)
        timer = KernelTimer(stream)
        for k in range(Wm + K):
            t = k >= Wm
            plan._load(Xu, Xuv)
            plan.grads[plan.passes & 1].copy_(gY)
            if t:
                timer.mark()
            plan._gf.replay()
            if t:
                timer.mark("fwd_graph")
            plan._gb.replay()
            if t:
                timer.mark("bwd_graph")
                timer.marks.append((None, timer.marks[-1][1]))
        torch.cuda.synchronize()
        un_re = {lb: round(ms / K, 4) for lb, ms in timer.totals().items()}
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        Yk, Yv = torch.empty_like(Xu), torch.empty_like(Xuv)
        gXr = torch.empty_like(gY)
        perm = torch.empty(N, dtype=torch.int16, device=dev)
        for rep in range(3):
            ev[0].record(stream)
            api.sort_runs(Xu, Xuv, key_type="u64", out=(Yk, Yv))
            ev[1].record(stream)
            api.sort_runs_backward(Xu, gY, key_type="u64", out=gXr)
            ev[2].record(stream)
            api.sort_runs_record(Xu, Xuv, key_type="u64", out=(Yk, Yv), perm=perm)
            ev[3].record(stream)
            api.sort_runs_backward_recorded(perm, gY, out=gXr)
            ev[4].record(stream)
        torch.cuda.synchronize()
        tms = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]

        def row(ms, bpe):
            gbs = bpe * N / (ms / 1e3) / 1e9
            return {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
        # run formation alone (the recorded chain's first stage is
        # sort_runs_record's launch).  Bytes per element: keys + payloads in
        # and out; backward replay reads keys and gY, writes gX; the recorded
        # forms add / read the 2-byte permutation instead of the keys
        unsorted = {"stages": stages_un, "passes": len(stages_un),
                    "fwd_graph_ms": un["fwd_graph"], "bwd_graph_ms": un["bwd_graph"],
                    "elements_per_s": N / ((un["fwd_graph"] + un["bwd_graph"]) / 1e3),
                    "recompute": {"fwd_graph_ms": un_re["fwd_graph"],
                                  "bwd_graph_ms": un_re["bwd_graph"],
                                  "elements_per_s":
                                      N / ((un_re["fwd_graph"] + un_re["bwd_graph"]) / 1e3)},
                    "sort_runs_run": api.sort_run_length(),
                    "sort_runs": row(tms[0], 24), "sort_runs_backward": row(tms[1], 16),
                    "sort_runs_record": row(tms[2], 26),
                    "sort_runs_backward_recorded": row(tms[3], 10)}
        del plan, Xu, Xuv, Yk, Yv, gXr, perm
        torch.cuda.empty_cache()
        P = len(per_pass["record"])
        rec = rows["record"]
        extra = {"stages": P, "backward": "record",
                 "recompute": {}, "unsorted_input": unsorted, "per_pass": per_pass,
                 "note": "each graph replays its stages' launches (the recorded form merges "
                         "widths below 4096 in one shared-memory stage); bytes are summed over "
                         "stages; value and the kernels rows are the recorded form"}
        for label, ms in rows["recompute"].items():
            b = alg["recompute"][0 if label == "fwd_graph" else 1]
            gbs = b / (ms / K / 1e3) / 1e9
            extra["recompute"][label] = {"ms": round(ms / K, 4), "gbs": round(gbs, 1),
                                         "frac": round(gbs / peak, 4)}
        return finish(rec, {"fwd_graph": int(alg["record"][0]),
                            "bwd_graph": int(alg["record"][1])}, "sort_u64_f32", N,
                      extra, combos=[("uint64+f32", 3, 4)])
    raise ValueError(args.workload)


# ---------------------------------------------------------------------------
# CPU oracle as a baseline / the reference arm
# ---------------------------------------------------------------------------
def _host_inputs(merges):
    out = []
    for mg in merges:
        dt = np.uint64 if mg["kt"] == "u64" else np.int32
        out.append((mg["name"], mg["A"].cpu().numpy().view(dt), mg["B"].cpu().numpy().view(dt)))
    return out


def time_oracle(host_inputs, threads: int):
    import oracle
    t0 = time.perf_counter()
    n = 0
    for _, a, b in host_inputs:
        oracle.parallel_merge(a, b, threads)
        n += len(a) + len(b)
    dt = time.perf_counter() - t0
    return n / dt, dt


def cpu_baseline_from(merges):
    """The oracle's Algorithm 2 on all host cores over full steps of the same
    inputs: one warm-up step, then steps until about 10 core-seconds of work
    (at most 20); elements over the summed step times."""
    hi = _host_inputs(merges)
    cores = os.cpu_count() or 1
    elems = sum(len(a) + len(b) for _, a, b in hi)
    time_oracle(hi, cores)
    total, reps = 0.0, 0
    while reps < 20 and (reps == 0 or total * cores < 10.0):
        _, secs = time_oracle(hi, cores)
        total += secs
        reps += 1
    return {"value": reps * elems / total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} full steps (all three merges, {elems} elements each) on the CPU "
                      f"oracle's Algorithm 2 with {cores} POSIX threads after one warm-up "
                      f"step; {total:.2f} s wall, about {total * cores:.0f} core-seconds"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import torch
    import oracle
    oracle.build()
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    # Each reference step merges the same three full-size workloads (the
    # oracle's Algorithm 2 takes about 0.2 s per step on 16 cores, so K + W
    # steps finish well within minutes).
    merges = make_inputs(dev, args.shift)
    elems = sum(mg["m"] + mg["n"] for mg in merges)
    hi = _host_inputs(merges)
    del merges
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        time_oracle(hi, cores)
    total, n = 0.0, 0
    for _ in range(args.steps):
        v, dt = time_oracle(hi, cores)
        total += dt
        n += sum(len(a) + len(b) for _, a, b in hi)
    value = n / total
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32+uint64 keys",
            "data": "synthetic (seeded, sorted; device-generated)", "impl": "reference",
            "config": {"workload": WORKLOAD, "merges": [m[0] for m in MERGES],
                       "elements_per_step": elems, "l2": "inputs larger than L2 (no flush)",
                       "size_shift": args.shift, "parallelism": f"replicas x{world}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full steps (the three merges, {elems} "
                                       "elements each step) of the CPU oracle's Algorithm 2 "
                                       f"on {cores} POSIX threads after {args.warmup} "
                                       "warm-up steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    rank, world, local, dist = dist_setup(args.gpus)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload != WORKLOAD:
        line = run_row(args) if rank == 0 else None
    else:
        line = run_ours(args, rank, world, local, dist)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
