"""ctypes binding of libcorank.so (include/corank.h).

Argument marshalling only: every step of the merge path runs inside the
library's CUDA kernels.  If the library is missing this module raises; there
is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcorank.so")

_lock = threading.RLock()
_lib = None

P = ctypes.c_void_p
I64 = ctypes.c_int64
INT = ctypes.c_int
SZ = ctypes.c_size_t

# name -> (argtypes, restype); mirrors include/corank.h
SIGNATURES = {
    "cr_status_string": ([INT], ctypes.c_char_p),
    "cr_last_error": ([], ctypes.c_char_p),
    "cr_abi_version": ([], INT),
    "cr_tile_size": ([INT, INT], I64),
    "cr_tile_shape_count": ([], INT),
    "cr_tile_shape_info": ([INT, ctypes.POINTER(INT), ctypes.POINTER(INT),
                            ctypes.POINTER(INT)], INT),
    "cr_set_tile_shape": ([INT, INT, INT], INT),
    "cr_get_tile_shape": ([INT, INT], INT),
    "cr_set_tile_shape_for": ([INT, INT, INT, INT], INT),
    "cr_get_tile_shape_for": ([INT, INT, INT], INT),
    "cr_tile_size_for": ([INT, INT, I64, I64], I64),
    "cr_tile_size_class": ([INT, INT, INT], I64),
    "cr_co_rank": ([INT, P, I64, P, I64, I64, ctypes.POINTER(I64), ctypes.POINTER(I64), P], INT),
    "cr_co_rank_async": ([INT, P, I64, P, I64, I64, P, P], INT),
    "cr_co_rank_many": ([INT, P, I64, P, I64, P, I64, P, P, P], INT),
    "cr_merge_workspace_size": ([INT, INT, I64, I64, ctypes.POINTER(SZ)], INT),
    "cr_stable_merge": ([INT, P, I64, P, I64, P, P, P, SZ, P], INT),
    "cr_stable_merge_kv": ([INT, INT, P, P, I64, P, P, I64, P, P, P, P, SZ, P], INT),
    "cr_stable_merge_kv_backward": ([INT, INT, P, I64, P, I64, P, P, P, P, SZ, P], INT),
    "cr_merge_partition": ([INT, INT, P, I64, P, I64, P, SZ, P], INT),
    "cr_merge_partition_alg2": ([INT, INT, P, I64, P, I64, P, SZ, P], INT),
    "cr_merge_tiles": ([INT, INT, P, P, I64, P, P, I64, P, P, P, P, SZ, P], INT),
    "cr_merge_tiles_backward": ([INT, INT, P, I64, P, I64, P, P, P, P, SZ, P], INT),
    "cr_batched_workspace_size": ([INT, INT, I64, I64, I64, ctypes.POINTER(SZ)], INT),
    "cr_batched_merge_kv": ([INT, INT, I64, P, P, P, P, I64, P, P, I64, P, P, P, SZ, P], INT),
    "cr_batched_merge_kv_backward": ([INT, INT, I64, P, P, P, I64, P, I64, P, P, P, P, SZ, P],
                                     INT),
    "cr_merge_pass_workspace_size": ([INT, INT, I64, I64, ctypes.POINTER(SZ)], INT),
    "cr_merge_pass": ([INT, INT, P, P, I64, I64, P, P, P, SZ, P], INT),
    "cr_merge_pass_backward": ([INT, INT, P, I64, I64, P, P, P, SZ, P], INT),
    "cr_merge_pass_record_size": ([INT, INT, I64, I64, ctypes.POINTER(SZ), ctypes.POINTER(SZ)],
                                  INT),
    "cr_merge_pass_record": ([INT, INT, P, P, I64, I64, P, P, P, SZ, P, SZ, P], INT),
    "cr_merge_pass_backward_recorded": ([INT, INT, I64, I64, P, SZ, P, P, P, SZ, P], INT),
    "cr_workspace_status": ([P, P], INT),
    "cr_selftest_bounded_wait": ([P, SZ, ctypes.c_uint64, P, P], INT),
    "cr_check_sorted": ([INT, P, I64, P, P, SZ, P], INT),
    "cr_merge_runs_block_length": ([], I64),
    "cr_merge_runs_block": ([INT, INT, P, P, I64, I64, P, P, P, P], INT),
    "cr_merge_runs_block_backward_recorded": ([INT, I64, P, P, P, P], INT),
    "cr_sort_run_length": ([], I64),
    "cr_sort_runs": ([INT, INT, P, P, I64, P, P, P], INT),
    "cr_sort_runs_record": ([INT, INT, P, P, I64, P, P, P, P], INT),
    "cr_sort_runs_backward_recorded": ([INT, I64, P, P, P, P], INT),
    "cr_sort_runs_backward": ([INT, INT, P, I64, P, P, P], INT),
    "cr_stable_merge_noalloc": ([INT, P, I64, P, I64, P, P, P], INT),
    "cr_dist_co_rank_init": ([I64, I64, P, I64, P, P], INT),
    "cr_dist_co_rank_probes": ([I64, I64, P, I64, P, P, P], INT),
    "cr_dist_co_rank_answer": ([INT, P, I64, I64, P, I64, P, P], INT),
    "cr_dist_co_rank_step": ([INT, I64, I64, P, P, P, I64, P], INT),
    "cr_dist_co_rank_result": ([P, I64, P, P, P, P], INT),
}

STATUS = {0: "CR_OK", 1: "CR_EINVAL", 2: "CR_EALIAS", 3: "CR_EALIGN", 4: "CR_ENOSPACE",
          5: "CR_ECUDA", 6: "CR_ETIMEOUT", 7: "CR_EUNSUPPORTED", 8: "CR_EINTERNAL",
          9: "CR_EBADSEG"}

KEY_TYPES = {"i32": 0, "u32": 1, "i64": 2, "u64": 3, "f32": 4, "f64": 5, "pair_u32": 6,
             "pair_i32": 7}
KEY_DESC = 256       # flag: descending order


def key_code(key_type) -> int:
    """C-ABI key type of a name: "i32", "u32", "i64", "u64", "f32", "f64"
    (floats in IEEE-754 totalOrder), "pair_u32", "pair_i32" (lexicographic
    (major, minor) pairs in one 64-bit word, major in the high half), with
    ":desc" for descending order, or an int code passed through."""
    if isinstance(key_type, int):
        return key_type
    base, _, mod = str(key_type).partition(":")
    if base not in KEY_TYPES or mod not in ("", "desc", "asc"):
        raise ValueError(f"key_type must be one of {sorted(KEY_TYPES)}, optionally with ':desc'")
    return KEY_TYPES[base] | (KEY_DESC if mod == "desc" else 0)


def key_bytes(key_type) -> int:
    code = key_code(key_type) & ~KEY_DESC
    return 4 if code in (0, 1, 4) else 8


class CorankError(RuntimeError):
    """A libcorank call returned a status other than CR_OK."""

    def __init__(self, status: int, detail: str):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{self.name}: {detail}")


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libcorank.so (built by ``paper_1303_4312_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"libcorank.so not found at {p}: build it first with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(p)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
            # select the tile shapes tuned for this GPU, when a table exists
            from . import autotune
            autotune.apply(lib)
    return _lib


def check(status: int) -> None:
    if status != 0:
        detail = load().cr_last_error().decode(errors="replace")
        raise CorankError(status, detail)
