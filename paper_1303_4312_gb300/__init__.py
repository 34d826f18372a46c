"""GB300 (sm_103a) co-rank and perfectly load-balanced stable merge.

Implements Siebert & Traeff, "Perfectly load-balanced, optimal, stable,
parallel merge": Algorithm 1 (co_rank) and Algorithm 2 (parallel stable
merge with equal output blocks), as CUDA kernels behind the C ABI declared in
``include/corank.h`` (``lib/libcorank.so``).

Importing this package does not load the library; the first call does, and
fails loudly if it has not been built.  ``workloads`` (seeded synthetic
inputs) needs neither the library nor a GPU.
"""
from importlib import import_module

__all__ = [
    "co_rank", "co_rank_many", "merge", "merge_kv", "merge_kv_backward", "MergeKV",
    "merge_kv_autograd", "batched_merge_kv", "batched_merge_kv_backward", "merge_pass",
    "merge_pass_backward", "workspace_status", "tile_size", "CorankError", "merge_sort",
    "MergeSortPlan", "MergeMany", "merge_many", "HostMerger", "sort_runs", "sort_runs_backward",
    "sort_run_length", "PassRecord", "merge_pass_record", "merge_pass_backward_recorded",
    "merge_pass_record_bytes", "sort_runs_record", "sort_runs_backward_recorded",
    "check_sorted", "merge_runs_block", "merge_runs_block_backward_recorded",
    "merge_runs_block_length", "merge_workspace_bytes", "merge_pass_workspace_bytes",
    "new_pass_record", "BatchedMergeGraph", "co_rank_async", "DistCoRank", "host_empty",
]


_SUBMODULES = ("api", "shard", "workloads", "autotune", "build", "_lib")


def __getattr__(name):
    if name == "CorankError":
        return import_module("._lib", __name__).CorankError
    if name in _SUBMODULES:
        return import_module("." + name, __name__)
    if name in __all__:
        return getattr(import_module(".api", __name__), name)
    raise AttributeError(name)
