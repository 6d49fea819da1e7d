"""B300-native SM-based SPARQL BGP join (arXiv 1807.07691).

The compute path is libgsmat.so (CUDA for sm_103a, C ABI in
include/gsmat.h); ``gsmat`` is its ctypes binding.  Build the library with
``python -m paper_1807_07691_b300.build``.  The library is loaded on first
use of any binding name (so the build module imports without it); a missing
library raises ImportError then.
"""

_BINDING_NAMES = {
    "COUNT_ONLY", "NO_INTERSECT", "PLAN_COST", "PLAN_COST_MAX", "PLAN_ORDER", "SORTED", "GsmatError", "Store",
    "Table", "Batch", "batch_autotune",
    "Server", "exclusive_scan_i32", "exclusive_scan_i32_noalloc", "exclusive_scan_i32_noalloc_max",
    "header_functions", "launch_count", "lib", "plan", "profile_enable", "profile_read", "radix_sort_u64", "sort_rows",
    "SORT_CARRY", "SORT_GATHER", "use_torch_allocator", "Dictionary", "Sparql",
    "merge_tables", "gather_rows", "gather_shards",
}


def __getattr__(name):
    if name in _BINDING_NAMES:
        from . import gsmat

        return getattr(gsmat, name)
    raise AttributeError(name)


def __dir__():
    return sorted(_BINDING_NAMES | {"build", "gsmat"})
