"""B300-native SM-based SPARQL BGP join (arXiv 1807.07691).

The compute path is libgsmat.so (CUDA for sm_103a, C ABI in
include/gsmat.h); ``gsmat`` is its ctypes binding.  Build the library with
``python -m paper_1807_07691_b300.build``.
"""

from .gsmat import (  # noqa: F401
    COUNT_ONLY,
    PLAN_ORDER,
    SORTED,
    GsmatError,
    Store,
    Table,
    exclusive_scan_i32,
    header_functions,
    lib,
    plan,
    profile_enable,
    profile_read,
    radix_sort_u64,
    use_torch_allocator,
)
