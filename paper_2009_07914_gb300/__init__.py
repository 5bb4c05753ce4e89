"""GB300-native bulk GPU hash tables after WarpCore (arXiv 2009.07914).

The compute path is libwc.so (hand-written CUDA for sm_103a behind the C ABI of
include/wc.h).  `api` exposes one Python function per C entry point; `table` wraps a
table handle in an object.  Nothing here computes on the CPU.
"""
from . import api
from ._binding import (WC_FLAG_COUNT_OVERFLOW, WC_FLAG_DUPLICATE_KEY, WC_FLAG_INVALID_KEY, WC_FLAG_POOL_EXHAUSTED,
                       WC_FLAG_PROBE_LIMIT, WC_FLAG_QUEUE_TIMEOUT, WC_MULTI_VALUE, WC_OP_COUNT, WC_OP_ERASE,
                       WC_OP_INSERT, WC_OP_RETRIEVE, WC_SCHEME_AUTO, WC_SCHEME_BLOCKED, WC_SCHEME_DEDUP, WC_SCHEME_DIRECT,
                       WC_SINGLE_VALUE, WC_MULTI_VALUE_OA, WC_OPT_OVERFLOW_BITS, WC_OPT_SOA, WC_HASH_SET, WC_COUNTING,
                       WC_BLOOM_FILTER, WcError, lib)
from .api import *  # noqa: F401,F403  (the C-ABI names)
from .table import (BloomFilterTable, CountingTable, HashSetTable, MultiValueOATable, MultiValueTable,
                    SingleValueTable)

__all__ = ["api", "lib", "WcError", "SingleValueTable", "MultiValueTable", "MultiValueOATable", "CountingTable",
           "HashSetTable", "BloomFilterTable"] + list(api.__all__)
