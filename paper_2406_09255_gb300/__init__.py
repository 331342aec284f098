"""Compact parallel hash tables for GB300 (sm_103a).

Batched lockless insert, find and find-or-put on compact (quotiented)
bucketed cuckoo and two-level iceberg hash tables, after Hegeman et al.,
"Compact Parallel Hash Tables on the GPU". The compute path is the C-ABI
library libcht.so (include/cht.h); this package is its Python binding.
"""
from ._lib import (CUCKOO, ERROR, FOUND, FULL, ICEBERG, INVALID, NOT_FOUND, PUT,  # noqa: F401
                   ChtError)
from .table import Table, resolve_config, table_bytes  # noqa: F401
from .kv import KVMap  # noqa: F401
