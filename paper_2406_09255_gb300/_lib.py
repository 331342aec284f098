"""ctypes declarations for libcht.so (include/cht.h).

The library is built in-tree by paper_2406_09255_gb300/build.py. Loading
fails loudly when it is missing: there is no CPU or PyTorch fallback for any
table operation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcht.so")

CHT_OK, CHT_ERR_INVALID, CHT_ERR_UNSUPPORTED, CHT_ERR_CUDA, CHT_ERR_CAPACITY, CHT_ERR_TIMEOUT = range(6)
NOT_FOUND, FOUND, PUT, FULL, INVALID, ERROR = range(6)
CUCKOO, ICEBERG = 0, 1
HEADER_BYTES = 256
BUCKET_BYTES = 128


class Config(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("compact", ctypes.c_int32),
        ("key_bits", ctypes.c_int32),
        ("key_bytes", ctypes.c_int32),
        ("num_buckets", ctypes.c_uint64),
        ("num_buckets_backyard", ctypes.c_uint64),
        ("fields_per_word", ctypes.c_int32),
        ("fields_per_word_backyard", ctypes.c_int32),
        ("num_hashes", ctypes.c_int32),
        ("max_chain", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("tile", ctypes.c_int32),
        ("items_per_thread", ctypes.c_int32),
        ("cta_threads", ctypes.c_int32),
        ("max_ctas", ctypes.c_int32),
        ("max_tiles", ctypes.c_int32),
        ("lookups_in_flight", ctypes.c_int32),
        ("retry_limit", ctypes.c_int32),
        ("stash_slots", ctypes.c_int32),
        ("bucket_words", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Counters(ctypes.Structure):
    _fields_ = [("probes", ctypes.c_uint64), ("writes", ctypes.c_uint64),
                ("cas_fail", ctypes.c_uint64), ("ops", ctypes.c_uint64)]


# every entry point declared in include/cht.h: name -> (restype, argtypes)
_vp, _sz, _u64p = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)
_cfgp = ctypes.POINTER(Config)
SIGNATURES = {
    "cht_resolve_config": (ctypes.c_int, [_cfgp, _cfgp]),
    "cht_table_bytes": (ctypes.c_size_t, [_cfgp]),
    "cht_create": (ctypes.c_int, [_cfgp, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "cht_destroy": (ctypes.c_int, [_vp]),
    "cht_clear": (ctypes.c_int, [_vp, _vp]),
    "cht_get_config": (ctypes.c_int, [_vp, _cfgp]),
    "cht_set_launch": (ctypes.c_int, [_vp, _cfgp]),
    "cht_insert": (ctypes.c_int, [_vp, _vp, _sz, _vp, _vp, _vp]),
    "cht_find": (ctypes.c_int, [_vp, _vp, _sz, _vp, _vp]),
    "cht_find_or_put": (ctypes.c_int, [_vp, _vp, _sz, _vp, _vp]),
    "cht_enumerate": (ctypes.c_int, [_vp, _vp, _sz, _vp, _vp]),
    "cht_set_counters": (ctypes.c_int, [_vp, _vp]),
    "cht_error_flags": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint32), _vp]),
    "cht_batch_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "cht_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                        ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_vp),
                                        ctypes.c_int, ctypes.c_int, _vp, _sz, _vp,
                                        ctypes.POINTER(_vp)]),
    "cht_batch_set_launch": (ctypes.c_int, [_vp, _cfgp]),
    "cht_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "cht_batch_capture": (ctypes.c_int, [_vp, _vp]),
    "cht_batch_replay": (ctypes.c_int, [_vp, _vp]),
    "cht_batch_clear": (ctypes.c_int, [_vp, _vp]),
    "cht_batch_destroy": (ctypes.c_int, [_vp]),
    "cht_batch_find_or_put_static": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                                    ctypes.POINTER(ctypes.c_size_t),
                                                    ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "cht_last_error": (ctypes.c_char_p, []),
    "cht_version": (ctypes.c_char_p, []),
    "cht_random_read": (ctypes.c_int, [_vp, _sz, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                       _vp, _vp]),
    "cht_random_claim": (ctypes.c_int, [_vp, _sz, ctypes.c_uint64, ctypes.c_uint64, _vp, _vp]),
    "cht_find_or_put_slots": (ctypes.c_int, [_vp, _vp, _sz, _vp, _vp, _vp]),
    "cht_find_slots": (ctypes.c_int, [_vp, _vp, _sz, _vp, _vp, _vp]),
    "cht_values_scatter": (ctypes.c_int, [_vp, _sz, _vp, ctypes.c_int, _vp, ctypes.c_uint64, _vp]),
    "cht_values_gather": (ctypes.c_int, [_vp, _sz, _vp, ctypes.c_int, ctypes.c_uint64, _vp, _vp]),
    "cht_kv_put": (ctypes.c_int, [_vp, _vp, _sz, _vp, ctypes.c_int, _vp, ctypes.c_uint64, _vp,
                                  _vp]),
    "cht_kv_get": (ctypes.c_int, [_vp, _vp, _sz, _vp, ctypes.c_int, ctypes.c_uint64, _vp, _vp,
                                  _vp]),
}

_lock = threading.Lock()
_lib = None


class ChtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"cht error {code}: {msg}")
        self.code = code


def load() -> ctypes.CDLL:
    """Load libcht.so (built in-tree); raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` "
                    "(there is no fallback implementation)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(code: int) -> None:
    if code != CHT_OK:
        raise ChtError(code, load().cht_last_error().decode())
