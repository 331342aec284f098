"""Fused multi-table batches: one persistent launch over many iceberg tables,
optionally captured once in a CUDA graph and replayed (binding of the
cht_batch_* entry points; argument marshalling only)."""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import Config, check
from .table import Table, _stream_handle

OP_FIND_OR_PUT = 0
OP_FIND = 1


class Batch:
    """One operation over many (table, keys) pairs in a single kernel launch.

    tables: list of iceberg Table objects (same primary packing; a table may
    repeat only in a lookup batch);
    keys: list of device key tensors (each of its table's key dtype);
    statuses: optional list of uint8 device tensors (allocated if omitted).
    The descriptor scratch is a device tensor owned by this object.
    """

    def __init__(self, tables, keys, statuses=None, op: int = OP_FIND_OR_PUT, stream=None):
        self._L = _lib.load()
        self.op = op
        assert len(tables) == len(keys) and len(tables) > 0
        self.tables = list(tables)
        self.keys = [k.contiguous() for k in keys]
        for t, k in zip(self.tables, self.keys):
            if k.dtype != t.key_dtype or k.device != t.device:
                raise ValueError("keys must match their table's key dtype and device")
        if statuses is None:
            statuses = [torch.empty(k.numel(), dtype=torch.uint8, device=k.device)
                        for k in self.keys]
        self.statuses = statuses
        self._create([k.data_ptr() for k in self.keys], [k.numel() for k in self.keys],
                     [s.data_ptr() for s in self.statuses], stream)

    @classmethod
    def from_pointers(cls, tables, key_ptrs, counts, status_ptrs, op: int = OP_FIND_OR_PUT,
                      stream=None):
        """A batch over raw device addresses (key_ptrs[i]: counts[i] keys of
        tables[i]'s key dtype; status_ptrs[i]: counts[i] bytes), for callers
        that place many requests in one device buffer. The caller keeps that
        memory alive while the batch is used; keys and statuses are not
        held."""
        b = cls.__new__(cls)
        b._L = _lib.load()
        b.op = op
        b.tables = list(tables)
        b.keys = b.statuses = None
        b._create(list(key_ptrs), list(counts), list(status_ptrs), stream)
        return b

    def _create(self, key_ptrs, counts, status_ptrs, stream):
        count = len(self.tables)
        nbytes = int(self._L.cht_batch_scratch_bytes(count))
        if nbytes == 0:
            raise ValueError(f"unsupported batch size {count}")
        self.scratch = torch.empty(nbytes, dtype=torch.uint8, device=self.tables[0].device)
        vp = ctypes.c_void_p
        T = (vp * count)(*[t.handle for t in self.tables])
        K = (vp * count)(*key_ptrs)
        N = (ctypes.c_size_t * count)(*counts)
        S = (vp * count)(*status_ptrs)
        self._h = vp()
        check(self._L.cht_batch_create(T, K, N, S, count, self.op, self.scratch.data_ptr(),
                                       nbytes, _stream_handle(stream), ctypes.byref(self._h)))
        self.n_keys = sum(counts)

    def set_launch(self, tile=0, items_per_thread=0, cta_threads=0, max_ctas=0):
        c = Config()
        c.tile, c.items_per_thread, c.cta_threads, c.max_ctas = (tile, items_per_thread,
                                                                  cta_threads, max_ctas)
        check(self._L.cht_batch_set_launch(self._h, ctypes.byref(c)))

    def launch(self, stream=None):
        check(self._L.cht_batch_launch(self._h, _stream_handle(stream)))
        return self.statuses

    def capture(self, stream=None):
        check(self._L.cht_batch_capture(self._h, _stream_handle(stream)))

    def replay(self, stream=None):
        check(self._L.cht_batch_replay(self._h, _stream_handle(stream)))
        return self.statuses

    def clear(self, stream=None):
        """Empty every table of the batch (one launch)."""
        check(self._L.cht_batch_clear(self._h, _stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.cht_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def per_table(tables, keys, statuses, op: int = OP_FIND_OR_PUT, stream=None):
    """The unfused baseline: one launch per table."""
    for t, k, s in zip(tables, keys, statuses):
        if op == OP_FIND_OR_PUT:
            t.find_or_put(k, status=s, stream=stream)
        else:
            t.find(k, status=s, stream=stream)
    return statuses
