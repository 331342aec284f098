"""Key-value map over an iceberg table: values live in a device array indexed
by the stable slot of their key (iceberg entries never move once placed). A
put is a find-or-put whose answering lane also writes the value to the key's
slot, and a get is a lookup whose answering lane reads it: one kernel each
(cht_kv_put / cht_kv_get)."""
from __future__ import annotations

import torch

from . import _lib
from .table import Table, _stream_handle

_VALUE_BYTES = {torch.int32: 4, torch.float32: 4, torch.int64: 8, torch.float64: 8}


class KVMap:
    def __init__(self, table: Table, value_dtype=torch.int64):
        if table.cfg.kind != 1:
            raise ValueError("a key-value map needs an iceberg table (stable slots)")
        if value_dtype not in _VALUE_BYTES:
            raise ValueError(f"value dtype must be one of {list(_VALUE_BYTES)}")
        self.table = table
        self.value_bytes = _VALUE_BYTES[value_dtype]
        self.values = torch.zeros(table.slots, dtype=value_dtype, device=table.device)
        self._L = _lib.load()

    def put(self, keys: torch.Tensor, values: torch.Tensor, status=None, stream=None):
        """Insert or assign, in one kernel (cht_kv_put). Returns the status
        per key. A key given twice in one call keeps one of its values, which
        one is unspecified. FULL keys store nothing. A get on another stream
        that overlaps this put may find a key before its value is written
        (it then reads the slot's previous value); order them on one stream."""
        if values.dtype != self.values.dtype or values.numel() != keys.numel():
            raise ValueError("one value of the map's dtype per key")
        keys, status = self.table._prep(keys, status)
        values = values.contiguous()
        _lib.check(self._L.cht_kv_put(self.table._h, keys.data_ptr(), keys.numel(),
                                      values.data_ptr(), self.value_bytes, self.values.data_ptr(),
                                      self.values.numel(), status.data_ptr(),
                                      _stream_handle(stream)))
        return status

    def get(self, keys: torch.Tensor, status=None, out=None, stream=None):
        """Values by key, in one kernel (cht_kv_get). Returns (values, status):
        zero values for keys not found."""
        keys, status = self.table._prep(keys, status)
        if out is None:
            out = torch.empty(keys.numel(), dtype=self.values.dtype, device=self.table.device)
        _lib.check(self._L.cht_kv_get(self.table._h, keys.data_ptr(), keys.numel(),
                                      self.values.data_ptr(), self.value_bytes,
                                      self.values.numel(), out.data_ptr(), status.data_ptr(),
                                      _stream_handle(stream)))
        return out, status
