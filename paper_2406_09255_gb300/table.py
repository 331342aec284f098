"""Python binding of the C-ABI table: argument marshalling only.

PyTorch supplies device memory (the table storage, key and status tensors)
and streams; every table operation runs in libcht.so's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import CUCKOO, ICEBERG, Config, Counters, check

__all__ = ["Table", "CUCKOO", "ICEBERG", "resolve_config", "table_bytes"]


def _make_config(kind, key_bits, num_buckets, num_buckets_backyard=0, *, compact=True,
                 key_bytes=8, fields_per_word=0, fields_per_word_backyard=0, num_hashes=0,
                 max_chain=0, seed=0, tile=0, items_per_thread=0, cta_threads=0, max_ctas=0,
                 max_tiles=0, lookups_in_flight=0, retry_limit=0, stash_slots=0,
                 bucket_words=0) -> Config:
    c = Config()
    c.kind, c.compact, c.key_bits, c.key_bytes = kind, int(compact), key_bits, key_bytes
    c.num_buckets, c.num_buckets_backyard = num_buckets, num_buckets_backyard
    c.fields_per_word, c.fields_per_word_backyard = fields_per_word, fields_per_word_backyard
    c.num_hashes, c.max_chain = num_hashes, max_chain
    c.seed = seed & 0xFFFFFFFFFFFFFFFF
    c.tile, c.items_per_thread, c.cta_threads = tile, items_per_thread, cta_threads
    c.max_ctas, c.max_tiles = max_ctas, max_tiles
    c.lookups_in_flight = lookups_in_flight
    c.retry_limit = retry_limit
    c.stash_slots = stash_slots
    c.bucket_words = bucket_words
    return c


def resolve_config(*args, **kw) -> Config:
    """The configuration with defaults filled in; raises ChtError if invalid."""
    c = _make_config(*args, **kw)
    out = Config()
    check(_lib.load().cht_resolve_config(ctypes.byref(c), ctypes.byref(out)))
    return out


def table_bytes(*args, **kw) -> int:
    c = _make_config(*args, **kw)
    return int(_lib.load().cht_table_bytes(ctypes.byref(c)))


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _key_dtype(key_bytes: int):
    return torch.int64 if key_bytes == 8 else torch.int32


class Table:
    """A compact (or whole-key) cuckoo or iceberg table in device memory.

    Same arguments as cht_config (include/cht.h). The storage is a uint8
    torch tensor on `device` owned by this object.
    """

    def __init__(self, kind, key_bits, num_buckets, num_buckets_backyard=0, *, device=None,
                 stream=None, **kw):
        self._L = _lib.load()
        self.requested = _make_config(kind, key_bits, num_buckets, num_buckets_backyard, **kw)
        self.cfg = Config()
        check(self._L.cht_resolve_config(ctypes.byref(self.requested), ctypes.byref(self.cfg)))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = int(self._L.cht_table_bytes(ctypes.byref(self.cfg)))
        self.storage = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self._L.cht_create(ctypes.byref(self.cfg), self.storage.data_ptr(), nbytes,
                                     _stream_handle(stream), ctypes.byref(self._h)))
        self.counters = None

    # -- lifecycle ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.cht_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    @property
    def key_dtype(self):
        return _key_dtype(self.cfg.key_bytes)

    @property
    def slots(self) -> int:
        c = self.cfg
        wpb = c.bucket_words
        n = c.num_buckets * wpb * c.fields_per_word
        if c.kind == ICEBERG:
            n += c.num_buckets_backyard * wpb * c.fields_per_word_backyard + c.stash_slots
        return n

    def clear(self, stream=None):
        check(self._L.cht_clear(self._h, _stream_handle(stream)))

    def set_launch(self, tile=0, items_per_thread=0, cta_threads=0, max_ctas=0, max_tiles=0,
                   lookups_in_flight=0):
        """Change the launch shape of later calls (contents stay)."""
        c = Config()
        c.tile, c.items_per_thread, c.cta_threads = tile, items_per_thread, cta_threads
        c.max_ctas, c.max_tiles, c.lookups_in_flight = max_ctas, max_tiles, lookups_in_flight
        check(self._L.cht_set_launch(self._h, ctypes.byref(c)))
        check(self._L.cht_get_config(self._h, ctypes.byref(self.cfg)))

    # -- operations -----------------------------------------------------------
    def _prep(self, keys: torch.Tensor, out):
        """Keys on the table's device, or in page-locked host memory: the
        kernels then read them (and write the statuses, which must be
        page-locked host memory too) directly over the CPU-GPU link. As with
        device outputs, host outputs are valid once the stream has been
        synchronised."""
        host = keys.device.type == "cpu"
        if host and not keys.is_pinned():
            raise ValueError("host keys must be in page-locked memory (pin_memory())")
        if not host and keys.device != self.device:
            raise ValueError(f"keys must be on {self.device} or pinned host memory "
                             f"(got {keys.device})")
        if keys.dtype != self.key_dtype:
            raise ValueError(f"keys must be {self.key_dtype} for {self.cfg.key_bytes}-byte keys")
        if not keys.is_contiguous():
            if host:
                raise ValueError("pinned host keys must be contiguous")
            keys = keys.contiguous()
        if out is None:
            out = (torch.empty(keys.numel(), dtype=torch.uint8, pin_memory=True) if host
                   else torch.empty(keys.numel(), dtype=torch.uint8, device=self.device))
        elif host != (out.device.type == "cpu") or (host and not out.is_pinned()):
            raise ValueError("statuses must live where the keys live (device or pinned host)")
        return keys, out

    def insert(self, keys: torch.Tensor, status=None, dropped=None, stream=None):
        """Insert keys. Returns the status tensor (uint8). For cuckoo tables
        pass a `dropped` int64 tensor to receive dropped keys of FULL puts."""
        keys, status = self._prep(keys, status)
        dp = dropped.data_ptr() if dropped is not None else None
        check(self._L.cht_insert(self._h, keys.data_ptr(), keys.numel(), status.data_ptr(), dp,
                                 _stream_handle(stream)))
        return status

    def _slots(self, n: int, slots):
        if slots is None or slots is True:
            return torch.empty(n, dtype=torch.int64, device=self.device)
        if slots.dtype != torch.int64 or slots.device != self.device or slots.numel() < n:
            raise ValueError("slots must be an int64 tensor on the table's device")
        return slots

    def find(self, keys: torch.Tensor, status=None, stream=None, slots=None):
        """Lookups. With slots (True, or an int64 tensor to fill) on an iceberg
        table, also returns each found key's slot (-1 when not found)."""
        keys, status = self._prep(keys, status)
        if slots is None or slots is False:
            check(self._L.cht_find(self._h, keys.data_ptr(), keys.numel(), status.data_ptr(),
                                   _stream_handle(stream)))
            return status
        slots = self._slots(keys.numel(), slots)
        check(self._L.cht_find_slots(self._h, keys.data_ptr(), keys.numel(), status.data_ptr(),
                                     slots.data_ptr(), _stream_handle(stream)))
        return status, slots

    def find_or_put(self, keys: torch.Tensor, status=None, stream=None, slots=None):
        """Find-or-put (iceberg). With slots (True, or an int64 tensor to fill),
        also returns the slot of each FOUND / PUT key (-1 otherwise): a handle
        that stays valid until clear()."""
        keys, status = self._prep(keys, status)
        if slots is None or slots is False:
            check(self._L.cht_find_or_put(self._h, keys.data_ptr(), keys.numel(),
                                          status.data_ptr(), _stream_handle(stream)))
            return status
        slots = self._slots(keys.numel(), slots)
        check(self._L.cht_find_or_put_slots(self._h, keys.data_ptr(), keys.numel(),
                                            status.data_ptr(), slots.data_ptr(),
                                            _stream_handle(stream)))
        return status, slots

    def enumerate(self, cap: int | None = None, out=None, count=None, stream=None):
        """All stored keys (unspecified order), trimmed to the stored count."""
        if cap is None:
            cap = self.slots
        if out is None:
            out = torch.empty(max(cap, 1), dtype=self.key_dtype, device=self.device)
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=self.device)
        check(self._L.cht_enumerate(self._h, out.data_ptr(), cap, count.data_ptr(),
                                    _stream_handle(stream)))
        n = int(count.item())
        return out[: min(n, cap)], n

    def attach_counters(self) -> torch.Tensor:
        """Attach zeroed device counters (probes, writes, cas_fail, ops)."""
        self.counters = torch.zeros(4, dtype=torch.int64, device=self.device)
        check(self._L.cht_set_counters(self._h, self.counters.data_ptr()))
        return self.counters

    def detach_counters(self):
        check(self._L.cht_set_counters(self._h, None))
        self.counters = None

    def error_flags(self, stream=None) -> int:
        f = ctypes.c_uint32(0)
        check(self._L.cht_error_flags(self._h, ctypes.byref(f), _stream_handle(stream)))
        return f.value

    # -- inspection -------------------------------------------------------------
    def words(self, level: int = 0) -> torch.Tensor:
        """The bucket words of a level as an int64 view of the storage
        (level 2: the iceberg stash's slots)."""
        c = self.cfg
        w = self.storage[_lib.HEADER_BYTES:].view(torch.int64)
        n0 = c.num_buckets * c.bucket_words
        if level == 0:
            return w[:n0]
        n1 = c.num_buckets_backyard * c.bucket_words
        if level == 1:
            return w[n0: n0 + n1]
        # level 2: the iceberg stash (whole keys, 0 = empty)
        return w[n0 + n1: n0 + n1 + c.stash_slots]
