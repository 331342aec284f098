"""Host-buffer entry points: run a table operation on keys that live in
(pinned) host memory, streaming them through the GPU.

Keys are cut into chunks that cycle through `depth` device staging buffers.
Host->device copies run on one copy stream, the table operation on the
compute stream and device->host copies of the statuses on a third stream, so
both directions of the host link and the kernels overlap. Events order each
buffer's reuse: a chunk's keys may be overwritten only after the kernel that
read them finished, and its statuses only after they were copied out.
"""
from __future__ import annotations

import torch

from .table import Table


class HostPipeline:
    def __init__(self, table: Table, chunk_keys: int = 1 << 24, depth: int = 3):
        self.t = table
        self.chunk = int(chunk_keys)
        self.depth = depth
        dev = table.device
        self.h2d = torch.cuda.Stream(device=dev)
        self.compute = torch.cuda.Stream(device=dev)
        self.d2h = torch.cuda.Stream(device=dev)
        kd = table.key_dtype
        self.d_keys = [torch.empty(self.chunk, dtype=kd, device=dev) for _ in range(depth)]
        self.d_st = [torch.empty(self.chunk, dtype=torch.uint8, device=dev) for _ in range(depth)]
        self.ev_loaded = [torch.cuda.Event() for _ in range(depth)]
        self.ev_done = [torch.cuda.Event() for _ in range(depth)]
        self.ev_drained = [torch.cuda.Event() for _ in range(depth)]
        self.h2d_bytes = 0
        self.d2h_bytes = 0
        self.launches = 0
        self._used = [False] * depth
        self._slot = 0

    def run(self, op: str, keys_host: torch.Tensor, status_host: torch.Tensor,
            wait: bool = True):
        """op in {"insert", "find", "find_or_put"}; keys_host / status_host are
        contiguous (ideally pinned) CPU tensors of equal length. With wait the
        call returns once every status has landed in status_host; otherwise
        call sync() before reading them."""
        assert keys_host.device.type == "cpu" and status_host.device.type == "cpu"
        n = keys_host.numel()
        fn = getattr(self.t, op)
        for lo in range(0, n, self.chunk):
            hi = min(n, lo + self.chunk)
            m = hi - lo
            b = self._slot
            self._slot = (b + 1) % self.depth
            if self._used[b]:
                # the kernel that read this buffer, and the copy-out of its
                # statuses, must be done before the buffer is refilled
                self.h2d.wait_event(self.ev_done[b])
                self.compute.wait_event(self.ev_drained[b])
            self._used[b] = True
            with torch.cuda.stream(self.h2d):
                self.d_keys[b][:m].copy_(keys_host[lo:hi], non_blocking=True)
                self.ev_loaded[b].record(self.h2d)
            self.compute.wait_event(self.ev_loaded[b])
            fn(self.d_keys[b][:m], status=self.d_st[b][:m], stream=self.compute)
            self.ev_done[b].record(self.compute)
            self.d2h.wait_event(self.ev_done[b])
            with torch.cuda.stream(self.d2h):
                status_host[lo:hi].copy_(self.d_st[b][:m], non_blocking=True)
                self.ev_drained[b].record(self.d2h)
            self.h2d_bytes += m * keys_host.element_size()
            self.d2h_bytes += m
            self.launches += 1
        if wait:
            self.sync()
        return status_host

    def sync(self):
        self.d2h.synchronize()
        self.compute.synchronize()
        self.h2d.synchronize()
