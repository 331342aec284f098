"""Host-buffer entry points: run a table operation on keys that live in
(pinned) host memory, streaming them through the GPU.

Keys are cut into chunks. While chunk i is processed on the compute stream,
chunk i+1 is copied host->device and the statuses of chunk i-1 are copied
device->host on a copy stream, so the link and the kernels overlap. Two
staging buffers per direction are allocated once per pipeline (by PyTorch's
allocator) and reused.
"""
from __future__ import annotations

import torch

from .table import Table


class HostPipeline:
    def __init__(self, table: Table, chunk_keys: int = 1 << 26):
        self.t = table
        self.chunk = int(chunk_keys)
        dev = table.device
        self.compute = torch.cuda.Stream(device=dev)
        self.copy = torch.cuda.Stream(device=dev)
        kd = table.key_dtype
        self.d_keys = [torch.empty(self.chunk, dtype=kd, device=dev) for _ in range(2)]
        self.d_st = [torch.empty(self.chunk, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.d_drop = None
        self.h2d_bytes = 0
        self.d2h_bytes = 0
        self.launches = 0

    def run(self, op: str, keys_host: torch.Tensor, status_host: torch.Tensor):
        """op in {"insert", "find", "find_or_put"}; keys_host / status_host are
        contiguous (ideally pinned) CPU tensors of equal length. Returns once
        every status has landed in status_host."""
        assert keys_host.device.type == "cpu" and status_host.device.type == "cpu"
        n = keys_host.numel()
        fn = getattr(self.t, op)
        loaded = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        drained = [torch.cuda.Event() for _ in range(2)]
        for e in drained:
            e.record(self.copy)
        nchunks = (n + self.chunk - 1) // self.chunk
        for i in range(nchunks):
            b = i & 1
            lo, hi = i * self.chunk, min(n, (i + 1) * self.chunk)
            m = hi - lo
            with torch.cuda.stream(self.copy):
                # the staging buffer is free once its previous statuses left
                self.copy.wait_event(drained[b])
                self.copy.wait_event(done[b]) if i >= 2 else None
                self.d_keys[b][:m].copy_(keys_host[lo:hi], non_blocking=True)
                loaded[b].record(self.copy)
            self.compute.wait_event(loaded[b])
            fn(self.d_keys[b][:m], status=self.d_st[b][:m], stream=self.compute)
            done[b].record(self.compute)
            with torch.cuda.stream(self.copy):
                self.copy.wait_event(done[b])
                status_host[lo:hi].copy_(self.d_st[b][:m], non_blocking=True)
                drained[b].record(self.copy)
            self.h2d_bytes += m * keys_host.element_size()
            self.d2h_bytes += m
            self.launches += 1
        self.copy.synchronize()
        self.compute.synchronize()
        return status_host
