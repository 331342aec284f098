"""Autotuner for the launch shape of table operations and fused batches.

For a given operation it times every candidate (threads per bucket tile,
items per thread), restoring the tables' contents before each trial so that
every candidate sees the same state, and keeps the fastest. Results are cached
in a JSON file (CHT_TUNE_CACHE, default ~/.cache/cht_tune.json) under a key
built from the device, the operation, the table kind, the primary packing and
the size class (log2 of the largest primary bucket count), so later runs of
the same shape skip the sweep.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

import torch

TILES = (4, 8, 16)
ITEMS = (1, 2, 4, 8)

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("CHT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "cht_tune.json"))


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(key: str, value: dict) -> None:
    with _lock:
        c = _load_cache()
        c[key] = value
        p = cache_path()
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, p)


def shape_key(op: str, tables) -> str:
    c = tables[0].cfg
    size_class = max(int(math.log2(max(t.cfg.num_buckets, 1))) for t in tables)
    dev = torch.cuda.get_device_name(tables[0].device)
    return f"{dev}|{op}|kind{c.kind}|compact{c.compact}|fpw{c.fields_per_word}|lg{size_class}|n{len(tables)}"


def _time(fn, reps: int) -> float:
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_batch(batch, reps: int = 3, use_cache: bool = True, tiles=TILES, items=ITEMS) -> dict:
    """Pick (tile, items_per_thread) for a fused Batch; applies and returns it.

    The tables' storage is snapshotted first and restored before every trial
    (find-or-put changes the tables), and once more at the end."""
    from .batch import OP_FIND
    op = "batch_find" if getattr(batch, "op", None) == OP_FIND else "batch_fop"
    key = shape_key(op, batch.tables)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            batch.set_launch(tile=hit["tile"], items_per_thread=hit["items"])
            return dict(hit, cached=True)
    snap = [t.storage.clone() for t in batch.tables]

    def restore():
        for t, s in zip(batch.tables, snap):
            t.storage.copy_(s)

    results = []
    for T in tiles:
        for I in items:
            batch.set_launch(tile=T, items_per_thread=I)

            def trial():
                batch.launch()

            ms = []
            for _ in range(reps):
                restore()
                torch.cuda.synchronize()
                ms.append(_time(trial, 1))
            results.append((statistics.median(ms), T, I))
    restore()
    torch.cuda.synchronize()
    best = min(results)
    out = {"tile": best[1], "items": best[2], "ms": best[0],
           "sweep": [{"tile": T, "items": I, "ms": m} for m, T, I in results]}
    batch.set_launch(tile=best[1], items_per_thread=best[2])
    if use_cache:
        _store(key, {k: out[k] for k in ("tile", "items", "ms")})
    return dict(out, cached=False)


def table_candidates(kind: int, op: str, current_in_flight: int, tiles=TILES, items=ITEMS,
                     in_flight=None) -> list[tuple[int, int, int]]:
    """(tile, items_per_thread, lookups_in_flight) shapes tune_table tries:
    on cuckoo tables the chunk forms (one load in flight, every items value)
    and the stream forms (4 or 8 loads in flight, items unused); iceberg
    operations keep the table's in-flight setting, which they ignore, and
    try every items value."""
    if in_flight is None:
        in_flight = (1, 4, 8) if (kind == 0 and op != "find_or_put") else (current_in_flight,)
    cands = []
    for P in in_flight:
        # items_per_thread matters to the chunk forms: cuckoo with one load in
        # flight, and every iceberg operation
        sweep_items = P == 1 or kind == 1
        for T in tiles:
            for I in (items if sweep_items else (1,)):
                cands.append((T, I, P))
    return cands


def tune_table(table, op: str, keys: torch.Tensor, reps: int = 3, use_cache: bool = True,
               tiles=TILES, items=ITEMS, in_flight=None) -> dict:
    """Pick the launch shape for one operation on one table ("find", "insert"
    or "find_or_put"); applies and returns it. The candidates are those of
    table_candidates: every (tile, items_per_thread) pair for iceberg
    operations and for cuckoo's one-load form, plus each tile with 4 or 8
    loads in flight on cuckoo tables (the stream kernels, which take no
    items_per_thread)."""
    key = shape_key(op, [table])
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            table.set_launch(tile=hit["tile"], items_per_thread=hit["items"],
                             lookups_in_flight=hit.get("in_flight",
                                                       table.cfg.lookups_in_flight))
            return dict(hit, cached=True)
    cands = table_candidates(table.cfg.kind, op, table.cfg.lookups_in_flight, tiles, items,
                             in_flight)
    snap = table.storage.clone()
    status = torch.empty(keys.numel(), dtype=torch.uint8, device=keys.device)
    fn = getattr(table, op)
    results = []
    for T, I, P in cands:
        table.set_launch(tile=T, items_per_thread=I, lookups_in_flight=P)
        ms = []
        for _ in range(reps):
            table.storage.copy_(snap)
            torch.cuda.synchronize()
            ms.append(_time(lambda: fn(keys, status=status), 1))
        results.append((statistics.median(ms), T, I, P))
    table.storage.copy_(snap)
    torch.cuda.synchronize()
    best = min(results)
    table.set_launch(tile=best[1], items_per_thread=best[2], lookups_in_flight=best[3])
    out = {"tile": best[1], "items": best[2], "in_flight": best[3], "ms": best[0]}
    if use_cache:
        _store(key, out)
    return dict(out, cached=False,
                sweep=[{"tile": T, "items": I, "in_flight": P, "ms": m} for m, T, I, P in results])
