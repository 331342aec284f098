"""Autotuner for the launch shape of table operations and fused batches, and
for the slot packing of new tables.

For a given operation it times every candidate (threads per bucket tile,
items per thread), restoring the tables' contents before each trial so that
every candidate sees the same state, and keeps the fastest. Results are cached
in a JSON file (CHT_TUNE_CACHE, default ~/.cache/cht_tune.json) under a key
built from the device, the operation, the table kind, the packing of both
levels and the size class (log2 of the largest primary bucket count), so
later runs of the same shape skip the sweep.

Tiles are 4, 8 or 16 lanes: a lane owns whole 64-bit words of the bucket
(slots are fields of a word and a claim is a compare-and-swap of one word's
field), and a 16-word bucket split over 32 lanes would leave a lane half a
word. Items per lane are 1, 2 or 4, the counts the kernels are built for
(larger settings run the 4-key form).

tune_packing chooses, for a table about to be created, between the densest
packing that holds its entries and the next wider one (fewer, wider fields
per word: 16- or 32-bit fields take a native compare-and-swap of their own
width, 21-bit fields a retried 64-bit one), by timing the operation on a
fresh table of each packing with the same bucket counts.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

import torch

TILES = (4, 8, 16)
ITEMS = (1, 2, 4)

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
    return (f"{dev}|{op}|kind{c.kind}|compact{c.compact}|fpw{c.fields_per_word}"
            f"/{c.fields_per_word_backyard}|wpb{c.bucket_words}|lg{size_class}|n{len(tables)}")


def _fits(body_bits: int, tag_bits: int, fpw: int) -> bool:
    return body_bits + tag_bits <= 64 // fpw


def packing_candidates(kind: int, key_bits: int, num_buckets: int,
                       num_buckets_backyard: int = 0, compact: bool = True) -> list:
    """(fields_per_word, fields_per_word_backyard) pairs tune_packing tries:
    per level the densest packing whose fields hold an entry (remainder of
    key_bits - log2(buckets) bits, or the whole key, plus the tag: 2 bits
    for cuckoo and iceberg secondary entries, 1 for iceberg primary ones)
    and the next wider one, when there is one."""
    def level(nb: int, tag: int) -> list:
        if not compact:
            return [1]
        body = key_bits - max(0, math.ceil(math.log2(max(nb, 1))))
        dense = max(f for f in (1, 2, 3, 4) if _fits(body, tag, f))
        return [dense] if dense == 1 else [dense, dense - 1]
    if kind == 0:
        return [(f, 0) for f in level(num_buckets, 2)]
    return [(f0, f1) for f0 in level(num_buckets, 1) for f1 in level(num_buckets_backyard, 2)]


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


def tune_packing(kind: int, key_bits: int, num_buckets: int, num_buckets_backyard: int,
                 keys: torch.Tensor, op: str, reps: int = 3, use_cache: bool = True,
                 **table_kw) -> dict:
    """Choose the slot packing of a new table by measurement.

    Every candidate of packing_candidates gets a fresh table with the given
    bucket counts, and `op` ("insert", "find_or_put") over `keys` is timed
    on it from empty, reps times. A candidate whose run reports more FULL
    keys than the densest packing's is dropped (a wider packing holds fewer
    slots). Returns {"fields_per_word", "fields_per_word_backyard", "ms",
    "sweep", "cached"}; the choice is cached under the operation, kind, key
    width, bucket counts and key count."""
    from . import Table
    dev = keys.device
    lg0 = int(math.log2(max(num_buckets, 1)))
    lg1 = int(math.log2(max(num_buckets_backyard, 1))) if num_buckets_backyard else 0
    key = (f"{torch.cuda.get_device_name(dev)}|packing|{op}|kind{kind}|w{key_bits}|lg{lg0}/{lg1}"
           f"|n{int(math.log2(max(keys.numel(), 1)))}")
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return dict(hit, cached=True)
    results = []
    full_dense = None
    for f0, f1 in packing_candidates(kind, key_bits, num_buckets, num_buckets_backyard,
                                     table_kw.get("compact", True)):
        t = Table(kind, key_bits, num_buckets, num_buckets_backyard, fields_per_word=f0,
                  fields_per_word_backyard=f1, device=dev, **table_kw)
        status = torch.empty(keys.numel(), dtype=torch.uint8, device=dev)
        fn = getattr(t, op)
        ms = []
        for _ in range(reps):
            t.clear()
            torch.cuda.synchronize()
            ms.append(_time(lambda: fn(keys, status=status), 1))
        full = int((status == 3).sum().item())
        if full_dense is None:
            full_dense = full
        results.append({"fields_per_word": f0, "fields_per_word_backyard": f1,
                        "ms": statistics.median(ms), "full": full})
        del t
    ok = [r for r in results if r["full"] <= full_dense]
    best = min(ok, key=lambda r: r["ms"])
    out = {"fields_per_word": best["fields_per_word"],
           "fields_per_word_backyard": best["fields_per_word_backyard"], "ms": best["ms"]}
    if use_cache:
        _store(key, out)
    return dict(out, cached=False, sweep=results)
