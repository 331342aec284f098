"""Served request loop over resident tables: continuous batching.

Requests (lookup, find-or-put or insert batches against one of several
resident iceberg tables) arrive over time. The server admits every request
that has arrived when it forms the next *wave*, as far as the free device
memory budget and each table's headroom allow, and runs each wave as at most
two fused multi-table launches (one lookup batch, one find-or-put batch). A
wave is issued while the previous one is still on the GPU, on the other of
two streams, so their work overlaps unless they touch a common table with a
write, in which case the later wave waits for the earlier one's event.

Per-table semantics equal running the requests one at a time in admission
order: in one wave a table receives either a run of consecutive lookups
(lookups commute) or a single write request, and waves that conflict on a
table are ordered by events. A request's result is therefore the same alone
and in the mix; the only freedom is which of several copies of one new key
inside one find-or-put request reports PUT (the others report FOUND), as for
any concurrent find-or-put.

Keys are planned in arrival order and generated on the device before serving
starts (Server.plan), from each table's counter-based key sequence
(workloads.keys_at): fresh keys take the table's next indices (capped by its
headroom, so a table admits writes only while it has room), re-queries draw
uniformly among the indices the table has been given before the request. The
served inputs are thus resident in HBM when a request arrives.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import workloads as W
from .batch import OP_FIND, OP_FIND_OR_PUT, Batch
from .table import Table

FIND, FOP, INSERT = "find", "find_or_put", "insert"


@dataclasses.dataclass
class Request:
    rid: int
    table: int
    op: str
    n: int
    arrival: float          # seconds from the start of the run
    requery_frac: float = 0.4
    # filled in by the server
    n_fresh: int = 0
    fresh_start: int = 0
    admitted: float = -1.0
    done: float = -1.0
    keys: torch.Tensor | None = None
    status: torch.Tensor | None = None


def form_wave(pending: list, budget: int) -> tuple[list, list]:
    """Split the pending requests (in admission order) into the next wave and
    the rest. Per table the wave takes a run of consecutive lookups or one
    write request, and no request is taken past an earlier one of its table
    that stays behind, so every table sees its requests in admission order.
    The wave holds at most budget keys, but always at least one request.
    Linear in the number of pending requests."""
    wave, rest, used, taken = [], [], 0, {}
    blocked = set()  # tables with an earlier request left for a later wave
    for r in pending:
        kind = "r" if r.op == FIND else "w"
        cur = taken.get(r.table)
        fits = used + r.n <= budget or not wave
        ok = fits and (cur is None or (cur == "r" and kind == "r"))
        if ok and r.table not in blocked:
            wave.append(r)
            used += r.n
            taken[r.table] = kind
        else:
            rest.append(r)
            blocked.add(r.table)
    return wave, rest


@dataclasses.dataclass
class TableState:
    table: Table
    seed: int
    key_bits: int
    capacity: int            # keys the table may receive before it counts as full
    next_index: int = 0      # next fresh key index of this table's sequence
    absent_base: int = 1 << 40


class Server:
    """Continuous-batching request loop over resident iceberg tables."""

    def __init__(self, tables: list[Table], seeds: list[int], *, fill_cap: float = 0.85,
                 max_wave_keys: int = 1 << 25, hbm_reserve: float = 0.1, device=None):
        self.dev = device or tables[0].device
        self.states = []
        for t, s in zip(tables, seeds):
            cap = int(fill_cap * t.slots)
            self.states.append(TableState(t, s, t.cfg.key_bits, cap,
                                          absent_base=1 << (t.cfg.key_bits - 2)))
        self.max_wave_keys = max_wave_keys
        self.hbm_reserve = hbm_reserve
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(2)]
        self.waves = 0
        self.launches = 0
        self._budget = None  # (keys, time taken)

    # -- admission ------------------------------------------------------------
    def _budget_keys(self, refresh_s: float = 0.01) -> int:
        """Keys a wave may admit given free HBM (re-read at most every
        refresh_s: the query is a driver call that costs the served loop)."""
        now = time.perf_counter()
        if self._budget is None or now - self._budget[1] > refresh_s:
            free, total = torch.cuda.mem_get_info(self.dev)
            usable = max(0, free - self.hbm_reserve * total)
            # per admitted key: its status byte plus staging of fused launches
            self._budget = (int(min(self.max_wave_keys, usable // 16)), now)
        return self._budget[0]

    def plan(self, requests: list[Request], seed: int = 0) -> list[Request]:
        """Give every request its keys, in arrival order: fresh keys take the
        table's next indices (capped by its headroom), lookups' fresh keys are
        never-inserted ones, re-queries draw uniformly among the indices the
        table has been given before the request. Keys are generated on the
        device, one vectorised pass per table, and stay resident."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        per_table: dict[int, list] = {}
        for r in reqs:
            st = self.states[r.table]
            want = int(round((1 - r.requery_frac) * r.n))
            if r.op == FIND:
                r.n_fresh, r.fresh_start = want, -1
                hi = st.next_index
            else:
                r.n_fresh = min(want, max(0, st.capacity - st.next_index))
                r.fresh_start = st.next_index
                hi = st.next_index
                st.next_index += r.n_fresh
            per_table.setdefault(r.table, []).append((r, hi))
        g = torch.Generator(device=self.dev)
        g.manual_seed(seed)
        for tid, items in per_table.items():
            st = self.states[tid]
            idx_parts = []
            for r, hi in items:
                n_re = r.n - r.n_fresh
                if r.op == FIND:
                    base = st.absent_base + r.rid * (1 << 23)
                    fresh = torch.arange(base, base + r.n_fresh, device=self.dev)
                else:
                    fresh = torch.arange(r.fresh_start, r.fresh_start + r.n_fresh,
                                         device=self.dev)
                if hi > 0:
                    u = torch.rand(n_re, generator=g, device=self.dev, dtype=torch.float64)
                    re = (u * hi).to(torch.int64).clamp_(max=hi - 1)
                else:  # nothing given yet: re-queries become misses
                    base = st.absent_base + r.rid * (1 << 23) + (1 << 22)
                    re = torch.arange(base, base + n_re, device=self.dev)
                idx_parts.append(torch.cat([fresh, re]))
            allk = W.keys_at(torch.cat(idx_parts), st.key_bits, st.seed)
            off = 0
            for r, _ in items:
                r.keys = allk[off: off + r.n]
                off += r.n
        return reqs

    # -- running --------------------------------------------------------------
    def run(self, requests: list[Request], *, realtime: bool = True):
        """Serve planned requests (see plan). With realtime, a request is
        visible only once the wall clock passes its arrival time. Returns the
        requests with admitted/done times and status tensors filled in."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending: list[Request] = []
        inflight = []   # (event, requests, write_tables, all_tables)
        nxt = 0
        t0 = time.perf_counter()
        slot = 0
        while nxt < len(reqs) or pending or inflight:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                pending.append(reqs[nxt])
                nxt += 1
            # retire finished waves
            still = []
            for ev, rs, wt, at in inflight:
                if ev.query():
                    tdone = time.perf_counter() - t0
                    for r in rs:
                        r.done = tdone
                else:
                    still.append((ev, rs, wt, at))
            inflight = still
            if not pending or len(inflight) >= 2:
                if not pending and nxt < len(reqs) and not inflight and realtime:
                    # idle: sleep towards the next arrival, but spin through
                    # its last 200 us (sleeping is too coarse to admit on time)
                    gap = reqs[nxt].arrival - now
                    if gap > 2e-4:
                        time.sleep(min(0.001, gap - 2e-4))
                continue
            wave, pending = form_wave(pending, self._budget_keys())
            tnow = time.perf_counter() - t0
            for r in wave:
                r.admitted = tnow
            self._issue(wave, slot, inflight)
            slot ^= 1
        torch.cuda.synchronize()
        return reqs

    def _issue(self, wave, slot, inflight):
        s = self.streams[slot]
        writes = {r.table for r in wave if r.op != FIND}
        touched = {r.table for r in wave}
        # order after in-flight waves that conflict on a table with a write
        for ev, rs, wt, at in inflight:
            if (writes & at) or (wt & touched):
                s.wait_event(ev)
        with torch.cuda.stream(s):
            for r in wave:
                r.status = torch.empty(r.n, dtype=torch.uint8, device=self.dev)
            finds = [r for r in wave if r.op == FIND and r.n]
            fops = [r for r in wave if r.op != FIND and r.n]
            for group, op in ((finds, OP_FIND), (fops, OP_FIND_OR_PUT)):
                if not group:
                    continue
                if len(group) == 1:
                    # a lone request needs no fused plan: one direct launch
                    r = group[0]
                    t = self.states[r.table].table
                    if op == OP_FIND:
                        t.find(r.keys, status=r.status, stream=s)
                    else:
                        t.find_or_put(r.keys, status=r.status, stream=s)
                    self.launches += 1
                    continue
                # one fused launch; several lookups of one table are
                # concatenated into one entry (lookups commute)
                by_table: dict[int, list[Request]] = {}
                for r in group:
                    by_table.setdefault(r.table, []).append(r)
                tabs, keys, sts, splits = [], [], [], []
                for tid, rs in by_table.items():
                    tabs.append(self.states[tid].table)
                    if len(rs) == 1:
                        keys.append(rs[0].keys)
                        sts.append(rs[0].status)
                    else:
                        keys.append(torch.cat([r.keys for r in rs]))
                        sts.append(torch.empty(sum(r.n for r in rs), dtype=torch.uint8,
                                               device=self.dev))
                        splits.append((sts[-1], rs))
                b = Batch(tabs, keys, sts, op=op, stream=s)
                b.launch(stream=s)
                self.launches += 1
                for big, rs in splits:
                    off = 0
                    for r in rs:
                        r.status.copy_(big[off: off + r.n])
                        off += r.n
            ev = torch.cuda.Event()
            ev.record(s)
        self.waves += 1
        inflight.append((ev, wave, writes, touched))


def run_sequential(server: Server, requests: list[Request], *, realtime: bool = True):
    """Baseline: one synchronous launch per request, in arrival order (the
    requests must have been planned by `server`)."""
    reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
    t0 = time.perf_counter()
    for r in reqs:
        if realtime:
            while time.perf_counter() - t0 < r.arrival:
                pass
        r.admitted = time.perf_counter() - t0
        t = server.states[r.table].table
        if r.n:
            r.status = t.find(r.keys) if r.op == FIND else t.find_or_put(r.keys)
        else:
            r.status = torch.empty(0, dtype=torch.uint8, device=server.dev)
        torch.cuda.synchronize()
        r.done = time.perf_counter() - t0
    return reqs


def make_requests(n: int, n_tables: int, rate_per_s: float, *, min_size: int = 256,
                  max_size: int = 4 << 20, mix=(0.6, 0.3, 0.1), requery_frac: float = 0.4,
                  rng_seed: int = W.SEED_BASE + 5) -> list[Request]:
    """Poisson arrivals, log-uniform sizes, op mix (find, find-or-put, insert)."""
    rng = np.random.default_rng(rng_seed)
    arr = W.poisson_arrivals(n, rate_per_s, rng_seed + 1) if rate_per_s > 0 else np.zeros(n)
    sizes = W.log_uniform_sizes(n, min_size, max_size, rng_seed + 2)
    tables = rng.integers(0, n_tables, n)
    u = rng.random(n)
    ops = np.where(u < mix[0], FIND, np.where(u < mix[0] + mix[1], FOP, INSERT))
    return [Request(i, int(tables[i]), str(ops[i]), int(sizes[i]), float(arr[i]), requery_frac)
            for i in range(n)]


def latency_stats(reqs: list[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs if r.done >= 0])
    keys = sum(r.n for r in reqs)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "mops": keys / span / 1e6, "requests": len(reqs),
            "keys": keys, "span_s": span}
