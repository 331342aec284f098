"""Served request loop over resident tables: continuous batching.

Requests (lookup, find-or-put or insert batches against one of several
resident iceberg tables) arrive over time. The server admits the requests
that have arrived when it forms the next *wave*, and runs each wave as at
most two fused multi-table launches (one lookup batch, one find-or-put
batch). A wave is issued while the previous one is still on the GPU, on the
other of two streams, so their work overlaps unless they touch a common table
with a write, in which case the later wave waits for the earlier one's event.

Admission is by device memory and by table headroom:
  - a request's keys and statuses live in a fixed key arena (device memory
    sized from the free HBM when the server starts); a request is admitted
    only when its keys fit in the arena next to the in-flight requests, and
    its space returns when its wave completes. Requests are admitted in
    arrival order: one that has to wait for memory holds back the ones behind
    it, so a large request is not starved by small ones; a request larger
    than the whole arena is rejected;
  - a write request reserves its fresh keys against its table's headroom (a
    share of the table's slots, max_fill) when it is admitted; one whose fresh
    keys exceed the headroom left is rejected (a table never frees slots);
  - a request with a deadline that is still waiting when the deadline passes
    is cancelled (not run), e.g. one held back for memory too long.
The arena's size is halved when the device cannot allocate it (alloc_arena).
Each wave is an NVTX range, so a profiler's timeline shows the waves.
Admitted requests get their keys generated on the device into their arena
space (one generator launch per wave, from each request's key recipe), so the
device holds only the keys of admitted requests.

Per-table semantics equal running the requests one at a time in admission
order: in one wave a table receives either a run of consecutive lookups
(lookups commute) or a single write request, and waves that conflict on a
table are ordered by events. A request's result is therefore the same alone
and in the mix; the only freedom is which of several copies of one new key
inside one find-or-put request reports PUT (the others report FOUND), as for
any concurrent find-or-put.

Key recipes (Server.plan, host only, O(1) per request): fresh keys take the
table's next indices of its key sequence (capped at fill_cap of its slots,
after which fresh draws become re-queries), lookups' fresh keys are
never-inserted ones, re-queries draw uniformly among the indices the table
has been given before the request (workloads.request_keys defines the keys).
"""
from __future__ import annotations

import collections
import dataclasses
import heapq
import time

import numpy as np
import torch

from . import workloads as W
from .batch import OP_FIND, OP_FIND_OR_PUT, Batch
from .table import Table

FIND, FOP, INSERT = "find", "find_or_put", "insert"
OK, WAIT, REJECT = "ok", "wait", "reject"


@dataclasses.dataclass
class Request:
    rid: int
    table: int
    op: str
    n: int
    arrival: float          # seconds from the start of the run
    requery_frac: float = 0.4
    deadline: float = -1.0  # give up if not admitted by then (seconds; < 0: never)
    # key recipe (Server.plan)
    n_fresh: int = 0
    fresh_base: int = 0
    re_hi: int = 0
    re_seed: int = 0
    miss_base: int = 0
    # filled in by the server
    admitted: float = -1.0
    done: float = -1.0
    rejected: str = ""      # why it was not served: headroom, size, cancelled
    off: int = -1           # position of the request's keys in the key arena
    keys: torch.Tensor | None = None    # kept with keep_results
    status: torch.Tensor | None = None  # kept with keep_results

    def recipe(self, key_bits: int, seed: int) -> dict:
        return dict(n=self.n, n_fresh=self.n_fresh, fresh_base=self.fresh_base,
                    re_hi=self.re_hi, re_seed=self.re_seed, miss_base=self.miss_base,
                    key_bits=key_bits, seed=seed)


class PendingQueues:
    """Requests waiting for a wave, one queue per table (each in arrival
    order), and the wave-forming rule over them.

    Per table a wave takes a run of consecutive lookups or one write
    request, and never a request past an earlier one of its table that stays
    behind, so every table sees its requests in admission order. Across
    tables, the requests that could join (each table's next ones) are taken
    in arrival order; the wave holds at most `budget` keys, but always at
    least one request, and the first of those requests that would overflow
    the budget ends the wave, as does reaching max_requests. Forming a wave
    examines only the requests it takes plus one per table, however many are
    waiting.

    admit(r), if given, is asked for each request the wave could take: OK
    takes it (its resources are then reserved), REJECT drops it (the caller
    has marked it), WAIT leaves it and ends the wave, so that no later
    request overtakes one held back for memory."""

    def __init__(self, requests=()):
        self.q: dict[int, collections.deque] = {}
        self.n = 0
        for r in requests:
            self.add(r)

    def add(self, r: Request) -> None:
        self.q.setdefault(r.table, collections.deque()).append(r)
        self.n += 1

    def __len__(self) -> int:
        return self.n

    def requests(self) -> list[Request]:
        """Every waiting request, in arrival order."""
        return sorted((r for q in self.q.values() for r in q), key=lambda r: (r.arrival, r.rid))

    def form_wave(self, budget: int, admit=None, max_requests: int = 4096) -> list[Request]:
        wave, used = [], 0
        took: dict[int, str] = {}  # table -> "r" (took lookups) or "w" (took a write)
        # the heap holds each table's next request while it may still join
        heads = [(q[0].arrival, q[0].rid, t) for t, q in self.q.items() if q]
        heapq.heapify(heads)
        while heads:
            _, _, t = heapq.heappop(heads)
            q = self.q[t]
            r = q[0]
            if wave and (used + r.n > budget or len(wave) >= max_requests):
                break
            verdict = admit(r) if admit is not None else OK
            if verdict == WAIT:
                break
            q.popleft()
            self.n -= 1
            if verdict != REJECT:
                wave.append(r)
                used += r.n
                took[t] = "r" if r.op == FIND else "w"
            k = took.get(t)
            if q and (k is None or (k == "r" and q[0].op == FIND)):
                heapq.heappush(heads, (q[0].arrival, q[0].rid, t))
        return wave


def form_wave(pending: list, budget: int, admit=None) -> tuple[list, list]:
    """The wave rule of PendingQueues over a list in arrival order: returns
    (wave, rest), rest being the requests not taken, in arrival order."""
    pq = PendingQueues(pending)
    wave = pq.form_wave(budget, admit)
    return wave, pq.requests()


class KeyArena:
    """A ring of `cap` key positions handed out in admission order and given
    back in any order; space is reused once every earlier allocation has been
    given back. Host bookkeeping only."""

    def __init__(self, cap: int):
        self.cap = cap
        self.live = collections.deque()  # [start, end, freed] in allocation order
        self.tail = 0                    # where the next allocation may start

    def used(self) -> int:
        return sum(e - s for s, e, _ in self.live)

    def alloc(self, n: int):
        """Start of n free consecutive positions, or None (-1 for n = 0:
        nothing to hold)."""
        if n > self.cap:
            return None
        if n == 0:
            return -1
        if not self.live:
            self.tail = start = 0
        else:
            head = self.live[0][0]
            if self.tail > head:
                # in use: [head, tail); free: [tail, cap), then [0, head)
                if self.tail + n <= self.cap:
                    start = self.tail
                elif n <= head:
                    start = 0
                else:
                    return None
            else:
                # wrapped: in use [head, cap) and [0, tail); free: [tail, head)
                if self.tail + n <= head:
                    start = self.tail
                else:
                    return None
        self.live.append([start, start + n, False])
        self.tail = start + n
        return start

    def free(self, start: int) -> None:
        if start < 0:
            return
        for item in self.live:
            if item[0] == start and not item[2]:
                item[2] = True
                break
        while self.live and self.live[0][2]:
            self.live.popleft()


@dataclasses.dataclass
class TableState:
    table: Table
    seed: int
    key_bits: int
    capacity: int            # fresh keys the workload gives the table (fill_cap)
    limit: int               # keys the server lets requests reserve (max_fill)
    next_index: int = 0      # next fresh key index of this table's sequence (plan)
    reserved: int = 0        # fresh keys reserved by admitted write requests
    absent_base: int = 1 << 40


def alloc_arena(keys: int, device, min_keys: int = 1 << 20, alloc=torch.empty):
    """The key arena's buffers (int64 keys, uint8 statuses) for `keys`
    positions; when the device runs out of memory, half as many, down to
    min_keys (below that the error propagates). Returns (keys, statuses)."""
    n = keys
    while True:
        try:
            k = alloc(n, dtype=torch.int64, device=device)
            st = alloc(n, dtype=torch.uint8, device=device)
            return k, st
        except torch.cuda.OutOfMemoryError:
            if n // 2 < min_keys:
                raise
            n //= 2


class Server:
    """Continuous-batching request loop over resident iceberg tables."""

    def __init__(self, tables: list[Table], seeds: list[int], *, fill_cap: float = 0.85,
                 max_fill: float = 0.95, arena_keys: int | None = None,
                 hbm_fraction: float = 0.25, max_wave_keys: int = 1 << 25,
                 keep_results: bool = False, device=None):
        self.dev = device or tables[0].device
        self.states = []
        for t, s in zip(tables, seeds):
            self.states.append(TableState(t, s, t.cfg.key_bits, int(fill_cap * t.slots),
                                          int(max_fill * t.slots),
                                          absent_base=1 << (t.cfg.key_bits - 2)))
        if arena_keys is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            arena_keys = int(min(1 << 28, hbm_fraction * free / 9))  # 8 B key + 1 B status
        self.keys, self.status = alloc_arena(arena_keys, self.dev)
        self.arena = KeyArena(self.keys.numel())
        self.max_wave_keys = max_wave_keys
        self.keep_results = keep_results
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(2)]
        self.waves = 0
        self.launches = 0
        self.rejected = 0
        self.held_for_memory = set()  # requests that had to wait for arena space

    # -- key recipes ---------------------------------------------------------
    def plan(self, requests: list[Request], seed: int = 0) -> list[Request]:
        """Give every request its key recipe, in arrival order: fresh keys
        take the table's next indices (capped at fill_cap of its slots),
        lookups' fresh keys are never-inserted ones, re-queries draw uniformly
        among the indices the table has been given before the request. Host
        arithmetic only: keys are generated when a request is admitted."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in reqs:
            st = self.states[r.table]
            want = int(round((1 - r.requery_frac) * r.n))
            r.re_hi = st.next_index
            r.re_seed = W.splitmix(seed, r.rid)
            r.miss_base = st.absent_base + r.rid * (1 << 23) + (1 << 22)
            if r.op == FIND:
                r.n_fresh = want
                r.fresh_base = st.absent_base + r.rid * (1 << 23)
            else:
                r.n_fresh = min(want, max(0, st.capacity - st.next_index))
                r.fresh_base = st.next_index
                st.next_index += r.n_fresh
        return reqs

    def request_keys(self, r: Request, device="cpu") -> torch.Tensor:
        """Request r's keys computed with torch (the generator's definition)."""
        st = self.states[r.table]
        return W.request_keys(r.n, r.n_fresh, r.fresh_base, r.re_hi, r.re_seed, r.miss_base,
                              st.key_bits, st.seed, device)

    # -- admission -------------------------------------------------------------
    def _admit(self, r: Request, now: float) -> str:
        st = self.states[r.table]
        if 0 <= r.deadline < now:
            r.rejected = "cancelled"
        elif r.op != FIND and r.n_fresh > st.limit - st.reserved:
            r.rejected = "table headroom"
        elif r.n > self.arena.cap:
            r.rejected = "larger than the key arena"
        if r.rejected:
            r.admitted = r.done = now
            self.rejected += 1
            return REJECT
        off = self.arena.alloc(r.n)
        if off is None:
            self.held_for_memory.add(r.rid)
            return WAIT
        r.off = off
        if r.op != FIND:
            st.reserved += r.n_fresh
        return OK

    # -- running -------------------------------------------------------------
    def run(self, requests: list[Request], *, realtime: bool = True):
        """Serve planned requests (see plan). With realtime, a request is
        visible only once the wall clock passes its arrival time. Returns the
        requests with admitted/done times (and, with keep_results, their keys
        and statuses) filled in."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = PendingQueues()
        inflight = []   # (event, requests, write_tables, all_tables)
        nxt = 0
        t0 = time.perf_counter()
        slot = 0
        while nxt < len(reqs) or pending or inflight:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                pending.add(reqs[nxt])
                nxt += 1
            # retire finished waves
            still = []
            for ev, rs, wt, at in inflight:
                if ev.query():
                    tdone = time.perf_counter() - t0
                    for r in rs:
                        r.done = tdone
                        self.arena.free(r.off)
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
            tnow = time.perf_counter() - t0
            wave = pending.form_wave(self.max_wave_keys, lambda r: self._admit(r, tnow))
            if not wave:
                continue  # held for memory (or all rejected): wait for a wave to finish
            for r in wave:
                r.admitted = tnow
            self._issue(wave, slot, inflight)
            slot ^= 1
        torch.cuda.synchronize()
        return reqs

    def _generate(self, wave: list, stream) -> None:
        """The wave's keys into the arena: one generator launch per 128
        requests (positions in arena order)."""
        recs = []
        for r in sorted(wave, key=lambda r: r.off):
            if r.n:
                st = self.states[r.table]
                recs.append(dict(r.recipe(st.key_bits, st.seed), out_off=r.off))
        # a launch covers a contiguous span of the arena; requests that
        # wrapped around its end go into a launch of their own
        span = []
        for d in recs:
            if span and d["out_off"] < span[-1]["out_off"] + span[-1]["n"]:
                W.request_keys_device(span, self.keys, stream)
                span = []
            span.append(d)
        if span:
            W.request_keys_device(span, self.keys, stream)

    def _issue(self, wave, slot, inflight):
        torch.cuda.nvtx.range_push(f"wave {self.waves}: {len(wave)} requests")
        try:
            self._issue_wave(wave, slot, inflight)
        finally:
            torch.cuda.nvtx.range_pop()

    def _issue_wave(self, wave, slot, inflight):
        s = self.streams[slot]
        writes = {r.table for r in wave if r.op != FIND}
        touched = {r.table for r in wave}
        with torch.cuda.stream(s):
            # the keys go into arena space that no in-flight wave uses, so
            # their generation need not wait for anything
            self._generate(wave, s)
            # the table work waits for in-flight waves that conflict on a
            # table with a write
            for ev, rs, wt, at in inflight:
                if (writes & at) or (wt & touched):
                    s.wait_event(ev)
            kbase, sbase = self.keys.data_ptr(), self.status.data_ptr()
            kb = self.keys.element_size()
            finds = [r for r in wave if r.op == FIND and r.n]
            fops = [r for r in wave if r.op != FIND and r.n]
            for group, op in ((finds, OP_FIND), (fops, OP_FIND_OR_PUT)):
                if not group:
                    continue
                if len(group) == 1:
                    # a lone request needs no fused plan: one direct launch
                    r = group[0]
                    t = self.states[r.table].table
                    k, st = self.keys[r.off: r.off + r.n], self.status[r.off: r.off + r.n]
                    if op == OP_FIND:
                        t.find(k, status=st, stream=s)
                    else:
                        t.find_or_put(k, status=st, stream=s)
                    self.launches += 1
                    continue
                # one fused launch with an entry per request, in place in the
                # arena (a lookup batch may list a table several times; a
                # wave holds at most one write request per table)
                b = Batch.from_pointers([self.states[r.table].table for r in group],
                                        [kbase + kb * r.off for r in group],
                                        [r.n for r in group],
                                        [sbase + r.off for r in group], op=op, stream=s)
                b.launch(stream=s)
                self.launches += 1
            if self.keep_results:
                for r in wave:
                    r.keys = self.keys[r.off: r.off + r.n].clone()
                    r.status = self.status[r.off: r.off + r.n].clone()
            ev = torch.cuda.Event()
            ev.record(s)
        self.waves += 1
        inflight.append((ev, wave, writes, touched))


def run_sequential(server: Server, requests: list[Request], *, realtime: bool = True):
    """Baseline: one synchronous launch per request, in arrival order (the
    requests must have been planned by `server`; same admission rules, the
    arena holding one request at a time)."""
    reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
    t0 = time.perf_counter()
    s = torch.cuda.current_stream(server.dev)
    for r in reqs:
        if realtime:
            while time.perf_counter() - t0 < r.arrival:
                pass
        r.admitted = time.perf_counter() - t0
        if server._admit(r, r.admitted) == REJECT:
            continue
        if r.n:
            server._generate([r], s)
            k, st = server.keys[r.off: r.off + r.n], server.status[r.off: r.off + r.n]
            t = server.states[r.table].table
            if r.op == FIND:
                t.find(k, status=st)
            else:
                t.find_or_put(k, status=st)
            if server.keep_results:
                r.keys, r.status = k.clone(), st.clone()
        elif server.keep_results:
            r.keys = torch.empty(0, dtype=torch.int64, device=server.dev)
            r.status = torch.empty(0, dtype=torch.uint8, device=server.dev)
        torch.cuda.synchronize()
        r.done = time.perf_counter() - t0
        server.arena.free(r.off)
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
    served = [r for r in reqs if r.done >= 0 and not r.rejected]
    lat = np.array([r.done - r.arrival for r in served])
    keys = sum(r.n for r in served)
    span = max(r.done for r in served) - min(r.arrival for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "mops": keys / span / 1e6, "requests": len(served),
            "rejected": len(reqs) - len(served), "keys": keys, "span_s": span}
