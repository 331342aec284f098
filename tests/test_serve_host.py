"""The served loop's wave formation (host logic, no GPU): per table a run of
consecutive lookups or one write, admission order kept per table, the key
budget respected, and every request eventually served."""
import random

import torch

from paper_2406_09255_gb300.serve import (FIND, FOP, INSERT, OK, REJECT, WAIT, PendingQueues,
                                          Request, form_wave)


def reqs(spec):
    return [Request(i, t, op, n, 0.0) for i, (t, op, n) in enumerate(spec)]


def test_runs_of_lookups_or_one_write_per_table():
    p = reqs([(0, FIND, 10), (0, FIND, 10), (1, FOP, 5), (0, FOP, 7), (1, FIND, 3),
              (2, INSERT, 4), (2, INSERT, 4), (0, FIND, 2)])
    wave, rest = form_wave(p, 10 ** 9)
    assert [r.rid for r in wave] == [0, 1, 2, 5]
    # table 0's write waits, and so does its later lookup (no overtaking);
    # table 1's lookup waits behind its write; table 2 takes one write
    assert [r.rid for r in rest] == [3, 4, 6, 7]
    wave2, rest2 = form_wave(rest, 10 ** 9)
    assert [r.rid for r in wave2] == [3, 4, 6]
    assert [r.rid for r in form_wave(rest2, 10 ** 9)[0]] == [7]


def test_budget_and_progress():
    p = reqs([(0, FIND, 100), (1, FIND, 100), (2, FIND, 100)])
    wave, rest = form_wave(p, 150)
    assert [r.rid for r in wave] == [0] and len(rest) == 2
    # a request larger than the budget still goes out alone
    wave, rest = form_wave(reqs([(0, FOP, 1000)]), 10)
    assert len(wave) == 1 and not rest


def test_random_streams_keep_per_table_order_and_drain():
    rnd = random.Random(3)
    spec = [(rnd.randrange(4), rnd.choice([FIND, FIND, FOP, INSERT]), rnd.randrange(1, 50))
            for _ in range(400)]
    pending = reqs(spec)
    served, waves = [], 0
    while pending:
        wave, pending = form_wave(pending, rnd.randrange(20, 200))
        assert wave, "every wave makes progress"
        per_table = {}
        for r in wave:
            per_table.setdefault(r.table, []).append(r)
        for rs in per_table.values():
            # one write alone, or only lookups
            assert (len(rs) == 1) or all(r.op == FIND for r in rs)
        served += wave
        waves += 1
    assert len(served) == 400
    for t in range(4):
        ids = [r.rid for r in served if r.table == t]
        assert ids == sorted(ids), "a table sees its requests in admission order"


def _reference_wave(pending, budget, admit):
    """The wave rule written as one plain pass over the requests in arrival
    order (O(n)): a table closes once it took a write or left a request
    behind; the first candidate over the budget, or one that must wait,
    ends the wave."""
    wave, rest, used, took, closed, stopped = [], [], 0, {}, set(), False
    for r in pending:
        if stopped or r.table in closed:
            rest.append(r)
            continue
        if took.get(r.table) == "r" and r.op != FIND:
            closed.add(r.table)
            rest.append(r)
            continue
        if wave and used + r.n > budget:
            stopped = True
            rest.append(r)
            continue
        v = admit(r)
        if v == WAIT:
            stopped = True
            rest.append(r)
            continue
        if v == REJECT:
            continue
        wave.append(r)
        used += r.n
        took[r.table] = "r" if r.op == FIND else "w"
        if r.op != FIND:
            closed.add(r.table)
    return wave, rest


def test_per_table_queues_match_the_plain_rule():
    """The per-table queues take the same wave, and leave the same requests
    in the same order, as the plain pass over every waiting request."""
    rnd = random.Random(11)
    for trial in range(400):
        nt = rnd.randrange(1, 6)
        spec = [(rnd.randrange(nt), rnd.choice([FIND, FIND, FOP, INSERT]), rnd.randrange(1, 50))
                for _ in range(rnd.randrange(1, 120))]
        budget = rnd.randrange(20, 400)
        verdict = {i: rnd.choice([OK] * 12 + [REJECT, WAIT]) for i in range(len(spec))}
        ref_wave, ref_rest = _reference_wave(reqs(spec), budget, lambda r: verdict[r.rid])
        pq = PendingQueues(reqs(spec))
        wave = pq.form_wave(budget, lambda r: verdict[r.rid])
        assert [r.rid for r in wave] == [r.rid for r in ref_wave]
        assert [r.rid for r in pq.requests()] == [r.rid for r in ref_rest]
        assert len(pq) == len(ref_rest)
    # a table that left a write behind takes none of its later lookups
    p = reqs([(0, FOP, 5), (1, FIND, 3), (1, FOP, 4), (1, FIND, 1), (0, FIND, 1)])
    wave, rest = form_wave(p, 10 ** 9)
    assert [r.rid for r in wave] == [0, 1] and [r.rid for r in rest] == [2, 3, 4]


def test_wave_request_cap():
    """At most max_requests requests join a wave (a fused launch holds one
    entry per request); the rest stay in arrival order."""
    p = reqs([(i % 3, FIND, 1) for i in range(50)])
    pq = PendingQueues(p)
    wave = pq.form_wave(10 ** 9, max_requests=16)
    assert [r.rid for r in wave] == list(range(16))
    assert [r.rid for r in pq.requests()] == list(range(16, 50)) and len(pq) == 34


def test_admission_wait_keeps_arrival_order_and_reject_drops():
    p = reqs([(0, FIND, 10), (1, FOP, 500), (2, FIND, 10), (3, FOP, 7)])
    verdicts = {0: OK, 1: WAIT, 2: OK, 3: OK}
    wave, rest = form_wave(p, 10 ** 9, lambda r: verdicts[r.rid])
    # the request that waits for memory holds back everything behind it
    assert [r.rid for r in wave] == [0] and [r.rid for r in rest] == [1, 2, 3]
    verdicts = {0: OK, 1: REJECT, 2: OK, 3: OK}
    wave, rest = form_wave(p, 10 ** 9, lambda r: verdicts[r.rid])
    assert [r.rid for r in wave] == [0, 2, 3] and rest == []


def test_key_arena_never_overlaps_and_reuses_space():
    from paper_2406_09255_gb300.serve import KeyArena
    rnd = random.Random(1)
    a = KeyArena(100)
    live = {}
    for _ in range(20000):
        if live and rnd.random() < 0.5:
            s = rnd.choice(list(live))
            a.free(s)
            del live[s]
        else:
            n = rnd.randrange(0, 60)
            s = a.alloc(n)
            if s is None or n == 0:
                continue
            assert 0 <= s and s + n <= 100
            for t, m in live.items():
                assert s + n <= t or t + m <= s
            live[s] = n
    for s in list(live):
        a.free(s)
    assert a.used() == 0 and a.alloc(100) == 0
    assert a.alloc(1) is None      # full
    assert a.alloc(101) is None    # larger than the arena


def test_key_arena_waits_for_the_oldest_allocation():
    from paper_2406_09255_gb300.serve import KeyArena
    a = KeyArena(10)
    x, y = a.alloc(6), a.alloc(4)
    assert (x, y) == (0, 6)
    a.free(y)                # freed out of order: space comes back only once
    assert a.alloc(4) is None  # the older allocation x is given back too
    a.free(x)
    assert a.alloc(10) == 0


def test_request_keys_definition():
    """Fresh keys at consecutive indices, re-queries at floor(h * hi / 2^64)
    with h = splitmix64(re_seed, j), misses at consecutive indices when
    nothing was given yet; keys are the key sequence at those indices."""
    from paper_2406_09255_gb300 import workloads as W
    idx = W.request_indices(10, 3, 100, 12345, 777, 1 << 40)
    want = list(range(100, 103)) + [(W.splitmix(777, j) * 12345) >> 64 for j in range(7)]
    assert idx.tolist() == want
    idx = W.request_indices(5, 2, 7, 0, 3, 1000)
    assert idx.tolist() == [7, 8, 1000, 1001, 1002]
    k = W.request_keys(10, 3, 100, 12345, 777, 1 << 40, 48, 99)
    assert k.tolist() == W.keys_at(torch.tensor(want), 48, 99).tolist()


def test_arena_allocation_halves_on_out_of_memory():
    from paper_2406_09255_gb300.serve import alloc_arena
    tried = []

    def fake_alloc(n, dtype, device):
        tried.append(n)
        if n > 1000:
            raise torch.cuda.OutOfMemoryError("fake")
        return torch.empty(n, dtype=dtype, device=device)

    k, st = alloc_arena(8000, "cpu", min_keys=100, alloc=fake_alloc)
    assert k.numel() == st.numel() == 1000 and k.dtype == torch.int64
    assert tried[:4] == [8000, 4000, 2000, 1000]
    try:
        alloc_arena(8000, "cpu", min_keys=4000, alloc=fake_alloc)
        assert False, "below the minimum the error propagates"
    except torch.cuda.OutOfMemoryError:
        pass


def test_deadline_cancels_a_waiting_request():
    """A request still waiting past its deadline is dropped as cancelled
    when it is next considered (the host rule; the GPU test runs it)."""
    from paper_2406_09255_gb300.serve import OK, REJECT, WAIT
    p = reqs([(0, FOP, 10), (1, FIND, 10)])
    p[1].deadline = 0.5
    calls = []

    def admit(r, now=1.0):
        calls.append(r.rid)
        if 0 <= r.deadline < now:
            r.rejected = "cancelled"
            return REJECT
        return OK

    wave, rest = form_wave(p, 10 ** 9, admit)
    assert [r.rid for r in wave] == [0] and rest == [] and p[1].rejected == "cancelled"
