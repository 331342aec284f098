"""The served loop's wave formation (host logic, no GPU): per table a run of
consecutive lookups or one write, admission order kept per table, the key
budget respected, and every request eventually served."""
import random

from paper_2406_09255_gb300.serve import FIND, FOP, INSERT, Request, form_wave


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
