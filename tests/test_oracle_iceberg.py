"""Pins of the oracle's iceberg find-or-put (Algorithm 5) and lookup.

Pinned against (1) the worked ranks of the slot-ordering figure, (2) an
independent restatement of Algorithm 1 (two loops, least-full choice, slot
counts) which the appendix states is indistinguishable from Algorithm 5 when
run sequentially, and (3) Theorem 1 (a)-(e) checked on every input order of
small key multisets over tiny tables.
"""
import itertools

import numpy as np
import pytest

import oracle
from conftest import read_golden

FOUND, PUT, FULL, NOT_FOUND, INVALID = (oracle.FOUND, oracle.PUT, oracle.FULL,
                                        oracle.NOT_FOUND, oracle.INVALID)


def test_prec_matches_figure_ranks():
    rows = [(int(x), int(y), int(r)) for x, y, r in read_golden("slot_order_fig.txt")]
    B0, B1 = 3, 2
    S = [(0, y) for y in range(B0)] + [(x, y) for x in (1, 2) for y in range(B1)]
    # rank of each slot = 1 + number of slots that precede it
    rank = {s: 1 + sum(oracle.prec(*t, *s) for t in S if t != s) for s in S}
    assert {(x, y): r for x, y, r in rows} == rank


@pytest.mark.parametrize("B0,B1", [(3, 2), (4, 4), (1, 3), (8, 2)])
def test_prec_is_strict_total_order(B0, B1):
    S = [(0, y) for y in range(B0)] + [(x, y) for x in (1, 2) for y in range(B1)]
    for a in S:
        assert not oracle.prec(*a, *a)
        for b in S:
            if a != b:
                assert oracle.prec(*a, *b) != oracle.prec(*b, *a)
            for c in S:
                if oracle.prec(*a, *b) and oracle.prec(*b, *c):
                    assert oracle.prec(*a, *c)


class Alg1Model:
    """Algorithm 1 restated on python lists: level-1 loop, then the level-2
    loop that checks both secondaries and takes the strictly-less-full one
    (ties to the second). Entries are (x, key) pairs; a write only succeeds on
    an empty slot (the CAS). Uses the oracle only for a_x(k)."""

    def __init__(self, t: oracle.Table):
        self.t = t
        c = t.cfg
        self.T0 = [[None] * t.slots_per_bucket(0) for _ in range(c.nb[0])]
        self.T1 = [[None] * t.slots_per_bucket(1) for _ in range(c.nb[1])]

    def fop(self, k):
        t = self.t
        a0, a1, a2 = t.address(0, 0, k), t.address(1, 0, k), t.address(1, 1, k)
        while True:  # level 1
            b = list(self.T0[a0])
            if (0, k) in b:
                return FOUND
            if all(s is not None for s in b):
                break
            i = b.index(None)
            if self.T0[a0][i] is None:
                self.T0[a0][i] = (0, k)
                return PUT
        while True:  # level 2
            b1 = list(self.T1[a1])
            if (1, k) in b1:
                return FOUND
            b2 = list(self.T1[a2])
            if (2, k) in b2:
                return FOUND
            load1 = sum(s is not None for s in b1)
            load2 = sum(s is not None for s in b2)
            i = 1 if load1 < load2 else 2
            b, row = (b1, self.T1[a1]) if i == 1 else (b2, self.T1[a2])
            if all(s is not None for s in b):
                return FULL
            j = b.index(None)
            if row[j] is None:
                row[j] = (i, k)
                return PUT

    def expected_slot(self, x_level, entry):
        """Slot bits of the documented encoding for a model entry."""
        if entry is None:
            return 0
        x, k = entry
        t = self.t
        if x == 0:
            return (t.remainder(0, 0, k) << 1) | 1
        return (t.remainder(1, x - 1, k) << 2) | x


def _assert_same_table(model, t):
    c = t.cfg
    for a in range(c.nb[0]):
        for y in range(t.slots_per_bucket(0)):
            assert t.slot(0, a, y) == model.expected_slot(0, model.T0[a][y]), (0, a, y)
    for a in range(c.nb[1]):
        for y in range(t.slots_per_bucket(1)):
            assert t.slot(1, a, y) == model.expected_slot(1, model.T1[a][y]), (1, a, y)


TINY = [
    # (w, nb0, nb1, wpb, fpw0, fpw1): slots per bucket = wpb * fpw
    (8, 1, 2, 1, 2, 1),   # one primary bucket of 2, two secondaries of 1
    (8, 2, 2, 1, 3, 1),   # 2 x 3 primary, 2 x 1 secondary
    (10, 2, 4, 2, 2, 1),  # 2 x 4 primary, 4 x 2 secondary
    (9, 1, 1, 1, 2, 2),   # a single secondary bucket: a_1 = a_2 always
]


@pytest.mark.parametrize("geom", TINY)
def test_alg5_equals_alg1_sequentially(geom):
    w, nb0, nb1, wpb, f0, f1 = geom
    rng = np.random.default_rng(sum(geom))
    for trial in range(40):
        t = oracle.Table(oracle.ICEBERG, w, nb0, nb1, wpb=wpb, fpw0=f0, fpw1=f1,
                         seed=trial * 31 + 5)
        m = Alg1Model(t)
        keys = rng.integers(1, 1 << w, rng.integers(1, 24), dtype=np.uint64)
        keys = np.concatenate([keys, keys[rng.integers(0, len(keys), len(keys))]])
        rng.shuffle(keys)
        got = t.insert(keys)
        want = [m.fop(int(k)) for k in keys]
        assert list(got) == want
        _assert_same_table(m, t)


def _theorem1_checks(t, keys, st):
    """Theorem 1 for a sequential composition, plus the no-duplicates lemma."""
    stored = t.enumerate()
    stored_set = set(int(k) for k in stored)
    # (a) well-formed: valid entries, order property, no duplicates
    assert t.check_entries() == 0
    assert t.check_order_property() == 0
    assert len(stored_set) == len(stored)
    assert t.check_prefix() == 0
    seen_put = {}
    for k, s in zip(keys, st):
        k = int(k)
        # (b) every call returns found, full or put
        assert s in (FOUND, FULL, PUT)
        # (c) found/put iff k is in the table afterwards
        assert (s in (FOUND, PUT)) == (k in stored_set)
        # (d) put iff this call inserted k: exactly one put per stored key,
        #     and it comes before any found of that key
        if s == PUT:
            assert k not in seen_put
            seen_put[k] = True
        if s == FOUND:
            assert k in seen_put
    assert set(seen_put) == stored_set
    # (e) full: all three buckets are full and lack k
    for k, s in zip(keys, st):
        if s == FULL:
            k = int(k)
            assert k not in stored_set
            for x in range(3):
                lvl, j = (0, 0) if x == 0 else (1, x - 1)
                a = t.address(lvl, j, k)
                for y in range(t.slots_per_bucket(lvl)):
                    assert t.slot(lvl, a, y) != 0


@pytest.mark.parametrize("geom", TINY[:3])
def test_theorem1_all_orders_tiny(geom):
    w, nb0, nb1, wpb, f0, f1 = geom
    rng = np.random.default_rng(7)
    for trial in range(6):
        base = [int(k) for k in rng.integers(1, 1 << w, 4, dtype=np.uint64)]
        multiset = base + [base[0], base[1]]
        for order in set(itertools.permutations(multiset)):
            t = oracle.Table(oracle.ICEBERG, w, nb0, nb1, wpb=wpb, fpw0=f0, fpw1=f1,
                             seed=trial)
            st = t.insert(np.array(order, dtype=np.uint64))
            _theorem1_checks(t, order, st)
            # lookups agree with membership
            probe = np.array(sorted(set(order)) + [int(k) for k in
                             rng.integers(1, 1 << w, 4, dtype=np.uint64)], dtype=np.uint64)
            members = set(int(k) for k in t.enumerate())
            f = t.find(probe)
            assert [s == FOUND for s in f] == [int(k) in members for k in probe]


def test_theorem1_at_scale_with_full():
    # 32-slot primary buckets, 32-slot secondary buckets (two 32-bit fields
    # per word), driven past capacity so FULL occurs
    rng = np.random.default_rng(3)
    t = oracle.Table(oracle.ICEBERG, 36, 1 << 8, 1 << 5, fpw0=2, fpw1=1, seed=17)
    cap = (1 << 8) * 32 + (1 << 5) * 16
    fresh = rng.integers(1, 1 << 36, int(cap * 1.05), dtype=np.uint64)
    keys = np.concatenate([fresh, fresh[rng.integers(0, len(fresh), len(fresh) // 2)]])
    rng.shuffle(keys)
    st = t.insert(keys)
    assert (st == FULL).sum() > 0
    _theorem1_checks(t, keys, st)


def test_no_full_below_capacity_and_probe_counts():
    # Section 5.2: two-level tables with 32-slot primary buckets fill to ~0.9
    rng = np.random.default_rng(4)
    nb0, nb1 = 1 << 10, 1 << 7
    t = oracle.Table(oracle.ICEBERG, 40, nb0, nb1, fpw0=2, fpw1=1, seed=5)
    slots = nb0 * 32 + nb1 * 16
    keys = rng.integers(1, 1 << 40, int(0.85 * slots), dtype=np.uint64)
    st = t.insert(keys)
    assert (st == PUT).all()
    # probes: 1 per op decided by the primary, 3 for each spill to level 2
    spilled = t.probes - len(keys)
    assert spilled % 2 == 0
    primary_count = sum(1 for a in range(nb0) for y in range(t.slots_per_bucket(0)) if t.slot(0, a, y))
    assert len(keys) - spilled // 2 == primary_count


def test_invalid_keys():
    t = oracle.Table(oracle.ICEBERG, 20, 4, 2, fpw0=2, fpw1=2, seed=1)
    st = t.insert(np.array([0, 1 << 20, 5, (1 << 20) - 1], dtype=np.uint64))
    assert list(st) == [INVALID, INVALID, PUT, PUT]
    assert list(t.find(np.array([0, 5, 1 << 21], dtype=np.uint64))) == [INVALID, FOUND, INVALID]


@pytest.mark.parametrize("wpb,f0,f1", [(16, 2, 2), (4, 3, 1), (2, 4, 2)])
def test_locate_closed_form_single_buckets(wpb, f0, f1):
    """Slot index (the key-value extension's handle), pinned by a closed form:
    with one primary and one secondary bucket, sequential puts fill the
    primary's slots in slot order (first empty slot, Algorithm 1), so the i-th
    key sits at slot i; the next B1 keys go to the one secondary bucket, whose
    slots follow the primary level's B0 slots. Keys past B0 + B1 are FULL and
    located nowhere."""
    w = 15  # remainders of 15 bits fit every packing here, 16-bit slots included
    t = oracle.Table(oracle.ICEBERG, w, 1, 1, wpb=wpb, fpw0=f0, fpw1=f1, seed=5)
    B0, B1 = t.slots_per_bucket(0), t.slots_per_bucket(1)
    assert B0 == wpb * f0 and B1 == wpb * f1
    keys = np.arange(1, B0 + B1 + 4, dtype=np.uint64) * np.uint64(211)
    assert int(keys.max()) < (1 << w)
    st = t.find_or_put(keys)
    assert (st[: B0 + B1] == oracle.PUT).all() and (st[B0 + B1:] == oracle.FULL).all()
    got = t.locate(keys)
    want = np.concatenate([np.arange(B0 + B1, dtype=np.uint64),
                           np.full(3, np.iinfo(np.uint64).max, dtype=np.uint64)])
    assert np.array_equal(got, want)
    # the located slot holds the key's own entry: r'_0 at level 0, r'_{1+i} at level 1
    for k, s in zip(keys[: B0 + B1].tolist(), got[: B0 + B1].tolist()):
        if s < B0:
            assert t.slot(0, 0, s) == (t.remainder(0, 0, k) << 1) | 1
        else:
            e = t.slot(1, 0, s - B0)
            i = (e & 3) - 1
            assert e >> 2 == t.remainder(1, i, k)


def test_locate_bucket_offsets():
    """Level-0 slot indices are a * B0 + y for the key's primary bucket a;
    absent and invalid keys locate to 2^64 - 1."""
    w = 32
    t = oracle.Table(oracle.ICEBERG, w, 1 << 6, 1 << 3, fpw0=2, fpw1=2, seed=9)
    B0 = t.slots_per_bucket(0)
    keys = np.arange(1, 400, dtype=np.uint64) * np.uint64(104729)
    assert (t.find_or_put(keys) == oracle.PUT).all()
    got = t.locate(keys)
    for k, s in zip(keys.tolist(), got.tolist()):
        a = t.address(0, 0, k)
        assert a * B0 <= s < (a + 1) * B0  # nothing spilled at this load
    absent = t.locate(np.array([0, 3, 1 << 40], dtype=np.uint64))
    assert (absent == np.iinfo(np.uint64).max).all()
