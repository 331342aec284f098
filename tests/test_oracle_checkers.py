"""Pins of the oracle's invariant checkers.

Every GPU claim about concurrent runs (Theorem 1 (a): well-formed tables; the
prefix property of Section 3; the cuckoo chain of Section 4.4; no key held
twice) rests on these checkers returning 0 on a device dump. A checker that
always returned 0 would pass every such test, so here each checker is given
tables built by hand that break exactly one invariant a known number of
times, and must return exactly that count; the same table without the planted
fault must give 0.

Counts: prefix = buckets with a filled slot after an empty one; entries =
stored fields that do not decode to a valid key of their bucket and tag;
order property = stored entries with a preceding slot (Definition 1) that is
empty or holds the same key; cuckoo chain = entries under hash j with one of
a_0 .. a_{j-1} not full; duplicates = stored entries minus distinct keys.
"""
import numpy as np
import pytest

import oracle

ICE = dict(kind=oracle.ICEBERG, key_bits=8, nb0=1, nb1=2, wpb=1, fpw0=2, fpw1=2)
CUC = dict(kind=oracle.CUCKOO, key_bits=8, nb0=4, wpb=1, fpw0=2, num_hashes=3)


def _table(spec, seed=3, **kw):
    s = dict(spec)
    s.update(kw)
    kind, w, nb0 = s.pop("kind"), s.pop("key_bits"), s.pop("nb0")
    nb1 = s.pop("nb1", 0)
    return oracle.Table(kind, w, nb0, nb1, seed=seed, **s)


def _keys(w):
    return range(1, 1 << w)


def _put(t, x, k, y):
    """Store key k's entry for choice x at slot y of its bucket."""
    level = 0 if (t.cfg.kind == oracle.CUCKOO or x == 0) else 1
    t.set_slot(level, t.bucket_of(x, k), y, t.entry_of(x, k))


def _clean(t):
    """Every checker on a table that should be well formed."""
    assert t.check_prefix() == 0
    assert t.check_entries() == 0
    assert t.check_duplicates() == 0
    if t.cfg.kind == oracle.ICEBERG:
        assert t.check_order_property() == 0
    else:
        assert t.check_cuckoo_chain() == 0


# ---------------------------------------------------------------------------
# prefix
# ---------------------------------------------------------------------------
def test_prefix_counts_buckets_with_gaps():
    # 4 buckets of 4 slots; slot contents only need to be nonzero
    t = _table(CUC, nb0=4, wpb=2, fpw0=2)
    assert t.slots_per_bucket(0) == 4
    t.set_slot(0, 0, 0, 5)
    t.set_slot(0, 0, 1, 6)                 # [x x . .] fine
    assert t.check_prefix() == 0
    t.set_slot(0, 1, 0, 5)
    t.set_slot(0, 1, 2, 6)
    t.set_slot(0, 1, 3, 7)                 # [x . x x]: one bucket, two late slots
    assert t.check_prefix() == 1
    t.set_slot(0, 2, 3, 9)                 # [. . . x]
    assert t.check_prefix() == 2
    t.set_slot(0, 1, 1, 4)                 # bucket 1 repaired: [x x x x]
    assert t.check_prefix() == 1


def test_prefix_reaches_the_secondary_level():
    t = _table(ICE)
    t.set_slot(1, 1, 1, 3)                 # secondary bucket 1: [. x]
    assert t.check_prefix_level(0) == 0
    assert t.check_prefix_level(1) == 1
    assert t.check_prefix() == 1
    t.set_slot(0, 0, 1, 3)                 # primary: [. x]
    assert t.check_prefix_level(0) == 1
    assert t.check_prefix() == 2


# ---------------------------------------------------------------------------
# entries
# ---------------------------------------------------------------------------
def test_entries_cuckoo_tags():
    t = _table(CUC, num_hashes=2)
    k1 = 11
    k2 = next(k for k in _keys(8) if k != k1 and t.bucket_of(1, k) != t.bucket_of(0, k1))
    _put(t, 0, k1, 0)
    _put(t, 1, k2, 0)
    assert t.check_entries() == 0
    # tag 0 with a nonzero body: no hash index
    a = t.bucket_of(0, k1)
    e = t.slot(0, a, 0)
    assert e >> 2, "needs a nonzero remainder"
    t.set_slot(0, a, 0, e & ~3)
    assert t.check_entries() == 1
    # tag 3 = hash index 2, outside H = 2
    b = t.bucket_of(1, k2)
    t.set_slot(0, b, 0, t.slot(0, b, 0) | 3)
    assert t.check_entries() == 2


def test_entries_whole_key_in_the_wrong_bucket():
    t = _table(CUC, compact=False)
    k = next(k for k in _keys(8) if t.bucket_of(0, k) == 1)
    _put(t, 0, k, 0)
    assert t.check_entries() == 0
    t.set_slot(0, 1, 0, 0)
    t.set_slot(0, 2, 0, t.entry_of(0, k))  # the same field, another bucket
    assert t.check_entries() == 1


def test_entries_iceberg_flags_and_tags():
    t = _table(ICE)
    p = next(k for k in _keys(8) if t.entry_of(0, k) >> 1)
    _put(t, 0, p, 0)
    q = next(k for k in _keys(8) if k != p)
    _put(t, 2, q, 0)
    assert t.check_entries() == 0
    # primary entry without its occupancy bit
    t.set_slot(0, 0, 0, t.entry_of(0, p) & ~1)
    assert t.check_entries() == 1
    # secondary entry with tag 3 (no such choice): only the secondary level has it
    b = t.bucket_of(2, q)
    t.set_slot(1, b, 0, t.entry_of(2, q) | 3)
    assert t.check_entries() == 2
    t.set_slot(0, 0, 0, t.entry_of(0, p))  # repair the primary
    assert t.check_entries() == 1
    t.set_slot(1, b, 0, t.entry_of(2, q) & ~3)  # tag 0
    assert t.check_entries() == 1


def test_entries_whole_key_iceberg_secondary_in_the_wrong_bucket():
    t = _table(ICE, compact=False)
    k = next(k for k in _keys(8) if t.bucket_of(1, k) == 0)
    t.set_slot(1, 1, 0, t.entry_of(1, k))
    assert t.check_entries() == 1
    t.set_slot(1, 1, 0, 0)
    t.set_slot(1, 0, 0, t.entry_of(1, k))
    assert t.check_entries() == 0


# ---------------------------------------------------------------------------
# order property (Definition 1, Appendix A) and duplicates
# ---------------------------------------------------------------------------
def _ice_parts(t):
    """Two keys p1, p2 that fill the single primary bucket, and the keys whose
    two secondary choices are different buckets, by choice-1 bucket."""
    allk = list(_keys(8))
    split = [k for k in allk if t.bucket_of(1, k) != t.bucket_of(2, k)]
    p1, p2 = allk[-1], allk[-2]
    return p1, p2, split


def test_order_secondary_while_primary_has_room():
    t = _table(ICE)
    p1, p2, split = _ice_parts(t)
    k = next(k for k in split if k not in (p1, p2))
    _put(t, 0, p1, 0)
    _put(t, 2, k, 0)                        # (0, 1) is still empty
    assert t.check_order_property() == 1
    _put(t, 0, p2, 1)                       # fill the primary
    _clean(t)


def test_order_ties_go_to_the_second_choice():
    t = _table(ICE)
    p1, p2, split = _ice_parts(t)
    k = next(k for k in split if k not in (p1, p2))
    _put(t, 0, p1, 0)
    _put(t, 0, p2, 1)
    # (2, 0) precedes (1, 0): k at choice 1 slot 0 with its choice-2 bucket empty
    _put(t, 1, k, 0)
    assert t.check_order_property() == 1
    # the mirror placement is the correct one
    t.set_slot(1, t.bucket_of(1, k), 0, 0)
    _put(t, 2, k, 0)
    _clean(t)


def test_order_earlier_secondary_slot_empty():
    t = _table(ICE)
    p1, p2, split = _ice_parts(t)
    _put(t, 0, p1, 0)
    _put(t, 0, p2, 1)
    # k at (1, 1) on top of q at (2, 0) of the same bucket; k's choice-2
    # bucket is the other one and empty, and (2, 0), (2, 1) precede (1, 1)
    k, q = next((k, q) for k in split for q in split
                if len({k, q, p1, p2}) == 4 and t.bucket_of(2, q) == t.bucket_of(1, k))
    _put(t, 2, q, 0)
    _clean(t)
    _put(t, 1, k, 1)
    assert t.check_order_property() == 1
    assert t.check_prefix() == 0
    # a second, independent violation adds one: k2 at (2, 1) of the empty
    # bucket, whose slot (2, 0) precedes it (this also breaks the prefix)
    k2 = next(x for x in split if x not in (k, q, p1, p2)
              and t.bucket_of(2, x) != t.bucket_of(1, k))
    b = t.bucket_of(2, k2)
    assert t.slot(1, b, 0) == 0
    t.set_slot(1, b, 1, t.entry_of(2, k2))
    assert t.check_order_property() == 2
    assert t.check_prefix() == 1


def test_order_and_duplicates_catch_a_key_stored_twice():
    t = _table(ICE)
    p1, p2, split = _ice_parts(t)
    _put(t, 0, p1, 0)
    _put(t, 0, p2, 1)
    _clean(t)
    # p1 again in a secondary bucket: its primary entry precedes every
    # secondary slot, so the second copy violates the order property
    _put(t, 2, p1, 0)
    assert t.check_order_property() == 1
    assert t.check_duplicates() == 1
    assert t.check_entries() == 0


def _stored(t):
    """(level, bucket, slot, key) of every stored entry, in the order the
    oracle's enumeration walks them (level by level, bucket by bucket)."""
    pos = []
    levels = ((0, t.cfg.nb[0]), (1, t.cfg.nb[1])) if t.cfg.kind == oracle.ICEBERG \
        else ((0, t.cfg.nb[0]),)
    for level, nb in levels:
        for a in range(nb):
            for y in range(t.slots_per_bucket(level)):
                if t.slot(level, a, y):
                    pos.append((level, a, y))
    keys = [int(k) for k in t.enumerate()]
    assert len(keys) == len(pos)
    return [p + (k,) for p, k in zip(pos, keys)]


def test_order_property_counts_each_violating_entry():
    # a table filled by the oracle is clean; clearing the last slot of a full
    # primary bucket turns every secondary entry whose primary it is into a
    # violation (that primary now has room), and nothing else
    t = oracle.Table(oracle.ICEBERG, 12, 2, 4, wpb=1, fpw0=2, fpw1=2, seed=9)
    rng = np.random.default_rng(1)
    keys = np.unique(rng.integers(1, 1 << 12, 60, dtype=np.uint64))
    t.insert(keys)
    _clean(t)
    sec = [(a, k) for level, a, y, k in _stored(t) if level == 1]
    assert t.slot(0, 0, 1) != 0, "primary bucket 0 should be full"
    expect = sum(1 for a, k in sec if t.bucket_of(0, k) == 0)
    assert expect > 0
    t.set_slot(0, 0, 1, 0)
    assert t.check_order_property() == expect


# ---------------------------------------------------------------------------
# cuckoo chain (Section 4.4) and duplicates
# ---------------------------------------------------------------------------
def _cuckoo_pick(t):
    """k with a_0, a_1, a_2 distinct, and fillers f1, f2 with a_0 = a_0(k)."""
    allk = list(_keys(8))
    for k in allk:
        a = [t.bucket_of(j, k) for j in range(3)]
        if len(set(a)) < 3:
            continue
        f = [x for x in allk if x != k and t.bucket_of(0, x) == a[0]]
        g = [x for x in allk if x not in [k] + f[:2] and t.bucket_of(0, x) == a[1]]
        if len(f) >= 2 and len(g) >= 2:
            return k, f[:2], g[:2]
    raise AssertionError("no key with three distinct buckets")


def test_chain_entry_under_second_hash_with_room_before():
    t = _table(CUC)
    k, f, g = _cuckoo_pick(t)
    _put(t, 1, k, 0)                        # a_0(k) is empty
    assert t.check_cuckoo_chain() == 1
    _put(t, 0, f[0], 0)
    assert t.check_cuckoo_chain() == 1      # a_0(k) still has a free slot
    _put(t, 0, f[1], 1)                     # a_0(k) full
    _clean(t)                               # a_1(k) itself may have room


def test_chain_entry_under_third_hash():
    t = _table(CUC)
    k, f, g = _cuckoo_pick(t)
    _put(t, 0, f[0], 0)
    _put(t, 0, f[1], 1)                     # a_0(k) full
    _put(t, 2, k, 0)                        # a_1(k) empty
    assert t.check_cuckoo_chain() == 1
    _put(t, 0, g[0], 0)
    _put(t, 0, g[1], 1)                     # a_1(k) full
    _clean(t)


def test_cuckoo_duplicates():
    t = _table(CUC)
    k, f, g = _cuckoo_pick(t)
    _put(t, 0, k, 0)
    _put(t, 0, f[0], 1)                     # a_0(k) = {k, f0}: full
    _clean(t)
    _put(t, 1, k, 0)                        # k again under hash 1
    assert t.check_duplicates() == 1
    assert t.check_cuckoo_chain() == 0
    _put(t, 2, k, 0)                        # and under hash 2
    assert t.check_duplicates() == 2


def test_duplicates_of_the_smallest_and_only_key():
    t = _table(CUC)
    k = next(k for k in _keys(8) if t.bucket_of(0, k) != t.bucket_of(1, k))
    _put(t, 0, k, 0)
    assert t.check_duplicates() == 0
    _put(t, 1, k, 0)
    assert t.check_duplicates() == 1
    t2 = _table(ICE)
    _put(t2, 0, 1, 0)
    _put(t2, 2, 1, 0)
    _put(t2, 0, 2, 1)
    assert t2.check_duplicates() == 1


# ---------------------------------------------------------------------------
# the order property against a plain restatement, on perturbed tables
# ---------------------------------------------------------------------------
def _order_violations(t):
    """Definition 1 read directly: for every stored entry at (x, y) of key k,
    some slot (x2, y2) preceding it in k's three buckets is empty or holds
    k's own entry for x2."""
    B = [t.slots_per_bucket(0), t.slots_per_bucket(1), t.slots_per_bucket(1)]
    bad = 0
    for level, a, y, k in _stored(t):
        e = t.slot(level, a, y)
        x = 0 if level == 0 else (e & 3)
        for x2, y2 in [(xx, v) for xx in range(3) for v in range(B[xx])]:
            if not oracle.prec(x2, y2, x, y):
                continue
            s = t.slot(0 if x2 == 0 else 1, t.bucket_of(x2, k), y2)
            if s == 0 or s == t.entry_of(x2, k):
                bad += 1
                break
    return bad


@pytest.mark.parametrize("seed", range(6))
def test_order_property_matches_definition_on_perturbed_tables(seed):
    rng = np.random.default_rng(seed)
    t = oracle.Table(oracle.ICEBERG, 12, 2, 4, wpb=1, fpw0=2, fpw1=2, seed=seed)
    keys = np.unique(rng.integers(1, 1 << 12, 40, dtype=np.uint64))
    t.insert(keys)
    assert _order_violations(t) == 0 == t.check_order_property()
    for _ in range(4):
        # clear a random filled slot (entries stay valid; the order may break)
        filled = [(lv, a, y) for lv, nb in ((0, 2), (1, 4)) for a in range(nb)
                  for y in range(2) if t.slot(lv, a, y)]
        lv, a, y = filled[rng.integers(len(filled))]
        t.set_slot(lv, a, y, 0)
        assert t.check_order_property() == _order_violations(t)
