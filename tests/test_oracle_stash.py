"""Pins of the oracle's iceberg level-3 overflow stash.

Section 2.3 describes a third level for keys whose primary and both
secondary buckets are full; the paper's implementation leaves it out
(Section 3). This library's design: a fixed stash of whole-key slots, an
open-addressing table with linear probing from a hash of the key, reached
only when the three buckets are full. Pinned by:
  - a closed form on one primary and one secondary bucket, where the keys
    overflow in input order: the stash then holds exactly the keys a
    textbook linear-probing table holds after inserting the overflow, at the
    same positions;
  - Theorem 1 on brute-force tiny tables, extended to the stash (one PUT per
    distinct key, FULL only when the stash is full, no duplicates, lookups
    equal membership, the stash invariant checker clean);
  - planted violations for the stash checker;
  - the threaded model with compare-and-swap claims on stash slots.
"""
import numpy as np
import pytest

import oracle
from paper_2406_09255_gb300 import workloads as W

FOUND, PUT, FULL, NOT_FOUND = oracle.FOUND, oracle.PUT, oracle.FULL, oracle.NOT_FOUND


def _home(seed, S, k):
    """Home position restated from its definition: the splitmix64 finaliser
    of k xor output 16 of the seed's splitmix64 sequence, modulo S."""
    return W.mix64(k ^ W.splitmix(seed, 16)) & (S - 1)


def _textbook_linear_probing(keys, S, seed):
    t = [0] * S
    for k in keys:
        p = _home(seed, S, k)
        while t[p]:
            p = (p + 1) % S
        t[p] = k
    return t


@pytest.mark.parametrize("S", [1, 4, 16, 64])
@pytest.mark.parametrize("w,fpw", [(20, (2, 2)), (19, (3, 3)), (20, (1, 1))])
def test_closed_form_single_buckets(S, w, fpw):
    # one primary bucket of B0 slots and one secondary bucket (a_1 = a_2) of
    # B1: the first B0 distinct keys fill the primary, the next B1 the
    # secondary, the next S the stash, the rest are FULL
    wpb = 2
    f0, f1 = fpw
    rng = np.random.default_rng(S * 10 + f0)
    for trial in range(5):
        t = oracle.Table(oracle.ICEBERG, w, 1, 1, wpb=wpb, fpw0=f0, fpw1=f1, seed=trial,
                         stash=S)
        B0, B1 = wpb * f0, wpb * f1
        n = B0 + B1 + S + 7
        keys = np.unique(rng.integers(1, 1 << w, 3 * n, dtype=np.uint64))[:n]
        rng.shuffle(keys)
        st = t.insert(keys)
        cap = B0 + B1 + S
        assert list(st) == [PUT] * cap + [FULL] * (n - cap)
        over = [int(k) for k in keys[B0 + B1: cap]]
        assert t.stash.tolist() == _textbook_linear_probing(over, S, trial)
        assert (t.find(keys[:cap]) == FOUND).all()
        assert (t.find(keys[cap:]) == NOT_FOUND).all()
        assert sorted(t.enumerate().tolist()) == sorted(keys[:cap].tolist())
        assert t.check_stash() == 0 and t.check_order_property() == 0
        assert t.check_duplicates() == 0
        # repeats are found, wherever they live
        assert (t.insert(keys[:cap]) == FOUND).all()
        # slot indices: stash position p is slot B0 + B1 + p
        loc = t.locate(np.array(over, dtype=np.uint64))
        pos = {k: i for i, k in enumerate(t.stash.tolist()) if k}
        assert loc.tolist() == [B0 + B1 + pos[k] for k in over]


def test_without_a_stash_nothing_changes():
    rng = np.random.default_rng(3)
    keys = rng.integers(1, 1 << 16, 400, dtype=np.uint64)
    a = oracle.Table(oracle.ICEBERG, 16, 4, 2, wpb=1, fpw0=2, fpw1=2, seed=4)
    b = oracle.Table(oracle.ICEBERG, 16, 4, 2, wpb=1, fpw0=2, fpw1=2, seed=4, stash=0)
    assert np.array_equal(a.insert(keys), b.insert(keys))
    assert np.array_equal(a.t1, b.t1)


TINY = [
    # (w, nb0, nb1, wpb, fpw0, fpw1, stash)
    (8, 1, 2, 1, 2, 1, 2),
    (8, 2, 2, 1, 3, 1, 4),
    (10, 2, 4, 2, 2, 1, 1),
    (9, 1, 1, 1, 2, 2, 8),
]


@pytest.mark.parametrize("geom", TINY)
def test_theorem1_with_stash_brute_force(geom):
    w, nb0, nb1, wpb, f0, f1, S = geom
    rng = np.random.default_rng(sum(geom))
    slots = nb0 * wpb * f0 + nb1 * wpb * f1
    for trial in range(200):
        t = oracle.Table(oracle.ICEBERG, w, nb0, nb1, wpb=wpb, fpw0=f0, fpw1=f1,
                         seed=trial, stash=S)
        distinct = np.unique(rng.integers(1, 1 << w, rng.integers(1, slots + S + 6),
                                          dtype=np.uint64))
        keys = np.concatenate([distinct, distinct[rng.integers(0, len(distinct), len(distinct))]])
        rng.shuffle(keys)
        st = t.insert(keys)
        stored = set(int(k) for k in t.enumerate())
        assert t.check_entries() == 0 and t.check_order_property() == 0
        assert t.check_prefix() == 0 and t.check_stash() == 0 and t.check_duplicates() == 0
        for k in distinct:
            mine = st[keys == k]
            if int(k) in stored:
                assert (mine == PUT).sum() == 1 and ((mine == PUT) | (mine == FOUND)).all()
            else:
                assert (mine == FULL).all()
        if (st == FULL).any():
            assert (t.stash != 0).all(), "FULL only once the stash is full"
        allk = np.arange(1, 1 << w, dtype=np.uint64)
        f = t.find(allk)
        assert [s == FOUND for s in f] == [int(k) in stored for k in allk]


def _ice_full_buckets(S=4):
    """A table whose single primary and single secondary bucket are full of
    keys 1..B0+B1, plus the next keys for the stash."""
    t = oracle.Table(oracle.ICEBERG, 12, 1, 1, wpb=1, fpw0=2, fpw1=2, seed=1, stash=S)
    keys = np.arange(1, 5, dtype=np.uint64)
    assert (t.insert(keys) == PUT).all()
    return t


def test_stash_checker_counts_planted_violations():
    t = _ice_full_buckets()
    k = 100
    p = t.stash_home(k)
    t.stash[p] = k
    assert t.check_stash() == 0
    # a gap between home and position
    t.stash[p] = 0
    t.stash[(p + 1) % 4] = k
    assert t.check_stash() == 1
    t.stash[(p + 1) % 4] = 0
    # a key whose buckets are not full
    t2 = oracle.Table(oracle.ICEBERG, 12, 1, 1, wpb=1, fpw0=2, fpw1=2, seed=1, stash=4)
    t2.stash[t2.stash_home(k)] = k
    assert t2.check_stash() == 1
    # a key that is also in a bucket
    t.stash[t.stash_home(3)] = 3
    assert t.check_stash() == 1 and t.check_duplicates() == 1


def test_stash_find_stops_at_the_first_empty_position():
    t = _ice_full_buckets(S=8)
    over = [200, 201, 202]
    assert (t.insert(np.array(over, dtype=np.uint64)) == PUT).all()
    absent = np.arange(300, 400, dtype=np.uint64)
    assert (t.find(absent) == NOT_FOUND).all()
    assert (t.find(np.array(over, dtype=np.uint64)) == FOUND).all()


@pytest.mark.parametrize("geom", TINY)
def test_threaded_model_with_stash(geom):
    w, nb0, nb1, wpb, f0, f1, S = geom
    rng = np.random.default_rng(50 + sum(geom))
    slots = nb0 * wpb * f0 + nb1 * wpb * f1
    for trial in range(40):
        t = oracle.Table(oracle.ICEBERG, w, nb0, nb1, wpb=wpb, fpw0=f0, fpw1=f1,
                         seed=trial, stash=S)
        distinct = np.unique(rng.integers(1, 1 << w, slots + S + 4, dtype=np.uint64))
        keys = np.concatenate([distinct] * 6)
        rng.shuffle(keys)
        st, _, ran, fails = t.insert_concurrent(keys, 8)
        assert (st != 5).all()
        stored = set(int(k) for k in t.enumerate())
        assert t.check_stash() == 0 and t.check_order_property() == 0
        assert t.check_duplicates() == 0 and t.check_prefix() == 0
        for k in distinct:
            mine = st[keys == k]
            if int(k) in stored:
                assert (mine == PUT).sum() == 1 and ((mine == PUT) | (mine == FOUND)).all()
            else:
                assert (mine == FULL).all()
