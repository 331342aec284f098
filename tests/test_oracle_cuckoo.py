"""Pins of the oracle's compact cuckoo put (Algorithm 4) and lookup (Section 4.4).

Pinned against set semantics that hold whatever the placement (every inserted
key is found exactly once, absent keys never are, enumerate returns the set,
stored plus dropped keys equal the input), the H = 1 special case that reduces
to a plain bucketed table with a closed-form overflow count, the exhaustive
lookup that ignores the early-stop rule, and brute force on tiny tables.
"""
import numpy as np
import pytest

import oracle

FOUND, PUT, FULL, NOT_FOUND, INVALID = (oracle.FOUND, oracle.PUT, oracle.FULL,
                                        oracle.NOT_FOUND, oracle.INVALID)


def test_single_hash_is_plain_bucketed_table():
    # H = 1: a key can only live in a_0(k); a bucket keeps min(n_b, B) keys and
    # every key past that is lost, whatever C is
    rng = np.random.default_rng(0)
    for C in (1, 5):
        t = oracle.Table(oracle.CUCKOO, 24, 64, fpw0=2, wpb=2, num_hashes=1,
                         max_chain=C, seed=C)
        B = t.slots_per_bucket(0)
        keys = np.unique(rng.integers(1, 1 << 24, 400, dtype=np.uint64))
        rng.shuffle(keys)
        st, dropped = t.insert(keys)
        a = t.perm_many(0, 0, keys)[1].astype(np.int64)
        n_b = np.bincount(a, minlength=64)
        assert (st == FULL).sum() == np.maximum(n_b - B, 0).sum()
        stored = t.enumerate()
        assert len(stored) == np.minimum(n_b, B).sum()
        lost = dropped[st == FULL]
        assert sorted(np.concatenate([stored, lost]).tolist()) == sorted(keys.tolist())


@pytest.mark.parametrize("w,N,fpw", [(32, 14, 3), (40, 12, 1), (24, 8, 3)])
def test_set_semantics_without_full(w, N, fpw):
    rng = np.random.default_rng(w + N)
    t = oracle.Table(oracle.CUCKOO, w, 1 << N, fpw0=fpw, seed=N)
    slots = (1 << N) * 16 * fpw
    keys = np.unique(rng.integers(1, 1 << w, int(0.85 * slots), dtype=np.uint64))
    rng.shuffle(keys)
    st, _ = t.insert(keys)
    assert (st == PUT).all()
    assert sorted(t.enumerate().tolist()) == sorted(keys.tolist())
    assert (t.find(keys) == FOUND).all()
    absent = np.setdiff1d(rng.integers(1, 1 << w, 5000, dtype=np.uint64), keys)
    fa = t.find(absent)
    assert (fa == NOT_FOUND).all()
    # the early stop never cuts a search short
    both = np.concatenate([keys[:5000], absent])
    assert (t.find(both) == t.find_exhaustive(both)).all()
    assert t.check_prefix() == 0
    assert t.check_entries() == 0
    assert t.check_cuckoo_chain() == 0


def test_brute_force_tiny_with_full():
    # 4 buckets of 2 slots, 6-bit keys: every run of a random subset, checked
    # for conservation (stored + dropped = input) and exact lookups
    rng = np.random.default_rng(11)
    allk = np.arange(1, 64, dtype=np.uint64)
    for trial in range(300):
        H = int(rng.integers(1, 4))
        C = int(rng.integers(1, 12))
        t = oracle.Table(oracle.CUCKOO, 6, 4, fpw0=2, wpb=1, num_hashes=H,
                         max_chain=C, seed=trial)
        keys = rng.permutation(allk)[: int(rng.integers(1, 14))]
        st, dropped = t.insert(keys)
        stored = t.enumerate()
        assert len(set(stored.tolist())) == len(stored)  # no duplicates
        lost = dropped[st == FULL]
        assert sorted(np.concatenate([stored, lost]).tolist()) == sorted(keys.tolist())
        members = set(stored.tolist())
        f = t.find(allk)
        assert [s == FOUND for s in f] == [int(k) in members for k in allk]
        assert (f == t.find_exhaustive(allk)).all()
        assert t.check_cuckoo_chain() == 0
        assert t.check_prefix() == 0
        assert t.check_entries() == 0


def test_failure_only_past_achievable_fill():
    # 48-slot buckets (three 21-bit fields per word): the paper reaches fill
    # 0.95 with 16- and 32-slot buckets (Section 5.2), so 0.9 must not fail;
    # at 0.99 with a short chain bound the build must report failures
    rng = np.random.default_rng(5)
    nb = 1 << 10
    slots = nb * 48
    keys = np.unique(rng.integers(1, 1 << 28, int(1.2 * slots), dtype=np.uint64))
    rng.shuffle(keys)
    t = oracle.Table(oracle.CUCKOO, 28, nb, fpw0=3, max_chain=128, seed=1)
    st, _ = t.insert(keys[: int(0.9 * slots)])
    assert (st == PUT).all()
    t = oracle.Table(oracle.CUCKOO, 28, nb, fpw0=3, max_chain=8, seed=1)
    st, dropped = t.insert(keys[: int(0.99 * slots)])
    assert (st == FULL).sum() > 0
    stored = t.enumerate()
    lost = dropped[st == FULL]
    assert sorted(np.concatenate([stored, lost]).tolist()) == sorted(keys[: int(0.99 * slots)].tolist())


def test_probe_and_write_counts():
    # with no evictions every put is one probe and one write; a find of a
    # present key at hash j costs j + 1 probes
    t = oracle.Table(oracle.CUCKOO, 30, 1 << 12, fpw0=3, seed=2)
    keys = np.arange(1, 1001, dtype=np.uint64) * np.uint64(104729)
    st, _ = t.insert(keys)
    assert (st == PUT).all() and t.probes == 1000 and t.writes == 1000
    t.find(keys)
    assert t.probes == 1000


def test_invalid_keys():
    t = oracle.Table(oracle.CUCKOO, 20, 4, fpw0=1, seed=1)
    st, _ = t.insert(np.array([0, 1 << 20, 7], dtype=np.uint64))
    assert list(st) == [INVALID, INVALID, PUT]
    assert list(t.find(np.array([0, 7, 8], dtype=np.uint64))) == [INVALID, FOUND, NOT_FOUND]
