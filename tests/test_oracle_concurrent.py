"""Pins of the host-threaded model of the packed-word claim.

The GPU kernels store several slots in one 64-bit word and claim a slot with
a compare-and-swap of one field (Section 4.5 notes that the atomic
instructions are too coarse for small slots). The oracle's threaded model
runs Algorithm 1 (iceberg find-or-put) and Algorithm 4 (cuckoo put) with the
same claim protocol on many CPU threads at once. Pinned here by:
  - one thread: identical tables and statuses to the sequential oracle
    (a claim on the first empty slot never loses when nobody races);
  - many threads on tiny tables with heavy duplication: Theorem 1 (one PUT
    per distinct key, the rest FOUND; FULL only for keys that are stored
    nowhere), the invariant checkers, and the sequential oracle's stored set
    whenever it reports no FULL;
  - cuckoo: conservation of keys (stored plus dropped = input) and exact
    lookups on the final table.
"""
import numpy as np
import pytest

import oracle

THREADS = 8
ERROR = 5

ICE_GEOMS = [
    # (w, nb0, nb1, wpb, fpw0, fpw1): slots per bucket = wpb * fpw
    (16, 4, 2, 2, 4, 3),   # 16-bit primary fields, 21-bit secondary fields
    (20, 2, 2, 4, 3, 3),   # 21-bit fields at both levels
    (30, 4, 4, 2, 2, 2),   # 32-bit fields
    (40, 2, 2, 2, 1, 1),   # one slot per word
]


def _ice(geom, seed):
    w, nb0, nb1, wpb, f0, f1 = geom
    return oracle.Table(oracle.ICEBERG, w, nb0, nb1, wpb=wpb, fpw0=f0, fpw1=f1, seed=seed)


def _stream(rng, w, distinct, copies):
    keys = np.unique(rng.integers(1, 1 << w, distinct * 2, dtype=np.uint64))[:distinct]
    rng.shuffle(keys)
    s = np.concatenate([keys] * copies)
    rng.shuffle(s)
    return keys, s


@pytest.mark.parametrize("geom", ICE_GEOMS)
def test_one_thread_equals_sequential_oracle(geom):
    rng = np.random.default_rng(sum(geom))
    w, nb0, nb1, wpb, f0, f1 = geom
    slots = nb0 * wpb * f0 + nb1 * wpb * f1
    for trial in range(10):
        _, s = _stream(rng, w, int(1.1 * slots), 2)
        a, b = _ice(geom, trial), _ice(geom, trial)
        st_seq = a.insert(s)
        st_mt, _, ran, fails = b.insert_concurrent(s, 1)
        assert ran == 1 and fails == 0
        assert np.array_equal(st_seq, st_mt)
        assert np.array_equal(a.t0, b.t0) and np.array_equal(a.t1, b.t1)


@pytest.mark.parametrize("fpw,H", [(3, 3), (2, 2), (4, 3)])
def test_one_thread_cuckoo_equals_sequential_oracle(fpw, H):
    rng = np.random.default_rng(fpw * 10 + H)
    w = 14
    for trial in range(10):
        a = oracle.Table(oracle.CUCKOO, w, 8, fpw0=fpw, wpb=2, num_hashes=H, max_chain=16,
                         seed=trial)
        b = oracle.Table(oracle.CUCKOO, w, 8, fpw0=fpw, wpb=2, num_hashes=H, max_chain=16,
                         seed=trial)
        keys = np.unique(rng.integers(1, 1 << w, 16 * 2 * fpw, dtype=np.uint64))
        rng.shuffle(keys)
        st_seq, dr_seq = a.insert(keys)
        st_mt, dr_mt, ran, _ = b.insert_concurrent(keys, 1)
        assert ran == 1
        assert np.array_equal(st_seq, st_mt)
        full = st_seq == oracle.FULL
        assert np.array_equal(dr_seq[full], dr_mt[full])
        assert np.array_equal(a.t0, b.t0)


def _theorem1(t, distinct, s, st):
    assert (st != ERROR).all(), "a bounded retry loop gave up"
    assert t.check_entries() == 0
    assert t.check_prefix() == 0
    assert t.check_order_property() == 0
    assert t.check_duplicates() == 0
    stored = set(int(k) for k in t.enumerate())
    for k in distinct:
        mine = st[s == k]
        n_put = int((mine == oracle.PUT).sum())
        if int(k) in stored:
            # exactly one copy inserted it, every other copy found it
            assert n_put == 1, (int(k), np.bincount(mine))
            assert ((mine == oracle.PUT) | (mine == oracle.FOUND)).all()
        else:
            # a FULL answer means its three buckets were full without it
            assert (mine == oracle.FULL).all(), (int(k), np.bincount(mine))
    return stored


@pytest.mark.parametrize("geom", ICE_GEOMS)
def test_threaded_find_or_put_theorem1(geom):
    rng = np.random.default_rng(7 + sum(geom))
    w, nb0, nb1, wpb, f0, f1 = geom
    slots = nb0 * wpb * f0 + nb1 * wpb * f1
    lost = 0
    trial = 0
    # at least 30 trials, and more (up to 600) until some compare-and-swap
    # has lost a race: on a loaded host the threads of a small trial may not
    # overlap at all
    while trial < 30 or (lost == 0 and trial < 600):
        # below capacity: equal to the sequential oracle's set
        d = int(0.6 * slots)
        distinct, s = _stream(rng, w, d, max(8, 256 // d))
        t = _ice(geom, trial)
        st, _, ran, fails = t.insert_concurrent(s, THREADS)
        lost += fails
        stored = _theorem1(t, distinct, s, st)
        seq = _ice(geom, trial)
        st_seq = seq.insert(s)
        if (st_seq == oracle.FULL).sum() == 0:
            assert stored == set(int(k) for k in distinct)
        # past capacity: FULL keys are stored nowhere, all others exactly once
        distinct, s = _stream(rng, w, int(1.5 * slots), 4)
        t = _ice(geom, 1000 + trial)
        st, _, ran, fails = t.insert_concurrent(s, THREADS)
        lost += fails
        stored = _theorem1(t, distinct, s, st)
        assert len(stored) <= slots
        assert (st == oracle.FULL).sum() > 0
        trial += 1
    assert lost > 0, "no compare-and-swap ever lost a race: the runs did not overlap"


@pytest.mark.parametrize("fpw", [3, 2, 4])
def test_threaded_cuckoo_put_conserves_keys(fpw):
    rng = np.random.default_rng(100 + fpw)
    w, nb = {2: 24, 3: 22, 4: 18}[fpw], 16
    B = 16 * fpw
    lost = 0
    trial = 0
    while trial < 20 or (lost == 0 and trial < 400):
        trial += 1
        t = oracle.Table(oracle.CUCKOO, w, nb, fpw0=fpw, num_hashes=3, max_chain=32,
                         seed=trial)
        fill = 0.8 if trial % 2 else 1.02
        keys = np.unique(rng.integers(1, 1 << w, int(fill * nb * B), dtype=np.uint64))
        rng.shuffle(keys)
        st, dropped, ran, fails = t.insert_concurrent(keys, THREADS)
        lost += fails
        assert (st != ERROR).all()
        assert t.check_entries() == 0 and t.check_prefix() == 0
        assert t.check_cuckoo_chain() == 0 and t.check_duplicates() == 0
        stored = t.enumerate()
        lost_keys = dropped[st == oracle.FULL]
        assert sorted(np.concatenate([stored, lost_keys]).tolist()) == sorted(keys.tolist())
        members = set(stored.tolist())
        f = t.find(keys)
        assert [s == oracle.FOUND for s in f] == [int(k) in members for k in keys]
        if fill > 1:
            assert (st == oracle.FULL).sum() > 0
    assert lost > 0, "no compare-and-swap ever lost a race: the runs did not overlap"
