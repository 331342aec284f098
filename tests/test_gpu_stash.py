"""GPU parity of the iceberg level-3 overflow stash (Section 2.3's third
level; this library's design: whole-key slots with linear probing, claimed by
compare-and-swap, reached only when a key's three buckets are full), through
the C ABI against the oracle.

- single-tile ordered runs: statuses and every word of the table, stash
  included, equal to the oracle's;
- concurrent runs with a stash large enough for every overflowing key: one
  PUT per distinct key, the oracle's stored set, a well-formed dump (stash
  invariant included), lookups equal to the oracle's on the GPU's own table;
- concurrent runs past the stash: FULL keys are stored nowhere and only
  once every stash slot is taken;
- slot indices of stash keys and the fused multi-table launch.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_09255_gb300 import workloads as W

from test_gpu_parity import DEV, cht, dev_keys, dump_into, level1_words, mirror, u64, words

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


GEOMS = [
    # (key_bits, key_bytes, log2 primary, log2 backyard, fpw0, fpw1, stash slots)
    (32, 4, 3, 1, 2, 1, 64),
    (40, 8, 3, 1, 1, 1, 32),
    (18, 4, 3, 1, 4, 2, 128),
]


def _stream(t, w, over, seed):
    """Distinct keys up to `over` times the two-level slots, with repeats."""
    c = t.cfg
    two_level = c.num_buckets * 16 * c.fields_per_word + \
        c.num_buckets_backyard * 16 * c.fields_per_word_backyard
    fresh = W.unique_keys(0, int(over * two_level), w, seed)
    rng = np.random.default_rng(seed)
    dup = fresh[torch.from_numpy(rng.integers(0, len(fresh), len(fresh) // 2))]
    keys = torch.cat([fresh, dup])
    return fresh, keys[torch.from_numpy(rng.permutation(len(keys)))]


@pytest.mark.parametrize("T", [4, 8])
@pytest.mark.parametrize("geom", GEOMS)
def test_sequential_stash_bit_exact(T, geom):
    w, kb, N0, N1, f0, f1, S = geom
    P = cht()
    t = P.Table(P.ICEBERG, w, 1 << N0, 1 << N1, key_bytes=kb, fields_per_word=f0,
                fields_per_word_backyard=f1, stash_slots=S, seed=31 + N0, tile=T,
                items_per_thread=2, max_tiles=1, cta_threads=64)
    o = mirror(t)
    fresh, keys = _stream(t, w, 1.25, 5 + T)
    st = t.find_or_put(dev_keys(keys, kb)).cpu().numpy()
    ost = o.insert(keys.numpy().astype(np.uint64))
    assert (st == ost).all()
    assert (o.stash != 0).sum() > 0, "the run should reach the stash"
    assert (ost == oracle.FULL).sum() > 0, "and fill it"
    assert np.array_equal(words(t, 0), o.t0)
    assert np.array_equal(level1_words(t), o.t1)
    q = W.unique_keys(0, len(fresh) + 500, w, 5 + T)
    assert (t.find(dev_keys(q, kb)).cpu().numpy() == o.find(q.numpy().astype(np.uint64))).all()
    stored, cnt = t.enumerate()
    assert cnt == len(o.enumerate())
    assert np.array_equal(np.sort(u64(stored)), np.sort(o.enumerate()))


@pytest.mark.parametrize("geom", GEOMS)
@pytest.mark.parametrize("T,items", [(4, 1), (8, 2), (4, 4)])
def test_concurrent_stash_parity(geom, T, items):
    w, kb, N0, N1, f0, f1, S = geom
    P = cht()
    # a stash big enough for every key the buckets cannot take
    t = P.Table(P.ICEBERG, w, 1 << N0, 1 << N1, key_bytes=kb, fields_per_word=f0,
                fields_per_word_backyard=f1, stash_slots=4 * S, seed=41 + N0, tile=T,
                items_per_thread=items)
    fresh, keys = _stream(t, w, 1.2, 11 + T + items)
    st = t.find_or_put(dev_keys(keys, kb)).cpu().numpy()
    o = mirror(t)
    kn = keys.numpy().astype(np.uint64)
    ost = o.insert(kn)
    assert (ost != oracle.FULL).all() and (st != P.FULL).all()
    assert t.error_flags() == 0
    uniq, inv = np.unique(kn, return_inverse=True)
    puts = np.bincount(inv, weights=(st == P.PUT), minlength=len(uniq))
    assert (puts == 1).all()
    assert ((st == P.PUT) | (st == P.FOUND)).all()
    stored, cnt = t.enumerate()
    assert np.array_equal(np.sort(u64(stored)), np.sort(o.enumerate()))
    d = dump_into(mirror(t), t)
    assert (d.stash != 0).sum() > 0
    assert d.check_entries() == 0 and d.check_order_property() == 0
    assert d.check_prefix() == 0 and d.check_stash() == 0 and d.check_duplicates() == 0
    q = W.unique_keys(0, len(fresh) + 2000, w, 11 + T + items)
    got = t.find(dev_keys(q, kb)).cpu().numpy()
    assert (got == d.find(q.numpy().astype(np.uint64))).all()
    assert (got[: len(fresh)] == P.FOUND).all() and (got[len(fresh):] == P.NOT_FOUND).all()


def test_concurrent_past_the_stash():
    P = cht()
    w = 32
    t = P.Table(P.ICEBERG, w, 1 << 3, 1 << 1, key_bytes=4, fields_per_word=2,
                stash_slots=16, seed=9)
    fresh, keys = _stream(t, w, 1.4, 99)
    kn = keys.numpy().astype(np.uint64)
    st = t.find_or_put(dev_keys(keys, 4)).cpu().numpy()
    assert (st == P.FULL).sum() > 0
    d = dump_into(mirror(t), t)
    assert (d.stash != 0).all(), "FULL only once every stash slot is taken"
    assert d.check_entries() == 0 and d.check_order_property() == 0
    assert d.check_stash() == 0 and d.check_duplicates() == 0
    stored = set(d.enumerate().tolist())
    uniq, inv = np.unique(kn, return_inverse=True)
    for i, k in enumerate(uniq):
        mine = st[inv == i]
        if int(k) in stored:
            assert (mine == P.PUT).sum() == 1 and ((mine == P.PUT) | (mine == P.FOUND)).all()
        else:
            assert (mine == P.FULL).all()


def test_stash_slots_and_values():
    P = cht()
    w = 40
    t = P.Table(P.ICEBERG, w, 1 << 3, 1 << 1, stash_slots=256, seed=13)
    c = t.cfg
    two_level = c.num_buckets * 16 * c.fields_per_word + \
        c.num_buckets_backyard * 16 * c.fields_per_word_backyard
    assert t.slots == two_level + 256
    keys = W.unique_keys(0, two_level + 200, w, 3)
    st, slots = t.find_or_put(keys.to(DEV), slots=True)
    st, slots = st.cpu().numpy(), slots.cpu().numpy()
    assert (st == P.PUT).all()
    d = dump_into(mirror(t), t)
    want = d.locate(keys.numpy().astype(np.uint64))
    assert np.array_equal(slots.view(np.uint64), want)
    assert (want >= two_level).sum() >= 200  # the overflow lives in the stash
    f, fs = t.find(keys.to(DEV), slots=True)
    assert (f.cpu().numpy() == P.FOUND).all()
    assert np.array_equal(fs.cpu().numpy().view(np.uint64), want)
    kv = P.KVMap(t, torch.int64)
    vals = torch.arange(len(keys), dtype=torch.int64, device=DEV) * 7
    kv.put(keys.to(DEV), vals)
    got, gst = kv.get(keys.to(DEV))
    assert torch.equal(got, vals)


def test_fused_batch_with_stash_tables():
    from paper_2406_09255_gb300.batch import Batch
    P = cht()
    tables, keys = [], []
    for i in range(6):
        t = P.Table(P.ICEBERG, 32, 1 << (3 + i % 3), 1 << 1, key_bytes=4, fields_per_word=2,
                    stash_slots=512, seed=70 + i)
        _, k = _stream(t, 32, 1.15, 200 + i)
        tables.append(t)
        keys.append(W.to_u32(k).to(DEV))
    b = Batch(tables, keys)
    b.launch()
    torch.cuda.synchronize()
    for t, k, s in zip(tables, keys, b.statuses):
        kn = u64(k)
        st = s.cpu().numpy()
        o = mirror(t)
        ost = o.insert(kn)
        assert (ost != oracle.FULL).all()
        uniq, inv = np.unique(kn, return_inverse=True)
        puts = np.bincount(inv, weights=(st == P.PUT), minlength=len(uniq))
        assert (puts == 1).all()
        stored, _ = t.enumerate()
        assert np.array_equal(np.sort(u64(stored)), np.sort(o.enumerate()))
        d = dump_into(mirror(t), t)
        assert d.check_stash() == 0 and d.check_order_property() == 0
