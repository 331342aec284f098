"""GPU parity of tables with 32- and 64-byte buckets (4 or 8 words; with
32-bit slots the 8- and 16-slot buckets that Section 5.1 sweeps beside 32),
through the C ABI against the oracle, which takes the bucket width as a
parameter:

- single-tile ordered runs: statuses and every table word equal to the
  oracle's (cuckoo with evictions and FULL, iceberg with spills and FULL);
- concurrent runs: cuckoo lookups exact, with the oracle's probe counts on
  the GPU's own table; iceberg find-or-put with duplicates meets the
  Theorem 1 contract; cuckoo past capacity conserves keys.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_09255_gb300 import workloads as W

from test_gpu_parity import DEV, cht, dev_keys, dump_into, mirror, u64, words

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("wpb", [4, 8])
@pytest.mark.parametrize("geom", [(24, 8, 6, 3), (32, 4, 6, 2), (20, 4, 6, 4), (40, 8, 6, 1)])
def test_sequential_cuckoo_small_buckets(wpb, geom):
    w, kb, N, fpw = geom
    P = cht()
    t = P.Table(P.CUCKOO, w, 1 << N, key_bytes=kb, fields_per_word=fpw, bucket_words=wpb,
                max_chain=16, seed=3 + N, max_tiles=1, cta_threads=64, items_per_thread=2)
    o = mirror(t)
    assert o.slots_per_bucket(0) == wpb * fpw
    keys = W.unique_keys(0, int(1.05 * t.slots), w, 21 + wpb)
    dropped = torch.zeros(len(keys), dtype=torch.int64, device=DEV)
    st = t.insert(dev_keys(keys, kb), dropped=dropped).cpu().numpy()
    ost, odr = o.insert(keys.numpy().astype(np.uint64))
    assert (st == ost).all()
    assert (ost == oracle.FULL).sum() > 0
    full = ost == oracle.FULL
    assert np.array_equal(u64(dropped)[full] & ((1 << w) - 1), odr[full])
    assert np.array_equal(words(t, 0), o.t0)
    q = W.unique_keys(0, len(keys) + 500, w, 21 + wpb)
    assert (t.find(dev_keys(q, kb)).cpu().numpy() == o.find(q.numpy().astype(np.uint64))).all()


@pytest.mark.parametrize("wpb", [4, 8])
@pytest.mark.parametrize("geom", [(32, 4, 4, 2, 2, 2), (40, 8, 4, 2, 1, 1), (19, 4, 4, 2, 4, 2)])
def test_sequential_iceberg_small_buckets(wpb, geom):
    w, kb, N0, N1, f0, f1 = geom
    P = cht()
    t = P.Table(P.ICEBERG, w, 1 << N0, 1 << N1, key_bytes=kb, fields_per_word=f0,
                fields_per_word_backyard=f1, bucket_words=wpb, seed=50 + N0, max_tiles=1,
                cta_threads=64, items_per_thread=2)
    o = mirror(t)
    fresh = W.unique_keys(0, int(1.1 * t.slots), w, 31 + wpb)
    rng = np.random.default_rng(wpb)
    dup = fresh[torch.from_numpy(rng.integers(0, len(fresh), len(fresh) // 2))]
    keys = torch.cat([fresh, dup])
    keys = keys[torch.from_numpy(rng.permutation(len(keys)))]
    st = t.find_or_put(dev_keys(keys, kb)).cpu().numpy()
    ost = o.insert(keys.numpy().astype(np.uint64))
    assert (st == ost).all()
    assert (ost == oracle.FULL).sum() > 0 and (ost == oracle.FOUND).sum() > 0
    assert np.array_equal(words(t, 0), o.t0)
    assert np.array_equal(words(t, 1), o.t1)
    q = W.unique_keys(0, len(fresh) + 300, w, 31 + wpb)
    assert (t.find(dev_keys(q, kb)).cpu().numpy() == o.find(q.numpy().astype(np.uint64))).all()
    stored, cnt = t.enumerate()
    assert np.array_equal(np.sort(u64(stored)), np.sort(o.enumerate()))


@pytest.mark.parametrize("wpb", [4, 8])
def test_concurrent_cuckoo_lookups_small_buckets(wpb):
    P = cht()
    w = 32
    t = P.Table(P.CUCKOO, w, 1 << 14, key_bytes=4, fields_per_word=2, bucket_words=wpb, seed=8)
    n = int(0.8 * t.slots)
    keys = W.unique_keys(0, n, w, 77)
    st = t.insert(W.to_u32(keys).to(DEV)).cpu().numpy()
    assert (st == P.PUT).all()
    stored, cnt = t.enumerate()
    assert np.array_equal(np.sort(u64(stored)), np.sort(keys.numpy().astype(np.uint64)))
    q, present = W.find_queries(n, 1 << 17, 0.5, w, 77, n)
    ctr = t.attach_counters()
    got = t.find(W.to_u32(q).to(DEV)).cpu().numpy()
    torch.cuda.synchronize()
    gprobes = int(ctr[0].item())
    t.detach_counters()
    assert np.array_equal(got == P.FOUND, present.numpy())
    d = dump_into(mirror(t), t)
    assert d.check_prefix() == 0 and d.check_entries() == 0 and d.check_cuckoo_chain() == 0
    assert d.check_duplicates() == 0
    assert (d.find(q.numpy().astype(np.uint64)) == got).all()
    assert d.probes == gprobes


@pytest.mark.parametrize("wpb", [4, 8])
def test_concurrent_iceberg_small_buckets(wpb):
    # 8- and 16-slot primary buckets overflow earlier than 32-slot ones
    # (Section 5.2): a stash takes the keys whose three buckets fill up
    P = cht()
    w = 40
    t = P.Table(P.ICEBERG, w, 1 << 10, 1 << 7, bucket_words=wpb, stash_slots=4096, seed=12)
    fresh = W.unique_keys(0, int(0.7 * t.slots), w, 5)
    rng = np.random.default_rng(2)
    keys = torch.cat([fresh, fresh[torch.from_numpy(rng.integers(0, len(fresh), len(fresh)))]])
    keys = keys[torch.from_numpy(rng.permutation(len(keys)))]
    kn = keys.numpy().astype(np.uint64)
    st = t.find_or_put(keys.to(DEV)).cpu().numpy()
    o = mirror(t)
    ost = o.insert(kn)
    assert (ost != oracle.FULL).all() and t.error_flags() == 0
    uniq, inv = np.unique(kn, return_inverse=True)
    puts = np.bincount(inv, weights=(st == P.PUT), minlength=len(uniq))
    assert (puts == 1).all() and ((st == P.PUT) | (st == P.FOUND)).all()
    stored, _ = t.enumerate()
    assert np.array_equal(np.sort(u64(stored)), np.sort(o.enumerate()))
    d = dump_into(mirror(t), t)
    assert d.check_entries() == 0 and d.check_order_property() == 0 and d.check_prefix() == 0
    assert d.check_duplicates() == 0 and d.check_stash() == 0
    q = W.unique_keys(0, len(fresh) + 5000, w, 5)
    got = t.find(q.to(DEV)).cpu().numpy()
    assert (got == d.find(q.numpy().astype(np.uint64))).all()


@pytest.mark.parametrize("wpb", [4, 8])
def test_cuckoo_small_buckets_past_capacity_conserves_keys(wpb):
    P = cht()
    w = 28
    t = P.Table(P.CUCKOO, w, 1 << 10, fields_per_word=3, bucket_words=wpb, max_chain=16, seed=2)
    keys = W.unique_keys(0, int(1.02 * t.slots), w, 8)
    dropped = torch.zeros(len(keys), dtype=torch.int64, device=DEV)
    st = t.insert(keys.to(DEV), dropped=dropped).cpu().numpy()
    assert (st == P.FULL).sum() > 0
    stored, _ = t.enumerate()
    lost = u64(dropped)[st == P.FULL]
    assert np.array_equal(np.sort(np.concatenate([u64(stored), lost])),
                          np.sort(keys.numpy().astype(np.uint64)))
    d = dump_into(mirror(t), t)
    assert d.check_prefix() == 0 and d.check_entries() == 0 and d.check_cuckoo_chain() == 0


def test_small_buckets_reject_what_they_do_not_offer():
    P = cht()
    t = P.Table(P.ICEBERG, 32, 1 << 6, 1 << 3, key_bytes=4, bucket_words=8, seed=1)
    k = torch.ones(4, dtype=torch.int32, device=DEV)
    with pytest.raises(P.ChtError):
        t.find_or_put(k, slots=True)
    from paper_2406_09255_gb300.batch import Batch
    with pytest.raises(P.ChtError):
        Batch([t], [k])
