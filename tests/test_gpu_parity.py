"""GPU parity: the CUDA path through the C ABI against the sequential oracle.

Contract (what is unique is compared exactly, the rest checked for validity):
  - A single tile (max_tiles = 1) processes keys strictly in input order, so
    its table must equal the oracle's word for word, with identical statuses
    and dropped keys.
  - Concurrent cuckoo build without FULL: every status PUT, the enumerated
    set equals the input, lookups equal the oracle's (they depend only on
    the key set), and the oracle run on the GPU's own table dump reproduces
    the GPU's lookups and probe counts exactly.
  - Concurrent cuckoo build with FULL: stored + dropped = input.
  - Concurrent iceberg find-or-put: exactly one PUT per distinct key, the
    rest FOUND; the stored set equals the oracle's; the dump is well formed
    (Theorem 1 (a)); FULL keys have all three buckets full and lack the key.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_09255_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0) if torch.cuda.is_available() else None


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def cht():
    import paper_2406_09255_gb300 as m
    return m


def u64(x: torch.Tensor) -> np.ndarray:
    """Device/host int tensor of keys -> numpy uint64 (4-byte keys zero-extended)."""
    a = x.detach().cpu().numpy()
    if a.dtype == np.int32:
        return a.view(np.uint32).astype(np.uint64)
    return a.view(np.uint64)


def dev_keys(keys64: torch.Tensor, key_bytes: int) -> torch.Tensor:
    k = W.to_u32(keys64) if key_bytes == 4 else keys64
    return k.to(DEV)


def words(t, level=0) -> np.ndarray:
    return t.words(level).cpu().numpy().view(np.uint64)


def mirror(t):
    """An oracle table with the resolved geometry of GPU table t."""
    c = t.cfg
    return oracle.Table(c.kind, c.key_bits, c.num_buckets, c.num_buckets_backyard,
                        compact=bool(c.compact), fpw0=c.fields_per_word,
                        fpw1=max(c.fields_per_word_backyard, 1), num_hashes=max(c.num_hashes, 1),
                        max_chain=max(c.max_chain, 1), seed=c.seed, stash=c.stash_slots,
                        wpb=c.bucket_words)


def level1_words(t) -> np.ndarray:
    """The secondary level's words followed by the stash (the oracle's t1)."""
    if t.cfg.stash_slots:
        return np.concatenate([words(t, 1), words(t, 2)])
    return words(t, 1)


def dump_into(o, t):
    o.load_words(words(t, 0), level1_words(t) if t.cfg.kind == 1 else None)
    return o


# --------------------------------------------------------------------------
# sequential single-tile runs: bit-exact tables
# --------------------------------------------------------------------------
CUCKOO_SEQ = [
    # (key_bits, key_bytes, log2 buckets, fpw, compact)
    (24, 8, 6, 3, True),
    (32, 4, 6, 2, True),
    (20, 4, 6, 4, True),
    (40, 8, 6, 1, True),
    (40, 8, 6, 1, False),
]


@pytest.mark.parametrize("T", [4, 8, 16])
@pytest.mark.parametrize("geom", CUCKOO_SEQ)
def test_sequential_cuckoo_bit_exact(T, geom):
    w, kb, N, fpw, compact = geom
    C = 24
    t = cht().Table(cht().CUCKOO, w, 1 << N, key_bytes=kb, fields_per_word=fpw, compact=compact,
                    max_chain=C, seed=1000 + N, tile=T, items_per_thread=3, max_tiles=1,
                    cta_threads=32)
    o = mirror(t)
    n = t.slots + 64  # more keys than slots: FULL must occur
    keys = W.unique_keys(0, n, w, 42 + T)
    # a few invalid keys in the stream
    keys[5] = 0
    keys[n // 2] = 1 << w if w < 62 and kb == 8 else 0
    dropped = torch.zeros(n, dtype=torch.int64, device=DEV)
    st = t.insert(dev_keys(keys, kb), dropped=dropped)
    ost, odr = o.insert(keys.numpy().astype(np.uint64))
    gst = st.cpu().numpy()
    assert (gst == ost).all()
    assert (ost == oracle.FULL).sum() > 0, "the case should exercise FULL"
    full = ost == oracle.FULL
    assert (dropped.cpu().numpy().view(np.uint64)[full] == odr[full]).all()
    assert np.array_equal(words(t), o.t0)
    # lookups on the same table are equal too
    q = W.unique_keys(0, n + 500, w, 42 + T)
    assert (t.find(dev_keys(q, kb)).cpu().numpy() == o.find(q.numpy().astype(np.uint64))).all()


ICEBERG_SEQ = [
    # (key_bits, key_bytes, log2 primary, log2 backyard, fpw0, fpw1, compact)
    (40, 8, 4, 2, 1, 1, True),
    (32, 4, 4, 2, 2, 2, True),
    (19, 4, 4, 2, 4, 2, True),
    (20, 4, 4, 2, 3, 2, True),
    (40, 8, 4, 2, 1, 1, False),
]


@pytest.mark.parametrize("T", [4, 8, 16])
@pytest.mark.parametrize("geom", ICEBERG_SEQ)
def test_sequential_iceberg_bit_exact(T, geom):
    w, kb, N0, N1, f0, f1, compact = geom
    t = cht().Table(cht().ICEBERG, w, 1 << N0, 1 << N1, key_bytes=kb, fields_per_word=f0,
                    fields_per_word_backyard=f1, compact=compact, seed=77 + N0, tile=T,
                    items_per_thread=2, max_tiles=1, cta_threads=64)
    o = mirror(t)
    fresh = W.unique_keys(0, int(1.1 * t.slots), w, 9 + T)
    rng = np.random.default_rng(T)
    dup = fresh[torch.from_numpy(rng.integers(0, len(fresh), len(fresh) // 2))]
    keys = torch.cat([fresh, dup])
    keys = keys[torch.from_numpy(rng.permutation(len(keys)))]
    keys[3] = 0
    st = t.find_or_put(dev_keys(keys, kb)).cpu().numpy()
    ost = o.insert(keys.numpy().astype(np.uint64))
    assert (st == ost).all()
    assert (ost == oracle.FULL).sum() > 0 and (ost == oracle.FOUND).sum() > 0
    assert np.array_equal(words(t, 0), o.t0)
    assert np.array_equal(words(t, 1), o.t1)
    q = W.unique_keys(0, len(fresh) + 300, w, 9 + T)
    assert (t.find(dev_keys(q, kb)).cpu().numpy() == o.find(q.numpy().astype(np.uint64))).all()


# --------------------------------------------------------------------------
# concurrent cuckoo
# --------------------------------------------------------------------------
@pytest.mark.parametrize("T,items,P", [(4, 1, 1), (8, 2, 1), (16, 8, 1), (8, 1, 4), (4, 3, 4), (16, 1, 4), (8, 1, 8), (4, 1, 8), (16, 2, 8)])
def test_cuckoo_2e14_fill_08_lookup_parity(T, items, P):
    """2^14 buckets x 48 slots, 32-bit keys, 629,145 keys (fill 0.8), then 2^20
    lookups, half present and half absent."""
    t = cht().Table(cht().CUCKOO, 32, 1 << 14, key_bytes=4, seed=0x2406_0925_5001, tile=T,
                    items_per_thread=items, lookups_in_flight=P)
    assert t.cfg.fields_per_word == 3 and t.slots == 786432
    n = 629145
    keys = W.unique_keys(0, n, 32, W.SEED_BASE + 1)
    st = t.insert(dev_keys(keys, 4)).cpu().numpy()
    assert (st == cht().PUT).all()
    assert t.error_flags() == 0
    stored, cnt = t.enumerate()
    assert cnt == n
    assert np.array_equal(np.sort(u64(stored)), np.sort(keys.numpy().astype(np.uint64)))

    q, present = W.find_queries(n, 1 << 20, 0.5, 32, W.SEED_BASE + 1, n)
    ctr = t.attach_counters()
    got = t.find(dev_keys(q, 4)).cpu().numpy()
    gprobes = int(ctr[0].item())
    t.detach_counters()
    assert np.array_equal(got == cht().FOUND, present.numpy())
    # the oracle on its own sequentially built table
    o = mirror(t)
    o.insert(keys.numpy().astype(np.uint64))
    assert (o.find(q.numpy().astype(np.uint64)) == got).all()
    # the oracle on the GPU's table: same answers and the same probe count
    d = dump_into(mirror(t), t)
    assert (d.find(q.numpy().astype(np.uint64)) == got).all()
    assert d.probes == gprobes
    assert d.check_prefix() == 0
    assert d.check_entries() == 0
    assert d.check_duplicates() == 0
    assert d.check_cuckoo_chain() == 0


@pytest.mark.parametrize("compact,P", [(True, 4), (False, 4), (True, 1), (True, 8)])
def test_cuckoo_past_capacity_conserves_keys(compact, P):
    """Puts past capacity (fill 0.99, C = 8): every key is stored or handed
    back as dropped, for the stream put (P = 4, 8) and the chunk put (P = 1)."""
    t = cht().Table(cht().CUCKOO, 28, 1 << 10, compact=compact, max_chain=8, seed=3,
                    lookups_in_flight=P)
    n = int(0.99 * t.slots)
    keys = W.unique_keys(0, n, 28, 99)
    dropped = torch.zeros(n, dtype=torch.int64, device=DEV)
    st = t.insert(keys.to(DEV), dropped=dropped).cpu().numpy()
    full = st == cht().FULL
    assert full.sum() > 0
    assert ((st == cht().PUT) | full).all()
    stored, cnt = t.enumerate()
    lost = dropped.cpu().numpy().view(np.uint64)[full]
    both = np.sort(np.concatenate([u64(stored), lost]))
    assert np.array_equal(both, np.sort(keys.numpy().astype(np.uint64)))
    d = dump_into(mirror(t), t)
    assert d.check_prefix() == 0 and d.check_entries() == 0 and d.check_cuckoo_chain() == 0
    assert d.check_duplicates() == 0
    # lookups are exact membership
    stored_set = set(u64(stored).tolist())
    got = t.find(keys.to(DEV)).cpu().numpy() == cht().FOUND
    assert np.array_equal(got, np.array([int(k) in stored_set for k in keys.numpy()]))


def test_cuckoo_noncompact_equal_slots_fastrange():
    # whole-key table with a bucket count that is not a power of two
    nb = 3 * (1 << 8)
    t = cht().Table(cht().CUCKOO, 40, nb, compact=False, seed=8)
    assert t.cfg.fields_per_word == 1
    n = int(0.85 * t.slots)
    keys = W.unique_keys(0, n, 40, 5)
    st = t.insert(keys.to(DEV)).cpu().numpy()
    assert (st == cht().PUT).all()
    q, present = W.find_queries(n, 20000, 0.5, 40, 5, n)
    got = t.find(q.to(DEV)).cpu().numpy()
    assert np.array_equal(got == cht().FOUND, present.numpy())
    d = dump_into(mirror(t), t)
    assert (d.find(q.numpy().astype(np.uint64)) == got).all()
    assert d.check_entries() == 0 and d.check_cuckoo_chain() == 0
    assert d.check_duplicates() == 0


# --------------------------------------------------------------------------
# concurrent iceberg find-or-put
# --------------------------------------------------------------------------
def _fop_contract(t, keys_np, st, o_stored):
    """Per-key flags and final set against the oracle's, for a run whose
    oracle replay had no FULL."""
    P = cht()
    assert ((st == P.PUT) | (st == P.FOUND)).all()
    uniq, inv = np.unique(keys_np, return_inverse=True)
    puts = np.bincount(inv, weights=(st == P.PUT), minlength=len(uniq))
    assert (puts == 1).all(), "each distinct key is put exactly once"
    stored, cnt = t.enumerate()
    assert np.array_equal(np.sort(u64(stored)), np.sort(o_stored))
    d = dump_into(mirror(t), t)
    assert d.check_entries() == 0
    assert d.check_duplicates() == 0
    assert d.check_order_property() == 0
    assert d.check_prefix() == 0
    return d


@pytest.mark.parametrize("T,items", [(4, 2), (8, 1), (16, 4)])
def test_iceberg_fop_duplicates_parity(T, items):
    w = 40
    t = cht().Table(cht().ICEBERG, w, 1 << 12, 1 << 9, seed=21, tile=T, items_per_thread=items)
    o = mirror(t)
    n_fresh = int(0.8 * t.slots)
    fresh = W.unique_keys(0, n_fresh, w, 55)
    keys = W.duplicate_stream(2 * n_fresh, n_fresh, w, 55, 0.5)
    # duplicate_stream draws its fresh keys from the same sequence
    assert set(keys.numpy().tolist()) == set(fresh.numpy().tolist())
    st = t.find_or_put(keys.to(DEV)).cpu().numpy()
    kn = keys.numpy().astype(np.uint64)
    ost = o.insert(kn)
    assert (ost != oracle.FULL).all()
    _fop_contract(t, kn, st, o.enumerate())
    # lookups after the batch are exact
    q, present = W.find_queries(n_fresh, 30000, 0.5, w, 55, 2 * n_fresh)
    got = t.find(q.to(DEV)).cpu().numpy()
    assert np.array_equal(got == cht().FOUND, present.numpy())
    assert (o.find(q.numpy().astype(np.uint64)) == got).all()
    # a second batch of the same keys finds everything
    st2 = t.find_or_put(keys.to(DEV)).cpu().numpy()
    assert (st2 == cht().FOUND).all()
    assert t.error_flags() == 0


@pytest.mark.parametrize("T,items", [(4, 1), (8, 2), (16, 4)])
def test_iceberg_copies_within_a_chunk(T, items):
    """Copies of a key next to each other, so that they race inside one
    warp's chunk: exactly one PUT per distinct key, the other copies FOUND,
    the oracle's stored set, and lookups whose copies all agree with
    membership."""
    w = 40
    t = cht().Table(cht().ICEBERG, w, 1 << 12, 1 << 9, seed=29, tile=T, items_per_thread=items)
    o = mirror(t)
    n = int(0.6 * t.slots)
    fresh = W.unique_keys(0, n, w, 61)
    rng = np.random.default_rng(61)
    # each key 1-6 times, copies placed next to each other
    reps = rng.integers(1, 7, n)
    keys = torch.from_numpy(np.repeat(fresh.numpy(), reps))
    st = t.find_or_put(keys.to(DEV)).cpu().numpy()
    kn = keys.numpy().astype(np.uint64)
    ost = o.insert(kn)
    assert (ost != oracle.FULL).all()
    _fop_contract(t, kn, st, o.enumerate())
    # lookups: present and absent keys, each in runs of copies
    q = torch.from_numpy(np.repeat(W.unique_keys(n - 2000, 4000, w, 61).numpy(), 5))
    got = t.find(q.to(DEV)).cpu().numpy()
    assert (o.find(q.numpy().astype(np.uint64)) == got).all()
    assert (got == cht().FOUND).sum() == 5 * 2000 and (got == cht().NOT_FOUND).sum() == 5 * 2000
    assert t.error_flags() == 0


@pytest.mark.parametrize("T,P", [(4, 4), (8, 4), (4, 8), (16, 8)])
def test_iceberg_stream_form_parity(T, P):
    """The stream form (level 1 in packed rounds with P loads in flight per
    tile, then a level-2 pass over the keys whose primary was full) meets the
    same contract as the chunk engine: one PUT per distinct key, the oracle's
    stored set, a well-formed dump, exact lookups (also in the stream form),
    and no key left pending."""
    w = 40
    t = cht().Table(cht().ICEBERG, w, 1 << 12, 1 << 9, seed=23, tile=T, lookups_in_flight=P)
    o = mirror(t)
    n_fresh = int(0.85 * t.slots)
    keys = W.duplicate_stream(2 * n_fresh, n_fresh, w, 57, 0.5)
    st = t.find_or_put(keys.to(DEV)).cpu().numpy()
    kn = keys.numpy().astype(np.uint64)
    ost = o.insert(kn)
    assert (ost != oracle.FULL).all() and (st != 6).all()
    _fop_contract(t, kn, st, o.enumerate())
    q, present = W.find_queries(n_fresh, 60000, 0.5, w, 57, 2 * n_fresh)
    got = t.find(q.to(DEV)).cpu().numpy()
    assert np.array_equal(got == cht().FOUND, present.numpy())
    d = dump_into(mirror(t), t)
    assert (d.find(q.numpy().astype(np.uint64)) == got).all()
    assert t.error_flags() == 0


@pytest.mark.parametrize("P", [4, 8])
def test_iceberg_stream_form_past_capacity_with_stash(P):
    w = 36
    t = cht().Table(cht().ICEBERG, w, 1 << 8, 1 << 5, seed=18, lookups_in_flight=P,
                    stash_slots=256)
    fresh = W.unique_keys(0, int(1.1 * t.slots), w, 4)
    rng = np.random.default_rng(3)
    keys = torch.cat([fresh, fresh[torch.from_numpy(rng.integers(0, len(fresh), len(fresh)))]])
    keys = keys[torch.from_numpy(rng.permutation(len(keys)))]
    kn = keys.numpy().astype(np.uint64)
    st = t.find_or_put(keys.to(DEV)).cpu().numpy()
    P_ = cht()
    assert (st == P_.FULL).sum() > 0 and (st != 6).all()
    d = dump_into(mirror(t), t)
    assert (d.stash != 0).all()
    assert d.check_entries() == 0 and d.check_order_property() == 0 and d.check_prefix() == 0
    assert d.check_stash() == 0 and d.check_duplicates() == 0
    stored = set(d.enumerate().tolist())
    uniq, inv = np.unique(kn, return_inverse=True)
    puts = np.bincount(inv, weights=(st == P_.PUT), minlength=len(uniq))
    assert set(uniq[puts == 1].tolist()) == stored and puts.max() == 1
    assert set(kn[st == P_.FULL].tolist()).isdisjoint(stored)
    got = t.find(keys.to(DEV)).cpu().numpy()
    assert (got == d.find(kn)).all()


def test_iceberg_hot_key_contention():
    # every key repeated 64 times in one batch: CAS races on the same slots
    t = cht().Table(cht().ICEBERG, 40, 1 << 6, 1 << 3, seed=4)
    base = W.unique_keys(0, 1000, 40, 7)
    keys = base.repeat(64)
    keys = keys[torch.from_numpy(np.random.default_rng(0).permutation(len(keys)))]
    st = t.find_or_put(keys.to(DEV)).cpu().numpy()
    o = mirror(t)
    ost = o.insert(keys.numpy().astype(np.uint64))
    assert (ost != oracle.FULL).all()
    _fop_contract(t, keys.numpy().astype(np.uint64), st, o.enumerate())


@pytest.mark.parametrize("P", [1, 4])
def test_bounded_retry_runs_out_and_reports_error(P):
    # One primary and one secondary bucket (16 + 16 slots of 64 bits for
    # 32-bit keys) and 64 distinct keys: in every round the tiles of a warp
    # race for the same first empty slot and all but one lose. With
    # retry_limit = 1 a key that loses twice gives up: CHT_ERROR status, the
    # table's error word set, and the kernel returns normally (no hang, no
    # trap). The keys that did get an answer follow Algorithm 1.
    M = cht()
    keys = W.to_u32(W.unique_keys(0, 64, 32, 9))
    t = M.Table(M.ICEBERG, 32, 1, 1, key_bytes=4, retry_limit=1, seed=3, lookups_in_flight=P)
    st = t.find_or_put(keys.to(DEV)).cpu().numpy()
    assert (st == M.ERROR).sum() > 0, np.bincount(st)
    assert ((st == M.ERROR) | (st == M.PUT) | (st == M.FULL)).all()
    assert t.error_flags() != 0
    stored, cnt = t.enumerate()
    kn = u64(keys)
    assert cnt == (st == M.PUT).sum()
    assert set(u64(stored).tolist()) == set(kn[st == M.PUT].tolist())
    d = dump_into(mirror(t), t)
    assert d.check_entries() == 0 and d.check_order_property() == 0 and d.check_prefix() == 0
    assert d.check_duplicates() == 0
    # the error word is cleared with the table; the built-in bound is never
    # reached on the same race
    t.clear()
    assert t.error_flags() == 0
    t2 = M.Table(M.ICEBERG, 32, 1, 1, key_bytes=4, seed=3)
    st2 = t2.find_or_put(keys.to(DEV)).cpu().numpy()
    assert (st2 != M.ERROR).all() and t2.error_flags() == 0
    assert (st2 == M.PUT).sum() == 32 and (st2 == M.FULL).sum() == 32


@pytest.mark.parametrize("compact", [True, False])
def test_iceberg_past_capacity_theorem1(compact):
    w = 36
    t = cht().Table(cht().ICEBERG, w, 1 << 8, 1 << 5, compact=compact, seed=17)
    fresh = W.unique_keys(0, int(1.08 * t.slots), w, 3)
    rng = np.random.default_rng(1)
    keys = torch.cat([fresh, fresh[torch.from_numpy(rng.integers(0, len(fresh), len(fresh)))]])
    keys = keys[torch.from_numpy(rng.permutation(len(keys)))]
    kn = keys.numpy().astype(np.uint64)
    st = t.find_or_put(keys.to(DEV)).cpu().numpy()
    P = cht()
    assert (st == P.FULL).sum() > 0
    stored, cnt = t.enumerate()
    s = u64(stored)
    assert len(np.unique(s)) == len(s), "no duplicates (Lemma, Appendix A)"
    d = dump_into(mirror(t), t)
    assert d.check_entries() == 0 and d.check_order_property() == 0 and d.check_prefix() == 0
    assert d.check_duplicates() == 0
    stored_set = set(s.tolist())
    # (c) found/put iff present afterwards; (d) one put per stored key
    present = np.array([int(k) in stored_set for k in kn])
    assert np.array_equal((st == P.FOUND) | (st == P.PUT), present)
    uniq, inv = np.unique(kn, return_inverse=True)
    puts = np.bincount(inv, weights=(st == P.PUT), minlength=len(uniq))
    assert set(uniq[puts == 1].tolist()) == stored_set and puts.max() == 1
    # (e) a FULL key's primary and both secondary buckets are full and lack it
    o = mirror(t)
    for k in np.unique(kn[st == P.FULL])[:200]:
        k = int(k)
        assert k not in stored_set
        for lvl, j in ((0, 0), (1, 0), (1, 1)):
            a = o.address(lvl, j, k)
            assert all(d.slot(lvl, a, y) != 0 for y in range(o.slots_per_bucket(lvl)))
    # stored + FULL keys = every distinct key
    full_set = set(kn[st == P.FULL].tolist())
    assert stored_set | full_set == set(uniq.tolist())


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 7, 1001])
@pytest.mark.parametrize("kind", [0, 1])
def test_ragged_and_empty_batches(n, kind):
    t = cht().Table(kind, 30, 1 << 8, 1 << 5 if kind else 0, key_bytes=4, seed=2, tile=8,
                    items_per_thread=3)
    keys = W.unique_keys(0, n, 30, 13)
    st = t.insert(dev_keys(keys, 4)).cpu().numpy()
    assert len(st) == n and (st == cht().PUT).all()
    f = t.find(dev_keys(keys, 4)).cpu().numpy()
    assert (f == cht().FOUND).all()
    stored, cnt = t.enumerate()
    assert cnt == n


def test_invalid_keys_and_capacity_of_enumerate():
    t = cht().Table(cht().ICEBERG, 30, 1 << 8, 1 << 5, seed=2)
    keys = torch.tensor([0, 1 << 30, 5, 6, (1 << 62), 7], dtype=torch.int64, device=DEV)
    st = t.find_or_put(keys).cpu().numpy().tolist()
    I, P = cht().INVALID, cht().PUT
    assert st == [I, I, P, P, I, P]
    out, cnt = t.enumerate(cap=2)
    assert cnt == 3 and len(out) == 2
    assert set(out.cpu().numpy().tolist()) <= {5, 6, 7}


def test_find_or_put_unsupported_on_cuckoo():
    t = cht().Table(cht().CUCKOO, 30, 1 << 8, seed=2)
    with pytest.raises(cht().ChtError) as e:
        t.find_or_put(torch.ones(4, dtype=torch.int64, device=DEV))
    assert e.value.code == 2


def test_clear_empties_table():
    t = cht().Table(cht().CUCKOO, 30, 1 << 8, seed=2)
    keys = W.unique_keys(0, 1000, 30, 1).to(DEV)
    t.insert(keys)
    t.clear()
    assert t.enumerate()[1] == 0
    assert (t.find(keys).cpu().numpy() == cht().NOT_FOUND).all()


# --------------------------------------------------------------------------
# full size: 2^24 buckets (2 GiB), the benchmark's launch configuration
# --------------------------------------------------------------------------
def test_cuckoo_2e24_full_size_sampled():
    P = cht()
    t = P.Table(P.CUCKOO, 40, 1 << 24, seed=2000)
    assert t.cfg.fields_per_word == 3 and t.slots == 805306368
    n = int(0.8 * t.slots)  # 644,245,094
    seed = W.SEED_BASE + 2
    keys = W.unique_keys(0, n, 40, seed, device=DEV)
    st = t.insert(keys)
    assert int((st != P.PUT).sum().item()) == 0
    del st
    # enumerate returns exactly the inserted set
    stored, cnt = t.enumerate()
    assert cnt == n
    assert torch.equal(torch.sort(stored)[0], torch.sort(keys)[0])
    del stored
    # lookups at 50 % hit: exact membership for all 402,653,184 queries
    nq = t.slots // 2
    q, present = W.find_queries(n, nq, 0.5, 40, seed, n, device=DEV)
    got = t.find(q)
    assert torch.equal(got == P.FOUND, present)
    # a sample re-checked by the oracle on the GPU's table
    d = dump_into(mirror(t), t)
    idx = torch.randint(0, nq, (200000,), generator=torch.Generator().manual_seed(0))
    qs = q[idx.to(DEV)].cpu().numpy().view(np.uint64)
    assert (d.find(qs) == got[idx.to(DEV)].cpu().numpy()).all()
    assert d.check_prefix() == 0


def test_random_read_utility_reads_every_block_size():
    """cht_random_read (a measurement utility) reads the blocks it should:
    over a buffer of seeded random words, the XOR-fold of every lane's word
    sums equals the value recomputed here from the block indices (splitmix64
    of seed + i * golden-ratio increment, masked to the block count)."""
    import ctypes
    from paper_2406_09255_gb300 import _lib
    L = _lib.load()
    nwords = 1 << 22  # 32 MiB of seeded random words
    host = np.random.default_rng(11).integers(0, 1 << 63, nwords, dtype=np.int64).view(np.uint64)
    buf = torch.from_numpy(host.view(np.int64)).to(DEV)
    M = (1 << 64) - 1

    def mix(z):
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9))
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB))
        return z ^ (z >> np.uint64(31))

    n, seed = 1 << 16, 7
    for bb, lanes, bpl in ((32, 2, 16), (64, 4, 16), (128, 8, 16), (256, 8, 32)):
        sink = torch.zeros(1, dtype=torch.int64, device=DEV)
        _lib.check(L.cht_random_read(buf.data_ptr(), nwords * 8, bb, n, seed,
                                     sink.data_ptr(), None))
        torch.cuda.synchronize()
        with np.errstate(over="ignore"):
            i = np.arange(n, dtype=np.uint64)
            blk = mix(np.uint64(seed) + i * np.uint64(0x9E3779B97F4A7C15)) & np.uint64(nwords * 8 // bb - 1)
            want = np.uint64(0)
            per = bpl // 8
            for lane in range(lanes):
                base = (blk * np.uint64(bb // 8) + np.uint64(lane * per)).astype(np.int64)
                tot = np.zeros(n, dtype=np.uint64)
                for k in range(per):
                    tot += host[base + k]
                want ^= np.bitwise_xor.reduce(tot)
        assert (int(sink.item()) & M) == int(want), bb


def test_random_claim_utility_claims_the_words_it_should():
    """cht_random_claim (the put-ceiling measurement) reads line i at
    splitmix64(seed + i * golden-ratio increment) masked to the line count and
    compare-and-swaps word (hash >> 40) & 15 of it from the value read to that
    value + 1. On a zeroed buffer with distinct targets every word ends at 1
    exactly where a target is, 0 elsewhere."""
    import ctypes
    from paper_2406_09255_gb300 import _lib
    L = _lib.load()
    nlines, n, seed = 1 << 16, 1 << 10, 5

    def mix(z):
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9))
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB))
        return z ^ (z >> np.uint64(31))

    with np.errstate(over="ignore"):
        i = np.arange(n, dtype=np.uint64)
        h = mix(np.uint64(seed) + i * np.uint64(0x9E3779B97F4A7C15))
        target = (h & np.uint64(nlines - 1)) * np.uint64(16) + ((h >> np.uint64(40)) & np.uint64(15))
    assert len(np.unique(target)) == n
    buf = torch.zeros(nlines * 16, dtype=torch.int64, device=DEV)
    sink = torch.zeros(1, dtype=torch.int64, device=DEV)
    _lib.check(L.cht_random_claim(buf.data_ptr(), nlines * 128, n, seed, sink.data_ptr(), None))
    torch.cuda.synchronize()
    want = np.zeros(nlines * 16, dtype=np.int64)
    want[target.astype(np.int64)] = 1
    assert np.array_equal(buf.cpu().numpy(), want)


def test_iceberg_2e22_full_size_stream():
    """The find-or-put stream workload at full size (2^22 + 2^19 buckets,
    150,994,944 slots, 48-bit keys; 80 % find-or-put / 20 % lookups, half
    first-seen keys, half Zipf repeats), in the benchmark's 2^22-op batches
    up to fill ~0.8: every find-or-put is PUT exactly once per distinct key
    and FOUND otherwise, every lookup answers membership at that point of
    the stream, the stored set is the set of keys put, Theorem 1's
    invariants hold on the GPU's table, and a sample re-checked by the
    oracle on that table agrees."""
    P = cht()
    t = P.Table(P.ICEBERG, 48, 1 << 22, 1 << 19, seed=3000)
    assert t.slots == 150994944
    max_distinct = int(0.8 * t.slots)
    n_ops = int(max_distinct / 0.4)
    keys, is_find, _ = W.fop_stream(n_ops, 48, W.SEED_BASE + 3, max_distinct=max_distinct,
                                    rng_seed=3, device=DEV)
    B = 1 << 22
    st = torch.empty(B, dtype=torch.uint8, device=DEV)
    seen = torch.empty(0, dtype=torch.int64, device=DEV)
    puts = 0
    for s0 in range(0, n_ops, B):
        k, f = keys[s0:s0 + B], is_find[s0:s0 + B]
        kf, kl = k[~f].contiguous(), k[f].contiguous()
        sf = t.find_or_put(kf, status=st[: kf.numel()])
        new = torch.unique(kf)
        fresh = new[~torch.isin(new, seen)]
        # exactly one PUT per key not seen before, FOUND for everything else
        assert bool(((sf == P.PUT) | (sf == P.FOUND)).all())
        put_keys = kf[sf == P.PUT]
        assert put_keys.numel() == fresh.numel()
        assert torch.equal(torch.sort(put_keys)[0], torch.sort(fresh)[0])
        puts += fresh.numel()
        seen = torch.sort(torch.cat([seen, fresh]))[0]
        sl = t.find(kl, status=st[kf.numel(): kf.numel() + kl.numel()])
        assert torch.equal(sl == P.FOUND, torch.isin(kl, seen))
    assert puts == seen.numel() and puts > 0.7 * t.slots
    stored, cnt = t.enumerate()
    assert cnt == puts
    assert torch.equal(torch.sort(stored)[0], seen)
    del stored, keys, is_find
    d = dump_into(mirror(t), t)
    assert d.check_entries() == 0 and d.check_order_property() == 0 and d.check_prefix() == 0
    assert d.check_duplicates() == 0
    g = torch.Generator(device=DEV)
    g.manual_seed(1)
    sample = torch.cat([seen[torch.randint(0, seen.numel(), (100000,), device=DEV, generator=g)],
                        W.keys_at(torch.arange(100000, device=DEV) + (1 << 46), 48,
                                  W.SEED_BASE + 3)])
    got = t.find(sample).cpu().numpy()
    assert (d.find(sample.cpu().numpy().view(np.uint64)) == got).all()
    assert t.error_flags() == 0


def test_host_resident_keys_and_statuses():
    """Key and status arrays in page-locked host memory: the kernels read the
    keys and write the statuses over the CPU-GPU link, with the same results
    as device-resident arrays (cuckoo put and lookup, iceberg find-or-put)."""
    from paper_2406_09255_gb300 import _lib
    L = _lib.load()
    P = cht()
    s = torch.cuda.current_stream().cuda_stream
    t = P.Table(P.CUCKOO, 40, 1 << 12, seed=77)
    n = int(0.8 * t.slots)
    keys = W.unique_keys(0, n, 40, 31)
    hk = keys.pin_memory()
    hs = torch.zeros(n, dtype=torch.uint8).pin_memory()
    _lib.check(L.cht_insert(t._h, hk.data_ptr(), n, hs.data_ptr(), None, s))
    torch.cuda.synchronize()
    assert bool((hs == P.PUT).all())
    q, present = W.find_queries(n, 50000, 0.5, 40, 31, n)
    hq, hqs = q.pin_memory(), torch.zeros(q.numel(), dtype=torch.uint8).pin_memory()
    _lib.check(L.cht_find(t._h, hq.data_ptr(), q.numel(), hqs.data_ptr(), s))
    torch.cuda.synchronize()
    assert torch.equal(hqs, t.find(q.to(DEV)).cpu())
    assert torch.equal(hqs == P.FOUND, present)
    ti = P.Table(P.ICEBERG, 40, 1 << 10, 1 << 7, seed=78)
    k2 = torch.cat([keys[:20000], keys[:5000]])
    hk2, hs2 = k2.pin_memory(), torch.zeros(k2.numel(), dtype=torch.uint8).pin_memory()
    _lib.check(L.cht_find_or_put(ti._h, hk2.data_ptr(), k2.numel(), hs2.data_ptr(), s))
    torch.cuda.synchronize()
    # one PUT per distinct key (which occurrence puts is up to the schedule)
    assert int((hs2 == P.PUT).sum()) == 20000
    assert bool(((hs2 == P.PUT) | (hs2 == P.FOUND)).all())


def test_table_methods_accept_pinned_host_tensors():
    """Table.insert / find / find_or_put / enumerate with page-locked host
    tensors give the same answers as with device tensors; unpinned host
    tensors are refused."""
    P = cht()
    t = P.Table(P.CUCKOO, 40, 1 << 10, seed=5)
    keys = W.unique_keys(0, 30000, 40, 77)
    # host results are valid once the stream has been synchronised
    st = t.insert(keys.pin_memory())
    torch.cuda.synchronize()
    assert st.device.type == "cpu" and st.is_pinned() and bool((st == P.PUT).all())
    q, present = W.find_queries(30000, 20000, 0.5, 40, 77, 30000)
    fq = t.find(q.pin_memory())
    torch.cuda.synchronize()
    assert torch.equal(fq == P.FOUND, present)
    out = torch.empty(t.slots, dtype=torch.int64).pin_memory()
    stored, cnt = t.enumerate(out=out)
    assert cnt == 30000 and torch.equal(torch.sort(stored)[0], torch.sort(keys)[0])
    with pytest.raises(ValueError):
        t.find(q)  # pageable host memory
    ti = P.Table(P.ICEBERG, 40, 1 << 9, 1 << 6, seed=6)
    k2 = torch.cat([keys[:5000], keys[:1000]]).pin_memory()
    s2 = ti.find_or_put(k2)
    torch.cuda.synchronize()
    assert int((s2 == P.PUT).sum()) == 5000 and bool(((s2 == P.PUT) | (s2 == P.FOUND)).all())
