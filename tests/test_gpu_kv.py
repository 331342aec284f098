"""Key-value extension on iceberg tables: the slot a find-or-put or a lookup
returns must be the slot that holds the key. Sequential single-tile runs
build the oracle's table bit for bit, so there the slots equal the oracle's
own locate() exactly; concurrent runs are checked by locating every key in
the GPU's table with the oracle. Then the value moves of KVMap."""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_09255_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0) if torch.cuda.is_available() else None
NONE = np.iinfo(np.uint64).max


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def P():
    import paper_2406_09255_gb300 as m
    return m


def dev_keys(keys64, key_bytes):
    return (W.to_u32(keys64) if key_bytes == 4 else keys64).to(DEV)


def words(t, level):
    return t.words(level).cpu().numpy().view(np.uint64)


def mirror(t):
    c = t.cfg
    return oracle.Table(c.kind, c.key_bits, c.num_buckets, c.num_buckets_backyard,
                        compact=bool(c.compact), fpw0=c.fields_per_word,
                        fpw1=max(c.fields_per_word_backyard, 1), seed=c.seed)


def dumped(t):
    o = mirror(t)
    o.load_words(words(t, 0), words(t, 1))
    return o


def as_u64(slots):
    return slots.cpu().numpy().view(np.uint64)


SEQ = [
    # (key_bits, key_bytes, log2 primary, log2 backyard, fpw0, fpw1, compact)
    (32, 4, 4, 2, 2, 2, True),
    (19, 4, 4, 2, 4, 2, True),
    (20, 4, 4, 2, 3, 2, True),
    (40, 8, 4, 2, 1, 1, False),
]


@pytest.mark.parametrize("T", [4, 8, 16])
@pytest.mark.parametrize("geom", SEQ)
def test_sequential_slots_equal_oracle_locate(T, geom):
    """One tile, keys in input order: the GPU table equals the oracle's bit
    for bit, and every returned slot equals the oracle's slot for the key
    (FULL and INVALID keys: none), for find-or-put and for lookups."""
    w, kb, N0, N1, f0, f1, compact = geom
    t = P().Table(P().ICEBERG, w, 1 << N0, 1 << N1, key_bytes=kb, fields_per_word=f0,
                  fields_per_word_backyard=f1, compact=compact, seed=31 + N0, tile=T,
                  items_per_thread=2, max_tiles=1, cta_threads=64)
    o = mirror(t)
    fresh = W.unique_keys(0, int(1.1 * t.slots), w, 70 + T)
    rng = np.random.default_rng(T)
    dup = fresh[torch.from_numpy(rng.integers(0, len(fresh), len(fresh) // 2))]
    keys = torch.cat([fresh, dup])
    keys = keys[torch.from_numpy(rng.permutation(len(keys)))]
    keys[7] = 0
    st, slots = t.find_or_put(dev_keys(keys, kb), slots=True)
    kn = keys.numpy().astype(np.uint64)
    ost = o.insert(kn)
    assert (st.cpu().numpy() == ost).all()
    assert (ost == oracle.FULL).sum() > 0
    assert np.array_equal(words(t, 0), o.t0) and np.array_equal(words(t, 1), o.t1)
    want = o.locate(kn)
    assert np.array_equal(as_u64(slots), np.where((ost == oracle.FOUND) | (ost == oracle.PUT),
                                                  want, NONE))
    # lookups: present keys return their slot, absent ones none
    q = W.unique_keys(0, int(1.3 * t.slots), w, 70 + T)
    fst, fslots = t.find(dev_keys(q, kb), slots=True)
    qn = q.numpy().astype(np.uint64)
    assert (fst.cpu().numpy() == o.find(qn)).all()
    assert np.array_equal(as_u64(fslots), o.locate(qn))


@pytest.mark.parametrize("T,items", [(4, 1), (4, 2), (8, 1), (16, 4), (8, 4)])
@pytest.mark.parametrize("f0", [2, 4])
def test_concurrent_slots_locate_their_keys(T, items, f0):
    """The warp-batched engine under contention (many repeats, a table
    driven past capacity): every FOUND / PUT slot holds its key in the
    GPU's table, repeats of one key share one slot, FULL keys get none, and
    a later lookup returns the same slots."""
    w = 25 if f0 == 4 else 36  # 16-bit primary slots hold remainders of 15 bits
    t = P().Table(P().ICEBERG, w, 1 << 10, 1 << 7, key_bytes=8, fields_per_word=f0,
                  fields_per_word_backyard=2, seed=5 + T, tile=T, items_per_thread=items)
    fresh = W.unique_keys(0, int(1.05 * t.slots), w, 300 + T)
    rng = np.random.default_rng(items)
    keys = torch.cat([fresh, fresh[torch.from_numpy(rng.integers(0, len(fresh), len(fresh)))]])
    keys = keys[torch.from_numpy(rng.permutation(len(keys)))]
    st, slots = t.find_or_put(keys.to(DEV), slots=True)
    st, s = st.cpu().numpy(), as_u64(slots)
    kn = keys.numpy().astype(np.uint64)
    Pm = P()
    ok = (st == Pm.FOUND) | (st == Pm.PUT)
    assert (st == Pm.FULL).sum() > 0 and ok.sum() > 0
    assert (s[~ok] == NONE).all()
    d = dumped(t)
    assert np.array_equal(s[ok], d.locate(kn[ok]))
    # repeats share the slot
    order = np.argsort(kn[ok], kind="stable")
    ks, ss = kn[ok][order], s[ok][order]
    same = ks[1:] == ks[:-1]
    assert (ss[1:][same] == ss[:-1][same]).all()
    fst, fslots = t.find(keys.to(DEV), slots=True)
    assert np.array_equal(as_u64(fslots)[ok], s[ok])
    assert t.error_flags() == 0


def test_kv_map_put_get_assign():
    """KVMap: values land at their keys' slots and come back by key; a second
    put assigns; absent keys read as zero with NOT_FOUND."""
    Pm = P()
    t = Pm.Table(Pm.ICEBERG, 40, 1 << 12, 1 << 9, seed=12)
    kv = Pm.KVMap(t, torch.int64)
    keys = W.unique_keys(0, 100_000, 40, 808).to(DEV)
    vals = torch.arange(100_000, dtype=torch.int64, device=DEV) * 3 + 1
    st = kv.put(keys, vals)
    assert bool((st == Pm.PUT).all())
    got, gst = kv.get(keys)
    assert bool((gst == Pm.FOUND).all()) and torch.equal(got, vals)
    half = keys[::2]
    st2 = kv.put(half, -vals[::2])
    assert bool((st2 == Pm.FOUND).all())
    got, _ = kv.get(keys)
    assert torch.equal(got[::2], -vals[::2]) and torch.equal(got[1::2], vals[1::2])
    absent = W.unique_keys(100_000, 1000, 40, 808).to(DEV)
    got, gst = kv.get(absent)
    assert bool((gst == Pm.NOT_FOUND).all()) and bool((got == 0).all())
    # float values of 4 bytes
    kv32 = Pm.KVMap(Pm.Table(Pm.ICEBERG, 40, 1 << 10, 1 << 7, seed=13), torch.float32)
    k2 = W.unique_keys(0, 20_000, 40, 809).to(DEV)
    v2 = torch.rand(20_000, device=DEV)
    kv32.put(k2, v2)
    assert torch.equal(kv32.get(k2)[0], v2)


def test_slots_unsupported_on_cuckoo():
    Pm = P()
    t = Pm.Table(Pm.CUCKOO, 32, 1 << 8, key_bytes=4, seed=1)
    k = dev_keys(W.unique_keys(0, 100, 32, 1), 4)
    with pytest.raises(Pm.ChtError):
        t.find(k, slots=True)
    with pytest.raises(ValueError):
        Pm.KVMap(t)


@pytest.mark.parametrize("T", [4, 8])
def test_kv_sequential_values_at_oracle_slots(T):
    """One tile, keys in input order (ordered engine): each value lands at
    the oracle's slot for its key, a repeated key keeps the value of its last
    occurrence, FULL keys store nothing, and get reads every stored value
    back (zero for keys never stored)."""
    Pm = P()
    t = Pm.Table(Pm.ICEBERG, 32, 1 << 4, 1 << 2, key_bytes=4, fields_per_word=2,
                 fields_per_word_backyard=2, seed=3, tile=T, max_tiles=1, cta_threads=64)
    kv = Pm.KVMap(t, torch.int64)
    o = mirror(t)
    fresh = W.unique_keys(0, int(1.1 * t.slots), 32, 5)
    rng = np.random.default_rng(2)
    keys = torch.cat([fresh, fresh[torch.from_numpy(rng.integers(0, len(fresh), 300))]])
    keys = keys[torch.from_numpy(rng.permutation(len(keys)))]
    vals = torch.arange(len(keys), dtype=torch.int64) * 7 + 11
    st = kv.put(dev_keys(keys, 4), vals.to(DEV)).cpu().numpy()
    kn = keys.numpy().astype(np.uint64)
    ost = o.insert(kn)
    assert (st == ost).all() and (ost == oracle.FULL).sum() > 0
    store = kv.values.cpu().numpy()
    last = {}
    for k, v, s_ in zip(kn.tolist(), vals.numpy().tolist(), ost.tolist()):
        if s_ in (oracle.FOUND, oracle.PUT):
            last[k] = v
    loc = o.locate(np.array(list(last), dtype=np.uint64))
    assert (store[loc.astype(np.int64)] == np.array(list(last.values()))).all()
    got, gst = kv.get(dev_keys(keys, 4))
    got, gst = got.cpu().numpy(), gst.cpu().numpy()
    want = np.array([last.get(k, 0) for k in kn.tolist()])
    assert (got == want).all()
    assert ((gst == Pm.FOUND) == np.array([k in last for k in kn.tolist()])).all()
