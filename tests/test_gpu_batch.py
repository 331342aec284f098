"""Fused multi-table batches (one persistent launch over many iceberg tables,
plain or replayed from a CUDA graph) against the per-table contract and the
oracle: for every table of the batch, exactly one PUT per distinct key, the
stored set equal to the oracle's, a well-formed table (Theorem 1 (a)), and
lookups that equal membership."""
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


def P():
    import paper_2406_09255_gb300 as m
    return m


def mirror(t):
    c = t.cfg
    return oracle.Table(c.kind, c.key_bits, c.num_buckets, c.num_buckets_backyard,
                        compact=bool(c.compact), fpw0=c.fields_per_word,
                        fpw1=c.fields_per_word_backyard, seed=c.seed)


def dump(t):
    o = mirror(t)
    o.load_words(t.words(0).cpu().numpy().view(np.uint64),
                 t.words(1).cpu().numpy().view(np.uint64))
    return o


def u64(x):
    a = x.detach().cpu().numpy()
    return a.view(np.uint32).astype(np.uint64) if a.dtype == np.int32 else a.view(np.uint64)


def make_tables(spec, key_bits=32, seed0=100):
    m = P()
    tables, keys = [], []
    for i, (e, size, distinct) in enumerate(spec):
        t = m.Table(m.ICEBERG, key_bits, 1 << e, 1 << (e - 3), key_bytes=4, fields_per_word=2,
                    seed=seed0 + i)
        k = W.duplicate_stream(size, distinct, key_bits, seed0 + 7 * i, 0.3)
        tables.append(t)
        keys.append(W.to_u32(k).to(DEV))
    return tables, keys


SPEC = [(8, 5000, 3500), (12, 100000, 70000), (9, 1, 1), (10, 20000, 14000), (14, 300000, 210000),
        (8, 1000, 700), (11, 0, 0), (13, 77777, 54443)]


def check_table(t, k, st):
    m = P()
    kn = u64(k)
    st = st.cpu().numpy()
    o = mirror(t)
    ost = o.insert(kn) if len(kn) else np.zeros(0, np.uint8)
    assert (ost != oracle.FULL).all()
    assert ((st == m.PUT) | (st == m.FOUND)).all()
    if len(kn):
        uniq, inv = np.unique(kn, return_inverse=True)
        puts = np.bincount(inv, weights=(st == m.PUT), minlength=len(uniq))
        assert (puts == 1).all()
    stored, cnt = t.enumerate()
    assert np.array_equal(np.sort(u64(stored)), np.sort(o.enumerate()))
    d = dump(t)
    assert d.check_entries() == 0 and d.check_order_property() == 0 and d.check_prefix() == 0
    assert d.check_duplicates() == 0


@pytest.mark.parametrize("tile,items", [(4, 2), (8, 1), (16, 8)])
def test_fused_batch_find_or_put(tile, items):
    m = P()
    from paper_2406_09255_gb300.batch import Batch, OP_FIND
    tables, keys = make_tables(SPEC)
    b = Batch(tables, keys)
    b.set_launch(tile=tile, items_per_thread=items)
    sts = b.launch()
    torch.cuda.synchronize()
    for t, k, s in zip(tables, keys, sts):
        check_table(t, k, s)
        assert t.error_flags() == 0
    # lookups of all keys plus absent ones, fused, are exact membership
    qk = [torch.cat([k, W.to_u32(W.unique_keys(10**6, 500, 32, 999 + i)).to(DEV)])
          for i, k in enumerate(keys)]
    bf = Batch(tables, qk, op=OP_FIND)
    fs = bf.launch()
    for t, q, s in zip(tables, qk, fs):
        stored = set(u64(t.enumerate()[0]).tolist())
        want = np.array([int(x) in stored for x in u64(q)])
        assert np.array_equal(s.cpu().numpy() == m.FOUND, want)


def test_graph_replay_matches_and_repeats():
    m = P()
    from paper_2406_09255_gb300.batch import Batch
    tables, keys = make_tables(SPEC, seed0=300)
    b = Batch(tables, keys)
    b.capture()
    for rep in range(2):
        b.clear()
        sts = b.replay()
        torch.cuda.synchronize()
        for t, k, s in zip(tables, keys, sts):
            check_table(t, k, s)
    # replay without clearing: everything is already there
    sts = b.replay()
    for s in sts:
        assert (s.cpu().numpy() == m.FOUND).all()


def test_fused_equals_per_table_sets():
    from paper_2406_09255_gb300.batch import Batch, per_table
    tables, keys = make_tables(SPEC, seed0=500)
    tables2, _ = make_tables(SPEC, seed0=500)
    b = Batch(tables, keys)
    b.launch()
    st2 = [torch.empty(k.numel(), dtype=torch.uint8, device=DEV) for k in keys]
    per_table(tables2, keys, st2)
    for t1, t2, s1, s2 in zip(tables, tables2, b.statuses, st2):
        assert np.array_equal(np.sort(u64(t1.enumerate()[0])), np.sort(u64(t2.enumerate()[0])))
        # the same number of PUTs (one per distinct key) on both paths
        assert int((s1 == 2).sum()) == int((s2 == 2).sum())


def test_batch_rejects_mixed_packing_and_cuckoo():
    m = P()
    from paper_2406_09255_gb300.batch import Batch
    a = m.Table(m.ICEBERG, 32, 1 << 8, 1 << 5, key_bytes=4, fields_per_word=2, seed=1)
    b = m.Table(m.ICEBERG, 32, 1 << 8, 1 << 5, key_bytes=4, fields_per_word=1, seed=1)
    c = m.Table(m.CUCKOO, 32, 1 << 8, key_bytes=4, seed=1)
    k = torch.ones(4, dtype=torch.int32, device=DEV)
    with pytest.raises(m.ChtError):
        Batch([a, b], [k, k])
    with pytest.raises(m.ChtError):
        Batch([a, c], [k, k])


def test_lookup_batch_may_repeat_a_table_find_or_put_may_not():
    """A lookup batch lists one table several times, each entry over its own
    keys placed in one buffer (Batch.from_pointers), and answers each entry
    as cht_find on that table; a find-or-put batch that lists a table twice
    is refused."""
    m = P()
    from paper_2406_09255_gb300.batch import OP_FIND, Batch
    tables, keys = make_tables(SPEC[:2], seed0=800)
    for t, k in zip(tables, keys):
        t.find_or_put(k)
    w = 32
    # half of each table's queries were put (its batch's distinct keys come
    # first in the same key sequence)
    q = [W.to_u32(W.unique_keys(lo, n, w, 800 + 7 * i)).to(DEV)
         for i, lo, n in ((0, 2000, 3000), (1, 67500, 5000))]
    # entries: table 0, table 1, table 0 again, table 1 again (one buffer)
    parts = [q[0][:1000], q[1][:2000], q[0][1000:], q[1][2000:]]
    buf = torch.cat(parts)
    st = torch.full((buf.numel(),), 255, dtype=torch.uint8, device=DEV)
    offs = np.cumsum([0] + [p.numel() for p in parts])[:-1]
    tabs = [tables[0], tables[1], tables[0], tables[1]]
    b = Batch.from_pointers(tabs, [buf.data_ptr() + 4 * int(o) for o in offs],
                            [p.numel() for p in parts], [st.data_ptr() + int(o) for o in offs],
                            op=OP_FIND)
    b.launch()
    want = torch.cat([t.find(p) for t, p in zip(tabs, parts)])
    assert torch.equal(st, want)
    assert int((want == m.FOUND).sum()) > 0 and int((want == m.NOT_FOUND).sum()) > 0
    with pytest.raises(m.ChtError):
        Batch([tables[0], tables[1], tables[0]], [keys[0], keys[1], keys[0]])


def test_tuner_picks_a_valid_shape(tmp_path, monkeypatch):
    monkeypatch.setenv("CHT_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2406_09255_gb300.batch import Batch
    from paper_2406_09255_gb300.tune import tune_batch
    tables, keys = make_tables(SPEC[:4], seed0=700)
    b = Batch(tables, keys)
    r = tune_batch(b, reps=1, tiles=(4, 8), items=(1, 2))
    assert r["tile"] in (4, 8) and r["items"] in (1, 2) and not r["cached"]
    # the tuner restored the empty tables: a launch now inserts everything
    sts = b.launch()
    for t, k, s in zip(tables, keys, sts):
        check_table(t, k, s)
    r2 = tune_batch(b, reps=1)
    assert r2["cached"] and r2["tile"] == r["tile"]


def test_table_tuner_sweeps_loads_in_flight(tmp_path, monkeypatch):
    """tune_table on a cuckoo table tries the chunk put (one load in flight,
    several items per lane) and the stream put (4 or 8 loads in flight),
    restores the table after every trial and applies the winner, which then
    stores every key."""
    monkeypatch.setenv("CHT_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2406_09255_gb300.tune import tune_table
    t = P().Table(P().CUCKOO, 32, 1 << 12, key_bytes=4, seed=44)
    n = int(0.85 * t.slots)
    keys = W.to_u32(W.unique_keys(0, n, 32, 4040)).to(DEV)
    r = tune_table(t, "insert", keys, reps=1, tiles=(4, 8), items=(1, 2))
    shapes = {(x["tile"], x["items"], x["in_flight"]) for x in r["sweep"]}
    assert shapes == {(4, 1, 1), (4, 2, 1), (8, 1, 1), (8, 2, 1),
                      (4, 1, 4), (8, 1, 4), (4, 1, 8), (8, 1, 8)}
    assert (r["tile"], r["items"], r["in_flight"]) in shapes and not r["cached"]
    assert t.cfg.lookups_in_flight == r["in_flight"]
    assert t.enumerate()[1] == 0  # restored to the empty table
    st = t.insert(keys).cpu().numpy()
    assert (st == P().PUT).all() and t.enumerate()[1] == n
    r2 = tune_table(t, "insert", keys, reps=1)
    assert r2["cached"] and r2["in_flight"] == r["in_flight"]


def test_packing_tuner_times_densest_and_wider(tmp_path, monkeypatch):
    """tune_packing times find-or-put on a fresh table of each candidate
    packing (densest, and one step wider per level) and returns one; a table
    built with the choice meets the find-or-put contract against the
    oracle."""
    monkeypatch.setenv("CHT_TUNE_CACHE", str(tmp_path / "tune.json"))
    import oracle
    from paper_2406_09255_gb300.tune import packing_candidates, tune_packing
    w, nb0, nb1 = 38, 1 << 12, 1 << 9  # 26 + 1 and 29 + 2 bits: 2 or 1 fields per level
    keys = W.unique_keys(0, 40000, w, 515)
    keys = torch.cat([keys, keys[:10000]]).to(DEV)
    r = tune_packing(1, w, nb0, nb1, keys, "find_or_put", reps=1, seed=5)
    cands = packing_candidates(1, w, nb0, nb1)
    assert len(r["sweep"]) == len(cands) == 4 and not r["cached"]
    assert (r["fields_per_word"], r["fields_per_word_backyard"]) in cands
    t = P().Table(P().ICEBERG, w, nb0, nb1, fields_per_word=r["fields_per_word"],
                  fields_per_word_backyard=r["fields_per_word_backyard"], seed=5)
    st = t.find_or_put(keys).cpu().numpy()
    kn = keys.cpu().numpy().view(np.uint64)
    o = oracle.Table(oracle.ICEBERG, w, nb0, nb1, fpw0=t.cfg.fields_per_word,
                     fpw1=t.cfg.fields_per_word_backyard, seed=t.cfg.seed)
    ost = o.insert(kn)
    assert (ost != oracle.FULL).all()
    uniq, inv = np.unique(kn, return_inverse=True)
    puts = np.bincount(inv, weights=(st == P().PUT), minlength=len(uniq))
    assert (puts == 1).all()
    r2 = tune_packing(1, w, nb0, nb1, keys, "find_or_put", reps=1, seed=5)
    assert r2["cached"] and r2["fields_per_word"] == r["fields_per_word"]


def test_config4_full_shape_fused_and_graph_replay():
    """The benchmark's 256-table batch at full shape (primary 2^8..2^18
    buckets, secondary 1/8, 32-bit keys, log-uniform 1K..1M-key batches with
    30 % duplicates), built exactly as the benchmark builds it, through one
    fused launch and then, from empty tables again, one CUDA-graph replay.
    Every table, both times: one PUT per distinct key, the rest FOUND. The
    graph replay stores the same set in every table as the fused launch. A
    sample of tables (the four largest batches into 2^18-bucket tables and
    every 32nd table) is checked against the oracle's sequential replay
    (stored set) and Theorem 1's invariants on the dump."""
    from paper_2406_09255_gb300.batch import Batch
    m = P()
    spec = W.multi_table_spec()
    assert len(spec) == 256 and max(e for e, _, _ in spec) == 18
    tables, keys = [], []
    for i, (e, size, distinct) in enumerate(spec):
        tables.append(m.Table(m.ICEBERG, 32, 1 << e, 1 << (e - 3), key_bytes=4,
                              fields_per_word=2, seed=4000 + i))
        keys.append(W.to_u32(W.duplicate_stream(size, distinct, 32, W.SEED_BASE + 4 + 7 * i,
                                                0.3, device=DEV)))
    big = sorted((i for i, (e, _, _) in enumerate(spec) if e == 18), key=lambda i: -spec[i][1])
    sample = sorted(set(big[:4]) | set(range(0, 256, 32)))
    b = Batch(tables, keys)
    stored = {}
    for mode in ("fused", "graph"):
        b.clear()
        if mode == "fused":
            b.launch()
        else:
            b.capture()
            b.replay()
        torch.cuda.synchronize()
        for i, (t, k, s) in enumerate(zip(tables, keys, b.statuses)):
            st = s.cpu().numpy()
            assert ((st == m.PUT) | (st == m.FOUND)).all(), (mode, i)
            kn = u64(k)
            if len(kn):
                uniq, inv = np.unique(kn, return_inverse=True)
                assert (np.bincount(inv, weights=(st == m.PUT), minlength=len(uniq)) == 1).all()
            got = torch.sort(t.enumerate()[0])[0]
            if mode == "fused":
                stored[i] = got
                if i in sample:
                    check_table(t, k, s)
            else:
                assert torch.equal(got, stored[i]), i
