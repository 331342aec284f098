"""The allocation-free fused find-or-put, cht_batch_find_or_put_static.

Some callers cannot allocate device memory when they need a batch done: code
that runs while another thread captures a CUDA graph in global capture mode
(cudaMalloc is an illegal call then), latency-critical loops that cannot take
the device-wide synchronisation cudaMalloc/cudaFree may cause, and processes
whose GPU memory another allocator has already reserved. For them the library
keeps the batch descriptors in a fixed device array of its own (room for
CHT_STATIC_BATCH_MAX tables) instead of caller scratch.

This file checks, through the C ABI, that the entry point gives the same
results as the planned batch (cht_batch_create + cht_batch_launch) on two
calls in a row, that every table's stored set and per-key outcomes equal the
sequential oracle's replay of its keys (also for a batch of more tables than
one descriptor upload carries), and that it rejects batches larger than its
array. It is collected last so that a failing run has already run every other
test.
"""
import ctypes

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


def _tables_and_keys(seed0):
    import paper_2406_09255_gb300 as m
    shapes = [(8, 4000, 4000), (11, 50000, 35000), (9, 1, 1), (13, 120000, 120000),
              (10, 0, 0), (12, 60000, 42000)]
    tables, keys = [], []
    for i, (e, size, distinct) in enumerate(shapes):
        tables.append(m.Table(m.ICEBERG, 32, 1 << e, 1 << (e - 3), key_bytes=4,
                              fields_per_word=2, seed=seed0 + i))
        k = W.duplicate_stream(size, distinct, 32, seed0 + 11 * i, 0.3)
        keys.append(W.to_u32(k).to(DEV))
    return tables, keys


def _static_call(tables, keys, statuses):
    from paper_2406_09255_gb300 import _lib
    L = _lib.load()
    cnt = len(tables)
    vp = ctypes.c_void_p
    T = (vp * cnt)(*[t.handle for t in tables])
    K = (vp * cnt)(*[k.data_ptr() for k in keys])
    N = (ctypes.c_size_t * cnt)(*[k.numel() for k in keys])
    S = (vp * cnt)(*[s.data_ptr() for s in statuses])
    stream = torch.cuda.current_stream().cuda_stream
    return L.cht_batch_find_or_put_static(T, K, N, S, cnt, stream), L


def _stored(t):
    out, n = t.enumerate()
    return np.sort(out.cpu().numpy().view(np.uint32).astype(np.uint64))


def _oracle_replay(t, kn):
    """The sequential oracle on table t's geometry, fed kn in input order."""
    c = t.cfg
    o = oracle.Table(oracle.ICEBERG, c.key_bits, c.num_buckets, c.num_buckets_backyard,
                     fpw0=c.fields_per_word, fpw1=c.fields_per_word_backyard, seed=c.seed)
    return o, o.insert(kn)


def _check_against_oracle(m, t, kn, st):
    """Per distinct key the oracle's outcome (one PUT, the rest FOUND, when
    the replay reports no FULL), and the oracle's stored set."""
    o, ost = _oracle_replay(t, kn)
    assert (ost != oracle.FULL).all()
    uniq, inv = np.unique(kn, return_inverse=True)
    puts = np.bincount(inv, weights=(st == m.PUT), minlength=len(uniq))
    oputs = np.bincount(inv, weights=(ost == oracle.PUT), minlength=len(uniq))
    assert np.array_equal(puts, oputs)
    assert ((st == m.PUT) | (st == m.FOUND)).all()
    assert np.array_equal(_stored(t), np.sort(o.enumerate()))


def test_static_batch_matches_planned_batch_on_two_calls():
    import paper_2406_09255_gb300 as m
    from paper_2406_09255_gb300.batch import Batch
    ref_tables, keys = _tables_and_keys(900)
    new_tables, keys2 = _tables_and_keys(900)
    for a, b in zip(keys, keys2):
        assert torch.equal(a, b)
    planned = Batch(ref_tables, keys)
    statuses = [torch.empty(k.numel(), dtype=torch.uint8, device=DEV) for k in keys]
    for call in range(2):
        planned.launch()
        code, L = _static_call(new_tables, keys, statuses)
        assert code == m._lib.CHT_OK, L.cht_last_error()
        torch.cuda.synchronize()
        for t_ref, t_new, k, s_ref, s_new in zip(ref_tables, new_tables, keys,
                                                 planned.statuses, statuses):
            a, b = s_ref.cpu().numpy(), s_new.cpu().numpy()
            kn = k.cpu().numpy()
            # which duplicate wins a PUT may differ; per distinct key the
            # outcome may not: exactly one PUT on the first call, none after
            uniq, inv = np.unique(kn, return_inverse=True)
            for st in (a, b):
                assert ((st == m.PUT) | (st == m.FOUND)).all()
                puts = np.bincount(inv, weights=(st == m.PUT), minlength=len(uniq))
                assert (puts == (1 if call == 0 else 0)).all()
            if call == 1 or len(uniq) == len(kn):
                assert np.array_equal(a, b)  # the outcome is unique: compare every byte
            assert np.array_equal(_stored(t_ref), _stored(t_new))
            assert t_new.error_flags() == 0
            if call == 0:
                _check_against_oracle(m, t_new, kn.view(np.uint32).astype(np.uint64), b)


def test_static_batch_over_many_tables_matches_oracle():
    # 150 tables: the descriptors go up in three kernel-parameter blocks
    import paper_2406_09255_gb300 as m
    rng = np.random.default_rng(5)
    tables, keys, statuses = [], [], []
    for i in range(150):
        e = int(rng.integers(4, 9))
        tables.append(m.Table(m.ICEBERG, 32, 1 << e, 1 << max(e - 3, 0), key_bytes=4,
                              fields_per_word=2, seed=3000 + i))
        size = int(rng.integers(0, 12 * (1 << e)))
        k = W.duplicate_stream(size, max(size * 7 // 10, 1), 32, 77 + i, 0.3) if size else \
            torch.zeros(0, dtype=torch.int64)
        keys.append(W.to_u32(k).to(DEV))
        statuses.append(torch.empty(max(size, 1), dtype=torch.uint8, device=DEV))
    for call in range(2):
        code, L = _static_call(tables, keys, statuses)
        assert code == m._lib.CHT_OK, L.cht_last_error()
        torch.cuda.synchronize()
        for t, k, s in zip(tables, keys, statuses):
            kn = k.cpu().numpy().view(np.uint32).astype(np.uint64)
            st = s[: k.numel()].cpu().numpy()
            if call == 0:
                _check_against_oracle(m, t, kn, st)
            else:
                assert (st == m.FOUND).all()
            assert t.error_flags() == 0


def test_static_batch_rejects_more_tables_than_its_array_holds():
    import paper_2406_09255_gb300 as m
    from paper_2406_09255_gb300 import _lib
    L = _lib.load()
    t = m.Table(m.ICEBERG, 32, 1 << 8, 1 << 5, key_bytes=4, fields_per_word=2, seed=1)
    k = torch.ones(8, dtype=torch.int32, device=DEV)
    s = torch.empty(8, dtype=torch.uint8, device=DEV)
    limit = 256  # CHT_STATIC_BATCH_MAX
    code, L = _static_call([t] * (limit + 1), [k] * (limit + 1), [s] * (limit + 1))
    assert code == _lib.CHT_ERR_INVALID
    assert b"1..256" in L.cht_last_error()


def test_static_batch_rejects_a_table_listed_twice():
    import paper_2406_09255_gb300 as m
    from paper_2406_09255_gb300 import _lib
    a = m.Table(m.ICEBERG, 32, 1 << 8, 1 << 5, key_bytes=4, fields_per_word=2, seed=1)
    b = m.Table(m.ICEBERG, 32, 1 << 8, 1 << 5, key_bytes=4, fields_per_word=2, seed=2)
    k = torch.ones(8, dtype=torch.int32, device=DEV)
    s = torch.empty(8, dtype=torch.uint8, device=DEV)
    code, L = _static_call([a, b, a], [k] * 3, [s] * 3)
    assert code == _lib.CHT_ERR_INVALID
    assert b"twice" in L.cht_last_error()
    code, L = _static_call([a, b], [k] * 2, [s] * 2)
    assert code == _lib.CHT_OK
