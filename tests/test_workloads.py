"""The seeded input generators shared by the oracle-side and GPU-side tests
and the benchmark (no GPU): the key sequence is a bijection onto the nonzero
w-bit keys, the tensor and scalar versions agree, absent keys are never
inserted keys, lookup mixes have the stated hit count, and the find-or-put
stream introduces each fresh key once."""
import numpy as np
import pytest
import torch

from paper_2406_09255_gb300 import workloads as W


@pytest.mark.parametrize("w", [8, 9, 12])
def test_key_sequence_is_a_bijection_onto_nonzero_keys(w):
    seed = 1234 + w
    keys = W.unique_keys(0, (1 << w) - 1, w, seed)
    k = keys.numpy()
    assert k.min() >= 1 and k.max() < (1 << w)
    assert len(np.unique(k)) == (1 << w) - 1  # every nonzero w-bit key once


def test_tensor_and_scalar_generators_agree():
    w, seed = 40, 77
    idx = torch.tensor([0, 1, 2, 12345, (1 << 39) - 5], dtype=torch.int64)
    t = W.keys_at(idx, w, seed)
    z = W.key_index_skip(w, seed)
    for i, k in zip(idx.tolist(), t.tolist()):
        j = i + (1 if i >= z else 0)
        assert k == W.g_scalar(j, w, seed)
        assert W.g_scalar(k, w, seed, inverse=True) == j
    # odd widths cycle-walk and stay in range
    t9 = W.keys_at(torch.arange(500, dtype=torch.int64), 9, 3)
    assert int(t9.max()) < 512 and int(t9.min()) >= 1


def test_unique_keys_windows_concatenate():
    a = W.unique_keys(0, 1000, 36, 9)
    b = W.unique_keys(1000, 500, 36, 9)
    assert torch.equal(torch.cat([a, b]), W.unique_keys(0, 1500, 36, 9))


def test_permutation_is_a_permutation():
    for n in (1, 2, 7, 1000, 4097):
        p = W.permutation(n, 5).numpy()
        assert np.array_equal(np.sort(p), np.arange(n))
    assert np.array_equal(W.permutation(4097, 5, start=100, count=50).numpy(),
                          W.permutation(4097, 5).numpy()[100:150])


@pytest.mark.parametrize("hit", [0.0, 0.5, 1.0])
def test_find_queries_hit_count_and_absence(hit):
    n, nq, w, seed = 5000, 3000, 32, 11
    inserted = set(W.unique_keys(0, n, w, seed).tolist())
    q, present = W.find_queries(n, nq, hit, w, seed, n)
    assert int(present.sum()) == int(hit * nq)
    ql = q.tolist()
    assert len(set(ql)) == nq  # distinct queries
    assert all((k in inserted) == bool(p) for k, p in zip(ql, present.tolist()))


def test_to_u32_keeps_the_low_bits():
    k = torch.tensor([1, (1 << 31) - 1, 1 << 31, (1 << 32) - 1], dtype=torch.int64)
    u = W.to_u32(k)
    assert u.dtype == torch.int32
    assert (u.numpy().view(np.uint32).astype(np.int64) == k.numpy()).all()


def test_duplicate_stream_repeats_only_fresh_keys():
    s = W.duplicate_stream(1000, 700, 32, 21, 0.3)
    fresh = set(W.unique_keys(0, 700, 32, 21).tolist())
    sl = s.tolist()
    assert len(sl) == 1000 and set(sl) == fresh


def test_fop_stream_introduces_each_fresh_key_once():
    n_ops, w, seed = 20000, 40, 31
    keys, is_find, seen = W.fop_stream(n_ops, w, seed, max_distinct=3000, rng_seed=4)
    k, f, c = keys.numpy(), is_find.numpy(), seen.numpy()
    fops = k[~f]
    distinct = len(np.unique(fops))
    # the fresh keys, plus the misses of ops that come before any key exists
    assert distinct <= 3000 + int((c == 0).sum())
    assert (np.diff(c) >= 0).all() and c.max() <= 3000
    # fresh lookups never ask for a key a find-or-put introduced
    absent_base = 1 << (w - 2)
    fresh_find = W.keys_at(torch.tensor([absent_base]), w, seed).item()
    assert fresh_find not in set(fops.tolist()) or c[0] == 0
    # uncapped, about half of the find-or-puts are repeats of earlier keys
    k2, f2, _ = W.fop_stream(n_ops, w, seed, rng_seed=5)
    fops2 = k2.numpy()[~f2.numpy()]
    assert 0.4 < 1 - len(np.unique(fops2)) / len(fops2) < 0.6
