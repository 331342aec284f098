"""The C-ABI library loads, exports every symbol include/cht.h declares, and
its host-only planner (configuration resolution, storage size) follows the
paper's bit budgets. No GPU needed: nothing here launches a kernel."""
import ctypes
import os
import re

import pytest

from conftest import ROOT, read_golden


@pytest.fixture(scope="module")
def lib():
    from paper_2406_09255_gb300 import build as B
    B.build()
    from paper_2406_09255_gb300 import _lib
    return _lib


def _declared():
    src = open(os.path.join(ROOT, "include", "cht.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cht_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    L = lib.load()
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), f"{name} declared in cht.h but not exported"
    # the binding declares exactly the header's entry points
    assert sorted(lib.SIGNATURES) == names


def test_binding_struct_matches_header_layout(lib):
    # 4 ints, 2 u64, 4 ints, u64, 6 launch ints, retry_limit, stash_slots,
    # bucket_words and one reserved int
    assert ctypes.sizeof(lib.Config) == 4 * 4 + 16 + 4 * 4 + 8 + 6 * 4 + 16
    assert ctypes.sizeof(lib.Counters) == 32


def _resolve(lib, **kw):
    from paper_2406_09255_gb300.table import _make_config
    c = _make_config(**kw)
    out = lib.Config()
    code = lib.load().cht_resolve_config(ctypes.byref(c), ctypes.byref(out))
    return code, out


def test_workload_layouts(lib):
    # compact cuckoo, 2^14 buckets, 32-bit keys: 18-bit remainders + 2 tag bits
    # -> three fields per word, 48 slots per bucket, 786,432 slots
    code, c = _resolve(lib, kind=0, key_bits=32, key_bytes=4, num_buckets=1 << 14)
    assert code == 0 and c.fields_per_word == 3 and c.num_hashes == 3
    assert c.lookups_in_flight == 4  # default: the stream form, four loads per tile
    assert (1 << 14) * 16 * c.fields_per_word == 786432
    # 2^24 buckets, 40-bit keys: 16 + 2 bits -> three per word (805,306,368 slots), 2 GiB
    code, c = _resolve(lib, kind=0, key_bits=40, num_buckets=1 << 24)
    assert code == 0 and c.fields_per_word == 3
    assert lib.load().cht_table_bytes(ctypes.byref(c)) == 256 + (1 << 24) * 128
    # iceberg, 48-bit keys, 2^22 primary (26-bit remainders + flag) and 2^19
    # secondary buckets (29 bits + 2 tag bits): two 32-bit fields per word
    code, c = _resolve(lib, kind=1, key_bits=48, num_buckets=1 << 22,
                       num_buckets_backyard=1 << 19)
    assert code == 0 and c.fields_per_word == 2 and c.fields_per_word_backyard == 2
    assert (1 << 22) * 32 + (1 << 19) * 32 == 150994944
    # whole-key table: 64-bit slots
    code, c = _resolve(lib, kind=0, key_bits=40, num_buckets=3 << 24, compact=0)
    assert code == 0 and c.fields_per_word == 1


def test_bit_budget_section_5_1(lib):
    g = {r[0]: int(r[1]) for r in read_golden("bit_budget.txt")}
    nb0 = 1 << g["primary_buckets_log2"]
    nb1 = 1 << g["secondary_buckets_log2"]
    # 16-bit primary slots (4 per word): the widest key that fits is 37 bits
    code, _ = _resolve(lib, kind=1, key_bits=g["max_key_bits"], num_buckets=nb0,
                       num_buckets_backyard=nb1, fields_per_word=4, fields_per_word_backyard=2)
    assert code == 0
    code, _ = _resolve(lib, kind=1, key_bits=g["max_key_bits"] + 1, num_buckets=nb0,
                       num_buckets_backyard=nb1, fields_per_word=4, fields_per_word_backyard=2)
    assert code == lib.CHT_ERR_INVALID
    # 37-bit keys do not fit 16-bit secondary slots, but fit 32-bit ones
    code, _ = _resolve(lib, kind=1, key_bits=g["max_key_bits"], num_buckets=nb0,
                       num_buckets_backyard=nb1, fields_per_word=4, fields_per_word_backyard=4)
    assert code == lib.CHT_ERR_INVALID


@pytest.mark.parametrize("kw,frag", [
    (dict(kind=2, key_bits=32, num_buckets=16), "kind"),
    (dict(kind=0, key_bits=40, key_bytes=4, num_buckets=16), "key_bits"),
    (dict(kind=0, key_bits=32, num_buckets=12), "power of two"),
    (dict(kind=0, key_bits=32, num_buckets=16, tile=32), "tile"),
    (dict(kind=0, key_bits=32, num_buckets=16, items_per_thread=9), "items"),
    (dict(kind=0, key_bits=32, num_buckets=16, cta_threads=48), "cta_threads"),
    (dict(kind=1, key_bits=32, num_buckets=16, num_buckets_backyard=0), "backyard"),
    (dict(kind=0, key_bits=62, num_buckets=4, fields_per_word=2), "bits"),
    (dict(kind=0, key_bits=32, num_buckets=16, lookups_in_flight=2), "lookups_in_flight"),
    (dict(kind=0, key_bits=60, num_buckets=1 << 33), "at most 2^32"),
    (dict(kind=0, key_bits=32, num_buckets=16, lookups_in_flight=16), "lookups_in_flight"),
    (dict(kind=1, key_bits=32, num_buckets=16, num_buckets_backyard=2, retry_limit=-1),
     "retry_limit"),
    (dict(kind=1, key_bits=32, num_buckets=16, num_buckets_backyard=2, retry_limit=40000),
     "retry_limit"),
    (dict(kind=0, key_bits=32, num_buckets=16, stash_slots=8), "stash"),
    (dict(kind=1, key_bits=32, num_buckets=16, num_buckets_backyard=2, stash_slots=12), "stash"),
    (dict(kind=0, key_bits=32, num_buckets=16, bucket_words=6), "bucket_words"),
    (dict(kind=0, key_bits=32, num_buckets=16, bucket_words=8, tile=8), "tile must be 0 or 4"),
])
def test_invalid_configs_rejected_with_message(lib, kw, frag):
    code, _ = _resolve(lib, **kw)
    assert code == lib.CHT_ERR_INVALID
    assert frag in lib.load().cht_last_error().decode()


def test_storage_sizes_of_stash_and_bucket_widths(lib):
    L = lib.load()
    from paper_2406_09255_gb300.table import _make_config
    c = _make_config(kind=1, key_bits=32, num_buckets=1 << 10, num_buckets_backyard=1 << 7)
    base = L.cht_table_bytes(ctypes.byref(c))
    assert base == 256 + ((1 << 10) + (1 << 7)) * 128
    # the stash: 8 bytes a slot, rounded up to 128-byte lines
    for slots, extra in ((2, 128), (16, 128), (32, 256), (1 << 20, 8 << 20)):
        c = _make_config(kind=1, key_bits=32, num_buckets=1 << 10, num_buckets_backyard=1 << 7,
                         stash_slots=slots)
        assert L.cht_table_bytes(ctypes.byref(c)) == base + extra
    for wpb in (4, 8):
        c = _make_config(kind=0, key_bits=32, num_buckets=1 << 10, bucket_words=wpb)
        assert L.cht_table_bytes(ctypes.byref(c)) == 256 + (1 << 10) * 8 * wpb
        code, r = _resolve(lib, kind=0, key_bits=32, num_buckets=1 << 10, bucket_words=wpb)
        assert code == 0 and r.bucket_words == wpb
    code, r = _resolve(lib, kind=0, key_bits=32, num_buckets=1 << 10)
    assert code == 0 and r.bucket_words == 16


def test_version(lib):
    assert b"sm_103a" in lib.load().cht_version()


def test_random_read_rejects_bad_arguments_without_a_launch(lib):
    """cht_random_read validates on the host before any CUDA call."""
    L = lib.load()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails validation
    sink = ctypes.c_void_p(1 << 21)
    assert L.cht_random_read(fake, 1 << 20, 100, 10, 0, sink, None) == lib.CHT_ERR_INVALID
    assert "block_bytes" in L.cht_last_error().decode()
    assert L.cht_random_read(None, 1 << 20, 128, 10, 0, sink, None) == lib.CHT_ERR_INVALID
    assert L.cht_random_read(fake, 3 * 128, 128, 10, 0, sink, None) == lib.CHT_ERR_INVALID
    assert "power of two" in L.cht_last_error().decode()
    assert L.cht_random_read(ctypes.c_void_p((1 << 20) + 8), 1 << 20, 128, 10, 0, sink,
                             None) == lib.CHT_ERR_INVALID


def test_random_claim_rejects_bad_arguments_without_a_launch(lib):
    L = lib.load()
    fake = ctypes.c_void_p(1 << 20)
    sink = ctypes.c_void_p(1 << 21)
    assert L.cht_random_claim(None, 1 << 20, 10, 0, sink, None) == lib.CHT_ERR_INVALID
    assert L.cht_random_claim(fake, 3 * 128, 10, 0, sink, None) == lib.CHT_ERR_INVALID
    assert "power of two" in L.cht_last_error().decode()
    assert L.cht_random_claim(ctypes.c_void_p((1 << 20) + 64), 1 << 20, 10, 0, sink,
                              None) == lib.CHT_ERR_INVALID
    assert L.cht_random_claim(fake, 1 << 20, 0, 0, sink, None) == lib.CHT_OK  # nothing to do


def test_value_moves_reject_bad_arguments_without_a_launch(lib):
    L = lib.load()
    fake = ctypes.c_void_p(1 << 20)
    assert L.cht_values_scatter(fake, 10, fake, 3, fake, 100, None) == lib.CHT_ERR_INVALID
    assert "value_bytes" in L.cht_last_error().decode()
    assert L.cht_values_gather(fake, 10, fake, 8, 100, None, None) == lib.CHT_ERR_INVALID
    assert L.cht_values_gather(ctypes.c_void_p((1 << 20) + 4), 10, fake, 8, 100, fake,
                               None) == lib.CHT_ERR_INVALID
    assert L.cht_values_scatter(fake, 0, fake, 8, fake, 100, None) == lib.CHT_OK  # empty: nothing to do


def test_null_handles_rejected_on_the_host(lib):
    """Every call taking a table or batch handle refuses NULL with
    CHT_ERR_INVALID before touching the GPU; destroy accepts NULL."""
    L = lib.load()
    z = ctypes.c_void_p(0)
    p = ctypes.c_void_p(1 << 20)  # never dereferenced: the handle check comes first
    INV = lib.CHT_ERR_INVALID
    calls = [
        lambda: L.cht_clear(z, None),
        lambda: L.cht_insert(z, p, 1, p, None, None),
        lambda: L.cht_find(z, p, 1, p, None),
        lambda: L.cht_find_or_put(z, p, 1, p, None),
        lambda: L.cht_find_or_put_slots(z, p, 1, p, p, None),
        lambda: L.cht_find_slots(z, p, 1, p, p, None),
        lambda: L.cht_kv_put(z, p, 1, p, 8, p, 10, p, None),
        lambda: L.cht_kv_get(z, p, 1, p, 8, 10, p, p, None),
        lambda: L.cht_enumerate(z, p, 1, p, None),
        lambda: L.cht_set_counters(z, None),
        lambda: L.cht_batch_launch(z, None),
        lambda: L.cht_batch_replay(z, None),
        lambda: L.cht_batch_clear(z, None),
        lambda: L.cht_batch_capture(z, None),
    ]
    for c in calls:
        assert c() == INV
        assert L.cht_last_error().decode()
    assert L.cht_destroy(z) == lib.CHT_OK
    assert L.cht_batch_destroy(z) == lib.CHT_OK


def test_batch_scratch_and_create_validation_on_the_host(lib):
    """cht_batch_scratch_bytes gives one fixed-size descriptor per table for
    1..16384 tables (a multiple of 16 bytes, so descriptors stay aligned) and
    0 outside; cht_batch_create checks its count, op, scratch alignment and
    size before it looks at any table."""
    L = lib.load()
    d = L.cht_batch_scratch_bytes(1)
    assert d > 0 and d % 16 == 0
    assert L.cht_batch_scratch_bytes(256) == 256 * d
    assert L.cht_batch_scratch_bytes(0) == 0 and L.cht_batch_scratch_bytes(16385) == 0
    p = ctypes.c_void_p(1 << 20)  # never dereferenced: every call fails validation
    arr = (ctypes.c_void_p * 1)(p)
    ns = (ctypes.c_size_t * 1)(10)
    out = ctypes.c_void_p(0)
    INV = lib.CHT_ERR_INVALID

    def create(count=1, op=0, scratch=p, nbytes=d):
        return L.cht_batch_create(arr, arr, ns, arr, count, op, scratch, nbytes, None,
                                  ctypes.byref(out))

    assert create(count=0) == INV and "count" in L.cht_last_error().decode()
    assert create(count=16385) == INV
    assert create(op=7) == INV and "op" in L.cht_last_error().decode()
    assert create(scratch=ctypes.c_void_p((1 << 20) + 8)) == INV
    assert create(nbytes=d - 1) == lib.CHT_ERR_CAPACITY
    assert out.value is None
