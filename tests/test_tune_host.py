"""The table tuner's candidate shapes (host logic, no GPU)."""
from paper_2406_09255_gb300.tune import ITEMS, packing_candidates, table_candidates


def test_cuckoo_candidates_cover_chunk_and_stream_forms():
    c = table_candidates(0, "find", 4, tiles=(4, 8), items=(1, 2))
    assert c == [(4, 1, 1), (4, 2, 1), (8, 1, 1), (8, 2, 1),
                 (4, 1, 4), (8, 1, 4), (4, 1, 8), (8, 1, 8)]
    assert len(set(c)) == len(c)


def test_iceberg_candidates_keep_the_in_flight_setting():
    c = table_candidates(1, "find_or_put", 4, tiles=(4, 8, 16), items=(1, 2, 4))
    assert {p for _, _, p in c} == {4} and len(c) == 9
    c = table_candidates(1, "find", 1, tiles=(4,), items=(1, 2))
    assert c == [(4, 1, 1), (4, 2, 1)]


def test_explicit_in_flight_list_is_used():
    assert table_candidates(0, "insert", 4, tiles=(4,), items=(1, 2), in_flight=(8,)) == [
        (4, 1, 8)]


def test_items_are_the_counts_the_kernels_are_built_for():
    assert ITEMS == (1, 2, 4)


def test_packing_candidates_densest_and_one_wider():
    # compact cuckoo, 2^24 buckets, 40-bit keys: 16 + 2 bits -> 3 fields
    # (21 bits) or 2 (32 bits)
    assert packing_candidates(0, 40, 1 << 24) == [(3, 0), (2, 0)]
    # 2^14 buckets, 32-bit keys: 18 + 2 = 20 bits -> 3 or 2
    assert packing_candidates(0, 32, 1 << 14) == [(3, 0), (2, 0)]
    # 2^22 buckets, 36-bit keys: 14 + 2 = 16 bits -> 4 (16-bit fields) or 3
    assert packing_candidates(0, 36, 1 << 22) == [(4, 0), (3, 0)]
    # whole keys: one 64-bit slot per word only
    assert packing_candidates(0, 40, 1 << 24, compact=False) == [(1, 0)]
    # iceberg, 48-bit keys, 2^22 + 2^19 buckets: 26 + 1 and 29 + 2 bits -> 2
    # or 1 per level
    assert packing_candidates(1, 48, 1 << 22, 1 << 19) == [(2, 2), (2, 1), (1, 2), (1, 1)]
    # 62-bit keys, 2 buckets: 61 + 2 bits need a whole word
    assert packing_candidates(0, 62, 2) == [(1, 0)]
