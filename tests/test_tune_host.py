"""The table tuner's candidate shapes (host logic, no GPU)."""
from paper_2406_09255_gb300.tune import table_candidates


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
