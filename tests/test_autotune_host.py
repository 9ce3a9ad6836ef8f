"""Host logic of the sort autotuner: which tunings it times."""
from paper_1308_2166_gb300 import autotune


def test_widths_only_where_a_pass_is_saved():
    # 25-bit ids: 8 -> 4 passes, 9 -> 3 (10 and 11 also 3: not timed)
    assert autotune._widths(25) == [8, 9]
    # 20 bits: 8 -> 3, 9 -> 3, 10 -> 2, 11 -> 2
    assert autotune._widths(20) == [8, 10]
    # 22 Step-3 bucket bits (w = 2^24): 8 -> 3, 11 -> 2
    assert autotune._widths(22) == [8, 11]
    assert autotune._widths(8) == [8]
    assert autotune._widths(32) == [8, 11]


def test_candidates_cover_every_useful_width_and_ranking():
    c = autotune.candidates(25, 1 << 24)
    assert len(c) == 2 * 2 * len(autotune.RANKINGS)
    assert (8, 8, 2) in c and (9, 11, 1) in c
    assert {rk for _, _, rk in c} == set(autotune.RANKINGS)
    # without the batch size every Step-3 width is timed
    assert len(autotune.candidates(20)) == 2 * len(autotune.DIGITS) * len(autotune.RANKINGS)


def test_tiny_vertex_ids_keep_8_bit_arc_digits():
    # with at most 8 id bits a wider arc digit would only add empty buckets
    c = autotune.candidates(8, 4096)
    assert all(ba == 8 for ba, _, _ in c)
