"""Host logic of the sort autotuner: which tunings it times."""
from paper_1308_2166_gb300 import autotune


def test_candidates_cover_every_width_and_ranking():
    c = autotune.candidates(20)
    assert len(c) == len(autotune.DIGITS) ** 2 * len(autotune.RANKINGS)
    assert (8, 8, 2) in c and (11, 11, 1) in c
    assert {rk for _, _, rk in c} == set(autotune.RANKINGS)


def test_tiny_vertex_ids_keep_8_bit_arc_digits():
    # with at most 8 id bits a wider arc digit would only add empty buckets
    c = autotune.candidates(8)
    assert all(ba == 8 for ba, _, _ in c)
    assert len(c) == len(autotune.DIGITS) * len(autotune.RANKINGS)
