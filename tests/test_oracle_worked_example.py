"""Oracle pins: the worked example of Figs. 1-3 (Sec. 4.3), exact values."""
import numpy as np

from golden_io import worked_example
from oracle import nbsi, nbsi_bulk

EX = worked_example()


def _batch():
    rows = sorted(EX["batch"], key=lambda r: r[2])
    assert [r[2] for r in rows] == [1, 2, 3, 4, 5]
    return [(min(a, b), max(a, b)) for a, b, _ in rows]


def test_rank_all_matches_fig2_scalar():
    F = nbsi.rank_all(_batch())
    got = [(a["src"], a["dst"], a["pos"] + 1, a["rank"]) for a in F]
    assert got == EX["rankall"]


def test_rank_all_matches_fig2_bulk():
    W = np.array([(a << 32) | b for a, b in _batch()], dtype=np.uint64)
    src, dst, pos, rank = nbsi_bulk.rank_all(W)
    got = list(zip(src.tolist(), dst.tolist(), (pos + 1).tolist(), rank.tolist()))
    assert got == EX["rankall"]


def test_rank_definition_matches_fig1():
    t = nbsi.RankTable(_batch())
    for x, y, rk in EX["rank"]:
        assert t.rank(x, y) == rk, (x, y)


def test_naming_system_matches_fig3():
    W = _batch()
    t = nbsi.RankTable(W)
    for u, v, phi, a, b in EX["name"]:
        arc = t.name(u, v, phi)
        assert W[arc["pos"]] == (min(a, b), max(a, b)), (u, v, phi)
        assert arc["src"] in (u, v)


def test_chi_plus_matches_fig3_caption():
    t = nbsi.RankTable(_batch())
    for u, v, chi in EX["chiplus"]:
        assert t.rank(u, v) + t.rank(v, u) == chi
