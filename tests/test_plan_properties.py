"""Properties of the ordered and narrow-integer planners over seeded random
shapes (no GPU): grid parts cover the reduced range exactly, warp ranges are
whole pieces and cover a part, load widths follow divisibility, and plans are
deterministic."""
import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb


def _describe(ext, r, op, prec, body="load", lm=None):
    n = hb.Nest(list(ext), r, op, prec, body, level_map=lm)
    try:
        return n.describe()
    finally:
        n.close()


def _shapes(seed, count):
    g = np.random.Generator(np.random.PCG64(seed))
    for _ in range(count):
        d = int(g.integers(2, 5))
        r = int(g.integers(1, d))
        ext = [int(g.integers(1, 40)) for _ in range(r)]
        # reduced levels: sizes from a few to millions
        ext += [int(2 ** g.uniform(0, 22 / (d - r))) for _ in range(d - r)]
        yield ext, r


@pytest.mark.parametrize("op", ["compose", "mat2", "last"])
def test_ordered_plans_cover_and_align(op):
    ib = 16 if op == "mat2" else 4
    seen = set()
    for ext, r in _shapes(41 + len(op), 60):
        d = _describe(ext, r, op, "f32")
        seen.add("parts" if d["grid_parts"] > 1 else d["team"])
        R = int(np.prod(ext[r:]))
        G, part, chunk, piece, V = d["grid_parts"], d["part"], d["chunk"], d["piece"], d["vec"]
        assert d["outputs"] == int(np.prod(ext[:r])) and d["reduced"] == R
        assert chunk % piece == 0 and chunk >= piece
        if R > 0:
            assert G * part >= R and (G - 1) * part < R, (ext, d)
        threads = 1 if d["team"] == "warp" else d["warps"]
        assert threads * chunk >= min(part, R) or R == 0, (ext, d)   # the warps cover a part
        per_load = max(1, 4 * V // ib)
        assert V in (1, 4, 8) and R % per_load == 0 and part % per_load == 0, (ext, d)
        if op != "mat2" and R % 8 == 0 and part % 8 == 0:
            assert V == 8
        assert d == _describe(ext, r, op, "f32")   # deterministic
    assert seen == {"warp", "block", "parts"}     # every team shape was exercised


@pytest.mark.parametrize("prec,op", [("i8", "sum"), ("i8", "max"), ("i16", "min")])
def test_narrow_plans_cover_and_align(prec, op):
    esize = 1 if prec == "i8" else 2
    seen = set()
    for ext, r in _shapes(77 + esize, 60):
        d = _describe(ext, r, op, prec)
        seen.add("parts" if d["grid_parts"] > 1 else d["team"])
        R = int(np.prod(ext[r:]))
        G, part = d["grid_parts"], d["part"]
        assert d["vec"] == 16 // esize and d["simd"] == 4 // esize
        if R > 0:
            assert G * part >= R and (G - 1) * part < R, (ext, d)
        if G > 1 and R % (16 // esize) == 0 and d["auto_map"]:
            assert part % (16 // esize) == 0   # parts of whole 16-byte pieces
        assert d == _describe(ext, r, op, prec)
    assert seen == {"warp", "block", "parts"}
