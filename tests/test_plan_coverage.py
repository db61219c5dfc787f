"""Host-side check of the level -> hardware lowering (no GPU).

For each plan the library describes, a model of the executor's index
arithmetic (per-thread slots from the cluster rank, warp, group and lane
coefficients; cyclic steps; vector slots; grid parts) enumerates which reduced
elements every thread of a team folds.  Every (output, element) pair must be
folded exactly once, and every address must stay inside A and w.
"""
import itertools

import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb


def team_coords(d):
    if d["team"] == "block":
        for rank in range(d["cluster"]):
            for warp in range(d["warps"]):
                for lane in range(32):
                    yield rank, warp, lane // d["group_lanes"], lane % d["group_lanes"]
    else:
        for lt in range(d["team_lanes"]):
            yield 0, 0, lt // d["group_lanes"], lt % d["group_lanes"]


def fold_item_model(d, o, g, coords):
    """Element offsets (within A) folded by one thread for item (o, g)."""
    lv = d["levels"]
    nv = len(lv)
    rank, warp, grp, lig = coords
    slot = [rank * L["c_rank"] + warp * L["c_warp"] + grp * L["c_group"] + lig * L["c_lane"] for L in lv]
    lo = [0] * nv
    hi = [L["n"] for L in lv]
    if d["grid_parts"] > 1 or (nv and d["tile"]):
        if d["tile"]:
            lo[0] = g * d["tile"]
            hi[0] = min(lv[0]["n"], lo[0] + d["tile"])
    ranges = []
    for v in range(nv):
        ranges.append(list(range(lo[v] + slot[v], hi[v], lv[v]["slots"])))
    out = []
    V = d["vec"]
    for xs in itertools.product(*ranges[:-1]):
        roff = sum(x * lv[v]["stride"] for v, x in enumerate(xs))
        for xi in ranges[-1]:
            for k in range(V):
                out.append((o * d["reduced"] + roff + xi + k, roff + xi + k))
    return out


MAPS = [
    ([37, 1029], 1, ["grid", "warp"]),
    ([37, 1028], 1, ["grid", "warp"]),
    ([37, 1029], 1, ["grid", "cta"]),
    ([9, 1028], 1, [("grid", 0, 0), ("cta", 4, 0)]),
    ([9, 70], 1, ["grid", "seq"]),
    ([9, 1028], 1, ["grid", ("subwarp", 8, 0)]),
    ([9, 1029], 1, ["grid", ("subwarp", 2, 0)]),
    ([9, 1028], 1, ["grid", ("lane", 4, 0)]),
    ([5, 1029], 1, ["grid", ("grid", 0, 300)]),
    ([5, 1028], 1, ["grid", ("grid", 0, 300)]),
    ([5, 1029], 1, [("grid", 0, 0), ("cluster", 4, 0)]),
    ([9, 100], 1, ["cta", "warp"]),
    ([9, 100], 1, [("cta", 4, 0), ("subwarp", 16, 0)]),
    ([9, 64], 1, ["warp", ("subwarp", 4, 0)]),
    ([3, 7, 16, 132], 2, [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 8, 0)]),
    ([2, 5, 11, 96], 2, [("grid", 0, 0), ("grid", 0, 0), ("cluster", 16, 0), ("cta", 4, 0)]),
    ([2, 5, 11, 96], 2, [("grid", 0, 0), ("grid", 0, 0), ("cluster", 2, 0), ("cta", 2, 0)]),
    ([2, 5, 11, 96], 2, ["grid", "grid", "cta", "warp"]),
    ([2, 5, 11, 96], 2, ["grid", "grid", ("grid", 0, 5), "cta"]),
    ([2, 5, 11, 96], 2, ["grid", "cta", "warp", "seq"]),
    ([2, 5, 11, 96], 2, ["grid", "grid", "warp", ("subwarp", 8, 0)]),
    ([2, 5, 11, 96], 2, ["grid", "grid", "seq", "seq"]),
    ([6, 16, 700], 1, ["grid", ("cluster", 4, 0), "cta"]),
    ([6, 16, 700], 1, ["grid", ("grid", 0, 3), "warp"]),
    ([32], 0, [("subwarp", 8, 0)]),
    ([7, 1 << 12], 1, [("grid", 0, 0), ("grid", 0, 1024)]),
    ([2, 3, 4, 5, 6], 0, None),
    ([9, 515], 1, None),
    ([4, 3, 2, 70], 1, None),
    ([300], 0, None),
    ([5, 0], 1, None),
    ([5, 0, 3], 1, ["grid", "cta", "cta"]),
]


@pytest.mark.parametrize("extents,r,level_map", MAPS, ids=lambda x: str(x))
def test_every_element_folded_once_in_bounds(extents, r, level_map):
    n = hb.Nest(extents, r, "sum", "f32", "dot_bcast", level_map=level_map)
    d = n.describe()
    n.close()
    total = int(np.prod(extents))
    R = d["reduced"]
    O = d["outputs"]
    G = d["grid_parts"]
    assert d["items"] == O * G
    coords = list(team_coords(d))
    for o in range(O):
        seen = np.zeros(R, dtype=np.int64)
        for g in range(G):
            for c in coords:
                for a_off, w_off in fold_item_model(d, o, g, c):
                    assert 0 <= a_off < total, (o, g, c, a_off)
                    assert 0 <= w_off < R, (o, g, c, w_off)
                    assert a_off - o * R == w_off
                    seen[w_off] += 1
        assert np.all(seen == 1), f"output {o}: elements folded {seen.min()}..{seen.max()} times"
