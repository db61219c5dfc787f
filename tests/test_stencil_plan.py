"""Stencil nests on the CPU: the planner's map sections (the paper's worked
example, Sec. 4), tiles, ghost widths and rejected descriptors; no GPU."""
import json
import os

import pytest

from oracle import stencil as so
from paper_2309_01906_gb300 import binding as hb

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_examples.json")


def test_paper_sections_from_the_planner():
    # Sec. 4: 1024^2 over 4 units; 'to' sections 513 x 513 at offsets 0 / 511, 'from' 512 x 512
    ex = json.load(open(GOLDEN))["ghost_map"]
    n, f = ex["array"][0], ex["from_size"]
    st = hb.Stencil(n, n, 1, [0.1] * 9, 1, section=(f, f))
    d = st.describe()
    st.close()
    ref = so.sections(n, n, f, f, 1, 1)
    assert len(d["sections"]) == ex["devices"] == len(ref)
    for got, want in zip(d["sections"], ref):
        assert [tuple(b) for b in got["to"]] == list(want["to"])
        assert [tuple(b) for b in got["from"]] == list(want["from"])
        assert got["to"][0][1] - got["to"][0][0] == ex["to_size"]


@pytest.mark.parametrize("r,T", [(0, 1), (1, 1), (1, 4), (2, 3), (4, 8)])
def test_ghost_border_and_box(r, T):
    st = hb.Stencil(3000, 2000, r, [0.0] * (2 * r + 1) ** 2, T)
    d = st.describe()
    st.close()
    h, hx = d["ghost"]
    assert h == r * T and hx % 4 == 0 and h <= hx < h + 4
    ty, tx = d["tile"]
    assert d["box"] == [ty + 2 * h, tx + 2 * hx] and max(d["box"]) <= 256
    assert d["smem"] <= 226 * 1024 and d["buffers"] == (2 if T > 1 else 1)
    assert d["tiles"] == -(-3000 // ty) * -(-2000 // tx)
    assert ty >= min(64, 2 * h)        # no tile much shorter than its ghost border


def test_sections_group_whole_tiles():
    st = hb.Stencil(1000, 1000, 1, [0.0] * 9, 2, section=(256, 512), tile=(64, 128))
    d = st.describe()
    st.close()
    assert d["section"] == [256, 512] and len(d["sections"]) == 4 * 2
    assert d["sections"][0] == {"to": [[0, 258], [0, 514]], "from": [[0, 256], [0, 512]]}


@pytest.mark.parametrize("kw,frag", [
    (dict(radius=5), "radius"),
    (dict(steps=0), "steps"),
    (dict(steps=9), "steps"),
    (dict(tile=(64, 130)), "multiple of 4"),
    (dict(tile=(250, 128), steps=4), "256 x 256"),
    (dict(section=(100, 128), tile=(64, 128)), "multiples of the tile"),
    (dict(ny=-1), ">= 0"),
])
def test_rejected_descriptors(kw, frag):
    args = dict(ny=100, nx=100, radius=1, steps=1, section=(0, 0), tile=(0, 0))
    args.update(kw)
    r = args["radius"]
    K = (2 * r + 1) ** 2 if 0 <= r <= 4 else 9
    with pytest.raises(hb.HPError) as e:
        hb.hp_stencil_create(args["ny"], args["nx"], r, [0.0] * K, args["steps"], args["section"], args["tile"])
    assert e.value.status == hb.HP_EINVAL
    assert frag in str(e.value)


def test_empty_array_plans_and_runs_nothing():
    st = hb.Stencil(0, 50, 1, [0.0] * 9, 1)
    assert st.describe()["tiles"] == 0
    st.run(0x1000, 0x2000)      # nothing to do: no device call
    st.close()
