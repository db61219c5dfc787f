"""Ordered (non-commutative) reductions on the CPU: the lowering's teams,
blocks and grid parts, and rejected descriptors (no GPU)."""
import pytest

from paper_2309_01906_gb300 import binding as hb


def plan(ext, r, lm=None):
    n = hb.Nest(ext, r, "compose", "f32", "load", level_map=lm)
    d = n.describe()
    n.close()
    return d


def test_auto_teams():
    # chunk: iterations per warp (whole pieces); a warp folds its range in rounds of
    # 32 pieces, one per lane
    d = plan([1000, 300], 1)
    assert d["kind"] == "ordered" and d["team"] == "warp" and d["grid_parts"] == 1
    assert d["piece"] == 8 and d["chunk"] == 304 and d["vec"] == 4   # 300 is a multiple of 4, not of 8
    d = plan([1000, 5000], 1)
    assert d["team"] == "block" and d["warps"] == 8 and d["grid_parts"] == 1 and d["chunk"] == 632   # 5000/8 -> 8s
    assert d["vec"] == 8
    d = plan([4, 1 << 22], 1)
    assert d["team"] == "block" and d["grid_parts"] > 1 and d["part"] * (d["grid_parts"] - 1) < (1 << 22)
    assert d["vec"] == 8 and d["chunk"] % d["piece"] == 0 and d["part"] % 8 == 0
    rounds = -(-d["chunk"] // (32 * d["piece"]))
    assert d["chain"] == d["piece"] + 5 + rounds + 5 + d["grid_parts"] - 1
    assert plan([64, 4096], 1, ["grid", ("cta", 8, 0)])["piece"] == 8


def test_pieces_per_operator():
    def p(op, R):
        n = hb.Nest([16, R], 1, op, "f32", "load")
        d = n.describe()
        n.close()
        return d
    assert p("mat2", 4096)["piece"] == 4 and p("mat2", 4096)["vec"] == 8 and p("mat2", 4095)["vec"] == 4
    assert p("last", 4096)["piece"] == 32 and p("last", 4096)["chunk"] % 32 == 0


def test_explicit_maps():
    d = plan([64, 3, 1000], 1, ["grid", ("cta", 4, 0), ("cta", 4, 0)])
    assert d["team"] == "block" and d["warps"] == 4 and d["chunk"] == 752   # 3000 / 4 warps -> 8s
    d = plan([64, 3, 1000], 1, ["grid", ("grid", 0, 1), "grid"])
    assert d["grid_parts"] == 3 and d["part"] == 1000
    d = plan([8, 100], 1, ["grid", "warp"])
    assert d["team"] == "warp" and d["chunk"] == 104
    d = plan([8, 102], 1, ["grid", "warp"])
    assert d["vec"] == 1 and d["chunk"] == 104


@pytest.mark.parametrize("kw,frag", [
    (dict(prec="f32_comp"), "HP_F32"),
    (dict(body="dot_bcast"), "HP_BODY_LOAD"),
    (dict(r=2), "red_level"),
    (dict(lm=["cta", "warp"]), "output levels on GRID"),
    (dict(lm=["grid", "subwarp"]), "WARP, CTA or GRID"),
])
def test_rejected(kw, frag):
    r = kw.get("r", 1)
    with pytest.raises(hb.HPError) as e:
        hb.Nest([8, 100], r, "compose", kw.get("prec", "f32"), kw.get("body", "load"), level_map=kw.get("lm"))
    assert e.value.status == hb.HP_EINVAL and frag in str(e.value)


def test_ordered_nests_are_not_batched_or_tuned():
    n = hb.Nest([8, 100], 1, "compose", "f32", "load")
    with pytest.raises(hb.HPError) as e:
        hb.hp_nest_run_batch([n.handle], [[0x1000, 0x2000]], [0x3000], 0)
    assert e.value.status == hb.HP_EUNSUPPORTED
    with pytest.raises(hb.HPError) as e:
        n.tune([0x1000, 0x2000], 0x3000)
    assert e.value.status == hb.HP_EUNSUPPORTED
    assert n.error_bound() == pytest.approx(2 * 99 * 2.0 ** -24, rel=1e-4)   # gamma_{2(R-1)}, R = 100
    n.close()


def test_error_bound_of_products_counts_every_combine():
    # gamma_{2(R-1)}: the relative errors of all R - 1 combines add, whatever the tree
    u = 2.0 ** -24
    for R in (1, 2, 1000, 1 << 20):
        n = hb.Nest([3, R], 1, "compose", "f32", "load")
        k2 = 2 * (R - 1)
        assert n.error_bound() == pytest.approx(k2 * u / (1 - k2 * u), rel=1e-12, abs=0.0)
        n.close()
        m = hb.Nest([3, R], 1, "mat2", "f32", "load")
        assert m.error_bound() == pytest.approx(k2 * u / (1 - k2 * u), rel=1e-12, abs=0.0)
        m.close()
    big = hb.Nest([1, (1 << 23) + 2], 1, "compose", "f32", "load")   # 2 (R - 1) u >= 1: no finite bound
    assert big.error_bound() == float("inf")
    big.close()
    last = hb.Nest([3, 1000], 1, "last", "f32", "load")
    assert last.error_bound() == 0.0
    last.close()
