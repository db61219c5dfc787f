"""Nests on 8- / 16-bit integers (SIMD-in-register sub-lanes) on the CPU: the
plan and rejected descriptors (no GPU)."""
import pytest

from paper_2309_01906_gb300 import binding as hb


def plan(ext, r, op="sum", prec="i8", body="load", lm=None):
    n = hb.Nest(ext, r, op, prec, body, level_map=lm)
    d = n.describe()
    n.close()
    return d


def test_plans():
    d = plan([1000, 4096], 1)
    assert d["kind"] == "narrow" and d["team"] == "warp" and d["vec"] == 16 and d["simd"] == 4
    d = plan([64, 1 << 16], 1, prec="i16", op="max")
    assert d["team"] == "block" and d["vec"] == 8 and d["simd"] == 2
    d = plan([4, 1 << 24], 1, body="dot_bcast")
    assert d["grid_parts"] > 1 and d["part"] % 16 == 0
    d = plan([64, 3, 1000], 1, lm=["grid", ("grid", 0, 1), "grid"])
    assert d["grid_parts"] == 3 and d["part"] == 1000


@pytest.mark.parametrize("kw,frag", [
    (dict(op="compose"), "SUM, MAX or MIN"),
    (dict(body="affine"), "LOAD or DOT_BCAST"),
    (dict(prec="i16", body="dot_bcast"), "HP_I8 with SUM"),
    (dict(op="max", body="dot_bcast"), "HP_I8 with SUM"),
    (dict(lm=["cta", "cta"]), "output levels on GRID"),
])
def test_rejected(kw, frag):
    with pytest.raises(hb.HPError) as e:
        plan([8, 100], 1, **kw)
    assert e.value.status == hb.HP_EINVAL and frag in str(e.value)
