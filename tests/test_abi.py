"""The C-ABI library on the CPU: it loads, exports every entry point
include/hp.h declares, validates descriptors and lowers level maps (no GPU)."""
import re
import os

import pytest

from paper_2309_01906_gb300 import binding as hb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hp_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = hb.lib()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), f"libhp.so does not export {n}"
    assert set(names) == set(hb.EXPORTED)
    assert hb.hp_version() == 100


def _err(fn, *a, **k):
    with pytest.raises(hb.HPError) as e:
        fn(*a, **k)
    return e.value


@pytest.mark.parametrize("kwargs,fragment", [
    (dict(extents=[4, 4], red_level=1, level_map=["warp", "warp"]), "below the output levels"),
    (dict(extents=[4, 4], red_level=1, level_map=["warp", "cta"]), "coarser hardware level"),
    (dict(extents=[4, 4], red_level=1, level_map=["grid", ("subwarp", 3, 0)]), "SUBWARP sub_width"),
    (dict(extents=[4, 4], red_level=1, level_map=[("grid", 0, 0), ("cluster", 17, 0)]), "CTAs per cluster"),
    (dict(extents=[4, 4], red_level=1, level_map=[("grid", 0, 0), ("cta", 33, 0)]), "warps per CTA"),
    (dict(extents=[4, 4], red_level=1, level_map=[("grid", 0, 0), ("lane", 2, 0)]), "vector slots"),
    (dict(extents=[4, 4], red_level=1, level_map=["auto", "warp"]), "HP_HW_AUTO"),
    (dict(extents=[4, 4], red_level=3), "red_level"),
    (dict(extents=[4, -1], red_level=1), ">= 0"),
    (dict(extents=[2] * 6, red_level=1), "depth"),
    (dict(extents=[1 << 40, 1 << 40], red_level=1), "2^62"),
    (dict(extents=[4, 4], red_level=1, op="hist"), "CSR"),
    (dict(extents=[4, 4], red_level=1, prec="i32", body="geometric",
          params=hb.hp_geometric_params(0.5, 8)), "FP body"),
    (dict(extents=[4, 4], red_level=1, body="geometric", params=hb.hp_geometric_params(0.5, 2000)), "m must be"),
    (dict(extents=[4, 4], red_level=1, body="affine", params=hb.hp_affine_params(1, 1, 0)), "m must be"),
])
def test_invalid_descriptors(kwargs, fragment):
    kw = dict(op="sum", prec="f32", body="load")
    kw.update(kwargs)
    e = _err(hb.Nest, kw.pop("extents"), **kw)
    assert e.status == hb.HP_EINVAL
    assert fragment in str(e), str(e)


def plan(extents, r, level_map=None, **kw):
    n = hb.Nest(extents, r, kw.get("op", "sum"), kw.get("prec", "f32_comp"), kw.get("body", "dot_bcast"),
                level_map=level_map, params=kw.get("params"))
    d = n.describe()
    n.close()
    return d


def test_plan_four_level_cluster_map():
    d = plan([64, 512, 16, 1024], 2, [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 8, 0)])
    assert d["team"] == "block" and d["cluster"] == 8 and d["warps"] == 8 and d["vec"] == 4
    assert d["outputs"] == 32768 and d["reduced"] == 16384 and d["grid_parts"] == 1
    j, k = d["levels"]
    # j over the 8 CTAs of the cluster (2 steps each); k over warps x lanes x 4 vector slots
    assert (j["n"], j["slots"], j["c_rank"], j["stride"]) == (16, 8, 1, 1024)
    assert (k["n"], k["slots"], k["c_warp"], k["c_lane"]) == (1024, 1024, 128, 4)
    assert d["kernel"] == "rect_block_pipe_cluster" and d["pipe"] == 1 and d["groups"] == 2
    hb.hp_set_option("pipeline", 0)
    try:
        d = plan([64, 512, 16, 1024], 2, [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 8, 0)])
        assert d["kernel"] == "rect_block_cluster" and d["pipe"] == 0
    finally:
        hb.hp_set_option("pipeline", 1)
    assert hb.hp_get_option("pipeline") == 1
    with pytest.raises(hb.HPError):
        hb.hp_set_option("no_such_option", 1)


def test_plan_collapse_and_split():
    d = plan([8, 4, 4, 100], 1, ["grid", "cta", "cta", "cta"])
    assert len(d["levels"]) == 1 and d["levels"][0]["n"] == 1600       # collapsed (Sec. 3.1)
    d = plan([3, 10000], 1, ["grid", ("grid", 0, 1000)])
    assert d["grid_parts"] == 10 and d["tile"] == 1000 and d["team"] == "block"
    d = plan([3, 10001], 1, ["grid", ("grid", 0, 0)])
    assert d["grid_parts"] >= 1 and d["items"] == 3 * d["grid_parts"]


def test_plan_partitioned_warp():
    # Sec. 3.8: warp split into 4 groups of 8 lanes, one output per group
    d = plan([100, 64], 1, ["warp", ("subwarp", 8, 0)])
    assert d["team"] == "lanes" and d["team_lanes"] == 8 and d["levels"][0]["slots"] == 32
    d = plan([10, 4, 64], 1, ["grid", "warp", ("subwarp", 8, 0)])
    j, k = d["levels"]
    assert d["team_lanes"] == 32 and j["slots"] == 4 and j["c_group"] == 1 and k["slots"] == 32


def test_plan_paper_examples():
    # Sec. 3.6: simd(8) over 32 values -> 8 lanes x 4 values, one step per lane
    d = plan([32], 0, [("subwarp", 8, 0)], prec="i64", body="load")
    assert d["team_lanes"] == 8 and d["vec"] == 4 and d["levels"][0]["slots"] == 32
    # Sec. 3.4: 128 x 64, outer loop bound to the outer parallel level, inner to the inner one
    d = plan([128, 64], 1, ["grid", "cta"], prec="i64", body="load")
    assert d["outputs"] == 128 and d["reduced"] == 64 and d["team"] == "block"


def test_auto_plans():
    assert plan([1024, 1024], 1)["team"] == "lanes"
    assert plan([64, 512, 16, 1024], 2)["team"] == "block"
    assert plan([2, 1 << 20], 1)["grid_parts"] > 1
    # teams sized for about 16 iterations per lane of every output
    assert plan([1000, 200], 1)["team_lanes"] == 8
    assert plan([1000, 16], 1)["team_lanes"] == 1 and plan([1000, 16], 1)["vec"] == 4
    assert plan([1000, 3], 1)["team_lanes"] == 1
    assert plan([1000, 512], 1)["team_lanes"] == 32
    assert plan([4, 5], 2)["team"] == "map"


def test_error_bounds():
    n = hb.Nest([100, 1000], 1, "sum", "f32_comp", "dot_bcast")
    b_comp = n.error_bound()
    n.close()
    n = hb.Nest([100, 1000], 1, "sum", "f32", "dot_bcast")
    b_plain = n.error_bound()
    n.close()
    n = hb.Nest([100, 1000], 1, "sum", "i32", "dot_bcast")
    assert n.error_bound() == 0.0
    n.close()
    assert 2.0 ** -24 <= b_comp < 1e-6 and b_comp < b_plain < 1e-4


def test_run_without_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    n = hb.Nest([4, 4], 1, "sum", "f32", "affine", params=hb.hp_affine_params(1, 1, 3))
    e = _err(n.run, [], 0x1000, 0)
    assert e.status == hb.HP_ECUDA
    n.close()


def test_serving_needs_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    e = _err(hb.hp_serve_create, 1 << 30, 8, 2)
    assert e.status == hb.HP_ECUDA
    e = _err(hb.hp_serve_create, 0, 8, 2)
    assert e.status == hb.HP_EINVAL
    hb.hp_set_option("serve_batching", 0)
    assert hb.hp_get_option("serve_batching") == 0
    hb.hp_set_option("serve_batching", 2)
    assert hb.hp_get_option("serve_batching") == 2
    hb.hp_set_option("serve_batching", 1)
    for bad in (-1, 3):
        assert _err(hb.hp_set_option, "serve_batching", bad).status == hb.HP_EINVAL
    assert hb.hp_get_option("serve_batching") == 1


def _header_enums():
    """name -> value of every enumerator in include/hp.h (explicit values and
    implicit successors, including 1u << k)."""
    text = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    vals = {}
    for body in re.findall(r"typedef enum\s*\w*\s*\{(.*?)\}", text, flags=re.S):
        nxt = 0
        for item in [x.strip() for x in body.split(",") if x.strip()]:
            if "=" in item:
                name, expr = [t.strip() for t in item.split("=", 1)]
                m = re.fullmatch(r"(\d+)u?\s*<<\s*(\d+)", expr)   # the header's two forms: N and 1u << k
                v = int(m.group(1)) << int(m.group(2)) if m else int(expr.rstrip("u"))
            else:
                name, v = item, nxt
            vals[name] = v
            nxt = v + 1
    return vals


def test_binding_enums_match_the_header():
    e = _header_enums()
    for name, v in hb.HW.items():
        assert e["HP_HW_" + name.upper()] == v
    ops = {"sum": "HP_RED_SUM", "max": "HP_RED_MAX", "min": "HP_RED_MIN", "hist": "HP_RED_HIST_COUNT",
           "compose": "HP_RED_AFFINE_COMPOSE", "mat2": "HP_RED_MAT2_PRODUCT", "last": "HP_RED_LAST_VALID"}
    assert set(ops) == set(hb.OPS)
    for k, name in ops.items():
        assert e[name] == hb.OPS[k], k
    for k, v in hb.PRECS.items():
        assert e["HP_" + k.upper()] == v, k
    for k, v in hb.BODIES.items():
        assert e["HP_BODY_" + k.upper()] == v, k
    for k, v in hb.PROPS.items():
        assert e["HP_PROP_" + k.upper()] == v, k
    for i, name in enumerate(hb.STATUS_NAMES):
        assert e[name] == i


def test_serve_clock_is_monotonic_and_host_only():
    # the serving clock needs no GPU; latency from scheduled arrival is measured on it
    import time
    a = hb.hp_serve_clock_us()
    time.sleep(0.002)
    b = hb.hp_serve_clock_us()
    assert b - a >= 1500.0
    # steady clock in microseconds: same epoch as the host's monotonic clock
    assert abs(hb.hp_serve_clock_us() - time.monotonic() * 1e6) < 1e6
