"""Checking level maps against per-level requirements (Sec. 3.2 sync clause,
Sec. 3.3 reserve clause): hand cases, and an exhaustive cross-check against
hp_level_select: over random requirement sets, selection succeeds exactly when
some map meets them, and the map it returns does.  No GPU."""
import itertools

import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb

# every map entry hp_level_select can produce
ENTRIES = [("grid", 0, 0), ("cluster", 0, 0), ("cta", 0, 0), ("warp", 0, 0), ("subwarp", 2, 0), ("subwarp", 4, 0),
           ("subwarp", 8, 0), ("subwarp", 16, 0), ("lane", 0, 0), ("seq", 0, 0)]


def ok(req, m):
    return hb.hp_level_check(req, m)[0]


def test_sync_properties_and_order():
    req = [{}, {"sync": ["barrier"]}]
    assert ok(req, ["grid", "cta"]) and ok(req, ["grid", "cluster"]) and ok(req, ["grid", "warp"])
    good, why = hb.hp_level_check(req, ["grid", "grid"])
    assert not good and "level 1" in why and "sync" in why
    good, why = hb.hp_level_check(req, ["cta", "grid"])
    assert not good and "coarser" in why
    assert not ok([{"sync": ["shuffle"]}], ["cta"]) and ok([{"sync": ["shuffle"]}], [("subwarp", 8, 0)])


def test_reserve():
    req = [{"reserve": ["barrier"]}, {"sync": ["barrier"]}]
    assert ok(req, ["grid", "cluster"]) and ok(req, ["grid", "cta"])
    assert not ok(req, ["grid", "grid"])          # the inner level must be strictly finer
    assert not ok(req, ["cluster", "cta"])        # the reserving level may not have a barrier itself
    assert not ok([{"reserve": ["lockstep"]}], ["lane"])
    assert not ok([{"reserve": ["localmem"]}], ["warp"])   # nothing finer than a warp has local memory


def test_min_num_counts_the_team_the_map_gives():
    req = [{}, {"sync": ["shuffle"], "min_num": 8}]
    assert ok(req, ["grid", ("subwarp", 8, 0)]) and ok(req, ["grid", "warp"])
    assert not ok(req, ["grid", ("subwarp", 4, 0)])
    assert ok([{}, {"min_num": 8}], ["grid", ("cta", 8, 0)]) and not ok([{}, {"min_num": 8}], ["grid", ("cta", 4, 0)])
    assert not ok([{"min_num": 5}], ["lane"])


def test_auto_and_bad_arguments_are_rejected():
    assert not ok([{}], ["auto"])
    good, why = hb.hp_level_check([{}] * 6, ["grid"] * 6)
    assert not good and "depth" in why


def test_selected_maps_pass_the_check():
    # the paper's examples and collapse under a sub-warp partition
    for req in ([{"sync": ["barrier"]}], [{"reserve": ["barrier"]}, {"sync": ["barrier"]}],
                [{"sync": ["shuffle"], "min_num": 4}, {"sync": ["shuffle"]}],
                [{"reserve": ["localmem"]}, {"sync": ["localmem"]}, {"sync": ["shuffle"]}]):
        m = hb.hp_level_select(req)
        assert ok(req, m), (req, m)


def _random_req(g, depth):
    names = list(hb.PROPS)
    req = []
    for _ in range(depth):
        r = {}
        if g.random() < 0.6:
            r["sync"] = [n for n in names if g.random() < 0.12]
        if g.random() < 0.2:
            r["reserve"] = [names[int(g.integers(len(names)))]]
        if g.random() < 0.4:
            r["min_num"] = int(g.choice([1, 2, 4, 5, 8, 16, 32, 64, 5000]))
        req.append(r)
    return req


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_select_succeeds_exactly_when_some_map_meets(depth):
    g = np.random.Generator(np.random.PCG64(100 + depth))
    maps = list(itertools.product(ENTRIES, repeat=depth))
    found = infeasible = 0
    for _ in range(150 if depth < 3 else 60):
        req = _random_req(g, depth)
        exists = any(ok(req, list(m)) for m in maps)
        try:
            m = hb.hp_level_select(req)
        except hb.HPError as e:
            assert e.status == hb.HP_EINVAL
            assert not exists, (req, [m for m in maps if ok(req, list(m))][:3])
            infeasible += 1
            continue
        assert exists and ok(req, m), (req, m, hb.hp_level_check(req, m))
        found += 1
    assert found > 10 and infeasible > 3   # both outcomes are exercised


def test_tuning_under_unsatisfiable_requirements_fails_on_the_host():
    # no map of a rectangular nest gives a reduced level lockstep and a barrier
    n = hb.Nest([1000, 4096], 1, "sum", "f32", "load")
    with pytest.raises(hb.HPError) as e:
        n.tune([0x1000], 0x2000, req=[{}, {"sync": ["lockstep", "barrier"]}])
    assert e.value.status == hb.HP_EINVAL and "level 1" in str(e.value)
    n.close()
    pure = hb.Nest([16, 16], 2, "sum", "f32", "load")   # nothing reduced: only the map is checked
    with pytest.raises(hb.HPError) as e:
        pure.tune([0x1000], 0x2000, req=[{}, {"sync": ["barrier"]}])
    assert e.value.status == hb.HP_EINVAL
    pure.tune([0x1000], 0x2000, req=[{}, {"sync": ["atomic"]}])   # met by the grid: nothing to do
    pure.close()
