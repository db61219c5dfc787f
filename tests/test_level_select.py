"""Selecting levels by property (Sec. 3.2 sync clause, Sec. 3.3 reserve
clause): the capability table of GB300's levels, the paper's examples, maps
that the planner accepts, and requirements no level meets.  No GPU except the
last test."""
import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb


def test_capability_table():
    grid, n_grid = hb.hp_level_properties("grid")
    assert "barrier" not in grid and {"dynamic", "oversub", "atomic", "globalmem"} <= grid and n_grid >= 152
    cl, n_cl = hb.hp_level_properties("cluster")
    assert {"barrier", "localmem", "progress"} <= cl and "shuffle" not in cl and n_cl == 8
    cta, _ = hb.hp_level_properties("cta")
    assert {"barrier", "localmem", "cache"} <= cta
    warp, n_warp = hb.hp_level_properties("warp")
    assert {"shuffle", "barrier", "groupmem"} <= warp and "localmem" not in warp and n_warp == 32
    lane, n_lane = hb.hp_level_properties("lane")
    assert "lockstep" in lane and "shuffle" not in lane and n_lane == 4


def test_paper_sync_barrier():
    # Sec. 3.2: `parallel sync(barrier)` runs on the coarsest level with a working barrier
    assert hb.hp_level_select([{"sync": ["barrier"]}]) == [("cluster", 0, 0)]


def test_paper_reserve():
    # Sec. 3.3: `parallel sync() reserve(sync(barrier))` over `parallel sync(barrier)`:
    # the outer level takes everything but a barrier level, the inner one gets it
    assert hb.hp_level_select([{"reserve": ["barrier"]}, {"sync": ["barrier"]}]) == [("grid", 0, 0), ("cluster", 0, 0)]
    # the reserved kind is left to the inner level: even with a barrier itself,
    # the outer level may not sit on a barrier level, nor the inner one on the outer's
    assert hb.hp_level_select([{"reserve": ["localmem"]}, {"sync": ["localmem"]}, {"sync": ["shuffle"]}]) == \
        [("grid", 0, 0), ("cluster", 0, 0), ("warp", 0, 0)]
    with pytest.raises(hb.HPError):   # progress without local memory is a warp: nothing finer has local memory
        hb.hp_level_select([{"sync": ["progress"], "reserve": ["localmem"]}, {"sync": ["localmem"]}])


@pytest.mark.parametrize("inner,want", [
    ({"sync": ["shuffle"]}, ("warp", 0, 0)),
    ({"sync": ["shuffle"], "min_num": 8}, ("subwarp", 8, 0)),      # Sec. 3.8: a partition of the warp
    ({"sync": ["shuffle"], "min_num": 5}, ("subwarp", 8, 0)),
    ({"sync": ["lockstep"]}, ("lane", 0, 0)),
    ({"sync": ["localmem", "cache"]}, ("cta", 0, 0)),
    ({}, ("grid", 0, 0)),                                          # no requirement: split over the grid
])
def test_reduction_nests_from_properties(inner, want):
    sel = hb.hp_level_select([{}, inner])
    assert sel[0] == ("grid", 0, 0) and sel[1] == want
    n = hb.Nest([64, 4096], 1, "sum", "f32_comp", "load", level_map=sel)   # the planner accepts the map
    d = n.describe()
    n.close()
    assert d["map"][1]["hw"] == want[0]


@pytest.mark.parametrize("reqs", [
    [{"sync": ["shuffle"]}, {"sync": ["localmem"]}],     # nothing below a warp has local memory
    [{"sync": ["barrier", "lockstep"]}],                 # no level has both
    [{"reserve": ["dynamic"]}, {}],                      # only the grid is dynamic: nothing finer keeps it
    [{"sync": ["shuffle"], "min_num": 64}],              # no level with shuffles runs 64 tasks
])
def test_unsatisfiable_requirements(reqs):
    with pytest.raises(hb.HPError) as e:
        hb.hp_level_select(reqs)
    assert e.value.status == hb.HP_EINVAL


@pytest.mark.gpu
def test_a_selected_map_runs():
    import torch

    from tests.hp_testutil import assert_close, oracle_rect
    sel = hb.hp_level_select([{}, {"sync": ["shuffle"], "min_num": 8}])
    A = np.random.Generator(np.random.PCG64(4)).standard_normal(300 * 200).astype(np.float32)
    n = hb.Nest([300, 200], 1, "sum", "f32_comp", "load", level_map=sel)
    dA = torch.from_numpy(A).cuda()
    out = torch.empty(300, dtype=torch.float32, device="cuda")
    n.run([dA.data_ptr()], out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref = oracle_rect([300, 200], 1, "sum", "f32_comp", "load", A=A)
    assert_close(out.cpu().numpy(), ref, "f32_comp", "sum", n.error_bound(), what="selected map")
    n.close()
