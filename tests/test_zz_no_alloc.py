"""The entry point that allocates nothing (hp_nest_run_static), on the GPU.

It serves callers that cannot allocate device memory at run time (serving
loops where cudaMalloc / cudaFree would synchronise the device, services whose
memory budget was handed out at start-up).  Its reductions split over grid
parts keep their partials in the library's fixed static array, so two calls
in a row reuse the array with whatever the previous call left in it; both must
give the outputs of the allocating entry point hp_nest_run.  This file is
collected last so that a failure here stops a -x run only after every other
test has run.
"""
import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb

pytestmark = pytest.mark.gpu

CASES = [
    # (extents, red_level, op, prec, body, level map): all split over grid parts
    ([7, 1 << 16], 1, "sum", "f32_comp", "dot_bcast", ["grid", ("grid", 0, 4096)]),
    ([7, 1 << 16], 1, "sum", "f32", "load", ["grid", ("grid", 0, 3000)]),
    ([5, 3, 10000], 1, "sum", "i64", "dot_bcast", ["grid", ("grid", 0, 1), "warp"]),
    ([4, 9, 700], 1, "max", "i32", "load", ["grid", ("grid", 0, 2), "cta"]),
    ([3, 200000], 1, "sum", "f32_comp", "load", None),
    # cluster teams (DSMEM) over grid parts: the launch sets the cluster
    # attributes on first use, here first through the static entry point
    ([3, 8, 16, 1024], 1, "sum", "f32_comp", "dot_bcast", ["grid", ("grid", 0, 4), ("cluster", 4, 0), ("cta", 4, 0)]),
    ([3, 4, 16, 512], 1, "sum", "f32", "dot_bcast", ["grid", ("grid", 0, 2), ("cluster", 16, 0), ("cta", 2, 0)]),
]

# expected plan fields per case (None = any): cluster size and grid parts
PLAN_FIELDS = {5: {"cluster": 4, "grid_parts": 2}, 6: {"cluster": 16, "grid_parts": 2}}


def _inputs(case, seed):
    import torch
    ext, r, op, prec, body, lm = case
    g = np.random.Generator(np.random.PCG64(seed))
    total = int(np.prod(ext))
    R = int(np.prod(ext[r:]))
    if prec in ("i32", "i64"):
        A = torch.from_numpy(g.integers(-1000, 1001, total).astype(np.int32)).cuda()
        w = torch.from_numpy(g.integers(-1000, 1001, R).astype(np.int32)).cuda()
        dt = torch.int32 if prec == "i32" else torch.int64
    else:
        A = torch.from_numpy(g.standard_normal(total).astype(np.float32)).cuda()
        w = torch.from_numpy(g.uniform(-1, 1, R).astype(np.float32)).cuda()
        dt = torch.float32
    return (A, w), dt


def _run(case, seed):
    import torch
    ext, r, op, prec, body, lm = case
    (A, w), dt = _inputs(case, seed)
    ins = [A.data_ptr()] + ([w.data_ptr()] if body == "dot_bcast" else [])
    O = int(np.prod(ext[:r]))
    stream = torch.cuda.current_stream().cuda_stream
    n_alloc = hb.Nest(ext, r, op, prec, body, level_map=lm)
    n_static = hb.Nest(ext, r, op, prec, body, level_map=lm)
    assert n_static.describe()["grid_parts"] > 1
    want = torch.empty(O, dtype=dt, device="cuda")
    n_alloc.run(ins, want.data_ptr(), stream)
    got = []
    for _ in range(2):   # two calls in a row share the static array
        out = torch.full((O,), 7, dtype=dt, device="cuda")
        n_static.run_static(ins, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got.append(out.cpu().numpy())
    torch.cuda.synchronize()
    ref = want.cpu().numpy()
    n_alloc.close()
    n_static.close()
    return ref, got


@pytest.mark.parametrize("idx", range(len(CASES)), ids=lambda i: f"{CASES[i][0]}-{CASES[i][2]}-{CASES[i][3]}")
def test_static_scratch_matches_allocating_entry_point(idx):
    case = CASES[idx]
    want = PLAN_FIELDS.get(idx, {})
    if want:
        ext, r, op, prec, body, lm = case
        n = hb.Nest(ext, r, op, prec, body, level_map=lm)
        d = n.describe()
        n.close()
        assert {k: d[k] for k in want} == want, d
    ref, got = _run(case, seed=11)
    for g in got:
        # same kernels and reduction tree: identical bits (the tolerance the
        # other parity tests use is looser than this)
        assert np.array_equal(g, ref), f"static-scratch run differs from hp_nest_run for {case}"


def test_static_scratch_rejects_plans_beyond_its_size():
    n = hb.Nest([1 << 16, 1 << 14], 1, "sum", "f32_comp", "load", level_map=["grid", ("grid", 0, 4)])
    need = n.describe()["items"] * 8
    assert need > (8 << 20)
    with pytest.raises(hb.HPError) as e:
        n.run_static([0x1000], 0x1000, 0)
    assert e.value.status == hb.HP_EINVAL and "static maximum" in str(e.value)
    n.close()


def test_static_then_allocating_run_on_one_nest():
    """One nest run first without allocating, then through hp_nest_run: the
    launch configuration the static call sized is reused and the bits agree."""
    import torch
    case = CASES[5]
    ext, r, op, prec, body, lm = case
    (A, w), dt = _inputs(case, seed=12)
    ins = [A.data_ptr(), w.data_ptr()]
    O = int(np.prod(ext[:r]))
    stream = torch.cuda.current_stream().cuda_stream
    n = hb.Nest(ext, r, op, prec, body, level_map=lm)
    outs = []
    for runner in (n.run_static, n.run, n.run_static):
        out = torch.full((O,), 7, dtype=dt, device="cuda")
        runner(ins, out.data_ptr(), stream)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    n.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
