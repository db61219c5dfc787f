"""GPU parity of the rectangular executor against the oracle, through the C ABI.

Sizes span several tiles and ragged tails; every hardware binding the planner
supports is exercised (grid / cluster / CTA / warp / sub-warp / lane / seq, grid
split with the second pass, collapse), for every precision and operator.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2309_01906_gb300 import synth
from tests.hp_testutil import assert_close, gpu_rect, oracle_rect, out_dtype

pytestmark = pytest.mark.gpu

RNG = np.random.Generator(np.random.PCG64(2024))


def _inputs(extents, red_level, prec, body):
    total = int(np.prod(extents))
    R = int(np.prod(extents[red_level:])) if red_level < len(extents) else 1
    if body not in ("load", "dot_bcast"):
        return None, None
    if prec in ("i32", "i64"):
        A = RNG.integers(-1000, 1001, max(total, 1)).astype(np.int32)
        w = RNG.integers(-1000, 1001, max(R, 1)).astype(np.int32)
    else:
        A = RNG.standard_normal(max(total, 1)).astype(np.float32)
        w = RNG.uniform(-1, 1, max(R, 1)).astype(np.float32)
    return A, (w if body == "dot_bcast" else None)


def check(extents, red_level, op, prec, body, level_map, params=None, A=None, w=None):
    if A is None and body in ("load", "dot_bcast"):
        A, w = _inputs(extents, red_level, prec, body)
    got, plan, bound = gpu_rect(extents, red_level, op, prec, body, level_map, A=A, w=w, params=params)
    ref = oracle_rect(extents, red_level, op, prec, body, A=A, w=w, params=params)
    assert_close(got, ref, prec, op, bound, what=f"{extents} r={red_level} {op} {prec} {body} {level_map}")
    return plan


MAPS_2L = [
    None,                                   # planner's choice
    ["grid", "warp"],                       # warp per output, lanes + vector over j
    ["grid", "cta"],                        # CTA per output
    [("grid", 0, 0), ("cta", 4, 0)],        # CTA of 4 warps
    ["grid", "seq"],                        # thread per output
    ["grid", ("subwarp", 8, 0)],            # 8-lane groups (Sec. 3.8 partition)
    ["grid", ("subwarp", 2, 0)],
    ["grid", ("lane", 4, 0)],               # one thread, 4 vector slots
    ["grid", ("lane", 1, 0)],
    ["grid", ("grid", 0, 300)],             # split over the grid + second pass
    [("grid", 0, 0), ("cluster", 4, 0)],    # cluster of 4 CTAs per output (DSMEM)
    ["cta", "warp"],                        # outputs over the warps of CTAs
    [("cta", 4, 0), ("subwarp", 16, 0)],
    ["warp", ("subwarp", 4, 0)],            # outputs over sub-warp groups
]


@pytest.mark.parametrize("level_map", MAPS_2L, ids=lambda m: str(m))
@pytest.mark.parametrize("prec,op", [("f32", "sum"), ("f32_comp", "sum"), ("i32", "sum"), ("f32", "max")])
def test_two_level_maps(level_map, prec, op):
    # 37 outputs x 1029 reduced: several warps/CTAs and a ragged tail
    check([37, 1029], 1, op, prec, "dot_bcast", level_map)
    check([37, 1028], 1, op, prec, "dot_bcast", level_map)   # vectorizable


MAPS_4L = [
    [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 8, 0)],   # the 4-level workload's map
    [("grid", 0, 0), ("grid", 0, 0), ("cluster", 16, 0), ("cta", 4, 0)],  # non-portable cluster of 16
    [("grid", 0, 0), ("grid", 0, 0), ("cluster", 2, 0), ("cta", 2, 0)],
    ["grid", "grid", "cta", "warp"],
    ["grid", "grid", ("grid", 0, 5), "cta"],                              # j split over grid parts
    ["grid", "cta", "warp", "seq"],
    ["grid", "grid", "warp", ("subwarp", 8, 0)],
    ["grid", "grid", "seq", "seq"],
    None,
]


@pytest.mark.parametrize("level_map", MAPS_4L, ids=lambda m: str(m))
@pytest.mark.parametrize("prec", ["f32", "f32_comp", "i64"])
def test_four_level_maps(level_map, prec):
    check([3, 7, 16, 132], 2, "sum", prec, "dot_bcast", level_map)
    check([2, 5, 11, 96], 2, "sum", prec, "dot_bcast", level_map)


@pytest.mark.parametrize("prec,op", list(itertools.product(["f32", "f32_comp", "i32", "i64"], ["sum", "max", "min"])))
@pytest.mark.parametrize("body", ["load", "dot_bcast", "affine"])
def test_precisions_ops_bodies(prec, op, body):
    params = (-3, 5, 7) if body == "affine" else None
    for ext, r in (([9, 515], 1), ([4, 3, 2, 70], 1), ([300], 0), ([6, 5], 2)):
        check(ext, r, op, prec, body, None, params=params)


@pytest.mark.parametrize("prec", ["f32", "f32_comp"])
def test_geometric_body(prec):
    for ext, r in (([5, 1000], 1), ([3, 4, 5, 6, 7], 2), ([100000], 0)):
        check(ext, r, "sum", prec, "geometric", None, params=(0.5, 24))
        check(ext, r, "sum", prec, "geometric", ["grid"] * r + ["warp"] * (len(ext) - r), params=(0.75, 13))


def test_affine_closed_form_large():
    # 2^26 iterations with no memory: int64 sums of an arithmetic sequence per output
    a, b, m = 11, -3, 1000003
    ext = [64, 1 << 20]
    got, _, _ = gpu_rect(ext, 1, "sum", "i64", "affine", None, params=(a, b, m))

    def F(N):
        q, s = divmod(N, m)
        return N * a + b * (q * m * (m - 1) // 2 + s * (s - 1) // 2)
    R = ext[1]
    want = np.array([F((o + 1) * R) - F(o * R) for o in range(ext[0])], dtype=np.int64)
    assert np.array_equal(got.astype(np.int64), want)


def test_edge_cases():
    # empty reduction -> identity; empty outputs -> nothing; r == 0; r == d; depth 5
    check([5, 0], 1, "sum", "f32_comp", "load", None, A=np.zeros(1, np.float32))
    check([5, 0], 1, "max", "i32", "load", None, A=np.zeros(1, np.int32))
    check([5, 0, 3], 1, "min", "f32", "load", ["grid", "cta", "cta"], A=np.zeros(1, np.float32))
    check([0, 7], 1, "sum", "f32", "load", None, A=np.zeros(1, np.float32))
    check([1], 0, "sum", "f32_comp", "load", None)
    check([1, 1, 1, 1, 1], 2, "sum", "i64", "dot_bcast", None)
    check([2, 3, 4, 5, 6], 0, "sum", "f32_comp", "dot_bcast", None)
    check([2, 3, 4, 5, 6], 5, "sum", "f32", "load", None)
    check([2, 3, 4, 5, 6], 5, "sum", "i64", "dot_bcast", None)
    check([7, 1 << 16], 1, "sum", "f32_comp", "load", [("grid", 0, 0), ("grid", 0, 4096)])


def test_deterministic_and_map_invariant():
    A, w = _inputs([6, 16, 700], 1, "i32", "dot_bcast")
    maps = [None, ["grid", "cta", "cta"], ["grid", "warp", ("subwarp", 8, 0)], ["grid", ("cluster", 4, 0), "cta"],
            ["grid", ("grid", 0, 3), "warp"], ["grid", "seq", "seq"]]
    outs = [gpu_rect([6, 16, 700], 1, "sum", "i32", "dot_bcast", m, A=A, w=w)[0] for m in maps]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    Af, wf = _inputs([6, 16, 700], 1, "f32_comp", "dot_bcast")
    for m in maps:
        runs, _, _ = gpu_rect([6, 16, 700], 1, "sum", "f32_comp", "dot_bcast", m, A=Af, w=wf, repeat=3)
        assert all(np.array_equal(runs[0], r) for r in runs[1:]), f"not bit-reproducible under {m}"


@pytest.mark.parametrize("prec", ["f32", "f32_comp", "i32", "i64"])
def test_pipelined_equals_plain_loads(prec):
    # the cp.async-pipelined block kernel folds in the same order: bit-identical
    from paper_2309_01906_gb300 import binding as hb
    for ext, r, lm in (([3, 7, 16, 132], 2, [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 8, 0)]),
                       ([40, 1028], 1, ["grid", ("cta", 4, 0)]),
                       ([3, 5, 16, 512], 2, [("grid", 0, 0), ("grid", 0, 0), ("cluster", 4, 0), ("cta", 2, 0)])):
        A, w = _inputs(ext, r, prec, "dot_bcast")
        got = {}
        for pipe in (1, 0):
            hb.hp_set_option("pipeline", pipe)
            try:
                got[pipe], plan, bound = gpu_rect(ext, r, "sum", prec, "dot_bcast", lm, A=A, w=w)
            finally:
                hb.hp_set_option("pipeline", 1)
            assert plan["pipe"] == pipe
        assert np.array_equal(got[0], got[1]), (ext, lm)
        ref = oracle_rect(ext, r, "sum", prec, "dot_bcast", A=A, w=w)
        assert_close(got[1], ref, prec, "sum", bound, what=f"pipelined {ext}")


def test_paper_simd8_example():
    # Sec. 3.6: 32 values, parallel level(simd(8)): 8 lanes, each sums 4 values
    A = np.arange(1, 33, dtype=np.int32)
    got, plan, _ = gpu_rect([32], 0, "sum", "i64", "load", [("subwarp", 8, 0)], A=A)
    assert int(got[0]) == 32 * 33 // 2
    assert plan["team_lanes"] == 8 and plan["vec"] == 4 and plan["levels"][0]["slots"] == 32


def test_gemv_workload_full_size():
    # 2-level nest 1024 x 1024, FP32 uniform[-1, 1] and int32 uniform [-100, 100]
    A, x = synth.gemv_f32()
    for prec in ("f32", "f32_comp"):
        check([1024, 1024], 1, "sum", prec, "dot_bcast", ["grid", "warp"], A=A, w=x)
    Ai, xi = synth.gemv_i32()
    check([1024, 1024], 1, "sum", "i32", "dot_bcast", ["grid", "warp"], A=Ai, w=xi)


@pytest.mark.slow
@pytest.mark.parametrize("which", ["bench_map", "cluster8_cta8"])
def test_four_level_workload_full_size(which):
    # 64 x 512 x 16 x 1024 (2 GiB), all 32768 outputs against the oracle, under
    # the map bench.py times (cluster of 4 CTAs x 4 warps x 4 vector slots, the
    # pipelined cluster kernel) and under a cluster of 8 x 8 warps
    import bench
    A, w = synth.nest4_f32()
    lm = bench.LEVEL_MAP if which == "bench_map" else [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 8, 0)]
    ref = oracle.rect([64, 512, 16, 1024], 2, "sum", "f32", "dot_bcast", A=A, w=w)
    for prec in ("f32_comp", "f32"):
        got, plan, bound = gpu_rect([64, 512, 16, 1024], 2, "sum", prec, "dot_bcast", lm, A=A, w=w)
        if which == "bench_map":
            assert (plan["cluster"], plan["warps"], plan["vec"], plan["grid_parts"], plan["pipe"]) == (4, 4, 4, 1, 1)
        assert_close(got, ref, prec, "sum", bound, what=f"4-level full {prec} {which}")


def test_kernel_attributes_shared_between_nests():
    # two nests on the same pipelined kernel with different shared-memory needs,
    # the larger one first: its later runs must still launch
    lm_a = [("grid", 0, 0), ("grid", 0, 0), ("cluster", 2, 0), ("cta", 8, 0)]   # 8 groups per thread
    lm_b = [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 8, 0)]   # 2 groups per thread
    A, w = _inputs([3, 7, 16, 1024], 2, "f32_comp", "dot_bcast")
    first = gpu_rect([3, 7, 16, 1024], 2, "sum", "f32_comp", "dot_bcast", lm_a, A=A, w=w)[0]
    gpu_rect([3, 7, 16, 1024], 2, "sum", "f32_comp", "dot_bcast", lm_b, A=A, w=w)
    again = gpu_rect([3, 7, 16, 1024], 2, "sum", "f32_comp", "dot_bcast", lm_a, A=A, w=w)[0]
    assert np.array_equal(first, again)


@pytest.mark.parametrize("ext,r,lm", [
    ([37, 1029], 1, None),
    ([37, 1028], 1, ["grid", "warp"]),
    ([3, 7, 16, 132], 2, [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 8, 0)]),   # pipelined cluster
    ([7, 1 << 16], 1, [("grid", 0, 0), ("grid", 0, 4096)]),                                    # FP64 grid combine
    ([5, 300], 1, ["grid", ("subwarp", 8, 0)]),
    ([6, 5], 2, None),                                                                          # no reduction
])
def test_compensation_output(ext, r, lm):
    # hp_nest_run_comp: the outputs are hp_nest_run's bits; comp is the exact
    # residual of each output's final rounding, so |comp| <= ulp/2 and out + comp
    # is far closer to the FP64 oracle than out alone
    import torch
    from paper_2309_01906_gb300 import binding as hb
    A, w = _inputs(ext, r, "f32_comp", "dot_bcast")
    O = int(np.prod(ext[:r]))
    n = hb.Nest(ext, r, "sum", "f32_comp", "dot_bcast", level_map=lm)
    try:
        dA, dw = torch.from_numpy(A).cuda(), torch.from_numpy(w).cuda()
        out = torch.empty(O, dtype=torch.float32, device="cuda")
        out2 = torch.empty_like(out)
        comp = torch.full((O,), float("nan"), dtype=torch.float32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        n.run([dA.data_ptr(), dw.data_ptr()], out.data_ptr(), s)
        n.run_comp([dA.data_ptr(), dw.data_ptr()], out2.data_ptr(), comp.data_ptr(), s)
        torch.cuda.synchronize()
        bound = n.error_bound()
    finally:
        n.close()
    o, o2, c = out.cpu().numpy(), out2.cpu().numpy(), comp.cpu().numpy()
    assert np.array_equal(o, o2)
    assert np.all(np.isfinite(c))
    ulp = np.spacing(np.abs(o).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(c.astype(np.float64)) <= 0.5 * ulp)
    ref = oracle_rect(ext, r, "sum", "f32_comp", "dot_bcast", A=A, w=w)
    dw_err = np.abs(o.astype(np.float64) + c.astype(np.float64) - ref.values)
    out_err = np.abs(o.astype(np.float64) - ref.values)
    # the two-word result carries the reduction tree's error only (no final FP32 rounding)
    lim = max(bound - 2.0 ** -24, 0.0) * ref.abs_sum + 2.0 ** -46 * np.abs(ref.values) + 1e-300
    assert np.all(dw_err <= lim), (dw_err.max(), lim.min())
    if r < len(ext):
        assert np.median(dw_err) <= 1e-3 * max(np.median(out_err), 1e-300) or np.median(out_err) == 0
    else:
        # one body value per output: out + comp is the exact FP32 x FP32 product
        assert np.all(dw_err == 0)


@pytest.mark.parametrize("ext,r,prec,lm", [
    ([3, 7, 16, 132], 2, "f32_comp", [("grid", 0, 0), ("grid", 0, 0), ("cluster", 4, 0), ("cta", 4, 0)]),  # pipelined cluster
    ([37, 1029], 1, "f32", ["grid", "warp"]),
    ([7, 1 << 16], 1, "f32_comp", [("grid", 0, 0), ("grid", 0, 4096)]),
    ([40, 1028], 1, "i32", ["grid", ("cta", 4, 0)]),
])
def test_run_host_matches_device_run(ext, r, prec, lm):
    # hp_nest_run_host with host buffers: the streamed input read in place from
    # page-locked memory (zero copy), through a staging copy (option off, and
    # pageable memory): the same bits as hp_nest_run on device copies
    import torch
    from paper_2309_01906_gb300 import binding as hb
    A, w = _inputs(ext, r, prec, "dot_bcast")
    O = int(np.prod(ext[:r]))
    dt = out_dtype(prec)
    n = hb.Nest(ext, r, "sum", prec, "dot_bcast", level_map=lm)
    try:
        s = torch.cuda.current_stream().cuda_stream
        dA, dw = torch.from_numpy(A).cuda(), torch.from_numpy(w).cuda()
        want = torch.empty(O, dtype=dt, device="cuda")
        n.run([dA.data_ptr(), dw.data_ptr()], want.data_ptr(), s)
        torch.cuda.synchronize()
        want = want.cpu()
        hA, hw = torch.from_numpy(A).pin_memory(), torch.from_numpy(w).pin_memory()
        for zero_copy, pinned in ((1, True), (0, True), (1, False)):
            hb.hp_set_option("host_zero_copy", zero_copy)
            try:
                out = torch.full((O,), 7, dtype=dt).pin_memory() if pinned else torch.full((O,), 7, dtype=dt)
                a_ptr = hA.data_ptr() if pinned else A.ctypes.data
                w_ptr = hw.data_ptr() if pinned else w.ctypes.data
                n.run_host([a_ptr, w_ptr], out.data_ptr(), s)
            finally:
                hb.hp_set_option("host_zero_copy", 1)
            assert torch.equal(out, want), (zero_copy, pinned)
    finally:
        n.close()
