"""GPU tests of hp_nest_run_batch: many uneven nests in one persistent launch
per arithmetic, replayed from a CUDA graph.  Each nest's outputs must equal
those of hp_nest_run on the same nest bit for bit (same plan, same reduction
tree) and match the oracle within the tolerances of the other parity tests."""
import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb
from paper_2309_01906_gb300 import synth
from tests.hp_testutil import assert_close, oracle_rect, out_dtype

pytestmark = pytest.mark.gpu

# (extents, red_level, op, prec, body, level map)
MIXED = [
    ([37, 1029], 1, "sum", "f32_comp", "dot_bcast", ["grid", "warp"]),
    ([37, 1028], 1, "sum", "f32", "dot_bcast", ["grid", "cta"]),
    ([9, 1028], 1, "sum", "f32_comp", "load", [("grid", 0, 0), ("cta", 4, 0)]),
    ([9, 70], 1, "max", "i32", "load", ["grid", "seq"]),
    ([9, 1028], 1, "sum", "i64", "dot_bcast", ["grid", ("subwarp", 8, 0)]),
    ([5, 1029], 1, "sum", "f32_comp", "load", ["grid", ("grid", 0, 300)]),
    ([5, 4096], 1, "min", "f32", "load", ["grid", ("grid", 0, 1024)]),
    ([3, 7, 16, 132], 2, "sum", "f32_comp", "dot_bcast", ["grid", "grid", "cta", "warp"]),
    ([2, 5, 11, 96], 2, "sum", "i32", "dot_bcast", ["grid", "grid", ("grid", 0, 5), "cta"]),
    ([2, 5, 11, 96], 2, "max", "i64", "load", ["grid", "cta", "warp", "seq"]),
    ([6, 5], 2, "sum", "f32", "load", None),
    ([2, 3, 4, 5, 6], 0, "sum", "f32_comp", "dot_bcast", None),
    ([300], 0, "max", "i32", "load", None),
    ([4, 3, 2, 70], 1, "min", "i64", "dot_bcast", None),
    ([7, 1 << 16], 1, "sum", "f32_comp", "load", None),
    ([11, 13], 1, "sum", "i32", "affine", None),
    ([1, 0], 1, "sum", "f32", "load", None),
]


def _make(case, rng):
    import torch
    ext, r, op, prec, body, lm = case
    total = int(np.prod(ext))
    R = int(np.prod(ext[r:])) if r < len(ext) else 1
    params = hb.hp_affine_params(-3, 5, 7) if body == "affine" else None
    n = hb.Nest(ext, r, op, prec, body, level_map=lm, params=params)
    if prec in ("i32", "i64"):
        A = rng.integers(-1000, 1001, max(total, 1)).astype(np.int32)
        w = rng.integers(-1000, 1001, max(R, 1)).astype(np.int32)
    else:
        A = rng.standard_normal(max(total, 1)).astype(np.float32)
        w = rng.uniform(-1, 1, max(R, 1)).astype(np.float32)
    dA, dw = torch.from_numpy(A).cuda(), torch.from_numpy(w).cuda()
    ins = {"load": [dA.data_ptr()], "dot_bcast": [dA.data_ptr(), dw.data_ptr()], "affine": []}[body]
    O = int(np.prod(ext[:r])) if r else 1
    return dict(nest=n, A=A, w=w, dA=dA, dw=dw, ins=ins, O=O, case=case, params=params)


def _out(item):
    import torch
    return torch.full((max(item["O"], 1),), 7, dtype=out_dtype(item["case"][3]), device="cuda")


def test_batch_equals_single_runs_and_oracle():
    import torch
    rng = np.random.Generator(np.random.PCG64(404))
    items = [_make(c, rng) for c in MIXED]
    s = torch.cuda.current_stream().cuda_stream
    singles = []
    for it in items:
        o = _out(it)
        it["nest"].run(it["ins"], o.data_ptr(), s)
        singles.append(o)
    for rep in range(2):   # two replays in a row: descriptors, counters and tickets start clean
        outs = [_out(it) for it in items]
        hb.hp_nest_run_batch([it["nest"].handle for it in items], [it["ins"] for it in items],
                             [o.data_ptr() for o in outs], s)
        torch.cuda.synchronize()
        for it, o, ref_o in zip(items, outs, singles):
            got = o[:it["O"]].cpu().numpy()
            assert np.array_equal(got, ref_o[:it["O"]].cpu().numpy()), f"batch != single for {it['case']}"
    for it, o in zip(items, singles):
        ext, r, op, prec, body, lm = it["case"]
        prm = (-3, 5, 7) if body == "affine" else None
        ref = oracle_rect(ext, r, op, prec, body, A=it["A"], w=it["w"], params=prm)
        assert_close(o[:it["O"]].cpu().numpy(), ref, prec, op, what=f"batch {it['case']}")
    for it in items:
        it["nest"].close()


def test_uneven_shapes_batch():
    import torch
    shapes = synth.uneven_shapes(n_nests=300, seed=9, mu=float(np.log(2.0 ** 10)), sigma=1.5, t_max=1 << 18)
    rng = np.random.Generator(np.random.PCG64(405))
    items = []
    for sh in shapes:
        items.append(_make((list(sh.extents), sh.red_level, sh.op, sh.prec, "load", None), rng))
    s = torch.cuda.current_stream().cuda_stream
    outs = [_out(it) for it in items]
    hb.hp_nest_run_batch([it["nest"].handle for it in items], [it["ins"] for it in items],
                         [o.data_ptr() for o in outs], s)
    torch.cuda.synchronize()
    for it, o in zip(items, outs):
        single = _out(it)
        it["nest"].run(it["ins"], single.data_ptr(), s)
        torch.cuda.synchronize()
        assert np.array_equal(o[:it["O"]].cpu().numpy(), single[:it["O"]].cpu().numpy()), it["case"]
    for it in items[:40]:
        ext, r, op, prec, body, _ = it["case"]
        ref = oracle_rect(ext, r, op, prec, "load", A=it["A"])
        assert_close(outs[items.index(it)][:it["O"]].cpu().numpy(), ref, prec, op, what=str(it["case"]))
    for it in items:
        it["nest"].close()


def test_batch_runs_cluster_teams_alone():
    # a cluster-team plan cannot run in the persistent kernel's single CTAs:
    # the batch runs it with its own launch, beside the batched nests, and
    # every output still equals hp_nest_run's
    import torch
    rng = np.random.Generator(np.random.PCG64(407))
    cases = [([3, 7, 16, 132], 2, "sum", "f32", "load", [("grid", 0, 0), ("grid", 0, 0), ("cluster", 4, 0), ("cta", 4, 0)]),
             MIXED[0], MIXED[3],
             ([2, 5, 16, 512], 2, "sum", "f32_comp", "dot_bcast", [("grid", 0, 0), ("grid", 0, 0), ("cluster", 8, 0), ("cta", 2, 0)])]
    items = [_make(c, rng) for c in cases]
    s = torch.cuda.current_stream().cuda_stream
    outs = [_out(it) for it in items]
    for _ in range(2):   # built, then replayed
        hb.hp_nest_run_batch([it["nest"].handle for it in items], [it["ins"] for it in items],
                             [o.data_ptr() for o in outs], s)
    torch.cuda.synchronize()
    for it, o in zip(items, outs):
        single = _out(it)
        it["nest"].run(it["ins"], single.data_ptr(), s)
        torch.cuda.synchronize()
        assert torch.equal(o[:it["O"]], single[:it["O"]]), it["case"]
        ext, r, op, prec, body, _ = it["case"]
        ref = oracle_rect(ext, r, op, prec, body, A=it["A"], w=it["w"])
        assert_close(o[:it["O"]].cpu().numpy(), ref, prec, op, what=f"batch {it['case']}")
        it["nest"].close()


def test_batch_after_destroy_and_recreate():
    # a destroyed nest's address may be reused by the next nest: the batch must
    # be rebuilt for the new nest's plan, never replayed from the old one
    import torch
    rng = np.random.Generator(np.random.PCG64(406))
    s = torch.cuda.current_stream().cuda_stream
    for case in (MIXED[3], MIXED[14], MIXED[0], MIXED[6]):
        it = _make(case, rng)
        out = _out(it)
        hb.hp_nest_run_batch([it["nest"].handle], [it["ins"]], [out.data_ptr()], s)
        single = _out(it)
        it["nest"].run(it["ins"], single.data_ptr(), s)
        torch.cuda.synchronize()
        assert torch.equal(out[:it["O"]], single[:it["O"]]), case
        it["nest"].close()


def test_stated_distribution_sample_against_oracle():
    # 256 nests drawn (seed 19) from the batched workload's own 10,000 shapes
    # (sigma 2, T up to 2^24, seed 9, inputs as the bench generates them), run
    # in one batch and compared with the oracle: FP32 compensated sums within
    # the normalized tolerance and the a-priori bound, int32 max bit for bit
    import torch
    from concurrent.futures import ThreadPoolExecutor
    shapes = synth.uneven_shapes(n_nests=10000, seed=9)
    g = np.random.Generator(np.random.PCG64(19))
    idxs = sorted(int(i) for i in g.choice(len(shapes), size=256, replace=False))
    assert max(shapes[i].size for i in idxs) > 1 << 20   # the long tail is in the sample
    nests, ins, outs, keep, hosts = [], [], [], [], []
    for i in idxs:
        sh = shapes[i]
        A = synth.nest_input(sh, i, 9)
        dA = torch.from_numpy(A).cuda()
        nests.append(hb.Nest(list(sh.extents), sh.red_level, sh.op, sh.prec, "load"))
        o = torch.full((max(sh.n_out, 1),), 7, dtype=out_dtype(sh.prec), device="cuda")
        ins.append([dA.data_ptr()])
        outs.append(o)
        keep.append(dA)
        hosts.append(A)
    s = torch.cuda.current_stream().cuda_stream
    hb.hp_nest_run_batch([n.handle for n in nests], ins, [o.data_ptr() for o in outs], s)
    torch.cuda.synchronize()

    def ref(k):
        sh = shapes[idxs[k]]
        return oracle_rect(list(sh.extents), sh.red_level, sh.op, sh.prec, "load", A=hosts[k])

    with ThreadPoolExecutor(8) as ex:
        refs = list(ex.map(ref, range(len(idxs))))
    for k, i in enumerate(idxs):
        sh = shapes[i]
        assert_close(outs[k][:sh.n_out].cpu().numpy(), refs[k], sh.prec, sh.op, nests[k].error_bound(),
                     what=f"nest {i} {sh.extents} r={sh.red_level}")
    for n in nests:
        n.close()
