"""GPU tests of the autotuner: candidates are timed on the caller's buffers, the
winner is installed and cached per shape class, later automatic nests of the
class take it, and results stay within the oracle tolerances."""
import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb
from tests.hp_testutil import assert_close, oracle_rect

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("batched", [False, True])
@pytest.mark.parametrize("ext,r,op,prec", [([200, 3000], 1, "sum", "f32_comp"), ([5000, 6], 1, "max", "i32"),
                                          ([3, 200000], 1, "sum", "f32"), ([64, 8, 100], 1, "sum", "i64")])
def test_tune_installs_and_caches(ext, r, op, prec, batched):
    # batched: candidates (and the planner's own map) timed in the batched executor
    import torch
    rng = np.random.Generator(np.random.PCG64(7))
    total = int(np.prod(ext))
    if prec in ("i32", "i64"):
        A = rng.integers(-1000, 1001, total).astype(np.int32)
        dt = torch.int32 if prec == "i32" else torch.int64
    else:
        A = rng.standard_normal(total).astype(np.float32)
        dt = torch.float32
    dA = torch.from_numpy(A).cuda()
    O = int(np.prod(ext[:r]))
    out = torch.empty(O, dtype=dt, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    n = hb.Nest(ext, r, op, prec, "load")
    n.tune([dA.data_ptr()], out.data_ptr(), s, retime=True, batched=batched)
    d = n.describe()
    assert d["tuned"]
    torch.cuda.synchronize()
    ref = oracle_rect(ext, r, op, prec, "load", A=A)
    assert_close(out.cpu().numpy(), ref, prec, op, n.error_bound(), what=f"tuned {ext}")
    # a later automatic nest of the same shape class takes the cached binding
    n2 = hb.Nest(ext, r, op, prec, "load")
    d2 = n2.describe()
    assert d2["tuned"] and d2["map"] == d["map"]
    out2 = torch.empty(O, dtype=dt, device="cuda")
    n2.run([dA.data_ptr()], out2.data_ptr(), s)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
    # batching after tuning uses the installed plan
    out3 = torch.empty(O, dtype=dt, device="cuda")
    hb.hp_nest_run_batch([n.handle], [[dA.data_ptr()]], [out3.data_ptr()], s)
    torch.cuda.synchronize()
    assert torch.equal(out, out3)
    n.close()
    n2.close()


@pytest.mark.parametrize("ext,req,allowed", [
    ([2000, 384], [{}, {"sync": ["shuffle"]}], {"warp", "subwarp"}),
    ([2000, 384], [{}, {"sync": ["barrier", "localmem"]}], {"cta", "cluster"}),
    ([4000, 64], [{}, {"sync": ["lockstep"]}], {"lane", "seq"}),
])
def test_tune_under_level_requirements(ext, req, allowed):
    # Sec. 3.2 requirements as the tuner's constraint language: only maps that
    # meet them are timed; the winner is cached under them alone
    import torch
    rng = np.random.Generator(np.random.PCG64(17))
    A = rng.standard_normal(int(np.prod(ext))).astype(np.float32)
    dA = torch.from_numpy(A).cuda()
    out = torch.empty(ext[0], dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    n = hb.Nest(ext, 1, "sum", "f32_comp", "load")
    n.tune([dA.data_ptr()], out.data_ptr(), s, retime=True, req=req)
    d = n.describe()
    assert d["tuned"] and d["map"][1]["hw"] in allowed, d["map"]
    assert hb.hp_level_check(req, [(m["hw"], m["sub_width"], m["tile"]) for m in d["map"]])[0]
    torch.cuda.synchronize()
    ref = oracle_rect(ext, 1, "sum", "f32_comp", "load", A=A)
    assert_close(out.cpu().numpy(), ref, "f32_comp", "sum", n.error_bound(), what=f"tuned under {req}")
    fresh = hb.Nest(ext, 1, "sum", "f32_comp", "load")   # an automatic nest of the class: not given the choice
    assert not fresh.describe()["tuned"]
    fresh.close()
    n.close()


def test_tuned_class_applies_across_depths():
    # a shape class (log2 outputs, log2 reduced size, ...) spans nests of
    # different depths: the binding tuned on a 4-level nest (with per-level
    # and cluster candidates) must give every later automatic nest of the
    # class a legal plan, or the planner's own map, and correct results
    import torch
    rng = np.random.Generator(np.random.PCG64(11))
    ext_a = [3, 5, 64, 1024]          # 15 outputs x 2^16 reduced, two reduced levels
    A = rng.standard_normal(int(np.prod(ext_a))).astype(np.float32)
    dA = torch.from_numpy(A).cuda()
    out = torch.empty(15, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    n = hb.Nest(ext_a, 2, "sum", "f32_comp", "load")
    n.tune([dA.data_ptr()], out.data_ptr(), s, retime=True)
    torch.cuda.synchronize()
    assert_close(out.cpu().numpy(), oracle_rect(ext_a, 2, "sum", "f32_comp", "load", A=A), "f32_comp", "sum",
                 n.error_bound(), what=f"tuned {n.describe()['map']}")
    n.close()
    for ext_b, r in (([15, 65536], 1), ([15, 2, 8, 4096], 1), ([5, 3, 65536], 2)):
        B = rng.standard_normal(int(np.prod(ext_b))).astype(np.float32)
        dB = torch.from_numpy(B).cuda()
        nb = hb.Nest(ext_b, r, "sum", "f32_comp", "load")
        ob = torch.empty(15, dtype=torch.float32, device="cuda")
        nb.run([dB.data_ptr()], ob.data_ptr(), s)
        torch.cuda.synchronize()
        assert_close(ob.cpu().numpy(), oracle_rect(ext_b, r, "sum", "f32_comp", "load", A=B), "f32_comp", "sum",
                     nb.error_bound(), what=f"{ext_b} {nb.describe()['map']}")
        nb.close()
