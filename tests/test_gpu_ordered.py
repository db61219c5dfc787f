"""GPU tests of ordered reductions with a non-commutative operator
(HP_RED_AFFINE_COMPOSE): parity with the oracle within gamma_{2k}, exact
results where FP32 arithmetic is exact (so the order of composition is
checked bit for bit), every team and split, ragged sizes and empty ranges."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ordered as oo
from paper_2309_01906_gb300 import binding as hb

pytestmark = pytest.mark.gpu


def _run(ext, r, a, b, lm=None, offset=0):
    import torch
    O = int(np.prod(ext[:r])) if r else 1
    n = hb.Nest(list(ext), r, "compose", "f32", "load", level_map=lm)
    total = a.size
    da = torch.zeros(total + offset + 4, dtype=torch.float32, device="cuda")
    db = torch.zeros(total + offset + 4, dtype=torch.float32, device="cuda")
    da[offset:offset + total] = torch.from_numpy(a.reshape(-1)).cuda()
    db[offset:offset + total] = torch.from_numpy(b.reshape(-1)).cuda()
    out = torch.full((2 * O + 2,), float("nan"), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    n.run([da.data_ptr() + 4 * offset, db.data_ptr() + 4 * offset], out.data_ptr(), s)
    torch.cuda.synchronize()
    d, bound = n.describe(), n.error_bound()
    n.close()
    got = out.cpu().numpy()
    assert np.isnan(got[2 * O:]).all()          # nothing written past the outputs
    return got[:2 * O].reshape(O, 2).astype(np.float64), d, bound


def _inputs(O, R, seed, lo=0.5, hi=1.0):
    g = np.random.Generator(np.random.PCG64(seed))
    return g.uniform(lo, hi, (O, R)).astype(np.float32), g.standard_normal((O, R)).astype(np.float32)


def _check(got, a, b, bound, what):
    A, B = oo.compose_rows(a.astype(np.float64), b.astype(np.float64))
    Aa, Ba = oo.abs_bound_rows(a.astype(np.float64), b.astype(np.float64))
    tiny = 1e-37   # FP32 underflow of long products of factors < 1
    assert np.all(np.abs(got[:, 0] - A) <= bound * Aa + tiny), what
    assert np.all(np.abs(got[:, 1] - B) <= bound * Ba + tiny), what


CASES = [
    ([1000, 300], 1, None),                                   # warp per output, 128-bit loads
    ([777, 301], 1, None),                                    # warp per output, scalar loads
    ([64, 5000], 1, None),                                    # CTA of 8 warps
    ([40, 3, 1001], 1, ["grid", ("cta", 4, 0), ("cta", 4, 0)]),
    ([40, 3, 1001], 1, ["grid", ("cta", 32, 0), ("cta", 32, 0)]),
    ([6, 7, 4000], 1, ["grid", ("grid", 0, 2), "grid"]),     # grid parts of 2 x 4000
    ([3, 100003], 1, ["grid", ("grid", 0, 4099)]),            # ragged last part, scalar loads
    ([4, 1 << 20], 1, None),                                  # automatic split
    ([2, 3, 5, 7], 2, None),                                  # two output levels, tiny reductions
    ([1, 1], 1, None),
    ([5, 33], 0, None),                                       # everything reduced into one output
]


@pytest.mark.parametrize("ext,r,lm", CASES)
def test_parity_with_the_oracle(ext, r, lm):
    O = int(np.prod(ext[:r])) if r else 1
    R = int(np.prod(ext[r:]))
    a, b = _inputs(O, R, O * 7 + R)
    got, d, bound = _run(ext, r, a, b, lm)
    _check(got, a, b, bound, f"{ext} {d['team']} parts={d['grid_parts']} chunk={d['chunk']}")


@pytest.mark.parametrize("ext,r,lm", [([300, 257], 1, None), ([16, 4096], 1, None),
                                      ([3, 5, 2000], 1, ["grid", ("grid", 0, 1), "grid"])])
def test_exact_when_the_arithmetic_is_exact(ext, r, lm):
    # a in {-1, +1}, b small integers: every product and sum is exact in FP32,
    # so the result must equal the exact composition in iteration order
    O = int(np.prod(ext[:r]))
    R = int(np.prod(ext[r:]))
    g = np.random.Generator(np.random.PCG64(R))
    a = g.choice([-1.0, 1.0], (O, R)).astype(np.float32)
    b = g.integers(-8, 9, (O, R)).astype(np.float32)
    got, d, _ = _run(ext, r, a, b, lm)
    for o in range(0, O, max(1, O // 16)):
        A, B = oo.compose_exact(a[o].astype(int).tolist(), b[o].astype(int).tolist())
        assert (got[o, 0], got[o, 1]) == (float(A), float(B)), (o, d["team"])
    # the reversed order gives a different B for these inputs: the executor kept the order
    Ar, Br = oo.compose_exact(a[0, ::-1].astype(int).tolist(), b[0, ::-1].astype(int).tolist())
    assert Br != Fraction(got[0, 1]) or Ar != Fraction(got[0, 0]) or R < 3


@pytest.mark.parametrize("offset", [1, 4])   # 4 bytes: scalar loads; 16 bytes: 128-bit loads
def test_misaligned_inputs_give_the_same_results(offset):
    a, b = _inputs(50, 4000, 3)
    aligned, d, _ = _run([50, 4000], 1, a, b)   # 32-byte aligned: 256-bit loads
    shifted, _, _ = _run([50, 4000], 1, a, b, offset=offset)
    assert d["vec"] == 8 and np.array_equal(aligned, shifted)


def test_empty_ranges_give_the_identity_map():
    got, _, _ = _run([7, 0], 1, np.zeros((7, 0), np.float32), np.zeros((7, 0), np.float32))
    assert np.array_equal(got, np.tile([1.0, 0.0], (7, 1)))


def test_repeated_runs_are_bit_identical():
    a, b = _inputs(4, 1 << 19, 5, 0.9, 1.1)
    first, d, _ = _run([4, 1 << 19], 1, a, b)
    second, _, _ = _run([4, 1 << 19], 1, a, b)
    assert d["grid_parts"] > 1 and np.array_equal(first, second)
