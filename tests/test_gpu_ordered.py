"""GPU tests of ordered reductions with a non-commutative operator
(HP_RED_AFFINE_COMPOSE, HP_RED_MAT2_PRODUCT, HP_RED_LAST_VALID): parity with
the oracle within the error bound of products (gamma_{2(R-1)}, or the
probabilistic bound for R - 1 combines when tighter), exact
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


def _tol(bound, R):
    # the library's worst-case bound (gamma_{2(R-1)}) or, tighter for long ranges,
    # the probabilistic bound for the same R - 1 combines (fails with probability
    # below 2 exp(-50) under the model of independent rounding errors)
    return min(bound, oo.prob_bound(R - 1))


def _check(got, a, b, bound, what):
    A, B = oo.compose_rows(a.astype(np.float64), b.astype(np.float64))
    Aa, Ba = oo.abs_bound_rows(a.astype(np.float64), b.astype(np.float64))
    tol = _tol(bound, a.shape[1])
    tiny = 1e-37   # FP32 underflow of long products of factors < 1
    assert np.all(np.abs(got[:, 0] - A) <= tol * Aa + tiny), what
    assert np.all(np.abs(got[:, 1] - B) <= tol * Ba + tiny), what


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


# ---------------------------------------------------------------- other ordered operators

def _run_op(ext, r, op, arrays, nout, lm=None, offset=0):
    """Run an ordered nest of operator `op` on FP32 `arrays` (each flattened),
    returning (O, nout) FP32 outputs and the plan."""
    import torch
    O = int(np.prod(ext[:r])) if r else 1
    n = hb.Nest(list(ext), r, op, "f32", "load", level_map=lm)
    ptrs, keep = [], []
    for arr in arrays:
        flat = np.ascontiguousarray(arr, np.float32).reshape(-1)
        d = torch.zeros(flat.size + offset + 8, dtype=torch.float32, device="cuda")
        d[offset:offset + flat.size] = torch.from_numpy(flat).cuda()
        keep.append(d)
        ptrs.append(d.data_ptr() + 4 * offset)
    out = torch.full((nout * O + 3,), 7.0, dtype=torch.float32, device="cuda")
    n.run(ptrs, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    d, bound = n.describe(), n.error_bound()
    n.close()
    got = out.cpu().numpy()
    assert np.all(got[nout * O:] == 7.0)             # nothing written past the outputs
    return got[:nout * O].reshape(O, nout), d, bound


def _markov(O, R, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    p, q = g.uniform(0.0, 1.0, (O, R)), g.uniform(0.0, 1.0, (O, R))
    return np.stack([1 - p, p, q, 1 - q], axis=-1).astype(np.float32)


@pytest.mark.parametrize("ext,r,lm", CASES)
def test_mat2_parity_with_the_oracle(ext, r, lm):
    O = int(np.prod(ext[:r])) if r else 1
    R = int(np.prod(ext[r:]))
    m = _markov(O, R, O * 11 + R)
    got, d, bound = _run_op(ext, r, "mat2", [m], 4, lm)
    want = oo.mat2_rows(m.astype(np.float64))
    scale = oo.mat2_abs_rows(m.astype(np.float64))   # = want: non-negative entries
    assert d["op"] == "mat2_product" and bound >= 0   # 0: a single matrix, no combine
    assert np.all(np.abs(got - want) <= _tol(bound, R) * scale + 1e-37), (ext, d["team"], d["vec"])


@pytest.mark.parametrize("ext,r,lm", [([300, 257], 1, None), ([16, 4096], 1, None), ([4, 1 << 18], 1, None),
                                      ([3, 5, 2000], 1, ["grid", ("grid", 0, 1), "grid"])])
def test_mat2_exact_in_order_on_signed_permutations(ext, r, lm):
    # the 8 signed 2x2 permutation matrices form a non-commutative group: every
    # FP32 operation is exact, so the product must equal the rational one
    O, R = int(np.prod(ext[:r])), int(np.prod(ext[r:]))
    group = np.array([[1, 0, 0, 1], [0, -1, 1, 0], [-1, 0, 0, -1], [0, 1, -1, 0],
                      [1, 0, 0, -1], [-1, 0, 0, 1], [0, 1, 1, 0], [0, -1, -1, 0]], np.float32)
    g = np.random.Generator(np.random.PCG64(R))
    m = group[g.integers(0, 8, (O, R))]
    got, d, _ = _run_op(ext, r, "mat2", [m], 4, lm)
    for o in range(0, O, max(1, O // 8)):
        want = oo.mat2_exact(m[o].astype(int).tolist())
        assert tuple(float(v) for v in want) == tuple(got[o]), (o, d["team"], d["grid_parts"])


def test_mat2_of_affine_maps_equals_the_affine_operator():
    # [[a, b], [0, 1]] composes like (a, b); with a = +-1 and small integer b every
    # FP32 operation of both operators is exact, whatever their trees
    g = np.random.Generator(np.random.PCG64(31))
    a = g.choice([-1.0, 1.0], (300, 4096)).astype(np.float32)
    b = g.integers(-8, 9, (300, 4096)).astype(np.float32)
    m = np.stack([a, b, np.zeros_like(a), np.ones_like(a)], axis=-1)
    got, dm, _ = _run_op([300, 4096], 1, "mat2", [m], 4)
    aff, da, _ = _run([300, 4096], 1, a, b)
    assert dm["piece"] != da["piece"]   # different trees (4 matrices, 8 maps per piece)
    assert np.array_equal(got[:, 2], np.zeros(300)) and np.array_equal(got[:, 3], np.ones(300))
    assert np.array_equal(got[:, :2].astype(np.float64), aff)


@pytest.mark.parametrize("offset", [1, 4])
def test_mat2_misaligned_inputs_give_the_same_results(offset):
    m = _markov(20, 3000, 5)
    aligned, d, _ = _run_op([20, 3000], 1, "mat2", [m], 4)
    shifted, _, _ = _run_op([20, 3000], 1, "mat2", [m], 4, offset=offset)
    assert d["vec"] == 8 and np.array_equal(aligned, shifted)


def _gappy(O, R, seed, p_nan):
    g = np.random.Generator(np.random.PCG64(seed))
    v = g.standard_normal((O, R)).astype(np.float32)
    v[g.random((O, R)) < p_nan] = np.nan
    return v


@pytest.mark.parametrize("p_nan", [0.3, 0.999])
@pytest.mark.parametrize("ext,r,lm", CASES)
def test_last_valid_bit_exact(ext, r, lm, p_nan):
    O = int(np.prod(ext[:r])) if r else 1
    R = int(np.prod(ext[r:]))
    v = _gappy(O, R, O * 3 + R, p_nan)
    got, d, bound = _run_op(ext, r, "last", [v], 1, lm)
    want = oo.last_valid_rows(v.reshape(O, R))
    got = got[:, 0]
    none = np.isnan(want)
    assert d["op"] == "last_valid" and bound == 0.0
    assert np.array_equal(got[~none].view(np.uint32), want[~none].view(np.uint32)), (ext, d["team"])
    assert np.all(got[none].view(np.uint32) == 0x7FC00000)


def test_last_valid_takes_the_last_value_not_the_largest_index_of_a_part():
    # one value per row, at a random place; everything else missing
    O, R = 64, 1 << 18
    v = np.full((O, R), np.nan, np.float32)
    g = np.random.Generator(np.random.PCG64(9))
    at = g.integers(0, R, O)
    v[np.arange(O), at] = np.arange(O, dtype=np.float32) + 0.5
    v[::2, 0] = -1.0                           # an earlier value in every other row must lose
    got, d, _ = _run_op([O, R], 1, "last", [v], 1)
    assert d["grid_parts"] > 1 and np.array_equal(got[:, 0], np.arange(O, dtype=np.float32) + 0.5)


@pytest.mark.parametrize("offset", [1, 4])
def test_last_valid_misaligned_and_empty(offset):
    v = _gappy(30, 4000, 6, 0.9)
    aligned, d, _ = _run_op([30, 4000], 1, "last", [v], 1)
    shifted, _, _ = _run_op([30, 4000], 1, "last", [v], 1, offset=offset)
    assert d["vec"] == 8 and np.array_equal(aligned.view(np.uint32), shifted.view(np.uint32))
    empty, _, _ = _run_op([5, 0], 1, "last", [np.zeros((5, 0), np.float32)], 1)
    assert np.all(empty.view(np.uint32) == 0x7FC00000)
