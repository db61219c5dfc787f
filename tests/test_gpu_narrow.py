"""GPU tests of nests on 8- / 16-bit integers with SIMD-in-register sub-lanes:
bit-exact against the oracle (the integer definition on the widened inputs:
sums modulo 2^32, max, min, int8 dot products) for every team, split and
alignment, ragged rows and empty reductions."""
import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb
from tests.hp_testutil import oracle_rect

pytestmark = pytest.mark.gpu

NP = {"i8": np.int8, "i16": np.int16}


def _run(ext, r, op, prec, body, A, w=None, lm=None, offset=0):
    import torch
    O = int(np.prod(ext[:r])) if r else 1
    n = hb.Nest(list(ext), r, op, prec, body, level_map=lm)
    tdt = torch.int8 if prec == "i8" else torch.int16
    esz = 1 if prec == "i8" else 2
    dA = torch.zeros(A.size + offset + 16, dtype=tdt, device="cuda")
    dA[offset:offset + A.size] = torch.from_numpy(A.reshape(-1)).cuda()
    ins = [dA.data_ptr() + esz * offset]
    if w is not None:
        dw = torch.from_numpy(w.reshape(-1)).cuda()
        ins.append(dw.data_ptr())
    out = torch.full((O + 1,), -7, dtype=torch.int32, device="cuda")
    n.run(ins, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    d = n.describe()
    n.close()
    got = out.cpu().numpy()
    assert got[O] == -7                      # nothing written past the outputs
    return got[:O].astype(np.int64), d


def _ref(ext, r, op, body, A, w=None):
    # the integer definition on the inputs widened to int32 (sums modulo 2^32)
    vals = oracle_rect(list(ext), r, op, "i32", "load" if body == "load" else "dot_bcast",
                       A=A.astype(np.int32).reshape(-1), w=None if w is None else w.astype(np.int32).reshape(-1))
    return np.asarray(vals.values if hasattr(vals, "values") else vals, dtype=np.int64)


def _data(shape, prec, seed, full_range=True):
    g = np.random.Generator(np.random.PCG64(seed))
    info = np.iinfo(NP[prec])
    lo, hi = (info.min, info.max) if full_range else (-100, 100)
    return g.integers(lo, hi + 1, shape).astype(NP[prec])


CASES = [
    ([1000, 4096], 1, None), ([300, 4097], 1, None), ([64, 1 << 16], 1, None), ([8, 3, 40000], 1, None),
    ([4, 1 << 21], 1, None), ([40, 3, 1000], 1, ["grid", ("cta", 4, 0), ("cta", 4, 0)]),
    ([6, 7, 4096], 1, ["grid", ("grid", 0, 2), "grid"]), ([2, 3, 5, 7], 2, None), ([5, 33], 0, None),
]


@pytest.mark.parametrize("prec", ["i8", "i16"])
@pytest.mark.parametrize("op", ["sum", "max", "min"])
@pytest.mark.parametrize("ext,r,lm", CASES)
def test_load_bit_exact(ext, r, lm, op, prec):
    A = _data(ext, prec, int(np.prod(ext)) % 9973 + len(op))
    got, d = _run(ext, r, op, prec, "load", A, lm=lm)
    ref = _ref(ext, r, op, "load", A)
    if op == "sum":
        ref = ((ref + 2 ** 31) % 2 ** 32) - 2 ** 31     # int32 results wrap like HP_I32
    assert np.array_equal(got, ref), (ext, op, prec, d["team"], d["grid_parts"])


@pytest.mark.parametrize("ext,r,lm", CASES[:6])
def test_int8_dot_bit_exact(ext, r, lm):
    R = int(np.prod(ext[r:]))
    A = _data(ext, "i8", 11)
    w = _data((R,), "i8", 12)
    got, d = _run(ext, r, "sum", "i8", "dot_bcast", A, w=w, lm=lm)
    ref = _ref(ext, r, "sum", "dot_bcast", A, w)
    ref = ((ref + 2 ** 31) % 2 ** 32) - 2 ** 31
    assert np.array_equal(got, ref), (ext, d["team"])


@pytest.mark.parametrize("prec", ["i8", "i16"])
def test_misaligned_rows_take_element_loads_with_the_same_results(prec):
    A = _data((50, 4096), prec, 3)
    for op in ("sum", "max"):
        aligned, _ = _run([50, 4096], 1, op, prec, "load", A)
        shifted, _ = _run([50, 4096], 1, op, prec, "load", A, offset=1)
        assert np.array_equal(aligned, shifted)


def test_empty_reductions_give_the_identities():
    for prec, lo, hi in (("i8", -128, 127), ("i16", -32768, 32767)):
        A = np.zeros((7, 0), NP[prec])
        assert np.array_equal(_run([7, 0], 1, "sum", prec, "load", A)[0], np.zeros(7))
        assert np.array_equal(_run([7, 0], 1, "max", prec, "load", A)[0], np.full(7, lo))
        assert np.array_equal(_run([7, 0], 1, "min", prec, "load", A)[0], np.full(7, hi))
