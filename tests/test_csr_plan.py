"""CSR nests on the CPU: descriptor validation and the row-class / chunk
arithmetic the kernels use (no GPU)."""
import numpy as np
import pytest

from paper_2309_01906_gb300 import binding as hb


def params(nnz=100, n_cols=50, shift=2, fuse=0, bins=13):
    return hb.hp_csr_params(nnz, n_cols, shift, fuse, bins)


def test_csr_plans():
    n = hb.Nest(csr_rows=10, red_level=1, op="sum", prec="f32_comp", body="csr_gather", params=params())
    d = n.describe()
    assert d["kind"] == "csr" and d["rows"] == 10 and d["fixed_class"] == -1 and d["chunk"] == 16384
    n.close()
    n = hb.Nest(csr_rows=10, red_level=1, op="sum", prec="f32", body="csr_gather", params=params(),
                level_map=["grid", "warp"])
    assert n.describe()["fixed_class"] == 2
    n.close()
    n = hb.Nest(csr_rows=10, red_level=0, op="hist", prec="i64", body="csr_gather", params=params())
    assert n.describe()["op"] == hb.HP_RED_HIST_COUNT
    n.close()


@pytest.mark.parametrize("kw,fragment", [
    (dict(red_level=0, op="sum"), "red_level 1"),
    (dict(red_level=1, op="hist"), "red_level 0"),
    (dict(red_level=1, op="sum", prec="i32"), "FP32"),
    (dict(red_level=1, op="sum", params=hb.hp_csr_params(-1, 5, 0, 0, 1)), "nnz"),
    (dict(red_level=1, op="sum", params=hb.hp_csr_params(10, 5, 0, 1, 0)), "n_bins"),
    (dict(red_level=1, op="sum", params=hb.hp_csr_params(10, 5, 40, 1, 4)), "shift"),
    (dict(red_level=1, op="sum", level_map=["warp", "warp"]), "rows are bound to the grid"),
    (dict(red_level=1, op="sum", level_map=["grid", ("subwarp", 4, 0)]), "groups of 8"),
])
def test_csr_invalid(kw, fragment):
    args = dict(prec="f32", body="csr_gather", params=params())
    args.update(kw)
    with pytest.raises(hb.HPError) as e:
        hb.Nest(csr_rows=10, **args)
    assert e.value.status == hb.HP_EINVAL and fragment in str(e.value)


def model_row_cover(length, lanes, chunk=16384, split=False):
    """Entries each lane folds (the kernels' arithmetic), relative to the row start."""
    seen = np.zeros(length, dtype=np.int64)
    ranges = [(c * chunk, min(length, (c + 1) * chunk)) for c in range(max(1, -(-length // chunk)))] if split \
        else [(0, length)]
    for s, e in ranges:
        for t in range(lanes):
            b = s + t
            while b < e:
                for u in range(4):
                    idx = b + u * lanes
                    if idx < e:
                        seen[idx] += 1
                b += 4 * lanes
    return seen


@pytest.mark.parametrize("length,lanes,split", [(0, 1, False), (1, 1, False), (4, 1, False), (5, 8, False),
                                                (32, 8, False), (33, 32, False), (1024, 32, False),
                                                (1025, 256, False), (16384, 256, False), (16385, 256, True),
                                                (40000, 256, True), (65536, 256, True)])
def test_row_cover_once(length, lanes, split):
    seen = model_row_cover(length, lanes, split=split)
    assert np.all(seen == 1)


def model_vec_cover(s, e, lanes):
    """Entries lanes fold in the 128-bit path (aligned middle, scalar head / tail)."""
    seen = {}
    g0, g1 = (s + 3) >> 2, e >> 2
    if g0 >= g1:
        return None
    for t in range(lanes):
        if t < 4 * g0 - s:
            seen[s + t] = seen.get(s + t, 0) + 1
        if t < e - 4 * g1:
            seen[4 * g1 + t] = seen.get(4 * g1 + t, 0) + 1
        g = g0 + t
        while g < g1:
            for gg in (g, g + lanes):
                if gg < g1 and (gg == g or True):
                    for k in range(4):
                        seen[4 * gg + k] = seen.get(4 * gg + k, 0) + 1
            g += 2 * lanes
    return seen


@pytest.mark.parametrize("s", [0, 1, 2, 3, 5, 1000, 1001])
@pytest.mark.parametrize("length,lanes", [(8, 32), (33, 32), (1024, 32), (1025, 256), (16385, 256), (7, 32)])
def test_vector_fold_covers_once(s, length, lanes):
    e = s + length
    seen = model_vec_cover(s, e, lanes)
    if seen is None:
        return   # short range: the scalar path (covered above)
    assert sorted(seen) == list(range(s, e)) and set(seen.values()) == {1}
