"""The bench line's per-result error statement (bench.fp_parity) on the CPU:
clause selection, the plain-FP32 scales and the a-priori bound check, against
errors planted in known places.  No GPU."""
import csv
import os

import numpy as np

import bench
import oracle


def _ref(values, abs_sum, sq_sum):
    return oracle.Result(np.asarray(values, np.float64), np.asarray(abs_sum, np.float64),
                         np.asarray(sq_sum, np.float64))


def test_clauses_and_worst_result():
    # result 0: well conditioned (relative clause); result 1: cond 2^22 (normalized clause)
    ref = _ref([2.0, 1.0], [4.0, 2.0 ** 22], [8.0, 2.0 ** 30])
    got = np.array([2.0 * (1 + 3e-7), 1.0 + 2.0 ** 22 * 2.0 ** -20 * 5e-7], np.float32)
    d = bench.fp_parity(got, ref, "f32_comp", 1e-6, 1e-6)
    assert d["n_checked"] == 2 and d["n_relative_clause"] == 1 and d["n_normalized_clause"] == 1
    assert 2e-7 < d["max_norm_err"] < 6e-7 and d["pass"]
    assert d["max_cond"] == 2.0 ** 22
    # a planted error of 2e-6 in the well-conditioned result fails the 1e-6 tolerance
    bad = got.copy()
    bad[0] = np.float32(2.0 * (1 + 2e-6))
    d = bench.fp_parity(bad, ref, "f32_comp", 1e-5, 1e-6)
    assert not d["pass"] and d["worst"]["index"] == 0


def test_a_priori_bound_is_checked():
    ref = _ref([1.0], [10.0], [10.0])
    got = np.array([1.0 + 1e-5], np.float32)
    assert not bench.fp_parity(got, ref, "f32_comp", 1e-7, 1.0)["within_a_priori_bound"]
    assert bench.fp_parity(got, ref, "f32_comp", 1e-5, 1.0)["within_a_priori_bound"]


def test_plain_scale_is_the_two_norm():
    # a cancelling plain sum: |ref| = 1e-3, sqrt(sum t^2) = 10 -> scaled error 1e-7
    ref = _ref([1e-3], [100.0], [100.0])
    got = np.array([1e-3 + 1e-6], np.float32)
    d = bench.fp_parity(got, ref, "f32", 1.0, 1e-5)
    assert d["max_norm_err_l2_scale"] < 1e-5 and d["pass"]
    assert d["max_plain_rel_err"] > 1e-4 and not d["pass_sum_abs_clause"]


def test_exact_zero_references():
    ref = _ref([0.0, 3.0], [0.0, 3.0], [0.0, 9.0])
    d = bench.fp_parity(np.array([0.0, 3.0], np.float32), ref, "f32_comp", 1e-6, 1e-6)
    assert d["n_exact_zero_ref"] == 1 and d["max_norm_err"] == 0.0 and d["pass"]
    d = bench.fp_parity(np.array([1e-30, 3.0], np.float32), ref, "f32_comp", 1e-6, 1e-6)
    assert not d["pass"]   # a nonzero result where every term is zero


def test_per_result_table(tmp_path):
    ref = _ref([2.0, 1.0], [4.0, 2.0 ** 22], [8.0, 2.0 ** 30])
    got = np.array([2.0, 1.0], np.float32)
    path = os.path.join(str(tmp_path), "parity.csv")
    bench.write_parity_table(path, np.array([5, 9]), got, ref)
    rows = list(csv.DictReader(open(path)))
    assert [int(r["output"]) for r in rows] == [5, 9]
    assert [r["clause"] for r in rows] == ["relative", "normalized"]
    assert float(rows[1]["cond"]) == 2.0 ** 22
