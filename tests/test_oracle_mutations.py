"""Planted mistakes in the oracle must fail at least one pin.

Each case builds the oracle C file with one planted mistake (a compile-time
switch that is 0 in every other build) into a temporary library and runs the
full pin battery against it.  A pin battery that let a dropped term, a flipped
sign, a transposed operand, a lost compensation or a wrong reduction level
through would not pin the oracle; nor would one that let an inflated or
misformed conditioning sum (sum|t|, sum t^2: the scales of every FP tolerance)
through.  CPU only.
"""
import os

import pytest

import oracle
from tests.oracle_pins import ALL_PINS

MUTATIONS = {
    1: "drops the last term of every innermost loop",
    2: "negates odd-indexed terms",
    3: "transposes the broadcast operand's two innermost indices",
    4: "drops the Neumaier compensation",
    5: "reduces one level too few",
    6: "doubles sum|t|",
    7: "adds |t| to sum t^2",
    8: "drops the absolute value in sum|t|",
}


@pytest.mark.parametrize("mutation", sorted(MUTATIONS), ids=lambda m: MUTATIONS[m].replace(" ", "_"))
def test_planted_mistake_fails_a_pin(mutation, tmp_path):
    path = os.path.join(str(tmp_path), f"liboracle_mut{mutation}.so")
    oracle.build(path, extra_flags=[f"-DORACLE_MUTATION={mutation}"])
    lib = oracle.load(path)
    caught = []
    for pin in ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError, ZeroDivisionError) as e:
            caught.append((pin.__name__, repr(e)[:80]))
    assert caught, f"mutation {mutation} ({MUTATIONS[mutation]}) passed every pin"
