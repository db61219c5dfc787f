"""The CPU oracle against its pins (closed forms, library routines, exact sums,
brute force, the paper's worked-example sizes).  No GPU."""
import pytest

import oracle
from tests.oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(oracle.load())
