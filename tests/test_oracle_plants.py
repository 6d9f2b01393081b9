"""Each planted mistake in the oracle (a dropped term, a wrong sign, a swapped
or off-by-one index, a missing a0 division, a dropped chain stage) must fail
at least one pin.  The mistakes are compiled into separate CPU-only builds of
``oracle/oracle.c`` (``-DORACLE_PLANT=k``); the oracle itself is unchanged.
Plant 7 sits in the gradient (VJP) code and must be caught by its pins."""
import numpy as np
import pytest

import oracle
from tests import pins

PLANTS = {
    1: "SOS b2 term dropped",
    2: "SOS a1 sign flipped",
    3: "FIR input index off by one",
    4: "SOS a0 division missing",
    5: "chain drops its last stage",
    6: "SOS a1/a2 swapped",
    7: "VJP: a1 sensitivity sign flipped",
    8: "sampled FIR drops its last tap",
}


@pytest.mark.parametrize("plant", sorted(PLANTS), ids=lambda k: PLANTS[k])
def test_planted_mistake_is_caught(plant):
    lib = oracle.load(plant)
    assert lib.lib.oracle_plant() == plant
    failures = []
    for pin in pins.ALL_PINS:
        try:
            pin(lib, np.random.default_rng(1234))
        except AssertionError:
            failures.append(pin.__name__)
    assert failures, f"no pin caught planted mistake {plant} ({PLANTS[plant]})"


def test_unplanted_build_passes_all_pins():
    lib = oracle.load(0)
    assert lib.lib.oracle_plant() == 0
    for pin in pins.ALL_PINS:
        pin(lib, np.random.default_rng(1234))
