"""Each planted mistake in the oracle (built with -DORACLE_MUTANT=k) must fail a pin.

Mutants: 1 R transposed, 2 shift ignored, 3 strict '<' instead of 'at most r',
4 a coordinate dropped from the distance, 5 truncation instead of floor, 6 pair stored
under the larger index, 7 last grid skipped, 8 self-pairs enumerated, 9 a query of a new
point examines only the first grid."""
import pytest

import oracle
import pins

MUTANTS = list(range(1, 10))
FAST_PINS = [p for p in pins.ALL_PINS if p is not pins.pin_table2_recall]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_mutant_is_caught(mutant):
    oracle.build(mutant)
    caught = []
    for pin in FAST_PINS:
        try:
            pin(mutant)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"planted mistake {mutant} passed every pin"
