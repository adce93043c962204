"""Every planted mistake in the oracle must fail at least one pin.

oracle.c compiles a known mistake when built with ORACLE_MUTANT=k (a
flipped twiddle sign, a dropped term, an index off by one, swapped
real/imaginary parts, a wrong butterfly sign, a skipped reordering, a
forgotten twiddle stride, wrong generator bits or counter, a conjugated
or truncated sampled-mode twiddle, a mis-reduced octant or quadrant).
The mutants are built into a temporary directory; the shipped library is
always built with ORACLE_MUTANT=0.
"""
import pytest

import oracle
from oracle_pins import ALL_PINS

MUTANTS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 13, 14]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_mutant_is_caught(mutant, tmp_path):
    o = oracle.Oracle(mutant=mutant, outdir=str(tmp_path))
    assert o._lib.oracle_mutant() == mutant
    caught = []
    for pin in ALL_PINS:
        try:
            pin(o)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
            break
    assert caught, f"mutant {mutant} passed every pin"


def test_real_oracle_is_not_a_mutant(orc):
    assert orc._lib.oracle_mutant() == 0
