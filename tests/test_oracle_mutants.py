"""Plants known mistakes in the oracle (on the CPU, via ORACLE_MUTANT) and
checks that the pins catch every one of them."""
import pytest

import oracle
import oracle_pins as P

MUTANTS = {
    1: "basis paired with indices in reverse order",
    2: "wrong sign of the fractional offset",
    3: "dropped constant term in B_2",
    4: "y offset drives the x weights",
    5: "l and m swapped in the grid read",
    6: "channels crossed",
    7: "adjoint scatters to the mirrored x neighbour",
    8: "adjoint drops the last z term",
    9: "resampling: x weights of the two taps exchanged",
    10: "resampling: sign of the z derivative flipped",
    11: "resampling: edge values repeated outside the image",
    12: "non-integer spacing: lattice shift with the wrong sign",
    13: "non-integer spacing adjoint: scatters to the mirrored x neighbour",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda m: MUTANTS[m].replace(" ", "_"))
def test_pins_catch_planted_mistake(mutant, tmp_path):
    path = oracle.build(tmp_path, mutant=mutant)
    lib = oracle.load(path)
    bad = P.failed_pins(lib)
    assert bad, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"
