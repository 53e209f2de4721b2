"""The CPU oracle against its pins (no GPU)."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("pin", P.CPU_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(orc, pin):
    pin(orc)


@pytest.mark.parametrize("pin", P.DATA_PINS, ids=lambda f: f.__name__)
def test_oracle_pin_on_small_day(orc, small_day, pin):
    pin(orc, small_day)


def test_oracle_pin_full_range_ids(orc):
    """Journey ids spread over all of int64 (the case that defeats a 64-bit packed key)."""
    import cvgen

    cols = cvgen.generate(cvgen.params("small_day", seed=4, n_journeys=300, jid_mode=1))
    assert cols["jid"].min() < -(2 ** 62) and cols["jid"].max() > 2 ** 62
    P.pin_invariants(orc, cols)
    P.pin_library_cross_check(orc, cols)
