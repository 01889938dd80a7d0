"""The CPU oracle against its pins (CPU only)."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)
