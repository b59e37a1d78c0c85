"""The velocity-variant oracle against its pins (CPU only)."""
import pytest

import oracle
from tests import variant_pins


@pytest.fixture(scope="module")
def o():
    oracle.build()
    return oracle._load()


@pytest.mark.parametrize("pin", variant_pins.ALL_VARIANT_PINS, ids=lambda f: f.__name__)
def test_variant_pin(o, pin):
    pin(o)
