"""Pins of the diffusion oracle (CPU only); the checks are in
``tests/diffusion_pins.py``."""
import pytest

import oracle
from tests import diffusion_pins as P


@pytest.fixture(scope="module")
def o():
    oracle.build()
    return oracle._load()


@pytest.mark.parametrize("shape,k", P.EIGEN_CASES)
def test_eigenmodes_decay_by_the_closed_form(o, shape, k):
    P.check_eigenmode(o, shape, k)


def test_mass_is_conserved_without_decay(o):
    P.pin_mass_conservation(o)


def test_constant_field_only_decays(o):
    P.pin_constant_decay(o)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_a_line_is_the_dense_tridiagonal_solve(o, axis):
    P.check_dense_line(o, axis)


def test_gradients_of_linear_and_quadratic_fields(o):
    P.pin_gradients(o)
