"""Substrate diffusion on the GPU against the diffusion oracle: the step uses
the oracle's operations in the oracle's order in FP64 (no contraction), so
densities and gradients must be equal bit for bit, for grids whose x lines
are staged in shared memory (nx <= 191) and grids whose x lines are walked
in global memory, several substrates, changing dt, and one-voxel axes."""
import numpy as np
import pytest

import oracle
from paper_2306_11544_gb300 import mech
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    H.lib()
    oracle.build()


def field(shape, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    S, nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = rng.random(shape)
    for s in range(S):  # a smooth bump plus noise: both the large and the small scales diffuse
        out[s] += 5.0 * np.exp(-((x - 0.3 * nx) ** 2 + (y - 0.6 * ny) ** 2 + (z - 0.5 * nz) ** 2) / (4.0 + s))
    return out


@pytest.mark.parametrize("shape", [(1, 75, 75, 75), (3, 20, 31, 9), (2, 5, 4, 200), (1, 1, 1, 64), (2, 7, 1, 1),
                                   (1, 1, 1, 1)])
def test_steps_and_gradients_equal_the_oracle(shape):
    S = shape[0]
    D = np.linspace(0.5, 40.0, S)
    lam = np.linspace(0.0, 0.1, S)
    dx = 20.0
    rho0 = field(shape, 3)
    with mech.Diffusion(shape[1:], dx, D, lam) as d:
        d.write(rho0)
        assert np.array_equal(d.read(), rho0)
        d.step(0.01, 3)
        d.step(0.02, 2)  # new coefficients
        out = d.read()
        g = d.gradient()
    ref = oracle.diffusion_step(oracle.diffusion_step(rho0, D, lam, dx, 0.01, 3), D, lam, dx, 0.02, 2)
    assert np.array_equal(out, ref)
    assert np.array_equal(g, oracle.diffusion_gradient(ref, dx))


def test_large_time_steps_stay_bounded_and_conserve_mass():
    """Implicit solves: a step far above the explicit stability limit stays
    bounded; without decay the total amount is kept (to rounding)."""
    shape = (1, 30, 30, 30)
    rho0 = field(shape, 4)
    with mech.Diffusion(shape[1:], 10.0, [1000.0], [0.0]) as d:
        d.write(rho0)
        d.step(5.0, 10)  # D dt / dx^2 = 50
        out = d.read()
    assert out.min() >= rho0.min() - 1e-12 and out.max() <= rho0.max() + 1e-12
    assert abs(out.sum() - rho0.sum()) <= 1e-12 * rho0.sum()


def test_invalid_arguments_are_refused():
    with pytest.raises(mech.MechError) as e:
        mech.Diffusion((0, 5, 5), 1.0, [1.0], [0.0])
    assert e.value.code == mech.MECH_E_ARG
    with pytest.raises(mech.MechError) as e:
        mech.Diffusion((5, 5, 5), 1.0, [-1.0], [0.0])
    assert e.value.code == mech.MECH_E_ARG
    with mech.Diffusion((3, 3, 3), 1.0, [1.0], [0.0]) as d:
        bad = np.zeros((1, 3, 3, 3))
        bad[0, 1, 1, 1] = np.inf
        with pytest.raises(mech.MechError) as e:
            d.write(bad)
        assert e.value.code == mech.MECH_E_NONFINITE
        with pytest.raises(mech.MechError) as e:
            d.step(-1.0)
        assert e.value.code == mech.MECH_E_ARG
