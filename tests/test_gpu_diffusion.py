"""Substrate diffusion on the GPU against the diffusion oracle, for grids
whose x lines are staged in shared memory (nx <= 189) and grids whose x lines
are walked in global memory, several substrates, changing dt, and one-voxel
axes.

Tolerance.  The oracle eliminates each line from its first row, dividing by
each Thomas pivot; the kernels eliminate from both ends toward the middle row
(the same pivots, mirrored), multiply by the pivots' reciprocals, rounded
once, and fuse each multiply-add.  Each step of a recurrence therefore
differs by at most about two units in the last place (u = 2^-53) of its
value.  For these systems (k = D dt / dx^2 <= 0.002) every pivot is within
1 % of 1 + 2k + e and both recurrences contract (|k / m_i|, |c_i| < 0.01), so
a difference does not grow along the line: a solve differs by a few u of
max |rho|, and a step (three solves) by about 10 u.  The tests take
8 u per solve, i.e. 24 u = 2.7e-15 per step, relative to max |rho|, times the
number of steps; gradients are differences of two densities divided by dx
(or 2 dx; the kernels multiply by the reciprocal), so they differ by at
most 2 / dx times the density bound plus a rounding of the quotient (2 ulp
of max |rho| / dx, a twelfth of that bound after one step)."""
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
    tol = density_tolerance(ref, 5)
    assert np.abs(out - ref).max() <= tol, (np.abs(out - ref).max(), tol)
    gref = oracle.diffusion_gradient(ref, dx)
    assert np.abs(g - gref).max() <= 2.0 * tol / dx, (np.abs(g - gref).max(), 2.0 * tol / dx)


def density_tolerance(ref, steps):
    """24 units in the last place of max |rho| per step (see the module notes)."""
    return steps * 24 * 2.0 ** -53 * np.abs(ref).max()


def test_handles_of_different_sizes_coexist():
    """A handle with long x lines keeps working after a handle with short x
    lines was created (no process-wide launch setting depends on a handle)."""
    big_shape, small_shape = (1, 6, 5, 150), (1, 4, 3, 9)
    rho_big, rho_small = field(big_shape, 5), field(small_shape, 6)
    with mech.Diffusion(big_shape[1:], 20.0, [30.0], [0.05]) as big:
        big.write(rho_big)
        big.step(0.01, 1)
        with mech.Diffusion(small_shape[1:], 20.0, [30.0], [0.05]) as small:
            small.write(rho_small)
            small.step(0.01, 2)
            out_small = small.read()
        big.step(0.01, 2)
        out_big = big.read()
    ref_big = oracle.diffusion_step(rho_big, [30.0], [0.05], 20.0, 0.01, 3)
    ref_small = oracle.diffusion_step(rho_small, [30.0], [0.05], 20.0, 0.01, 2)
    assert np.abs(out_big - ref_big).max() <= density_tolerance(ref_big, 3)
    assert np.abs(out_small - ref_small).max() <= density_tolerance(ref_small, 2)


def test_many_substrates_get_coefficients():
    """More (substrate, axis) pairs (330,000) than threads in the coefficient
    launch (at most 32 blocks of 64 threads per SM)."""
    shape = (110000, 1, 1, 2)
    S = shape[0]
    D = np.linspace(1.0, 80.0, S)
    lam = np.linspace(0.0, 0.2, S)
    rho0 = field(shape, 7)
    with mech.Diffusion(shape[1:], 20.0, D, lam) as d:
        d.write(rho0)
        d.step(0.01, 1)
        out = d.read()
    ref = oracle.diffusion_step(rho0, D, lam, 20.0, 0.01, 1)
    assert np.abs(out - ref).max() <= density_tolerance(ref, 1)


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
