"""Pins of the diffusion oracle: checks of what the statement fixes without
the oracle's own code, each a function of an oracle library object `o`
(anything with `diffusion_step` and `diffusion_gradient`), so that planted
mistakes in copies of the oracle can be run against them too.

* Eigenmodes.  On a line of n voxels with no-flux faces (mirrored
  neighbours), cos(pi k (i + 1/2) / n) is an eigenvector of the second
  difference with eigenvalue -4 sin^2(pi k / (2 n)) (the DCT-II basis), so one
  implicit solve along that axis divides it by 1 + e + 4 K sin^2(pi k / (2 n))
  (K = D dt / dx^2, e = lambda dt / 3) and a product of three such modes
  decays by the product of the three factors per step.
* With no decay the solves conserve the total amount (each column sum of the
  matrix is 1), up to rounding.
* A constant field only decays: by (1 + e)^-3 per step.
* A line equals numpy's dense solve of the tridiagonal matrix.
* Gradients of linear fields are exact everywhere, central differences of a
  quadratic are exact inside.
"""
import numpy as np


def mode(shape, k):
    nz, ny, nx = shape
    cx = np.cos(np.pi * k[0] * (np.arange(nx) + 0.5) / nx)
    cy = np.cos(np.pi * k[1] * (np.arange(ny) + 0.5) / ny)
    cz = np.cos(np.pi * k[2] * (np.arange(nz) + 0.5) / nz)
    return cz[:, None, None] * cy[None, :, None] * cx[None, None, :]


EIGEN_CASES = [((9, 11, 13), (3, 2, 1)), ((16, 16, 16), (5, 0, 7)), ((1, 8, 20), (19, 3, 0)), ((75, 1, 1), (0, 0, 4))]


def check_eigenmode(o, shape, k):
    D, lam, dx, dt, steps = 1.3, 0.07, 2.0, 0.9, 4
    K, e = D * dt / dx ** 2, lam * dt / 3
    f = 1.0
    for kd, nd in zip(k, shape[::-1]):
        f /= 1 + e + 4 * K * np.sin(np.pi * kd / (2 * nd)) ** 2
    rho0 = mode(shape, k)
    out = o.diffusion_step(rho0[None], [D], [lam], dx, dt, steps)[0]
    assert np.abs(out - rho0 * f ** steps).max() <= 1e-12 * np.abs(rho0).max(), (shape, k)


def pin_eigenmodes(o):
    for shape, k in EIGEN_CASES:
        check_eigenmode(o, shape, k)


def pin_mass_conservation(o):
    rng = np.random.default_rng(1)
    rho = rng.random((3, 12, 10, 14))
    out = o.diffusion_step(rho, [0.5, 2.0, 40.0], [0.0, 0.0, 0.0], 1.5, 0.3, 5)
    assert np.allclose(out.sum(axis=(1, 2, 3)), rho.sum(axis=(1, 2, 3)), rtol=1e-13, atol=0)
    assert not np.allclose(out, rho)  # it did diffuse


def pin_constant_decay(o):
    lam, dt, steps = 0.2, 0.5, 3
    out = o.diffusion_step(np.full((1, 5, 6, 7), 2.5), [3.0], [lam], 1.0, dt, steps)
    assert np.allclose(out, 2.5 * (1 + lam * dt / 3) ** (-3 * steps), rtol=1e-14, atol=0)


def check_dense_line(o, axis):
    n, D, lam, dx, dt = 23, 0.8, 0.05, 1.0, 0.7
    K, e = D * dt / dx ** 2, lam * dt / 3
    rng = np.random.default_rng(2)
    old = rng.random(n)
    T = np.diag(np.full(n, 1 + 2 * K + e)) - K * (np.eye(n, k=1) + np.eye(n, k=-1))
    T[0, 0] = T[-1, -1] = 1 + K + e
    shape = [1, 1, 1]
    shape[2 - axis] = n  # (z, y, x) array order
    out = o.diffusion_step(old.reshape(shape)[None], [D], [lam], dx, dt, 1)[0].reshape(n)
    ref = np.linalg.solve(T, old) / (1 + e) ** 2  # the two other axes are single voxels
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max(), axis


def pin_dense_lines(o):
    for axis in (0, 1, 2):
        check_dense_line(o, axis)


def pin_gradients(o):
    nz, ny, nx, dx = 6, 7, 8, 1.5
    z, y, x = np.meshgrid(np.arange(nz) * dx, np.arange(ny) * dx, np.arange(nx) * dx, indexing="ij")
    lin = 1.0 + 2.0 * x - 3.0 * y + 0.5 * z
    g = o.diffusion_gradient(lin[None], dx)[0]
    assert np.allclose(g[0], 2.0, atol=1e-12) and np.allclose(g[1], -3.0, atol=1e-12)
    assert np.allclose(g[2], 0.5, atol=1e-12)
    quad = x ** 2 - y * z
    g = o.diffusion_gradient(quad[None], dx)[0]
    assert np.allclose(g[0][:, :, 1:-1], 2 * x[:, :, 1:-1], atol=1e-12)
    assert np.allclose(g[1][:, 1:-1, :], -z[:, 1:-1, :], atol=1e-12)
    assert np.allclose(g[2][1:-1], -y[1:-1], atol=1e-12)
    assert np.allclose(g[0][:, :, 0], x[:, :, 1] + x[:, :, 0], atol=1e-12)  # one-sided at the face
    flat = o.diffusion_gradient(np.ones((1, 1, 1, 5)), 1.0)[0]
    assert np.array_equal(flat[1], np.zeros((1, 1, 5))) and np.array_equal(flat[2], np.zeros((1, 1, 5)))


ALL_DIFFUSION_PINS = [pin_eigenmodes, pin_mass_conservation, pin_constant_decay, pin_dense_lines, pin_gradients]
