"""Pins of the oracle's self-gravity Poisson solver (Sec. 2.1): red-black SOR for
(1/r) d/dr (r dPhi/dr) + d2Phi/dz2 = 4 pi G rho on an (r,z) grid, reflecting inner boundaries (axis,
z = 0 plane) and the Roche value -G M / sqrt(r^2 + z^2) on the outer ones.

The pins do not retype the solver: they check it against the closed-form potential of a uniform
sphere, the exact mass of a uniform cylinder, the mirror symmetry that the reflecting z = 0 plane must
reproduce, and properties of the iteration itself (the fixed point does not depend on omega, a converged
guess stops after one sweep, tol <= 0 runs exactly max_iters sweeps)."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_08549_gb300.workloads import AXIS, TRANSMISSIVE, REFLECT, Problem


def rz_problem(nx, ny, z0=0.0, z1=1.0, r1=1.0, zsym=True):
    return Problem("poisson", nx, ny, 0.0, r1, z0, z1, geometry=1,
                   bc=(AXIS, TRANSMISSIVE, REFLECT if zsym else TRANSMISSIVE, TRANSMISSIVE))


def centres(p):
    r = p.x0 + (np.arange(p.nx) + 0.5) * p.dx
    z = p.y0 + (np.arange(p.ny) + 0.5) * p.dy
    return np.meshgrid(r, z)


def uniform_sphere(p, R=0.5, rho0=1.0):
    r, z = centres(p)
    s = np.hypot(r, z)
    rho = np.where(s < R, rho0, 0.0)
    M = 4.0 / 3.0 * math.pi * R ** 3 * rho0
    exact = np.where(s <= R, -2.0 * math.pi * rho0 * (R * R - s * s / 3.0), -M / s)
    return rho, exact


@pytest.mark.parametrize("n,bound", [(32, 0.015), (64, 0.005), (128, 0.0025)])
def test_uniform_sphere_potential(n, bound):
    # Phi = -2 pi G rho0 (R^2 - s^2/3) inside, -G M / s outside (G = 1); omega near the optimum
    # 2 / (1 + pi / n) of the model problem
    p = rz_problem(n, n)
    rho, exact = uniform_sphere(p)
    phi, sweeps = oracle.poisson(p, rho, G=1.0, omega=2.0 / (1.0 + math.pi / n), tol=1e-10)
    assert 0 < sweeps < 20 * n
    err = np.max(np.abs(phi - exact)) / np.max(np.abs(exact))
    assert err < bound, err


def test_uniform_sphere_on_unequal_spacing():
    # dr != dz: the radial and vertical coefficients must each take their own spacing
    p = rz_problem(48, 32, z0=0.0, z1=1.0, r1=1.0)
    rho, exact = uniform_sphere(p)
    phi, _ = oracle.poisson(p, rho, omega=1.9, tol=1e-10)
    err = np.max(np.abs(phi - exact)) / np.max(np.abs(exact))
    assert err < 0.01, err


def test_sphere_error_falls_with_resolution():
    errs = []
    for n in (16, 32, 64):
        p = rz_problem(n, n)
        rho, exact = uniform_sphere(p)
        phi, _ = oracle.poisson(p, rho, omega=2.0 / (1.0 + math.pi / n), tol=1e-11)
        errs.append(np.max(np.abs(phi - exact)) / np.max(np.abs(exact)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 1.8


def test_potential_scales_with_G_and_rho():
    # the equation and the Roche boundary are both linear in G rho: Phi(G=3, 2 rho) = 6 Phi(1, rho)
    p = rz_problem(24, 24)
    rho, _ = uniform_sphere(p)
    a, _ = oracle.poisson(p, rho, G=1.0, omega=1.8, tol=1e-13)
    b, _ = oracle.poisson(p, 2.0 * rho, G=3.0, omega=1.8, tol=1e-13)
    np.testing.assert_allclose(b, 6.0 * a, rtol=1e-9)
    # the stopping test is a relative change, so it does not see the scale either
    _, n1 = oracle.poisson(p, rho, G=1.0, omega=1.8, tol=1e-9)
    _, n2 = oracle.poisson(p, rho, G=1e6, omega=1.8, tol=1e-9)
    assert n1 == n2


def test_mass_of_uniform_cylinder_is_exact():
    # midpoint rule in r is exact for the integrand 2 pi r: a uniform cylinder of radius R and height Z
    # has mass pi R^2 Z rho exactly (up to the rounding of the terms)
    p = rz_problem(40, 30, z0=0.0, z1=1.5, r1=0.75)
    rho = np.full((30, 40), 2.5)
    assert oracle.mass(p, rho) == pytest.approx(math.pi * 0.75 ** 2 * 1.5 * 2.5, rel=1e-14)
    # a sphere's mass converges to 4/3 pi R^3
    q = rz_problem(128, 128)
    rho_s, _ = uniform_sphere(q)
    assert oracle.mass(q, rho_s) * 2 == pytest.approx(4.0 / 3.0 * math.pi * 0.125, rel=5e-3)


def test_reflecting_plane_matches_mirrored_full_domain():
    # a density symmetric about z = 0 on [0,1] x [-1,1] (Roche on every outer face) has the same
    # potential as the upper half with a reflecting z = 0 plane and the mass doubled
    half = rz_problem(24, 24, z0=0.0, z1=1.0, zsym=True)
    full = rz_problem(24, 48, z0=-1.0, z1=1.0, zsym=False)
    rng = np.random.default_rng(7)
    rho_h = np.where(np.hypot(*centres(half)) < 0.6, 1.0 + 0.5 * rng.random((24, 24)), 0.0)
    rho_f = np.concatenate([rho_h[::-1], rho_h], axis=0)
    assert oracle.mass(full, rho_f) == pytest.approx(2.0 * oracle.mass(half, rho_h), rel=1e-15)
    a, _ = oracle.poisson(half, rho_h, omega=1.8, tol=1e-13)
    b, _ = oracle.poisson(full, rho_f, omega=1.8, tol=1e-13)
    np.testing.assert_allclose(b[24:], a, rtol=1e-9)
    np.testing.assert_allclose(b[:24][::-1], a, rtol=1e-9)


def test_fixed_point_does_not_depend_on_omega():
    p = rz_problem(20, 20)
    rho, _ = uniform_sphere(p, R=0.4)
    gs, n_gs = oracle.poisson(p, rho, omega=1.0, tol=1e-13, max_iters=200000)
    sor, n_sor = oracle.poisson(p, rho, omega=1.75, tol=1e-13)
    np.testing.assert_allclose(sor, gs, rtol=1e-9)
    assert n_sor * 4 < n_gs  # over-relaxation converges several times faster


def test_iteration_control():
    p = rz_problem(16, 16)
    rho, _ = uniform_sphere(p)
    phi, n = oracle.poisson(p, rho, omega=1.7, tol=1e-14)
    # the converged field changes by less than tol in one more sweep
    again, n1 = oracle.poisson(p, rho, omega=1.7, tol=1e-14, phi0=phi)
    assert n1 == 1
    np.testing.assert_allclose(again, phi, rtol=1e-13)
    # tol <= 0: exactly max_iters sweeps, and sweeps compose
    five, n5 = oracle.poisson(p, rho, omega=1.7, tol=0.0, max_iters=5)
    assert n5 == 5
    two, _ = oracle.poisson(p, rho, omega=1.7, tol=0.0, max_iters=2)
    three, _ = oracle.poisson(p, rho, omega=1.7, tol=0.0, max_iters=3, phi0=two)
    assert np.array_equal(three, five)
    zero, n0 = oracle.poisson(p, rho, omega=1.7, tol=0.0, max_iters=0)
    assert n0 == 0 and not zero.any()


def test_rejects_cartesian_grid():
    p = Problem("cart", 8, 8, 0.0, 1.0, 0.0, 1.0, geometry=0, bc=(REFLECT,) * 4)
    with pytest.raises(oracle.OracleError):
        oracle.poisson(p, np.ones((8, 8)))
