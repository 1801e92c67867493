"""Pins of the oracle's discrete adjoint (frozen alpha and dt) against central finite differences of
the oracle's own forward map and the dot-product identity <mu, J delta> = <J^T mu, delta>."""
import numpy as np
import pytest

import oracle
from paper_1507_08549_gb300 import workloads as wl


def test_weno5_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    for _ in range(20):
        v = rng.normal(size=5) * 10.0 ** rng.uniform(-2, 1)
        g = oracle.weno5_grad(*v)
        h = 1e-6 * max(1.0, np.abs(v).max())
        fd = np.array([(oracle.weno5(*(v + h * e)) - oracle.weno5(*(v - h * e))) / (2 * h) for e in np.eye(5)])
        np.testing.assert_allclose(g, fd, rtol=2e-5, atol=1e-7)


def _smooth_state(nx, ny, nf, seed, rz=False):
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(wl.centres(nx, 0, 1), wl.centres(ny, 0, 1))
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * X + 0.3) * np.cos(2 * np.pi * Y) + 0.02 * rng.random((ny, nx))
    u = 0.3 + 0.2 * np.cos(2 * np.pi * Y) + 0.01 * rng.random((ny, nx))
    v = -0.25 + 0.1 * np.sin(2 * np.pi * X)
    p = 1.0 + 0.1 * rng.random((ny, nx))
    phi = 0.3 - np.hypot(X - 0.45, Y - 0.55) + 0.1 * X
    return wl.conserved(1.4, rho, u, v, p, phi if nf == 5 else None)


def richardson(D, h=1e-6):
    """Central difference with one Richardson step: (4 D(h/2) - D(h)) / 3, error O(h^4)."""
    return (4.0 * D(h / 2) - D(h)) / 3.0


CASES = {
    "periodic": dict(),
    "rz_gravity_phi": dict(geometry=1, gravity=-0.8, nfields=5, flame_speed=0.07,
                           bc=(wl.AXIS, wl.TRANSMISSIVE, wl.REFLECT, wl.TRANSMISSIVE)),
    "walls_phi": dict(nfields=5, flame_speed=0.03, bc=(wl.REFLECT, wl.TRANSMISSIVE, wl.PERIODIC, wl.PERIODIC)),
}


def _problem(case, nx=19, ny=17):
    kw = CASES[case]
    p = wl.Problem(name=case, nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, **kw)
    return p.with_(U0=_smooth_state(nx, ny, p.nfields, 1))


@pytest.mark.parametrize("case", list(CASES))
def test_rhs_adjoint_dot_product(case):
    p = _problem(case)
    U = p.U0
    ax, ay = oracle.alpha(p, U)
    rng = np.random.default_rng(2)
    mu = rng.normal(size=U.shape)
    for trial in range(3):
        d = rng.normal(size=U.shape) * np.abs(U).mean(axis=(1, 2), keepdims=True)
        jd = richardson(lambda h: (oracle.rhs(p, U + h * d, ax, ay) - oracle.rhs(p, U - h * d, ax, ay)) / (2 * h))
        lhs = np.sum(mu * jd)
        rhs = np.sum(oracle.rhs_adjoint(p, U, ax, ay, mu) * d)
        assert abs(lhs - rhs) <= 5e-8 * max(abs(lhs), abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("case", list(CASES))
def test_step_adjoint_dot_product(case):
    p = _problem(case)
    U = p.U0
    _, _, _, dtl, al = oracle.step(p, U, 1, log=True)
    rng = np.random.default_rng(5)
    lam = rng.normal(size=U.shape)
    d = rng.normal(size=U.shape) * np.abs(U).mean(axis=(1, 2), keepdims=True)
    jd = richardson(lambda h: (oracle.step_frozen(p, U + h * d, dtl, al) - oracle.step_frozen(p, U - h * d, dtl, al))
                    / (2 * h))
    lhs = np.sum(lam * jd)
    rhs = np.sum(oracle.adjoint_step(p, U, lam, dtl[0], al[0]) * d)
    assert abs(lhs - rhs) <= 5e-8 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _kinetic(p, U):
    return np.sum(0.5 * (U[1] ** 2 + U[2] ** 2) / U[0]) * p.dx * p.dy


def _kinetic_grad(p, U):
    rho, mx, my = U[0], U[1], U[2]
    g = np.zeros_like(U)
    g[0] = -0.5 * (mx ** 2 + my ** 2) / rho ** 2 * p.dx * p.dy
    g[1] = mx / rho * p.dx * p.dy
    g[2] = my / rho * p.dx * p.dy
    return g


def test_kinetic_energy_gradient_wrt_initial_density_fd():
    """Gradient configuration at reduced size: 32^2 periodic Fourier-mode state, 20 steps; d KE(U^N) /
    d rho_0 with u, v, p held fixed, checked by central differences on 8 seeded cells."""
    p, (rho, u, v, pr) = wl.fourier_modes(32, nsteps=20)
    n = 20
    lamN = _kinetic_grad(p, oracle.step(p, p.U0, n)[0])
    lam0, UN, dtl, al = oracle.adjoint_run(p, p.U0, n, lamN)
    # chain rule to the primitive parameterisation: dU/drho = (1, u, v, |v|^2/2)
    grad_rho = lam0[0] + lam0[1] * u + lam0[2] * v + lam0[3] * 0.5 * (u * u + v * v)
    rng = np.random.default_rng(11)
    cells = rng.integers(0, 32, size=(8, 2))
    for (j, i) in cells:
        def D(h):
            rp = rho.copy(); rp[j, i] += h
            rm = rho.copy(); rm[j, i] -= h
            Jp = _kinetic(p, oracle.step_frozen(p, wl.conserved(1.4, rp, u, v, pr), dtl, al))
            Jm = _kinetic(p, oracle.step_frozen(p, wl.conserved(1.4, rm, u, v, pr), dtl, al))
            return (Jp - Jm) / (2 * h)
        fd = richardson(D, 1e-5)
        assert abs(fd - grad_rho[j, i]) <= 1e-7 * abs(fd) + 1e-13, (j, i, fd, grad_rho[j, i])
