"""Pins of the oracle's characteristic-wise WENO5 (scheme 1): Lax-Friedrichs split fluxes projected on
the eigenvectors of the Roe-averaged flux Jacobian at each face, reconstructed per characteristic field
and projected back (the "WENO-Roe" construction of Sec. 2.1, Jiang & Shu 1996).

The eigen-system is checked against the physics it must satisfy, not against its own formulas: L R = I;
R diag(lambda) L equals the flux Jacobian at the averaged state (complex-step derivative of the Euler
flux); and Roe's property A(U~) (U_r - U_l) = F(U_r) - F(U_l). The scheme is checked for fifth order on
smooth data, agreement with the component-wise scheme to high order where the data are smooth (a linear
reconstruction commutes with the projection), free-stream preservation, conservation, symmetry, the exact
Riemann solutions of Table Test1D, and the property that motivates it: far smaller spurious oscillations
at shocks and contacts than the component-wise scheme."""
import math

import numpy as np
import pytest

import oracle
from oracle import riemann_exact as rx
from paper_1507_08549_gb300 import workloads as wl


def euler_flux(U, direction, gamma, xp=np):
    rho, mx, my, E = U
    u, v = mx / rho, my / rho
    p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v))
    if direction == 0:
        return xp.array([mx, mx * u + p, my * u, (E + p) * u])
    return xp.array([my, mx * v, my * v + p, (E + p) * v])


def rotate(direction):
    """Permutation matrix from the frame (rho, m_x, m_y, tau) to the rotated (rho, m_n, m_t, tau)."""
    P = np.eye(4)
    if direction == 1:
        P = P[[0, 2, 1, 3]]
    return P


def random_state(rng, gamma=1.4):
    rho = rng.uniform(0.2, 3.0)
    u, v = rng.normal(0, 1.5, 2)
    p = rng.uniform(0.1, 5.0)
    return np.array([rho, rho * u, rho * v, p / (gamma - 1) + 0.5 * rho * (u * u + v * v)])


def jacobian(U, direction, gamma):
    """Flux Jacobian by complex-step differentiation (exact to rounding)."""
    J = np.zeros((4, 4))
    h = 1e-30
    for k in range(4):
        Z = U.astype(complex)
        Z[k] += 1j * h
        J[:, k] = euler_flux(Z, direction, gamma).imag / h
    return J


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_roe_eigen_system(direction, seed):
    gamma = 1.4
    rng = np.random.default_rng(seed)
    a, b = random_state(rng), random_state(rng)
    R, L, lam = oracle.roe_eigen(gamma, direction, a, b)
    assert np.abs(L @ R - np.eye(4)).max() < 1e-12
    P = rotate(direction)
    A = P.T @ R @ np.diag(lam) @ L @ P  # back in the (rho, m_x, m_y, tau) frame
    # Roe's property: the averaged Jacobian maps the jump of U onto the jump of F exactly
    dF = euler_flux(b, direction, gamma) - euler_flux(a, direction, gamma)
    assert np.abs(A @ (b - a) - dF).max() <= 1e-12 * (1 + np.abs(dF).max())
    # and A is the flux Jacobian at the averaged state: rho~ = 1 with the averaged v_n, v_t, H
    un, ut = lam[1], R[2, 0]
    c = lam[3] - lam[1]
    H = R[3, 0] + un * c
    q2 = un * un + ut * ut
    Ut = np.array([1.0, un, ut, (H + 0.5 * (gamma - 1) * q2) / gamma])  # rotated frame, rho = 1
    J = jacobian(P.T @ Ut, direction, gamma)
    assert np.abs(J - A).max() <= 1e-12 * np.abs(J).max()
    assert abs(c * c - (gamma - 1) * (H - 0.5 * q2)) <= 1e-12 * c * c
    assert lam[0] < lam[1] == lam[2] < lam[3]


def test_roe_eigen_rejects_imaginary_sound_speed():
    with pytest.raises(oracle.OracleError):
        oracle.roe_eigen(1.4, 0, [1.0, 0.0, 0.0, -1.0], [1.0, 0.0, 0.0, -1.0])


def _wave_error(n, t_end, scheme):
    prob = wl.advected_wave(n).with_(scheme=scheme)
    U, t = prob.U0, 0.0
    while t < t_end - 1e-15:
        dt = min(0.4 * prob.dx ** (5.0 / 3.0) / 3.0 * 32 ** (2.0 / 3.0), t_end - t)
        U = oracle.step_frozen(prob, U, [dt], [[3.0, 3.0]] * 3)
        t += dt
    X, Y = np.meshgrid(wl.centres(n, 0, 1), wl.centres(n, 0, 1))
    return np.mean(np.abs(U[0] - (1.0 + 0.2 * np.sin(2 * np.pi * (X + Y - 2 * t)))))


def test_fifth_order_on_advected_wave():
    errs = [_wave_error(n, 0.05, 1) for n in (32, 64)]
    assert math.log2(errs[0] / errs[1]) > 4.7, errs


def _smooth_state(n, gamma=1.4):
    X, Y = np.meshgrid(wl.centres(n, 0, 1), wl.centres(n, 0, 1))
    two_pi = 2 * np.pi
    rho = 1.0 + 0.3 * np.sin(two_pi * X) * np.cos(two_pi * Y)
    u = 0.5 + 0.2 * np.cos(two_pi * (X + 2 * Y))
    v = -0.3 + 0.25 * np.sin(two_pi * (2 * X - Y))
    p = 1.0 + 0.2 * np.cos(two_pi * (X - Y))
    return wl.conserved(gamma, rho, u, v, p)


def test_agrees_with_componentwise_on_smooth_data_to_high_order():
    # where the data are smooth the WENO weights are near the linear ones, and a linear reconstruction
    # commutes with the projection: the two schemes' operators differ by a high-order amount only (in L1;
    # near the critical points of each scheme's variables the JS weights leave the linear ones at O(1))
    diffs = []
    for n in (64, 128):
        prob = wl.advected_wave(n)
        U = _smooth_state(n)
        ax, ay = oracle.alpha(prob, U)
        a = oracle.rhs(prob, U, ax, ay)
        b = oracle.rhs(prob.with_(scheme=1), U, ax, ay)
        diffs.append(np.abs(a - b).mean() / np.abs(a).mean())
    assert diffs[0] < 2e-4 and diffs[1] < diffs[0] / 16, diffs


def test_free_stream_and_conservation():
    p = wl.advected_wave(16).with_(scheme=1)
    U = np.zeros((4, 16, 16))
    U[0], U[1], U[2], U[3] = 1.3, 1.3 * 0.7, -1.3 * 0.2, 2.0 / 0.4 + 0.5 * 1.3 * (0.49 + 0.04)
    assert not oracle.rhs(p, U, 3.0, 3.0).any()
    prob = wl.advected_wave(48).with_(scheme=1)
    U0 = _smooth_state(48)
    U, _, _ = oracle.step(prob, U0, 30)
    m0, m1 = oracle.totals(prob, U0), oracle.totals(prob, U)
    for f in range(4):
        assert abs(m1[f] - m0[f]) <= 1e-13 * abs(m0[f])


def test_symmetries():
    # x <-> y transposition is exact (the y faces use the same rotated arithmetic); mirror images change
    # the order of the projection sums, so they hold to rounding
    prob = wl.explosion(40).with_(scheme=1)
    U, _, _ = oracle.step(prob, prob.U0, 20)
    assert np.array_equal(U[0], U[0].T) and np.array_equal(U[1], U[2].T) and np.array_equal(U[3], U[3].T)
    prob = wl.blast(40, 60).with_(scheme=1)
    U, _, _ = oracle.step(prob, prob.U0, 20)
    scale = np.abs(U).max(axis=(1, 2))
    assert np.abs(U[0] - U[0, :, ::-1]).max() <= 1e-13 * scale[0]
    assert np.abs(U[0] - U[0, ::-1, :]).max() <= 1e-13 * scale[0]
    assert np.abs(U[1] + U[1, :, ::-1]).max() <= 1e-13 * scale[1]
    assert np.abs(U[2] + U[2, ::-1, :]).max() <= 1e-13 * scale[2]


def _run_to(prob, t_end):
    U, t = prob.U0, 0.0
    while t < t_end - 1e-14:
        U, t, _ = oracle.step(prob, U, 1, t)
    return U, t


def _tube(test, nx, scheme):
    prob = wl.shock_tube(test, nx=nx, ny=3).with_(scheme=scheme)
    t0, x0 = wl.TORO_TESTS[test][:2]
    U, t = _run_to(prob, t0)
    x = wl.centres(nx, 0.0, 1.0)
    rho_ex, u_ex, _ = rx.sample(wl.TORO_TESTS[test][2:5], wl.TORO_TESTS[test][5:8], x, t, x0)
    assert np.all(U[0] == U[0, :1])
    rho, u = U[0, 1], U[1, 1] / U[0, 1]
    tv_excess = np.abs(np.diff(rho)).sum() - np.abs(np.diff(rho_ex)).sum()
    return np.mean(np.abs(rho - rho_ex)), tv_excess, np.abs(np.diff(u)).sum() - np.abs(np.diff(u_ex)).sum()


@pytest.mark.parametrize("test,bound", [(1, 0.006), (3, 0.3), (4, 0.1)])
def test_shock_tubes_converge(test, bound):
    e100, _, _ = _tube(test, 100, 1)
    e200, _, _ = _tube(test, 200, 1)
    assert e200 < bound and e200 <= 0.75 * e100


@pytest.mark.parametrize("test,factor,factor_u", [(1, 0.1, 0.1), (3, 0.1, 0.3)])
def test_far_fewer_oscillations_than_componentwise(test, factor, factor_u):
    # total variation of rho and u above the exact solution's: spurious oscillations behind the shock and
    # at the contact, which the characteristic projection suppresses (Jiang & Shu 1996, Sec. 5)
    _, tv_c, tvu_c = _tube(test, 200, 0)
    _, tv_k, tvu_k = _tube(test, 200, 1)
    assert tv_k < factor * tv_c, (tv_k, tv_c)
    assert tvu_k < factor_u * tvu_c, (tvu_k, tvu_c)


def test_adjoint_is_for_the_componentwise_scheme_only():
    prob = wl.advected_wave(16).with_(scheme=1)
    with pytest.raises(oracle.OracleError):
        oracle.adjoint_step(prob, prob.U0, np.ones_like(prob.U0), 1e-3, np.full(6, 3.0))
