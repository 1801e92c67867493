"""GPU self-gravity Poisson solve (Sec. 2.1) and exact summation against the oracle, through the C ABI.

Every SOR operation is rounded once in the oracle's order and red-black sweeps are order-free within a
colour, so the potential after any number of sweeps is bitwise the oracle's; the stopping test takes the
same per-cell decision, so converged solves stop at the same sweep. The grid mass is a correctly rounded
sum on both sides (math.fsum in the oracle, a long accumulator on the GPU), so it is bitwise equal too."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_08549_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rz(nx, ny, z0=0.0, z1=1.0, r1=1.0, zsym=True, dtype=np.float64, rho=None, seed=3):
    p = wl.Problem(name="grav", nx=nx, ny=ny, x0=0.0, x1=r1, y0=z0, y1=z1, gamma=5.0 / 3.0, geometry=1,
                   bc=(wl.AXIS, wl.TRANSMISSIVE, wl.REFLECT if zsym else wl.TRANSMISSIVE, wl.TRANSMISSIVE))
    if rho is None:
        r = wl.centres(nx, 0.0, r1)
        z = wl.centres(ny, z0, z1)
        R, Z = np.meshgrid(r, z)
        s = np.hypot(R, Z)
        rng = np.random.default_rng(seed)
        rho = np.where(s < 0.5, 1.0 - (s / 0.5) ** 2, 0.0) + 1e-3 * (1.0 + rng.random((ny, nx)))
    rho = rho.astype(dtype).astype(np.float64)
    U = np.zeros((4, ny, nx))
    U[0] = rho
    U[3] = 1.0
    return p, U, rho


def _gpu_solve(p, U, dt, **kw):
    import torch
    from paper_1507_08549_gb300 import hydro
    h = hydro.Hydro(p, dtype=dt)
    try:
        Ud = h.state(U)
        phi0 = kw.pop("phi0", None)
        phi = None if phi0 is None else torch.as_tensor(phi0, dtype=torch.float64, device=h.device).contiguous()
        phi, n, m = h.poisson(Ud, phi=phi, **kw)
        return phi.cpu().numpy(), n, m
    finally:
        h.close()


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("shape,zsym", [((37, 29), True), ((300, 261), False), ((64, 64), True)])
def test_fixed_sweeps_bitwise(dt, shape, zsym):
    nx, ny = shape
    z0 = 0.0 if zsym else -1.0
    p, U, rho = _rz(nx, ny, z0=z0, z1=1.0, zsym=zsym, dtype=np.float32 if dt == "f32" else np.float64)
    for sweeps in (1, 2, 63, 64, 65, 130):  # across the 64-sweep chunk boundaries
        ref, n_ref = oracle.poisson(p, rho, G=0.7, omega=1.85, tol=0.0, max_iters=sweeps)
        got, n, m = _gpu_solve(p, U, dt, G=0.7, omega=1.85, tol=0.0, max_iters=sweeps)
        assert n == n_ref == sweeps
        assert np.array_equal(got, ref), (sweeps, np.abs(got - ref).max())
        assert m == oracle.mass(p, rho)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_converged_solve_bitwise_same_sweeps(dt):
    p, U, rho = _rz(96, 160, z1=1.6, dtype=np.float32 if dt == "f32" else np.float64)
    omega = 2.0 / (1.0 + math.pi / 128)
    ref, n_ref = oracle.poisson(p, rho, omega=omega, tol=1e-10)
    got, n, m = _gpu_solve(p, U, dt, omega=omega, tol=1e-10)
    assert n == n_ref and 64 < n < 100000
    assert np.array_equal(got, ref)
    # max_iters just below / at the converging sweep
    for cap in (n_ref - 1, n_ref, n_ref + 1):
        ref_c, nr = oracle.poisson(p, rho, omega=omega, tol=1e-10, max_iters=cap)
        got_c, ng, _ = _gpu_solve(p, U, dt, omega=omega, tol=1e-10, max_iters=cap)
        assert ng == nr == min(cap, n_ref)
        assert np.array_equal(got_c, ref_c)


@pytest.mark.parametrize("tol", [2.0 ** -30, 3.7e-9, 1e-6])
def test_stopping_test_takes_the_oracle_decision(tol):
    # a power-of-two tolerance and two others: the per-cell decision fl(|d| / |new|) >= tol is taken with
    # exponent and mantissa screens plus exact division near tol; the sweep count must be the oracle's
    p, U, rho = _rz(50, 70, z1=1.4)
    ref, n_ref = oracle.poisson(p, rho, omega=1.9, tol=tol)
    got, n, _ = _gpu_solve(p, U, "f64", omega=1.9, tol=tol)
    assert n == n_ref
    assert np.array_equal(got, ref)


def test_warm_start_and_uniform_sphere():
    # the analytic uniform sphere, and a converged guess stopping after one sweep
    n = 64
    p, U, _ = _rz(n, n)
    r, z = np.meshgrid(wl.centres(n, 0, 1), wl.centres(n, 0, 1))
    s = np.hypot(r, z)
    rho = np.where(s < 0.5, 1.0, 0.0)
    U[0] = rho
    exact = np.where(s <= 0.5, -2 * math.pi * (0.25 - s * s / 3), -(4 / 3 * math.pi * 0.125) / s)
    phi, sweeps, m = _gpu_solve(p, U, "f64", omega=2 / (1 + math.pi / n), tol=1e-10)
    assert np.abs(phi - exact).max() / np.abs(exact).max() < 0.005
    again, n1, _ = _gpu_solve(p, U, "f64", omega=2 / (1 + math.pi / n), tol=1e-10, phi0=phi)
    ref, nr = oracle.poisson(p, rho, omega=2 / (1 + math.pi / n), tol=1e-10, phi0=phi)
    assert n1 == nr == 1 and np.array_equal(again, ref)


def test_full_size_sweeps_bitwise():
    # the 1024 x 2048 (r,z) grid of the axisymmetric workload: three sweeps from a nonzero guess
    p, U, rho = _rz(1024, 2048, z1=2.0, dtype=np.float32)
    rng = np.random.default_rng(11)
    phi0 = -1.0 - rng.random((2048, 1024))
    ref, _ = oracle.poisson(p, rho, omega=1.95, tol=0.0, max_iters=3, phi0=phi0)
    got, n, m = _gpu_solve(p, U, "f32", omega=1.95, tol=0.0, max_iters=3, phi0=phi0)
    assert n == 3 and np.array_equal(got, ref)
    assert m == oracle.mass(p, rho)


def test_exact_sum_matches_fsum():
    import torch
    from paper_1507_08549_gb300 import hydro
    p, _, _ = _rz(8, 8)
    h = hydro.Hydro(p, dtype="f64")
    rng = np.random.default_rng(5)
    cases = [
        np.array([]), np.zeros(7), np.array([1e100, 1.0, -1e100]), np.array([1.0, 2.0 ** -53]),
        np.array([1.0, 2.0 ** -53, 2.0 ** -160]), np.array([1.0 + 2.0 ** -52, 2.0 ** -53]),
        np.array([5e-324, 5e-324, -1e-323, 2.2250738585072014e-308, -2.225073858507201e-308]),
        np.array([1.7976931348623157e308, -1.7976931348623157e308, 3.0]),
        np.array([-1.0, -2.0 ** -60, 2.0 ** -1074]),
        rng.standard_normal(100003) * np.exp(rng.uniform(-300, 300, 100003)),
        rng.random(1 << 20),
        np.concatenate([rng.standard_normal(5000) * 1e30, -rng.standard_normal(5000) * 1e30, [1e-30]]),
    ]
    big = rng.standard_normal(50000) * 1e20
    cases.append(np.concatenate([big, -big, [math.pi]]))
    try:
        for x in cases:
            got = h.exact_sum(torch.as_tensor(x, dtype=torch.float64, device=h.device).contiguous())
            want = math.fsum(x.tolist())
            assert got == want and math.copysign(1, got) == math.copysign(1, want) or (got == 0 and want == 0), \
                (x[:4], got, want)
        # order independence: a permutation gives the same bits
        x = rng.standard_normal(77777) * np.exp(rng.uniform(-50, 50, 77777))
        a = h.exact_sum(torch.as_tensor(x, device=h.device))
        b = h.exact_sum(torch.as_tensor(x[rng.permutation(x.size)].copy(), device=h.device))
        assert a == b == math.fsum(x.tolist())
        with pytest.raises(hydro.HydroError) as e:
            h.exact_sum(torch.as_tensor(np.array([1.0, np.inf]), device=h.device))
        assert e.value.code == hydro.ENONPHYSICAL
    finally:
        h.close()


def test_poisson_argument_errors():
    import torch
    from paper_1507_08549_gb300 import hydro
    p, U, _ = _rz(16, 16)
    h = hydro.Hydro(p, dtype="f64")
    try:
        Ud = h.state(U)
        for kw in ({"omega": 2.0}, {"omega": 0.0}, {"max_iters": -1}):
            with pytest.raises(hydro.HydroError) as e:
                h.poisson(Ud, **kw)
            assert e.value.code == hydro.EINVAL
        Ud[0, 3, 4] = float("nan")
        with pytest.raises(hydro.HydroError) as e:
            h.poisson(Ud, max_iters=2, tol=0.0)
        assert e.value.code == hydro.ENONPHYSICAL
    finally:
        h.close()
    cart = wl.Problem(name="c", nx=16, ny=16, x0=0, x1=1, y0=0, y1=1, bc=(wl.PERIODIC,) * 4)
    h = hydro.Hydro(cart, dtype="f64")
    try:
        with pytest.raises(hydro.HydroError) as e:
            h.poisson(h.state(np.ones((4, 16, 16))))
        assert e.value.code == hydro.EINVAL
    finally:
        h.close()
