"""The seeded synthetic inputs follow their stated recipes (the configurations' readings of the paper's
setups): checked as properties of the generated states, not by rebuilding them."""
import numpy as np
import pytest

from paper_1507_08549_gb300 import workloads as wl


def _prims(U, gamma):
    rho = U[0]
    u, v = U[1] / rho, U[2] / rho
    p = (gamma - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def test_rayleigh_taylor_recipe():
    p = wl.rayleigh_taylor(64, 128)
    assert (p.x0, p.x1, p.y0, p.y1, p.geometry, p.gravity, p.nfields) == (0.0, 0.5, 0.0, 1.0, 1, -1.0, 5)
    assert p.gamma == pytest.approx(5.0 / 3.0) and p.bc == (wl.AXIS, wl.TRANSMISSIVE, wl.TRANSMISSIVE, wl.TRANSMISSIVE)
    rho, u, v, pr = _prims(p.U0, p.gamma)
    z = wl.centres(128, 0.0, 1.0)
    heavy = z > 0.5
    assert np.all(rho[heavy] == 2.0) and np.all(rho[~heavy] == 1.0)
    np.testing.assert_allclose(u, 0.0, atol=1e-15)
    assert pr.min() >= 1.5 - 1e-12 and pr.max() <= 3.0 + 1e-12
    # hydrostatic: dp/dz = rho g on each side, continuous (2.5) at the interface
    dz = z[1] - z[0]
    np.testing.assert_allclose(np.diff(pr[:, 0])[heavy[1:] & heavy[:-1]], -2.0 * dz, rtol=1e-9)
    np.testing.assert_allclose(np.diff(pr[:, 0])[~heavy[1:] & ~heavy[:-1]], -1.0 * dz, rtol=1e-9)
    k = np.argmax(heavy)
    assert pr[k - 1, 0] - 2.5 == pytest.approx(0.5 - z[k - 1], abs=1e-12)
    assert pr[k, 0] - 2.5 == pytest.approx(-2.0 * (z[k] - 0.5), abs=1e-12)
    # v_z noise: amplitude at most 1e-2, confined to the band about the interface, not constant
    assert np.abs(v).max() <= 1e-2 and np.abs(v).max() > 5e-3
    assert np.abs(v[np.abs(z - 0.5) > 0.15]).max() < 1e-2 * np.exp(-(0.15 / 0.02) ** 2) * 1.01
    np.testing.assert_allclose(p.U0[4], (0.5 - z)[:, None] * np.ones((1, 64)), atol=1e-15)


def test_quadrant_ensemble_recipe():
    members = wl.quadrant_ensemble(64)
    assert len(members) == 64
    sizes = {(m.nx, m.ny) for m in members}
    assert all(nx in wl.ENSEMBLE_SIZES and ny in wl.ENSEMBLE_SIZES for nx, ny in sizes) and len(sizes) > 8
    for m in members[:12]:
        assert m.bc == (wl.TRANSMISSIVE,) * 4 and m.gamma == 1.4
        rho, u, v, pr = _prims(m.U0, m.gamma)
        X, Y = np.meshgrid(wl.centres(m.nx, 0, 1), wl.centres(m.ny, 0, 1))
        for qx in (False, True):
            for qy in (False, True):
                sel = ((X >= 0.5) == qx) & ((Y >= 0.5) == qy)
                for f, lo, hi in ((rho, 0.1, 2.0), (pr, 0.1, 2.0), (u, -1.0, 1.0), (v, -1.0, 1.0)):
                    vals = f[sel]
                    assert np.ptp(vals) <= 1e-12 * max(1.0, np.abs(vals).max())  # one state per quadrant
                    assert lo - 1e-12 <= vals[0] <= hi + 1e-12


def test_fourier_modes_recipe():
    p, (rho, u, v, pr) = wl.fourier_modes(64)
    # integer wavenumbers >= 1 on the periodic grid: every mode sums to zero over the cells
    assert rho.mean() == pytest.approx(1.0, abs=1e-14)
    assert abs(u.mean()) < 1e-14 and abs(v.mean()) < 1e-14
    assert 0.9 <= rho.min() and rho.max() <= 1.1 and np.abs(u).max() <= 0.1 and np.abs(v).max() <= 0.1
    assert np.all(pr == 1.0) and p.bc == (wl.PERIODIC,) * 4 and p.nsteps == 200
    assert np.ptp(rho) > 0.02  # not a constant state


def test_blobs_blast_recipe():
    p = wl.blobs_blast(256)
    rho, u, v, pr = _prims(p.U0, p.gamma)
    assert p.nfields == 5 and p.bc == (wl.PERIODIC,) * 4 and p.nsteps == 100
    assert np.all(p.U0[1] == 0) and np.all(p.U0[2] == 0)
    assert rho.min() >= 1.0 and rho.max() <= 1.0 + 16 * 0.5
    x = wl.centres(256, 0.0, 1.0)
    r = np.hypot(x[None, :] - 0.5, x[:, None] - 0.5)
    np.testing.assert_allclose(pr[r < 0.05], 100.0, rtol=1e-12)
    np.testing.assert_allclose(pr[r >= 0.05], rho[r >= 0.05], rtol=1e-12)
    np.testing.assert_allclose(p.U0[4], 0.05 - r, atol=1e-15)
