"""Pins of the oracle's level-set reinitialisation (Sec. 2.2) against closed forms: the blending
weight's stated properties, a plane front (already a signed distance: unchanged, one front point per
column), and a circle whose S is not a distance (far values become the signed distance to the circle,
values next to the front are kept), and a tilted straight front on a grid with dx != dy (geometric bounds
that an exchange of x and y, or of dx and dy, breaks)."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_08549_gb300 import workloads as wl


def test_blend_weight_properties():
    delta = 0.01
    H = lambda d: oracle.reinit_blend(d, delta)
    assert H(0.0) == 1.0
    assert abs(H(3 * delta) - 1.0 / (1.0 + math.tanh(9.0))) < 1e-15  # d = d0: about one half
    assert H(2 * delta) > 0.997  # the closest cells around the front keep their values
    assert H(10 * delta) < 1e-9
    ds = np.linspace(0, 10 * delta, 101)
    assert all(H(a) >= H(b) for a, b in zip(ds[:-1], ds[1:]))


def _ls(n, phi):
    p = wl.Problem(name="ls", nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, nfields=5,
                   bc=(wl.TRANSMISSIVE,) * 4)
    return p.with_(U0=wl.conserved(1.4, np.ones((n, n)), 0.0, 0.0, 1.0, phi))


def test_plane_front_is_unchanged():
    n = 48
    X, Y = np.meshgrid(wl.centres(n, 0, 1), wl.centres(n, 0, 1))
    p = _ls(n, 0.437 - Y)
    U, npts = oracle.reinit(p, p.U0)
    assert npts == n
    np.testing.assert_allclose(U[4], p.U0[4], rtol=0, atol=1e-14)
    assert np.array_equal(U[:4], p.U0[:4])


def test_circle_far_field_becomes_signed_distance():
    n, r0 = 96, 0.27
    X, Y = np.meshgrid(wl.centres(n, 0, 1), wl.centres(n, 0, 1))
    r = np.hypot(X - 0.5, Y - 0.5)
    p = _ls(n, 4.0 * (r0 - r))
    U, npts = oracle.reinit(p, p.U0)
    assert npts > 0
    delta = 1.0 / n
    sd = r0 - r
    far = np.abs(sd) > 8 * delta
    near = np.abs(sd) < 1.5 * delta
    # far: the distance to the interpolated front points (chords of the circle): O(delta^2 / r0) off
    assert np.max(np.abs(U[4][far] - sd[far])) < 0.05 * delta
    # near: weight H ~ 1 keeps the old values
    assert np.max(np.abs(U[4][near] - p.U0[4][near])) < 0.01 * np.max(np.abs(p.U0[4][near]))
    assert np.all(np.sign(U[4]) == np.sign(p.U0[4]))


def test_tilted_front_on_unequal_spacing():
    """A straight front 0.8 x + 0.6 y = c on a grid with dx != dy, with S = 2.5 x (signed distance), so not a
    distance itself. Linear interpolation of linear data puts every front point exactly on the line, so:
    (1) |S_new| >= the distance to the line everywhere (no front point is nearer than the line);
    (2) where the foot of the perpendicular lies well inside the domain, the nearest front point is at most
        half a gap g along the line away, so |S_new - sd| <= (g/2)^2 / (2 |sd|) + H |S_old - sd|, with g the
        smaller of the spacings of the line's crossings with the rows (dy / 0.8) and columns (dx / 0.6) of
        cell centres;
    (3) the number of front points is the number of those crossings that fall between the first and last
        centres of their row or column."""
    nx, ny, c = 72, 40, 0.7131
    p = wl.Problem(name="ls", nx=nx, ny=ny, x0=0.0, x1=1.2, y0=0.0, y1=0.8, gamma=1.4, nfields=5,
                   bc=(wl.TRANSMISSIVE,) * 4)
    xc, yc = wl.centres(nx, 0.0, 1.2), wl.centres(ny, 0.0, 0.8)
    X, Y = np.meshgrid(xc, yc)
    sd = c - 0.8 * X - 0.6 * Y
    p = p.with_(U0=wl.conserved(1.4, np.ones((ny, nx)), 0.0, 0.0, 1.0, 2.5 * sd))
    U, npts = oracle.reinit(p, p.U0)
    dx, dy = 1.2 / nx, 0.8 / ny
    delta = min(dx, dy)

    xs_row = (c - 0.6 * yc) / 0.8   # crossing of the line with the row y = y_j
    ys_col = (c - 0.8 * xc) / 0.6   # crossing with the column x = x_i
    expected = int(np.sum((xs_row > xc[0]) & (xs_row < xc[-1])) + np.sum((ys_col > yc[0]) & (ys_col < yc[-1])))
    assert npts == expected

    phi = U[4]
    assert np.all(np.sign(phi) == np.sign(sd))
    assert np.all(np.abs(phi) >= np.abs(sd) - 1e-13)

    g = min(dy / 0.8, dx / 0.6)
    fx, fy = X + 0.8 * sd, Y + 0.6 * sd   # foot of the perpendicular on the line
    inside = (fx > xc[0] + 2 * g) & (fx < xc[-1] - 2 * g) & (fy > yc[0] + 2 * g) & (fy < yc[-1] - 2 * g)
    far = inside & (np.abs(sd) > 4 * delta)
    assert far.sum() > nx * ny // 4
    H = np.vectorize(lambda d: oracle.reinit_blend(d, delta))(np.abs(sd[far]))
    bound = (g / 2) ** 2 / (2 * np.abs(sd[far])) + H * 1.5 * np.abs(sd[far]) + 1e-13
    assert np.all(np.abs(phi[far] - sd[far]) <= bound)
    # next to the front the weight is ~1 and the old values stay
    near = np.abs(sd) < 0.5 * delta
    assert np.max(np.abs(phi[near] - 2.5 * sd[near])) < 1e-3 * delta


def _grid(nx, ny, x1, y1, phi):
    p = wl.Problem(name="ls", nx=nx, ny=ny, x0=0.0, x1=x1, y0=0.0, y1=y1, gamma=1.4, nfields=5,
                   bc=(wl.TRANSMISSIVE,) * 4)
    return p.with_(U0=wl.conserved(1.4, np.ones((ny, nx)), 0.0, 0.0, 1.0, phi))


def test_no_front_leaves_everything_unchanged():
    rng = np.random.default_rng(wl.DEFAULT_SEED)
    fuel = -rng.random((16, 24))
    fuel[3, 5] = 0.0                                  # S = 0 counts as fuel: still no sign change
    for phi in (0.1 + rng.random((16, 24)), fuel):   # all ash; all fuel
        p = _grid(24, 16, 1.0, 1.0, phi)
        U, npts = oracle.reinit(p, p.U0)
        assert npts == 0
        assert np.array_equal(U, p.U0)


def test_single_fuel_cell_worked_by_hand():
    """S = 1 everywhere but S = -3 in the corner cell (0, 0) of a 6 x 6 grid with dx = 0.2, dy = 0.1. The two
    sign-changing pairs put front points a quarter of the way back from the neighbour, at
    (x_0 + 0.75 dx, y_0) and (x_0, y_0 + 0.75 dy); every cell's distance is the nearer of the two."""
    nx = ny = 6
    dx, dy = 0.2, 0.1
    phi = np.ones((ny, nx))
    phi[0, 0] = -3.0
    p = _grid(nx, ny, nx * dx, ny * dy, phi)
    U, npts = oracle.reinit(p, p.U0)
    assert npts == 2
    pts = [(0.5 * dx + 0.75 * dx, 0.5 * dy), (0.5 * dx, 0.5 * dy + 0.75 * dy)]
    delta = dy
    for j in range(ny):
        for i in range(nx):
            x, y = (i + 0.5) * dx, (j + 0.5) * dy
            d = min(math.hypot(x - a, y - b) for a, b in pts)
            H = oracle.reinit_blend(d, delta)
            s = phi[j, i]
            want = H * s + (1.0 - H) * (d if s > 0 else -d)
            assert abs(U[4][j, i] - want) <= 1e-15 * max(1.0, abs(want)), (i, j)
    # spot values: the fuel cell is 0.75 dy from the nearer point; cell (5, 5) is far, so it holds its distance
    assert abs(U[4][0, 0] - (-(0.75 * dy) * (1 - oracle.reinit_blend(0.75 * dy, delta))
                             - 3.0 * oracle.reinit_blend(0.75 * dy, delta))) < 1e-15
    far = math.hypot(5.5 * dx - 1.25 * dx, 5.5 * dy - 0.5 * dy)
    assert abs(U[4][5, 5] - far) < 1e-12
