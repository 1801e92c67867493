"""Pins of the oracle's level-set reinitialisation (Sec. 2.2) against closed forms: the blending
weight's stated properties, a plane front (already a signed distance: unchanged, one front point per
column), and a circle whose S is not a distance (far values become the signed distance to the circle,
values next to the front are kept)."""
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
