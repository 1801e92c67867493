"""Degenerate cases of the update on the GPU, through the C ABI, against the FP64 oracle: a step count of
zero (the state and the time come back unchanged), and grids smaller than one tile down to the smallest
the boundary accepts (3 cells, where every ghost layer of a periodic or reflecting face maps back into the
grid), with each boundary kind, the level set, gravity and the (r,z) axis."""
import numpy as np
import pytest

import oracle
from paper_1507_08549_gb300 import workloads as wl

from test_gpu_parity import F32_SHOCK, F64_TOL, _hydro, rel_l1, rel_linf, run_gpu

pytestmark = pytest.mark.gpu

P, T, R, A = wl.PERIODIC, wl.TRANSMISSIVE, wl.REFLECT, wl.AXIS


def _state(nx, ny, nfields, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.3 * rng.random((ny, nx))
    p = 1.0 + 0.5 * rng.random((ny, nx))
    u = 0.2 * (rng.random((ny, nx)) - 0.5)
    v = 0.2 * (rng.random((ny, nx)) - 0.5)
    phi = (np.arange(ny)[:, None] - 0.4 * ny + 0.3 * np.arange(nx)[None, :]) / ny if nfields == 5 else None
    return wl.conserved(1.4, rho, u, v, p, phi)


CASES = [
    # nx, ny, bc (x-lo, x-hi, y-lo, y-hi), geometry, nfields, gravity, flame speed
    (3, 3, (P, P, P, P), 0, 4, 0.0, 0.0),
    (4, 7, (R, R, T, T), 0, 5, -0.5, 0.05),
    (6, 5, (T, T, P, P), 0, 5, 0.0, 0.1),
    (5, 3, (A, T, R, R), 1, 4, -1.0, 0.0),
    (61, 16, (R, T, T, R), 0, 5, 0.3, 0.02),  # one column and one row past a 60 x 15 tile
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}" for c in CASES])
def test_grids_smaller_than_a_tile_match_the_oracle(case):
    nx, ny, bc, geom, nf, grav, sf = case
    prob = wl.Problem(name="tiny", nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=ny / nx, gamma=1.4, cfl=0.4,
                      geometry=geom, gravity=grav, bc=bc, nfields=nf, flame_speed=sf,
                      U0=_state(nx, ny, nf, 1000 + nx * 31 + ny))
    ref, t_ref, _ = oracle.step(prob, prob.U0, 6)
    got, t, _ = run_gpu(prob, 6, "f64")
    assert rel_linf(got, ref) <= F64_TOL
    assert np.array_equal(got, ref) and t == t_ref
    got32, _, _ = run_gpu(prob, 6, "f32")
    assert rel_l1(got32, ref) <= F32_SHOCK


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_zero_steps_return_the_state_and_time_unchanged(dtype):
    prob = wl.blobs_blast(96)
    h = _hydro().Hydro(prob, dtype=dtype)
    U = h.state(prob.U0)
    before = U.clone()
    t, _ = h.step(U, 0, 0.25)
    assert t == 0.25
    assert bool((U == before).all())
    h.close()
