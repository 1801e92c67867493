"""The allocation-free totals entry point (for callers that cannot allocate device memory) against the
context-based conserved_totals, called through the C ABI twice in a row, plus its size limit.

Collected last on purpose (file name), so a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_1507_08549_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problems():
    X = wl.advected_wave(96, ny=53)
    rt = wl.rayleigh_taylor(64, 128)
    return [(X, "f64"), (X, "f32"), (rt, "f64"), (rt, "f32")]


@pytest.mark.parametrize("k", range(4))
def test_noalloc_totals_match_conserved_totals_twice(k):
    import torch
    from paper_1507_08549_gb300 import hydro
    prob, dt = _problems()[k]
    h = hydro.Hydro(prob, dtype=dt)
    U = h.state(prob.U0)
    ref = h.totals(U)
    lib = hydro.load()
    code = hydro.HYDRO_F64 if dt == "f64" else hydro.HYDRO_F32
    # summation-order tolerance: 1e-14 of the sum of |U_f| dV (a total that cancels to ~0, like the level
    # set's, differs between reduction orders at that absolute level, not relative to itself)
    dv_max = prob.dx * prob.dy * (2 * np.pi * prob.x1 if prob.geometry == 1 else 1.0)
    scale = np.abs(prob.U0).sum(axis=(1, 2)) * dv_max
    scale = np.concatenate([scale, np.zeros(5 - scale.size)])
    for _ in range(2):  # the shared scratch keeps the previous call's contents: results must not depend on it
        out = np.full(5, np.nan)
        rc = lib.conserved_totals_noalloc(ctypes.c_void_p(U.data_ptr()), prob.nx, prob.ny, prob.nfields, code,
                                          prob.geometry, prob.x0, prob.x1, prob.y0, prob.y1,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert rc == hydro.OK
        assert np.all(np.abs(out - ref) <= 1e-14 * scale), (out, ref)
    h.close()


def _narrow(nx, ny, geometry, nfields, seed):
    """A narrow grid of seeded values: rows narrower than a warp, and more rows than the kernel has
    blocks (ny > 4096 takes the grid-stride row loop)."""
    rng = np.random.default_rng(seed)
    base = wl.advected_wave(16)
    bc = (wl.AXIS, wl.TRANSMISSIVE, wl.TRANSMISSIVE, wl.TRANSMISSIVE) if geometry == 1 else base.bc
    U0 = rng.uniform(0.5, 2.0, size=(nfields, ny, nx))
    U0[1:3] -= 1.25  # momenta of both signs
    U0[3] += 2.0     # energies well above the kinetic part
    return base.with_(name="narrow", nx=nx, ny=ny, x0=0.0, x1=0.25, y0=0.0, y1=2.0, geometry=geometry, bc=bc,
                      nfields=nfields, U0=U0)


@pytest.mark.parametrize("nx,ny,geometry,nfields,dt", [
    (8, 16384, 0, 4, "f32"),   # the largest allowed row count
    (8, 16384, 0, 5, "f64"),
    (5, 4100, 1, 4, "f64"),    # (r,z) weights, grid-stride rows, 27 of 32 lanes idle per row
    (5, 4100, 1, 5, "f32"),
])
def test_noalloc_totals_edge_sizes(nx, ny, geometry, nfields, dt):
    import torch
    from paper_1507_08549_gb300 import hydro
    prob = _narrow(nx, ny, geometry, nfields, seed=nx * 100003 + ny)
    h = hydro.Hydro(prob, dtype=dt)
    U = h.state(prob.U0)
    ref = h.totals(U)
    dv_max = prob.dx * prob.dy * (2 * np.pi * prob.x1 if geometry == 1 else 1.0)
    scale = np.abs(prob.U0).sum(axis=(1, 2)) * dv_max
    scale = np.concatenate([scale, np.zeros(5 - scale.size)])
    for _ in range(2):
        out = hydro.conserved_totals_noalloc(prob, U)
        assert np.all(np.abs(out - ref) <= 1e-14 * scale), (out, ref)
    h.close()


def test_noalloc_totals_reject_sizes_beyond_the_limit():
    import torch
    from paper_1507_08549_gb300 import hydro
    lib = hydro.load()
    U = torch.zeros(4 * 16385 * 3, dtype=torch.float32, device="cuda")
    out = np.zeros(5)
    rc = lib.conserved_totals_noalloc(ctypes.c_void_p(U.data_ptr()), 3, 16385, 4, hydro.HYDRO_F32, 0, 0.0, 1.0,
                                      0.0, 1.0, None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == hydro.ESIZE
    p = wl.advected_wave(16)
    Ug = torch.zeros((4, 16, 16), dtype=torch.float32, device="cuda")
    np.testing.assert_array_equal(hydro.conserved_totals_noalloc(p, Ug), np.zeros(5))
