"""GPU characteristic-wise WENO5 (Roe-averaged eigenvectors, scheme 1) against the oracle, through the C ABI.

FP64 performs the plain definition's operations in its order (products by the eigenvectors' 0 and 1
entries included), so FP64 states are compared bit for bit; FP32 by the relative L1 bars of the
component-wise scheme (1e-5 smooth, 1e-4 with shocks)."""
import numpy as np
import pytest

import oracle
from paper_1507_08549_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

F32_SMOOTH = 1e-5
F32_SHOCK = 1e-4


def _hydro():
    from paper_1507_08549_gb300 import hydro
    return hydro


def rel_l1(a, b, gamma=1.4):
    rho = b[0]
    u, v = b[1] / rho, b[2] / rho
    p = (gamma - 1.0) * (b[3] - 0.5 * rho * (u * u + v * v))
    mscale = np.sum(rho * np.sqrt(gamma * np.maximum(p, 0.0) / rho))
    errs = []
    for f in range(b.shape[0]):
        den = np.abs(b[f]).sum()
        if f in (1, 2):
            den = max(den, mscale)
        errs.append(np.abs(a[f] - b[f]).sum() / max(den, 1e-300))
    return max(errs)


def run_gpu(prob, nsteps, dtype, variant=None):
    h = _hydro().Hydro(prob, dtype=dtype)
    if variant is not None:
        h.set_tile_variant(variant)
    U = h.state(prob.U0)
    t, dtl = h.step(U, nsteps)
    out = U.double().cpu().numpy()
    h.close()
    return out, t


def _smooth(n):
    X, Y = np.meshgrid(wl.centres(n, 0, 1), wl.centres(n, 0, 1))
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    u = 0.5 + 0.2 * np.cos(2 * np.pi * (X + 2 * Y))
    v = -0.3 + 0.25 * np.sin(2 * np.pi * (2 * X - Y))
    p = 1.0 + 0.2 * np.cos(2 * np.pi * (X - Y))
    return wl.advected_wave(n).with_(scheme=1, U0=wl.conserved(1.4, rho, u, v, p))


def _ragged():
    x, y = wl.centres(131, 0, 1.5), wl.centres(77, 0, 1.5 * 77 / 131)
    X, Y = np.meshgrid(x, y)
    inside = (X - 0.3) ** 2 + (Y - 0.5) ** 2 < 0.09
    U0 = wl.conserved(1.4, np.where(inside, 1.0, 0.125), 0.1, -0.05, np.where(inside, 1.0, 0.1),
                      0.3 - np.sqrt((X - 0.3) ** 2 + (Y - 0.5) ** 2))
    return wl.explosion(131).with_(nx=131, ny=77, nfields=5, flame_speed=0.05, gravity=-0.5, y1=1.5 * 77 / 131,
                                   bc=(wl.REFLECT, wl.TRANSMISSIVE, wl.PERIODIC, wl.PERIODIC), U0=U0, scheme=1)


CASES = {
    "smooth_periodic": (lambda: _smooth(64), 20, F32_SMOOTH),
    "ragged_all_boundaries_phi_gravity": (_ragged, 12, F32_SHOCK),
    "rz_rayleigh_taylor": (lambda: wl.rayleigh_taylor(128, 256, nsteps=20).with_(scheme=1), 20, F32_SHOCK),
    "shock_tube_test3": (lambda: wl.shock_tube(3, nx=400, ny=3).with_(scheme=1), 60, F32_SHOCK),
}


@pytest.mark.parametrize("case", list(CASES))
def test_characteristic_matches_oracle(case, record_property):
    make, nsteps, tol32 = CASES[case]
    prob = make()
    ref, t_ref, _ = oracle.step(prob, prob.U0, nsteps)
    got, t = run_gpu(prob, nsteps, "f64")
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    assert t == t_ref
    got32, _ = run_gpu(prob, nsteps, "f32")
    err = rel_l1(got32, ref, prob.gamma)
    record_property("err:fp32_char_rel_l1", err)
    assert err <= tol32


def test_characteristic_rhs_bitwise_and_differs_from_componentwise():
    prob = _ragged()
    ax, ay = oracle.alpha(prob, prob.U0)
    ref = oracle.rhs(prob, prob.U0, ax, ay)
    h = _hydro().Hydro(prob, dtype="f64")
    L = h.rhs(h.state(prob.U0), ax, ay).cpu().numpy()
    h.close()
    assert np.array_equal(L, ref)
    comp = oracle.rhs(prob.with_(scheme=0), prob.U0, ax, ay)
    # the two schemes really differ on the hydro fields here (the level set's right-hand side is shared)
    assert np.abs(comp[:4] - ref[:4]).max() > 1e-4 * np.abs(ref[:4]).max()
    assert np.array_equal(comp[4], ref[4])


def test_characteristic_tile_variants_agree():
    prob = _ragged()
    outs = []
    for v in (0, 1, 2):
        outs.append(run_gpu(prob, 6, "f32", variant=v)[0])
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_characteristic_full_size_windows(record_property):
    """8192^2 blobs + blast, FP32, one step with the characteristic scheme: the state on sampled windows
    against the oracle stepping each window (9-cell margin) at the GPU's logged alphas and dt."""
    hydro = _hydro()
    prob = wl.blobs_blast(8192).with_(scheme=1)
    h = hydro.Hydro(prob, dtype="f32")
    h.record(2)
    U = h.state(prob.U0)
    h.step(U, 1)
    dtl, al = h.get_log()
    got = U.cpu().numpy()
    h.close()
    ax, ay = oracle.alpha(prob, prob.U0)
    assert abs(al[0, 0, 0] - ax) <= 1e-6 * ax and abs(al[0, 0, 1] - ay) <= 1e-6 * ay
    rng = np.random.default_rng(9)
    m, w = 9, 96
    for (j0, i0) in [(4096 - w // 2, 4096 - w // 2)] + [tuple(rng.integers(m, 8192 - w - m, 2)) for _ in range(2)]:
        sub = prob.U0[:, j0 - m:j0 + w + m, i0 - m:i0 + w + m]
        win = prob.with_(nx=w + 2 * m, ny=w + 2 * m, bc=(wl.TRANSMISSIVE,) * 4, x1=prob.x0 + (w + 2 * m) * prob.dx,
                         y1=prob.y0 + (w + 2 * m) * prob.dy)
        a6 = np.array([[ax, ay], al[0, 1], al[0, 2]])
        ref = oracle.step_frozen(win, sub, [float(dtl[0])], a6.reshape(1, 3, 2))
        err = rel_l1(got[:, j0:j0 + w, i0:i0 + w], ref[:, m:-m, m:-m])
        record_property(f"err:fp32_char_rel_l1_window_{j0}_{i0}", err)
        assert err <= F32_SHOCK


def test_characteristic_rejected_by_adjoint_and_batch():
    hydro = _hydro()
    prob = _smooth(32)
    h = hydro.Hydro(prob, dtype="f64")
    try:
        U = h.state(prob.U0)
        with pytest.raises(hydro.HydroError) as e:
            h.adjoint_step(U, U.clone(), 1e-3, np.full(6, 3.0))
        assert e.value.code == hydro.EINVAL
        with pytest.raises(hydro.HydroError) as e:
            h.forward_checkpointed(U, 4, 2)
        assert e.value.code == hydro.EINVAL
        with pytest.raises(hydro.HydroError) as e:
            hydro.hydro_batch_step([h], [U], 1)
        assert e.value.code == hydro.EINVAL
    finally:
        h.close()
