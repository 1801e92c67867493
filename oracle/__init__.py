"""Plain FP64 CPU oracle of the WENO5 / global Lax-Friedrichs / SSP-RK3 update of the 2D Euler
equations with a level-set scalar (Leung, Chu & Lin 2015, Sec. 2.1 Eq. euler2D, Sec. 2.2).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline leg may
use this package; the CUDA library and its Python binding never import it.

The arithmetic lives in ``hydro_oracle.c`` (plain C, FP64, compiled with ``-ffp-contract=off`` so the
x86 and Arm hosts round identically); this module compiles it with gcc on first use and wraps it with
ctypes. ``riemann_exact`` holds the exact Riemann solver used to pin the oracle.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhydro_oracle.so")
_SOURCES = ["hydro_oracle.c", "hydro_oracle.h", "hydro_oracle_adjoint.inc", "hydro_oracle_reinit.inc", "hydro_oracle_poisson.inc", "hydro_oracle_char.inc"]
_lock = threading.Lock()
_lib = None

PERIODIC, TRANSMISSIVE, REFLECT, AXIS = 0, 1, 2, 3
OK, EINVAL, ENONPHYSICAL = 0, -1, -3


class OracleError(RuntimeError):
    pass


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("geometry", ctypes.c_int), ("gravity", ctypes.c_double),
        ("bc", ctypes.c_int * 4), ("nfields", ctypes.c_int),
        ("flame_speed", ctypes.c_double), ("scheme", ctypes.c_int), ("rk_stages", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FP contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    src_mtime = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SOURCES)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= src_mtime:
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, os.path.join(_HERE, "hydro_oracle.c"), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        cp = ctypes.POINTER(_Config)
        lib.orc_validate.argtypes = [cp]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        lib.orc_weno5.argtypes = [ctypes.c_double] * 5
        lib.orc_weno5.restype = ctypes.c_double
        lib.orc_weno5_weights.argtypes = [ctypes.c_double] * 5 + [dp]
        lib.orc_weno5_grad.argtypes = [ctypes.c_double] * 5 + [dp]
        lib.orc_alpha.argtypes = [cp, dp, dp, dp]
        lib.orc_max_speed.argtypes = [cp, dp, dp]
        lib.orc_dt.argtypes = [cp, dp, dp]
        lib.orc_rhs.argtypes = [cp, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_step.argtypes = [cp, dp, ctypes.c_int, dp, dp, dp, dp]
        lib.orc_step_frozen.argtypes = [cp, dp, ctypes.c_int, dp, dp]
        lib.orc_totals.argtypes = [cp, dp, dp]
        lib.orc_adjoint_step.argtypes = [cp, dp, dp, ctypes.c_double, dp]
        lib.orc_rhs_adjoint.argtypes = [cp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_reinit.argtypes = [cp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.orc_reinit_blend.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_reinit_blend.restype = ctypes.c_double
        lib.orc_roe_eigen.argtypes = [ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, dp]
        lib.orc_poisson.argtypes = [cp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int)]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cfg(p) -> _Config:
    """Oracle config from any object with the problem attributes (nx, ny, x0, ... flame_speed)."""
    c = _Config()
    c.nx, c.ny = int(p.nx), int(p.ny)
    c.x0, c.x1, c.y0, c.y1 = float(p.x0), float(p.x1), float(p.y0), float(p.y1)
    c.gamma, c.cfl = float(p.gamma), float(p.cfl)
    c.geometry, c.gravity = int(p.geometry), float(p.gravity)
    for k in range(4):
        c.bc[k] = int(p.bc[k])
    c.nfields, c.flame_speed = int(p.nfields), float(p.flame_speed)
    c.scheme = int(getattr(p, "scheme", 0))
    c.rk_stages = int(getattr(p, "rk_stages", 3))
    return c


def _state(p, U) -> np.ndarray:
    a = np.ascontiguousarray(U, dtype=np.float64)
    if a.shape != (int(p.nfields), int(p.ny), int(p.nx)):
        raise OracleError(f"state shape {a.shape} != {(p.nfields, p.ny, p.nx)}")
    return a


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(f"{what} failed with code {rc}")


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def validate(p) -> int:
    c = _cfg(p)
    return int(_load().orc_validate(ctypes.byref(c)))


def weno5(a, b, c, d, e) -> float:
    return float(_load().orc_weno5(float(a), float(b), float(c), float(d), float(e)))


def weno5_weights(a, b, c, d, e) -> np.ndarray:
    w = np.zeros(3)
    _load().orc_weno5_weights(float(a), float(b), float(c), float(d), float(e), _ptr(w))
    return w


def weno5_grad(a, b, c, d, e) -> np.ndarray:
    g = np.zeros(5)
    _load().orc_weno5_grad(float(a), float(b), float(c), float(d), float(e), _ptr(g))
    return g


def alpha(p, U):
    U = _state(p, U)
    ax, ay = ctypes.c_double(), ctypes.c_double()
    _check(_load().orc_alpha(ctypes.byref(_cfg(p)), _ptr(U), ctypes.byref(ax), ctypes.byref(ay)), "alpha")
    return ax.value, ay.value


def max_speed(p, U) -> float:
    U = _state(p, U)
    s = ctypes.c_double()
    _check(_load().orc_max_speed(ctypes.byref(_cfg(p)), _ptr(U), ctypes.byref(s)), "max_speed")
    return s.value


def dt(p, U) -> float:
    U = _state(p, U)
    s = ctypes.c_double()
    _check(_load().orc_dt(ctypes.byref(_cfg(p)), _ptr(U), ctypes.byref(s)), "dt")
    return s.value


def rhs(p, U, ax: float, ay: float) -> np.ndarray:
    U = _state(p, U)
    L = np.zeros_like(U)
    _check(_load().orc_rhs(ctypes.byref(_cfg(p)), _ptr(U), float(ax), float(ay), _ptr(L)), "rhs")
    return L


def step(p, U, nsteps: int, t: float = 0.0, log: bool = False):
    """Advance ``nsteps`` steps (SSP-RK3, or the five-stage scheme for ``rk_stages`` = 5). Returns
    (U, t, dt_last) or, with ``log``, also the per-step dt log and the per-stage (alpha_x, alpha_y) log of
    shape (nsteps, stages, 2)."""
    U = _state(p, U).copy()
    ns = _stages(p)
    tt, dl = ctypes.c_double(t), ctypes.c_double(0.0)
    dtl = np.zeros(max(nsteps, 1))
    al = np.zeros(max(2 * ns * nsteps, 1))
    rc = _load().orc_step(ctypes.byref(_cfg(p)), _ptr(U), int(nsteps), ctypes.byref(tt), ctypes.byref(dl),
                          _ptr(dtl), _ptr(al))
    _check(rc, "step")
    if log:
        return U, tt.value, dl.value, dtl[:nsteps].copy(), al[: 2 * ns * nsteps].reshape(nsteps, ns, 2).copy()
    return U, tt.value, dl.value


def _stages(p) -> int:
    return 5 if int(getattr(p, "rk_stages", 3)) == 5 else 3


def step_frozen(p, U, dt_log, alpha_log) -> np.ndarray:
    """The same map as ``step`` with dt and the stage alphas frozen at logged values."""
    U = _state(p, U).copy()
    dtl = np.ascontiguousarray(dt_log, dtype=np.float64).ravel()
    al = np.ascontiguousarray(alpha_log, dtype=np.float64).ravel()
    if al.size != 2 * _stages(p) * dtl.size:
        raise OracleError(f"alpha log must hold {2 * _stages(p)} values per step")
    _check(_load().orc_step_frozen(ctypes.byref(_cfg(p)), _ptr(U), int(dtl.size), _ptr(dtl), _ptr(al)),
           "step_frozen")
    return U


def totals(p, U) -> np.ndarray:
    U = _state(p, U)
    out = np.zeros(5)
    _check(_load().orc_totals(ctypes.byref(_cfg(p)), _ptr(U), _ptr(out)), "totals")
    return out


def reinit(p, U):
    """Level-set reinitialisation (Sec. 2.2) of phi; returns (U, number of front points)."""
    U = _state(p, U).copy()
    npts = ctypes.c_int(0)
    _check(_load().orc_reinit(ctypes.byref(_cfg(p)), _ptr(U), ctypes.byref(npts)), "reinit")
    return U, npts.value


def roe_eigen(gamma: float, direction: int, a, b):
    """Roe average of the conserved states a, b and the eigen-system of the flux Jacobian along
    `direction` there (rotated frame rho, m_n, m_t, tau). Returns (R, L, lam): R[:, k] is right
    eigenvector k, L[k, :] left eigenvector k."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    R = np.zeros(16)
    L = np.zeros(16)
    lam = np.zeros(4)
    _check(_load().orc_roe_eigen(float(gamma), int(direction), _ptr(a), _ptr(b), _ptr(R), _ptr(L), _ptr(lam)),
           "roe_eigen")
    return R.reshape(4, 4), L.reshape(4, 4), lam


def mass(p, rho) -> float:
    """Mass of an (r,z) grid, sum over cells of rho 2 pi r dr dz (Sec. 2.1), each term rounded in that
    order and the sum correctly rounded (math.fsum)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if rho.shape != (int(p.ny), int(p.nx)):
        raise OracleError("rho shape mismatch")
    dr = (float(p.x1) - float(p.x0)) / int(p.nx)
    dz = (float(p.y1) - float(p.y0)) / int(p.ny)
    r = float(p.x0) + (np.arange(int(p.nx), dtype=np.float64) + 0.5) * dr
    terms = rho * (2.0 * np.pi) * r[None, :] * dr * dz
    return math.fsum(terms.ravel().tolist())


def poisson(p, rho, G=1.0, omega=1.9, tol=1e-8, max_iters=100000, phi0=None):
    """Self-gravity potential by red-black SOR (Sec. 2.1). Returns (phi, sweeps)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if rho.shape != (int(p.ny), int(p.nx)):
        raise OracleError("rho shape mismatch")
    phi = np.zeros_like(rho) if phi0 is None else np.ascontiguousarray(phi0, dtype=np.float64).copy()
    it = ctypes.c_int(0)
    _check(_load().orc_poisson(ctypes.byref(_cfg(p)), _ptr(rho), float(G), mass(p, rho), float(omega), float(tol),
                               int(max_iters), _ptr(phi), ctypes.byref(it)), "poisson")
    return phi, it.value


def reinit_blend(d: float, delta: float) -> float:
    return float(_load().orc_reinit_blend(float(d), float(delta)))


def rhs_adjoint(p, U, ax: float, ay: float, mu) -> np.ndarray:
    U = _state(p, U)
    mu = _state(p, mu)
    out = np.zeros_like(U)
    _check(_load().orc_rhs_adjoint(ctypes.byref(_cfg(p)), _ptr(U), float(ax), float(ay), _ptr(mu), _ptr(out)),
           "rhs_adjoint")
    return out


def adjoint_step(p, Un, lam, dt_: float, alpha6) -> np.ndarray:
    """Given dJ/dU^{n+1}, return dJ/dU^n of one SSP-RK3 step with frozen dt and stage alphas."""
    Un = _state(p, Un)
    lam = _state(p, lam).copy()
    a = np.ascontiguousarray(alpha6, dtype=np.float64).ravel()
    if a.size != 6:
        raise OracleError("alpha must hold 6 values")
    _check(_load().orc_adjoint_step(ctypes.byref(_cfg(p)), _ptr(Un), _ptr(lam), float(dt_), _ptr(a)),
           "adjoint_step")
    return lam


def adjoint_run(p, U0, nsteps: int, lam_final, checkpoint_every: int = 0):
    """Reverse sweep of ``nsteps`` steps from U0 with dt / alpha frozen at the forward run's values.
    Plain two-level scheme: the forward run keeps every state (or every ``checkpoint_every``-th and
    recomputes in between). Returns (dJ/dU0, U_final, dt_log, alpha_log)."""
    U0 = _state(p, U0).copy()
    states = [U0]
    U, _, _, dtl, al = step(p, U0, nsteps, log=True)
    # replay the frozen forward map once, keeping every state (plain; memory is small at test sizes)
    cur = U0
    for s in range(nsteps - 1):
        cur = step_frozen(p, cur, dtl[s:s + 1], al[s:s + 1])
        states.append(cur)
    lam = _state(p, lam_final).copy()
    for s in range(nsteps - 1, -1, -1):
        lam = adjoint_step(p, states[s], lam, dtl[s], al[s])
    return lam, U, dtl, al
