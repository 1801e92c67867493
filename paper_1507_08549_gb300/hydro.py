"""ctypes binding of the C ABI in include/hydro.h (argument marshalling only: every step of the update
runs in the library's CUDA kernels). Function names match the C entry points; ``Hydro`` wraps one
context for torch tensors.

The library is built in-tree by ``paper_1507_08549_gb300.build``; loading raises ``HydroError`` if it
cannot be built or loaded -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

HYDRO_F32, HYDRO_F64 = 0, 1
SCHEME_COMPONENT, SCHEME_CHARACTERISTIC = 0, 1
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECT, BC_AXIS = 0, 1, 2, 3
OK, EINVAL, ECUDA, ENONPHYSICAL, ETIMEOUT, ESTATE, ESIZE = 0, -1, -2, -3, -4, -5, -6
_NAMES = {EINVAL: "HYDRO_EINVAL", ECUDA: "HYDRO_ECUDA", ENONPHYSICAL: "HYDRO_ENONPHYSICAL",
          ETIMEOUT: "HYDRO_ETIMEOUT", ESTATE: "HYDRO_ESTATE", ESIZE: "HYDRO_ESIZE"}


class HydroError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class hydro_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("geometry", ctypes.c_int), ("gravity_y", ctypes.c_double),
        ("bc", ctypes.c_int * 4), ("nfields", ctypes.c_int),
        ("flame_speed", ctypes.c_double), ("dtype", ctypes.c_int), ("scheme", ctypes.c_int),
        ("rk_stages", ctypes.c_int),
    ]


EXPORTS = [
    "hydro_init", "hydro_destroy", "hydro_last_error", "hydro_set_stream", "hydro_step", "hydro_step_host",
    "hydro_rhs", "conserved_totals", "hydro_last_totals", "hydro_record", "hydro_get_log", "hydro_step_frozen",
    "hydro_adjoint_step", "hydro_forward_checkpointed", "hydro_adjoint_sweep", "hydro_forward_revolve",
    "hydro_batch_step",
    "hydro_tile_variants", "hydro_set_tile_variant", "hydro_set_adjoint_tile_rows", "hydro_tile_info", "hydro_autotune", "hydro_batch_autotune",
    "hydro_profile",
    "hydro_stage_timing", "hydro_launch_count", "conserved_totals_noalloc", "hydro_reinit",
    "hydro_poisson", "hydro_exact_sum", "hydro_wait_selftest", "hydro_fma_probe",
]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load (building first if needed) the CUDA library; raises HydroError if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_needed:
            try:
                path = _build.build()
            except Exception as e:  # no silent fallback: the CUDA library is the only implementation
                if not os.path.exists(path):
                    raise HydroError(ECUDA, f"CUDA library could not be built: {e}") from e
        if not os.path.exists(path):
            raise HydroError(ECUDA, f"CUDA library missing at {path}")
        lib = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        ctxp = ctypes.c_void_p
        sig = {
            "hydro_init": ([ctypes.POINTER(hydro_config), vp, ctypes.POINTER(ctxp)], ctypes.c_int),
            "hydro_destroy": ([ctxp], None),
            "hydro_last_error": ([ctxp], ctypes.c_char_p),
            "hydro_set_stream": ([ctxp, vp], ctypes.c_int),
            "hydro_step": ([ctxp, vp, ctypes.c_int, dp, dp], ctypes.c_int),
            "hydro_step_host": ([ctxp, vp, ctypes.c_int, dp, dp], ctypes.c_int),
            "hydro_rhs": ([ctxp, vp, ctypes.c_double, ctypes.c_double, vp], ctypes.c_int),
            "conserved_totals": ([ctxp, vp, dp], ctypes.c_int),
            "hydro_last_totals": ([ctxp, dp], ctypes.c_int),
            "hydro_record": ([ctxp, ctypes.c_int], ctypes.c_int),
            "hydro_get_log": ([ctxp, ctypes.c_int, dp, dp, ip], ctypes.c_int),
            "hydro_step_frozen": ([ctxp, vp, ctypes.c_int, dp, dp], ctypes.c_int),
            "hydro_adjoint_step": ([ctxp, vp, vp, ctypes.c_double, dp], ctypes.c_int),
            "hydro_forward_checkpointed": ([ctxp, vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "hydro_adjoint_sweep": ([ctxp, vp], ctypes.c_int),
            "hydro_forward_revolve": ([ctxp, vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)],
                                      ctypes.c_int),
            "hydro_batch_step": ([ctypes.POINTER(ctxp), ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, dp],
                                 ctypes.c_int),
            "hydro_tile_variants": ([ctxp, ip, ip], ctypes.c_int),
            "hydro_set_tile_variant": ([ctxp, ctypes.c_int], ctypes.c_int),
            "hydro_set_adjoint_tile_rows": ([ctxp, ctypes.c_int], ctypes.c_int),
            "hydro_tile_info": ([ctxp, ctypes.c_int, ip, ip, ip, ip], ctypes.c_int),
            "hydro_autotune": ([ctxp, vp, ctypes.c_int, dp], ctypes.c_int),
            "hydro_batch_autotune": ([ctypes.POINTER(ctxp), ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, dp, ip],
                                     ctypes.c_int),
            "hydro_profile": ([ctxp, ctypes.c_int], ctypes.c_int),
            "hydro_stage_timing": ([ctxp, ip, dp], ctypes.c_int),
            "hydro_launch_count": ([ctxp], ctypes.c_longlong),
            "hydro_reinit": ([ctxp, vp, ip], ctypes.c_int),
            "hydro_poisson": ([ctxp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, ip, dp],
                              ctypes.c_int),
            "hydro_exact_sum": ([ctxp, vp, ctypes.c_longlong, dp], ctypes.c_int),
            "hydro_wait_selftest": ([ctxp, ctypes.c_uint], ctypes.c_int),
            "hydro_fma_probe": ([ctxp, ctypes.c_int, ctypes.c_int, dp], ctypes.c_int),
            "conserved_totals_noalloc": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp, dp],
                                         ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def make_config(p, dtype: int) -> hydro_config:
    """C config from a problem description (any object with nx, ny, x0, x1, y0, y1, gamma, cfl, geometry,
    gravity, bc, nfields, flame_speed)."""
    c = hydro_config()
    c.nx, c.ny = int(p.nx), int(p.ny)
    c.x0, c.x1, c.y0, c.y1 = float(p.x0), float(p.x1), float(p.y0), float(p.y1)
    c.gamma, c.cfl = float(p.gamma), float(p.cfl)
    c.geometry, c.gravity_y = int(p.geometry), float(p.gravity)
    for k in range(4):
        c.bc[k] = int(p.bc[k])
    c.nfields, c.flame_speed, c.dtype = int(p.nfields), float(p.flame_speed), int(dtype)
    c.scheme = int(getattr(p, "scheme", 0))
    c.rk_stages = int(getattr(p, "rk_stages", 3))
    return c


def _torch():
    import torch
    return torch


def _dtype_code(dtype) -> int:
    torch = _torch()
    if dtype in (torch.float32, np.float32, "f32", "float32", HYDRO_F32):
        return HYDRO_F32
    if dtype in (torch.float64, np.float64, "f64", "float64", HYDRO_F64):
        return HYDRO_F64
    raise ValueError(f"unsupported dtype {dtype}")


class Hydro:
    """One solver context for a problem; states are CUDA torch tensors [nfields, ny, nx]."""

    def __init__(self, problem, dtype="f32", stream=None, device=None):
        torch = _torch()
        self.lib = load()
        self.problem = problem
        self.code = _dtype_code(dtype)
        self.torch_dtype = torch.float64 if self.code == HYDRO_F64 else torch.float32
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if dev.type != "cuda":
            raise HydroError(EINVAL, f"device must be a CUDA device, got {dev}")
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.cfg = make_config(problem, self.code)
            self.ctx = ctypes.c_void_p()
            rc = self.lib.hydro_init(ctypes.byref(self.cfg), ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.byref(self.ctx))
        if rc != OK:
            raise HydroError(rc, "hydro_init failed")
        self.shape = (int(problem.nfields), int(problem.ny), int(problem.nx))

    # -- helpers
    def _check(self, rc: int, what: str):
        if rc != OK:
            msg = self.lib.hydro_last_error(self.ctx)
            raise HydroError(rc, f"{what}: {msg.decode() if msg else ''}")

    def _ptr(self, U, name="U"):
        torch = _torch()
        if not isinstance(U, torch.Tensor) or not U.is_cuda:
            raise HydroError(EINVAL, f"{name} must be a CUDA tensor")
        if U.device != self.device:
            raise HydroError(EINVAL, f"{name} is on {U.device}; this context runs on {self.device}")
        if U.dtype != self.torch_dtype or tuple(U.shape) != self.shape or not U.is_contiguous():
            raise HydroError(EINVAL, f"{name} must be a contiguous {self.torch_dtype} tensor of shape {self.shape}")
        return ctypes.c_void_p(U.data_ptr())

    def state(self, U0) -> "torch.Tensor":
        torch = _torch()
        return torch.as_tensor(np.ascontiguousarray(U0), dtype=self.torch_dtype, device=self.device).contiguous()

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            self.lib.hydro_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    # -- entry points
    def step(self, U, nsteps: int, t: float = 0.0):
        tt, dl = ctypes.c_double(t), ctypes.c_double(0.0)
        self._check(self.lib.hydro_step(self.ctx, self._ptr(U), int(nsteps), ctypes.byref(tt), ctypes.byref(dl)),
                    "hydro_step")
        return tt.value, dl.value

    def step_host(self, U_host: np.ndarray, nsteps: int, t: float = 0.0):
        if U_host.dtype != (np.float64 if self.code == HYDRO_F64 else np.float32) or U_host.shape != self.shape \
                or not U_host.flags.c_contiguous:
            raise HydroError(EINVAL, "host state has the wrong dtype, shape or layout")
        tt, dl = ctypes.c_double(t), ctypes.c_double(0.0)
        self._check(self.lib.hydro_step_host(self.ctx, ctypes.c_void_p(U_host.ctypes.data), int(nsteps),
                                             ctypes.byref(tt), ctypes.byref(dl)), "hydro_step_host")
        return tt.value, dl.value

    def rhs(self, U, ax: float, ay: float):
        torch = _torch()
        L = torch.empty_like(U)
        self._check(self.lib.hydro_rhs(self.ctx, self._ptr(U), float(ax), float(ay), self._ptr(L, "L")), "hydro_rhs")
        return L

    def totals(self, U) -> np.ndarray:
        out = np.zeros(5)
        self._check(self.lib.conserved_totals(self.ctx, self._ptr(U), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "conserved_totals")
        return out

    def last_totals(self) -> np.ndarray:
        out = np.zeros(5)
        self._check(self.lib.hydro_last_totals(self.ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "hydro_last_totals")
        return out

    def record(self, max_steps: int):
        self._check(self.lib.hydro_record(self.ctx, int(max_steps)), "hydro_record")

    def get_log(self, n: int | None = None):
        cnt = ctypes.c_int(0)
        self._check(self.lib.hydro_get_log(self.ctx, 0, None, None, ctypes.byref(cnt)), "hydro_get_log")
        n = cnt.value if n is None else n
        dtl = np.zeros(max(n, 1))
        al = np.zeros(max(6 * n, 1))
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.hydro_get_log(self.ctx, int(n), dtl.ctypes.data_as(dp), al.ctypes.data_as(dp), None),
                    "hydro_get_log")
        return dtl[:n], al[: 6 * n].reshape(n, 3, 2)

    def step_frozen(self, U, dt_log, alpha_log):
        dtl = np.ascontiguousarray(dt_log, dtype=np.float64).ravel()
        al = np.ascontiguousarray(alpha_log, dtype=np.float64).ravel()
        if al.size != 6 * dtl.size:
            raise HydroError(EINVAL, "alpha log must hold 6 values per step")
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.hydro_step_frozen(self.ctx, self._ptr(U), int(dtl.size), dtl.ctypes.data_as(dp),
                                               al.ctypes.data_as(dp)), "hydro_step_frozen")

    def adjoint_step(self, U_n, lam, dt: float, alpha6):
        a = np.ascontiguousarray(alpha6, dtype=np.float64).ravel()
        self._check(self.lib.hydro_adjoint_step(self.ctx, self._ptr(U_n), self._ptr(lam, "lambda"), float(dt),
                                                a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "hydro_adjoint_step")

    def forward_checkpointed(self, U, nsteps: int, checkpoint_every: int = 0):
        self._check(self.lib.hydro_forward_checkpointed(self.ctx, self._ptr(U), int(nsteps), int(checkpoint_every)),
                    "hydro_forward_checkpointed")

    def forward_revolve(self, U, nsteps: int, snapshots: int) -> int:
        """Forward run for a binomial-schedule reverse sweep with `snapshots` state slots (hydro_forward_revolve);
        returns the forward steps the next adjoint_sweep will recompute."""
        n = ctypes.c_longlong(0)
        self._check(self.lib.hydro_forward_revolve(self.ctx, self._ptr(U), int(nsteps), int(snapshots), ctypes.byref(n)),
                    "hydro_forward_revolve")
        return n.value

    def adjoint_sweep(self, lam):
        self._check(self.lib.hydro_adjoint_sweep(self.ctx, self._ptr(lam, "lambda")), "hydro_adjoint_sweep")

    def reinit(self, U) -> int:
        """Level-set reinitialisation of phi in place (hydro_reinit); returns the front point count."""
        n = ctypes.c_int(0)
        self._check(self.lib.hydro_reinit(self.ctx, self._ptr(U), ctypes.byref(n)), "hydro_reinit")
        return n.value

    def poisson(self, U, G: float = 1.0, omega: float = 1.9, tol: float = 1e-8, max_iters: int = 100000, phi=None):
        """Self-gravity potential of rho = U[0] (hydro_poisson). ``phi`` (a CUDA float64 [ny, nx] tensor,
        updated in place) is the initial guess, zeros when None. Returns (phi, sweeps, grid mass)."""
        torch = _torch()
        shape = self.shape[1:]
        if phi is None:
            phi = torch.zeros(shape, dtype=torch.float64, device=self.device)
        if not isinstance(phi, torch.Tensor) or not phi.is_cuda or phi.dtype != torch.float64 \
                or tuple(phi.shape) != shape or not phi.is_contiguous():
            raise HydroError(EINVAL, f"phi must be a contiguous CUDA float64 tensor of shape {shape}")
        it, m = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self.lib.hydro_poisson(self.ctx, self._ptr(U), float(G), float(omega), float(tol), int(max_iters),
                                           ctypes.c_void_p(phi.data_ptr()), ctypes.byref(it), ctypes.byref(m)),
                    "hydro_poisson")
        return phi, it.value, m.value

    def exact_sum(self, x) -> float:
        """Correctly rounded sum of a CUDA float64 tensor (hydro_exact_sum)."""
        torch = _torch()
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise HydroError(EINVAL, "x must be a contiguous CUDA float64 tensor")
        out = ctypes.c_double(0.0)
        self._check(self.lib.hydro_exact_sum(self.ctx, ctypes.c_void_p(x.data_ptr()), int(x.numel()),
                                             ctypes.byref(out)), "hydro_exact_sum")
        return out.value

    def wait_selftest(self, polls: int = 1 << 16) -> int:
        """Run the bounded device wait on a barrier nothing completes (hydro_wait_selftest); returns the
        C return code (HYDRO_ETIMEOUT when the failure path works) without raising."""
        return int(self.lib.hydro_wait_selftest(self.ctx, int(polls)))

    def fma_probe(self, dtype="f32", iters: int = 4096) -> float:
        """Measured FMAs per second of this GPU in the given precision (hydro_fma_probe)."""
        out = ctypes.c_double(0.0)
        self._check(self.lib.hydro_fma_probe(self.ctx, _dtype_code(dtype), int(iters), ctypes.byref(out)),
                    "hydro_fma_probe")
        return out.value

    def tile_variants(self):
        n, cur = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.hydro_tile_variants(self.ctx, ctypes.byref(n), ctypes.byref(cur)), "hydro_tile_variants")
        return n.value, cur.value

    def set_tile_variant(self, v: int):
        self._check(self.lib.hydro_set_tile_variant(self.ctx, int(v)), "hydro_set_tile_variant")

    def set_adjoint_tile_rows(self, rows: int):
        """Line-adjoint tile rows: 16, 32 (FP32), or 0 for the default size rule (hydro_set_adjoint_tile_rows)."""
        self._check(self.lib.hydro_set_adjoint_tile_rows(self.ctx, int(rows)), "hydro_set_adjoint_tile_rows")

    def tile_info(self, v: int):
        a = [ctypes.c_int() for _ in range(4)]
        self._check(self.lib.hydro_tile_info(self.ctx, int(v), *[ctypes.byref(x) for x in a]), "hydro_tile_info")
        return dict(tile_x=a[0].value, tile_y=a[1].value, threads=a[2].value, smem=a[3].value)

    def autotune(self, U, steps: int = 3):
        n, _ = self.tile_variants()
        ms = np.zeros(n)
        self._check(self.lib.hydro_autotune(self.ctx, self._ptr(U), int(steps),
                                            ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "hydro_autotune")
        return ms

    def profile(self, enable: bool):
        self._check(self.lib.hydro_profile(self.ctx, 1 if enable else 0), "hydro_profile")

    def stage_timing(self):
        n, ms = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.hydro_stage_timing(self.ctx, ctypes.byref(n), ctypes.byref(ms)), "hydro_stage_timing")
        return n.value, ms.value

    def launch_count(self) -> int:
        return int(self.lib.hydro_launch_count(self.ctx))


def conserved_totals_noalloc(problem, U, stream=None) -> np.ndarray:
    """Totals of a CUDA tensor state through the allocation-free, context-free C entry point (for
    callers that cannot allocate device memory; see include/hydro.h)."""
    torch = _torch()
    # everything the kernel will read is checked on the host first: a smaller or narrower tensor would
    # otherwise be read past its end
    if not isinstance(U, torch.Tensor):
        raise HydroError(EINVAL, "U must be a torch tensor")
    if U.dtype not in (torch.float32, torch.float64):
        raise HydroError(EINVAL, f"U must be float32 or float64, got {U.dtype}")
    shape = (int(problem.nfields), int(problem.ny), int(problem.nx))
    if tuple(U.shape) != shape:
        raise HydroError(EINVAL, f"U has shape {tuple(U.shape)}, the problem needs {shape}")
    if not U.is_cuda or not U.is_contiguous():
        raise HydroError(EINVAL, "U must be a contiguous CUDA tensor")
    code = HYDRO_F64 if U.dtype == torch.float64 else HYDRO_F32
    lib = load()
    out = np.zeros(5)
    with torch.cuda.device(U.device):  # the scratch address is looked up in the current device's context
        s = stream if stream is not None else torch.cuda.current_stream(U.device)
        rc = lib.conserved_totals_noalloc(ctypes.c_void_p(U.data_ptr()), int(problem.nx), int(problem.ny),
                                          int(problem.nfields), code, int(problem.geometry), float(problem.x0),
                                          float(problem.x1), float(problem.y0), float(problem.y1),
                                          ctypes.c_void_p(s.cuda_stream),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != OK:
        raise HydroError(rc, "conserved_totals_noalloc")
    return out


def hydro_batch_step(members: list[Hydro], states: list, nsteps: int, t=None):
    """Advance an ensemble (one context per member) with one persistent launch per stage (C ABI
    hydro_batch_step). ``t``: optional list of member times, updated and returned."""
    n = len(members)
    if n == 0 or len(states) != n:
        raise HydroError(EINVAL, f"hydro_batch_step: {n} members and {len(states)} states")
    lib = members[0].lib
    ctxs = (ctypes.c_void_p * n)(*[m.ctx.value for m in members])
    ptrs = (ctypes.c_void_p * n)(*[m._ptr(U).value for m, U in zip(members, states)])
    tt = np.ascontiguousarray(np.zeros(n) if t is None else np.asarray(t, dtype=np.float64).ravel())
    if tt.size != n:
        raise HydroError(EINVAL, f"hydro_batch_step: {tt.size} member times for {n} members")
    rc = lib.hydro_batch_step(ctxs, ptrs, n, int(nsteps), tt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != OK:
        msg = lib.hydro_last_error(members[0].ctx)
        raise HydroError(rc, f"hydro_batch_step: {msg.decode() if msg else ''}")
    return tt


BATCH_TUNE_TRIALS = 18  # 3 tile variants x 2 grid sizes x 3 work-list layouts


def batch_trial(i: int) -> dict:
    """The plan of autotuner trial i: tile variant, CTA waves and work-list layout."""
    return {"variant": i // 6, "waves": (i // 3) % 2 + 1,
            "layout": ("runs_rows", "runs_columns", "interleaved")[i % 3]}


def hydro_batch_autotune(members: list, states: list, steps: int = 3):
    """Time every batch plan (tile variant x grid size x work-list layout) on this ensemble's work list and
    keep the fastest for later hydro_batch_step calls with these members (C ABI hydro_batch_autotune; the
    states are read, not written). Returns (ms per step of each of the 18 trials, -1 if it does not fit;
    the index kept)."""
    n = len(members)
    if n == 0 or len(states) != n:
        raise HydroError(EINVAL, f"hydro_batch_autotune: {n} members and {len(states)} states")
    lib = members[0].lib
    ctxs = (ctypes.c_void_p * n)(*[m.ctx.value for m in members])
    ptrs = (ctypes.c_void_p * n)(*[m._ptr(U).value for m, U in zip(members, states)])
    ms = np.full(BATCH_TUNE_TRIALS, -1.0)
    best = ctypes.c_int(-1)
    rc = lib.hydro_batch_autotune(ctxs, ptrs, n, int(steps), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.byref(best))
    if rc != OK:
        msg = lib.hydro_last_error(members[0].ctx)
        raise HydroError(rc, f"hydro_batch_autotune: {msg.decode() if msg else ''}")
    return ms, best.value


def _autograd():
    import torch

    class HydroRollout(torch.autograd.Function):
        """U_N = (nsteps SSP-RK3 steps)(U_0) with a discrete-adjoint backward: the forward run records dt
        and the stage alphas and keeps checkpoints -- every ``checkpoint_every`` steps (uniform two-level
        scheme, hydro_forward_checkpointed), or, with ``snapshots`` >= 0, only U_0 with a binomial
        (revolve) reverse schedule over that many state slots (hydro_forward_revolve); backward recomputes
        the states it needs and runs the adjoint stages in reverse (hydro_adjoint_sweep). dt and the
        alphas are held at their recorded values, so the gradient is that of the frozen map."""

        @staticmethod
        def forward(ctx, U0, solver, nsteps, checkpoint_every, snapshots):
            U = U0.detach().clone().contiguous()
            if snapshots is not None and snapshots >= 0:
                solver.forward_revolve(U, int(nsteps), int(snapshots))
            else:
                solver.forward_checkpointed(U, int(nsteps), int(checkpoint_every))
            ctx.solver = solver
            return U

        @staticmethod
        def backward(ctx, gU):
            lam = gU.detach().to(ctx.solver.torch_dtype).clone().contiguous()
            ctx.solver.adjoint_sweep(lam)
            return lam, None, None, None, None

    return HydroRollout


_ROLLOUT = None


def rollout(solver: Hydro, U0, nsteps: int, checkpoint_every: int = 0, snapshots: int | None = None):
    """Differentiable multi-step rollout through the discrete adjoint (see HydroRollout): uniform
    checkpoints every ``checkpoint_every`` steps, or a binomial schedule with ``snapshots`` state slots."""
    global _ROLLOUT
    if _ROLLOUT is None:
        _ROLLOUT = _autograd()
    return _ROLLOUT.apply(U0, solver, nsteps, checkpoint_every, snapshots)
