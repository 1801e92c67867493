"""Seeded synthetic initial conditions for the 2D Euler / level-set update.

This module only builds inputs: grids, boundary choices and initial primitive fields, converted to
the conserved state (rho, rho u, rho v, tau = p/(gamma-1) + rho |v|^2 / 2[, phi]). It holds none of
the update's arithmetic, so the CUDA path and the CPU oracle can both be fed from it.

Problems:
  * the paper's code tests (Sec. 5.1-5.2): Toro shock tubes (Table Test1D), Gresho vortex, Blast,
    Explosion and Kelvin-Helmholtz;
  * the five workload configurations: advected density wave (128^2, FP64), axisymmetric
    Rayleigh-Taylor with a level-set front (1024x2048), an ensemble of 64 quadrant Riemann problems
    of uneven sizes, the 256^2 Fourier-mode state used for gradients, and the 8192^2 blob + blast
    throughput state with a level set.
Random draws come from numpy's PCG64 stream for small parameter sets and from SplitMix64 of
(seed XOR cell index) for per-cell noise, so the same seed gives the same bits on every host.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

PERIODIC, TRANSMISSIVE, REFLECT, AXIS = 0, 1, 2, 3
DEFAULT_SEED = 20150730


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    gamma: float = 1.4
    cfl: float = 0.4
    geometry: int = 0          # 0 Cartesian (x, y); 1 axisymmetric (r, z), x = r
    gravity: float = 0.0       # constant acceleration along y (z)
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)  # x-lo, x-hi, y-lo, y-hi
    nfields: int = 4
    flame_speed: float = 0.0
    scheme: int = 0            # 0 component-wise WENO5, 1 characteristic-wise (Roe-averaged eigenvectors)
    rk_stages: int = 3         # 3: SSP-RK3; 5: the five-stage third-order scheme (Spiteri & Ruuth SSP(5,3))
    nsteps: int = 0            # step count of the workload definition
    seed: int = DEFAULT_SEED
    U0: np.ndarray = field(default=None, repr=False)  # float64 [nfields, ny, nx]

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014) on uint64 counters."""
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_cells(seed: int, n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n values uniform in [lo, hi) from SplitMix64(seed ^ index), 53-bit resolution."""
    idx = np.arange(n, dtype=np.uint64) ^ np.uint64(seed)
    bits = splitmix64(idx) >> np.uint64(11)
    return lo + (hi - lo) * (bits.astype(np.float64) * (1.0 / 9007199254740992.0))


def centres(n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * ((hi - lo) / n)


def symmetric_centres(n: int, half_width: float) -> np.ndarray:
    """Cell centres of [-half_width, half_width] computed so that the mirror image of every centre is
    exactly its negation (integer offsets from the middle times the spacing)."""
    return (np.arange(n, dtype=np.float64) + 0.5 - 0.5 * n) * (2.0 * half_width / n)


def conserved(gamma, rho, u, v, p, phi=None) -> np.ndarray:
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), shape)
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), shape)
    fields = [rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)]
    if phi is not None:
        fields.append(np.broadcast_to(np.asarray(phi, dtype=np.float64), shape))
    return np.ascontiguousarray(np.stack(fields))


# ------------------------------------------------------------------ the paper's code tests (Sec. 5)

# Table Test1D: (t0, x0, rho_L, v_L, p_L, rho_R, v_R, p_R)
TORO_TESTS = {
    1: (0.2, 0.3, 1.0, 0.75, 1.0, 0.125, 0.0, 0.1),
    2: (0.5, 0.5, 1.0, -2.0, 0.4, 1.0, 2.0, 0.4),
    3: (0.035, 0.4, 5.99924, 19.5975, 460.894, 5.99242, -6.19633, 46.0950),
    4: (0.012, 0.8, 1.0, -19.59745, 1000.0, 1.0, -19.59745, 0.01),
}


def shock_tube(test: int, nx: int = 2000, ny: int = 6, cfl: float = 0.5, table=None) -> Problem:
    """Toro shock tube as a strip: [0,1] in x with transmissive ends, ny periodic rows (Sec. 5.1)."""
    t0, xd, rl, ul, pl, rr, ur, pr = (table or TORO_TESTS)[test]
    x = centres(nx, 0.0, 1.0)
    left = x < xd
    rho = np.where(left, rl, rr)[None, :].repeat(ny, 0)
    u = np.where(left, ul, ur)[None, :].repeat(ny, 0)
    p = np.where(left, pl, pr)[None, :].repeat(ny, 0)
    return Problem(name=f"toro{test}", nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=ny / nx, gamma=1.4, cfl=cfl,
                   bc=(TRANSMISSIVE, TRANSMISSIVE, PERIODIC, PERIODIC), U0=conserved(1.4, rho, u, 0.0, p))


def gresho(n: int = 100, cfl: float = 0.5) -> Problem:
    """Gresho vortex on [-0.5, 0.5]^2 with free (transmissive) boundaries (Sec. 5.2)."""
    x = symmetric_centres(n, 0.5)
    X, Y = np.meshgrid(x, x)
    r = np.hypot(X, Y)
    vphi = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    with np.errstate(divide="ignore"):
        p = np.where(r < 0.2, 5.0 + 12.5 * r * r,
                     np.where(r < 0.4, 9.0 + 4.0 * np.log(np.maximum(r, 1e-300) / 0.2) + 12.5 * r * r - 20.0 * r,
                              3.0 + 4.0 * np.log(2.0)))
    rs = np.where(r > 0, r, 1.0)
    u = -vphi * Y / rs
    v = vphi * X / rs
    return Problem(name="gresho", nx=n, ny=n, x0=-0.5, x1=0.5, y0=-0.5, y1=0.5, gamma=1.4, cfl=cfl,
                   bc=(TRANSMISSIVE,) * 4, U0=conserved(1.4, np.ones_like(r), u, v, p))


def blast(nx: int = 512, ny: int = 768, cfl: float = 0.5) -> Problem:
    """Blast: [-0.5,0.5]x[-0.75,0.75], reflecting walls, p = 10 inside r < 0.1 else 1, rho = 1 (Sec. 5.2)."""
    x = symmetric_centres(nx, 0.5)
    y = symmetric_centres(ny, 0.75)
    X, Y = np.meshgrid(x, y)
    r2 = X * X + Y * Y
    p = np.where(r2 < 0.01, 10.0, 1.0)
    return Problem(name="blast", nx=nx, ny=ny, x0=-0.5, x1=0.5, y0=-0.75, y1=0.75, gamma=1.4, cfl=cfl,
                   bc=(REFLECT,) * 4, U0=conserved(1.4, np.ones_like(p), 0.0, 0.0, p))


def explosion(n: int = 512, cfl: float = 0.5, geometry: int = 0) -> Problem:
    """Explosion: [0,1.5]^2, reflecting inner and free outer faces; (rho, p) = (1, 1) inside r < 0.4,
    (0.125, 0.1) outside (Sec. 5.2). With geometry=1 the x = 0 face is the symmetry axis."""
    x = centres(n, 0.0, 1.5)
    X, Y = np.meshgrid(x, x)
    inside = X * X + Y * Y < 0.16
    rho = np.where(inside, 1.0, 0.125)
    p = np.where(inside, 1.0, 0.1)
    lo = AXIS if geometry == 1 else REFLECT
    return Problem(name="explosion", nx=n, ny=n, x0=0.0, x1=1.5, y0=0.0, y1=1.5, gamma=1.4, cfl=cfl,
                   geometry=geometry, bc=(lo, TRANSMISSIVE, REFLECT, TRANSMISSIVE),
                   U0=conserved(1.4, rho, 0.0, 0.0, p))


def kelvin_helmholtz(n: int = 256, amplitude: float = 0.01, shear: float = 0.5, cfl: float = 0.5) -> Problem:
    """Kelvin-Helmholtz on the periodic unit square: p = 1, rho = 2 in 0.25 < y < 0.75 else 1, the two
    layers streaming at +-shear along x, v_y = A (1 + cos 2 pi x)(1 + cos 2 pi y) (Sec. 5.2)."""
    x = centres(n, 0.0, 1.0)
    X, Y = np.meshgrid(x, x)
    band = (Y > 0.25) & (Y < 0.75)
    rho = np.where(band, 2.0, 1.0)
    u = np.where(band, shear, -shear)
    v = amplitude * (1.0 + np.cos(2 * np.pi * X)) * (1.0 + np.cos(2 * np.pi * Y))
    return Problem(name="kelvin_helmholtz", nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, cfl=cfl,
                   U0=conserved(1.4, rho, u, v, 1.0))


# ------------------------------------------------------------------------ workload configurations

def advected_wave(n: int = 128, ny: int | None = None, nsteps: int = 100, cfl: float = 0.4) -> Problem:
    """rho = 1 + 0.2 sin 2 pi (x + y), u = v = 1, p = 1 on the periodic unit square, gamma = 1.4.
    Exact solution: the density profile translated by (t, t)."""
    ny = n if ny is None else ny
    x = centres(n, 0.0, 1.0)
    y = centres(ny, 0.0, 1.0)
    X, Y = np.meshgrid(x, y)
    rho = 1.0 + 0.2 * np.sin(2.0 * np.pi * (X + Y))
    return Problem(name=f"advected_wave_{n}x{ny}", nx=n, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4,
                   cfl=cfl, nsteps=nsteps, U0=conserved(1.4, rho, 1.0, 1.0, 1.0))


def rayleigh_taylor(nr: int = 1024, nz: int = 2048, seed: int = DEFAULT_SEED, nsteps: int = 2000,
                    flame_speed: float = 0.05, cfl: float = 0.4) -> Problem:
    """Axisymmetric Rayleigh-Taylor: r in [0, 0.5], z in [0, 1], gamma = 5/3, g = -1 along z; heavy
    rho = 2 above light rho = 1 at z = 0.5 with hydrostatic p (2.5 at the interface); v_z noise of
    amplitude 1e-2 (SplitMix64 of seed ^ cell index) in a Gaussian band of width 0.02 about the
    interface; level set phi = 0.5 - z (ash below); symmetry axis at r = 0, outflow elsewhere."""
    gamma = 5.0 / 3.0
    r = centres(nr, 0.0, 0.5)
    z = centres(nz, 0.0, 1.0)
    R, Z = np.meshgrid(r, z)
    heavy = Z > 0.5
    rho = np.where(heavy, 2.0, 1.0)
    p = np.where(heavy, 2.5 - 2.0 * (Z - 0.5), 2.5 + (0.5 - Z))
    xi = uniform_cells(seed, nr * nz).reshape(nz, nr)
    vz = 1e-2 * xi * np.exp(-(((Z - 0.5) / 0.02) ** 2))
    phi = 0.5 - Z
    return Problem(name=f"rayleigh_taylor_{nr}x{nz}", nx=nr, ny=nz, x0=0.0, x1=0.5, y0=0.0, y1=1.0,
                   gamma=gamma, cfl=cfl, geometry=1, gravity=-1.0,
                   bc=(AXIS, TRANSMISSIVE, TRANSMISSIVE, TRANSMISSIVE), nfields=5, flame_speed=flame_speed,
                   nsteps=nsteps, seed=seed, U0=conserved(gamma, rho, 0.0, vz, p, phi))


def self_gravity_star(nr: int = 1024, nz: int = 2048, radius: float = 0.3, rho_c: float = 1.0,
                      seed: int = DEFAULT_SEED) -> Problem:
    """Density of a centrally condensed star for the self-gravity potential: r in [0, 0.5], z in [0, 1]
    (square cells on the 1024 x 2048 axisymmetric grid), z = 0 the equatorial symmetry plane (reflecting),
    the axis at r = 0; rho = rho_c (1 - (s/R)^2)^(3/2) inside s = sqrt(r^2 + z^2) < R, a floor of 1e-4 rho_c
    outside, times 1 + 1e-3 xi with xi the SplitMix64 uniform of the cell (seed ^ cell index); p = rho^(5/3)
    (only rho matters for the potential)."""
    gamma = 5.0 / 3.0
    r = centres(nr, 0.0, 0.5)
    z = centres(nz, 0.0, 1.0)
    R, Z = np.meshgrid(r, z)
    s = np.hypot(R, Z)
    core = np.clip(1.0 - (s / radius) ** 2, 0.0, None) ** 1.5
    xi = uniform_cells(seed, nr * nz).reshape(nz, nr)
    rho = rho_c * np.maximum(core, 1e-4) * (1.0 + 1e-3 * xi)
    p = rho ** gamma
    return Problem(name=f"self_gravity_star_{nr}x{nz}", nx=nr, ny=nz, x0=0.0, x1=0.5, y0=0.0, y1=1.0,
                   gamma=gamma, geometry=1, bc=(AXIS, TRANSMISSIVE, REFLECT, TRANSMISSIVE), nfields=4,
                   seed=seed, U0=conserved(gamma, rho, 0.0, 0.0, p))


ENSEMBLE_SIZES = (128, 256, 512, 1024)


def quadrant_ensemble(nmembers: int = 64, seed: int = DEFAULT_SEED, nsteps: int = 500,
                      sizes=ENSEMBLE_SIZES, cfl: float = 0.4) -> list[Problem]:
    """Independent 2D quadrant Riemann problems on [0,1]^2 with transmissive faces; nx and ny each drawn
    from ``sizes``; each quadrant's rho, p ~ U[0.1, 2] and u, v ~ U[-1, 1]; split at (0.5, 0.5)."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(nmembers):
        nx, ny = (int(s) for s in rng.choice(np.asarray(sizes), size=2))
        q_rho = rng.uniform(0.1, 2.0, 4)
        q_p = rng.uniform(0.1, 2.0, 4)
        q_u = rng.uniform(-1.0, 1.0, 4)
        q_v = rng.uniform(-1.0, 1.0, 4)
        x = centres(nx, 0.0, 1.0)
        y = centres(ny, 0.0, 1.0)
        X, Y = np.meshgrid(x, y)
        quad = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
        U = conserved(1.4, q_rho[quad], q_u[quad], q_v[quad], q_p[quad])
        out.append(Problem(name=f"quadrant_{m}_{nx}x{ny}", nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
                           gamma=1.4, cfl=cfl, bc=(TRANSMISSIVE,) * 4, nsteps=nsteps, seed=seed, U0=U))
    return out


def _fourier_sum(rng, X, Y, nmodes=8, kmax=4):
    s = np.zeros_like(X)
    for _ in range(nmodes):
        kx, ky = rng.integers(1, kmax + 1, size=2)
        a = rng.uniform(-1.0, 1.0)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        s += a * np.sin(2.0 * np.pi * (kx * X + ky * Y) + ph)
    return s / nmodes


def fourier_modes(n: int = 256, seed: int = DEFAULT_SEED, nsteps: int = 200, cfl: float = 0.4):
    """Periodic unit square: rho = 1 + 0.1 (8 seeded Fourier modes)/8, u, v = 0.1 (modes)/8 each,
    p = 1, gamma = 1.4. Returns the problem and the primitive fields (rho, u, v, p)."""
    rng = np.random.default_rng(seed)
    x = centres(n, 0.0, 1.0)
    X, Y = np.meshgrid(x, x)
    rho = 1.0 + 0.1 * _fourier_sum(rng, X, Y)
    u = 0.1 * _fourier_sum(rng, X, Y)
    v = 0.1 * _fourier_sum(rng, X, Y)
    p = np.ones_like(rho)
    prob = Problem(name=f"fourier_{n}", nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, cfl=cfl,
                   nsteps=nsteps, seed=seed, U0=conserved(1.4, rho, u, v, p))
    return prob, (rho, u, v, p)


def blobs_blast(n: int = 8192, seed: int = DEFAULT_SEED, nsteps: int = 100, nblobs: int = 16,
                amplitude: float = 0.5, width: float = 0.05, blast_radius: float = 0.05,
                blast_pressure: float = 100.0, flame_speed: float = 0.05, cfl: float = 0.4) -> Problem:
    """Periodic unit square, gamma = 1.4, 5 fields: rho and p = 1 plus ``nblobs`` Gaussian blobs
    (seeded centres, periodic distance), then p = blast_pressure inside r < blast_radius of the centre;
    level set phi = blast_radius - r (ash inside the blast). Fluid at rest."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0.0, 1.0, nblobs)
    cy = rng.uniform(0.0, 1.0, nblobs)
    x = centres(n, 0.0, 1.0)
    rho = np.ones((n, n))
    for k in range(nblobs):
        dxp = np.abs(x - cx[k])
        dxp = np.minimum(dxp, 1.0 - dxp)
        dyp = np.abs(x - cy[k])
        dyp = np.minimum(dyp, 1.0 - dyp)
        gx = np.exp(-((dxp / width) ** 2))
        gy = np.exp(-((dyp / width) ** 2))
        rho += amplitude * np.outer(gy, gx)
    p = rho.copy()
    dx0 = x - 0.5
    r = np.sqrt(dx0[None, :] ** 2 + dx0[:, None] ** 2)
    p[r < blast_radius] = blast_pressure
    phi = blast_radius - r
    return Problem(name=f"blobs_blast_{n}", nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, cfl=cfl,
                   nfields=5, flame_speed=flame_speed, nsteps=nsteps, seed=seed,
                   U0=conserved(1.4, rho, 0.0, 0.0, p, phi))
