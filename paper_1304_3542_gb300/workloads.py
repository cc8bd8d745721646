"""Seeded synthetic inputs for the FGA hot path (velocity models, initial data, shot sets).

This module only builds problem data and the method parameters a user would
choose; it contains none of the method's arithmetic (no FBI, no rays, no
reconstruction), so both the CUDA path and the CPU oracle can take their inputs
from here. It depends on numpy and scipy only.

Problems follow the acoustic wave equation u_tt = c(x)^2 Laplace(u) with Cauchy
data u(0) = f0, u_t(0) = f1 (Theory section, Eqs. wave, f0, f1). Lengths are
nondimensional for the two unit-square problems and in km (times in s,
velocities in km/s) for the layered-model problems.

Grids are x_i = origin + i*h per axis, arrays C-contiguous with the last axis
fastest; in 2D the axes are (x, z) with z the depth.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class Shot:
    """One set of initial data with its own FGA width parameter eps."""

    eps: float
    u0: np.ndarray  # f0 on the grid, float64, shape = grid shape
    u1: np.ndarray  # f1 on the grid, float64
    q_stride: Tuple[int, ...]  # q-grid stride in grid points per axis
    box: Tuple[int, ...]  # FBI box points per axis (even)
    source: Optional[Tuple[float, ...]] = None
    freq: Optional[float] = None


@dataclasses.dataclass
class Problem:
    name: str
    dim: int
    n: Tuple[int, ...]
    h: Tuple[float, ...]
    origin: Tuple[float, ...]
    periodic: Tuple[bool, ...]
    velocity: np.ndarray  # c on the grid, float64
    shots: List[Shot]
    T: float
    dt: float
    kappa: float  # reconstruction window half-width in units of sqrt(eps)
    tau: float  # relative threshold on |psi|
    keep_n: int = 0  # >0 selects the keep_n largest |psi| per branch instead of tau
    receivers: Optional[np.ndarray] = None  # [nr][dim] points
    record_every: int = 0  # steps between recorded trace samples

    @property
    def nsteps(self) -> int:
        return int(round(self.T / self.dt))

    @property
    def npoints(self) -> int:
        return int(np.prod(self.n))

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    def grid_axes(self) -> List[np.ndarray]:
        return [self.origin[k] + self.h[k] * np.arange(self.n[k]) for k in range(self.dim)]

    def grid_points(self) -> np.ndarray:
        axes = np.meshgrid(*self.grid_axes(), indexing="ij")
        return np.stack([a.ravel() for a in axes], axis=1)


def default_stride_box(eps: float, h: Sequence[float], n: Sequence[int],
                       periodic: Sequence[bool]) -> Tuple[Tuple[int, ...], Tuple[int, ...]]:
    """q-stride s = round(0.5 sqrt(eps)/h) and box n_b = ceil(12 sqrt(eps)/h) rounded up
    to a multiple of 32 (one period on periodic axes)."""
    se = math.sqrt(eps)
    s, nb = [], []
    for k in range(len(h)):
        sk = max(1, int(round(0.5 * se / h[k])))
        if periodic[k]:
            while n[k] % sk:
                sk -= 1
            nbk = n[k]
        else:
            nbk = int(math.ceil(12.0 * se / h[k]))
            nbk = 32 * ((nbk + 31) // 32)
        s.append(sk)
        nb.append(nbk)
    return tuple(s), tuple(nb)


# ---------------------------------------------------------------------------
# Unit-square problems
# ---------------------------------------------------------------------------

def periodic_1d(N: int = 512, eps: float = 1.0 / 128, T: float = 0.25, dt: float = 1e-3,
                k0: float = 40 * math.pi, width2: float = 0.005, s: int = 16,
                kappa: float = 8.0, tau: float = 0.0, c: float = 1.0) -> Problem:
    """1D constant-speed periodic problem on [0,1): right-going Gaussian packet
    u0 = exp(-(x-0.5)^2/width2) cos(k0 x), u1 = -c u0'."""
    h = 1.0 / N
    x = h * np.arange(N)
    env = np.exp(-((x - 0.5) ** 2) / width2)
    u0 = env * np.cos(k0 * x)
    du0 = env * (-2.0 * (x - 0.5) / width2 * np.cos(k0 * x) - k0 * np.sin(k0 * x))
    u1 = -c * du0
    shot = Shot(eps=eps, u0=u0, u1=u1, q_stride=(s,), box=(N,))
    return Problem(name="periodic_1d", dim=1, n=(N,), h=(h,), origin=(0.0,), periodic=(True,),
                   velocity=np.full(N, c), shots=[shot], T=T, dt=dt, kappa=kappa, tau=tau)


def lens_2d(N: int = 256, eps: float = 1.0 / 256, T: float = 0.5, dt: float = 1e-3,
            kappa: float = 6.0, tau: float = 1e-3, s: int = 8, box: int = 192,
            k0: float = 40 * math.pi, width2: float = 0.005,
            x0: Tuple[float, float] = (0.5, 0.2),
            center: Tuple[float, float] = (0.5, 0.5)) -> Problem:
    """2D smooth lens c = 1 + 0.3 exp(-|x - center|^2/0.02) on [0,1)^2 (open axes; the
    default center is (0.5, 0.5)), with a Gaussian-modulated plane-wave packet travelling
    in +z: u0 = exp(-|x-x0|^2/width2) cos(k0 (z - z0)), u1 = -c(x) du0/dz."""
    h = 1.0 / N
    ax = h * np.arange(N)
    X, Z = np.meshgrid(ax, ax, indexing="ij")
    c = 1.0 + 0.3 * np.exp(-((X - center[0]) ** 2 + (Z - center[1]) ** 2) / 0.02)
    env = np.exp(-((X - x0[0]) ** 2 + (Z - x0[1]) ** 2) / width2)
    u0 = env * np.cos(k0 * (Z - x0[1]))
    du0 = env * (-2.0 * (Z - x0[1]) / width2 * np.cos(k0 * (Z - x0[1]))
                 - k0 * np.sin(k0 * (Z - x0[1])))
    u1 = -c * du0
    shot = Shot(eps=eps, u0=u0, u1=u1, q_stride=(s, s), box=(box, box))
    return Problem(name="lens_2d", dim=2, n=(N, N), h=(h, h), origin=(0.0, 0.0),
                   periodic=(False, False), velocity=c, shots=[shot], T=T, dt=dt,
                   kappa=kappa, tau=tau)


def lens_3d(N: int = 20, eps: float = 0.003, T: float = 0.05, dt: float = 1e-3,
            kappa: float = 6.0, tau: float = 1e-2, s: int = 2, box: int = 16,
            k0: float = 6 * math.pi, width2: float = 0.01,
            x0: Tuple[float, float, float] = (0.5, 0.5, 0.35),
            center: Tuple[float, float, float] = (0.52, 0.48, 0.55)) -> Problem:
    """3D smooth lens c = 1 + 0.3 exp(-|x - center|^2/0.02) on [0,1)^3 (open axes; center
    off the grid's knot planes), with a Gaussian-modulated plane-wave packet travelling
    in +z: u0 = exp(-|x-x0|^2/width2) cos(k0 (z - z0)), u1 = -c(x) du0/dz."""
    h = 1.0 / N
    ax = h * np.arange(N)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    c = 1.0 + 0.3 * np.exp(-((X - center[0]) ** 2 + (Y - center[1]) ** 2 + (Z - center[2]) ** 2)
                           / 0.02)
    env = np.exp(-((X - x0[0]) ** 2 + (Y - x0[1]) ** 2 + (Z - x0[2]) ** 2) / width2)
    u0 = env * np.cos(k0 * (Z - x0[2]))
    du0 = env * (-2.0 * (Z - x0[2]) / width2 * np.cos(k0 * (Z - x0[2]))
                 - k0 * np.sin(k0 * (Z - x0[2])))
    u1 = -c * du0
    shot = Shot(eps=eps, u0=u0, u1=u1, q_stride=(s, s, s), box=(box, box, box))
    return Problem(name="lens_3d", dim=3, n=(N, N, N), h=(h, h, h), origin=(0.0, 0.0, 0.0),
                   periodic=(False, False, False), velocity=c, shots=[shot], T=T, dt=dt,
                   kappa=kappa, tau=tau)


def periodic_2d(N: int = 64, eps: float = 1.0 / 128, T: float = 0.0, dt: float = 1e-2,
                s: int = 2, kappa: float = 8.0, tau: float = 0.0, c: float = 1.0,
                k0: Tuple[float, float] = (8 * math.pi, 12 * math.pi), width2: float = 0.01,
                with_u1: bool = False) -> Problem:
    """2D constant-speed problem on the periodic unit square (box = one period)."""
    h = 1.0 / N
    ax = h * np.arange(N)
    X, Z = np.meshgrid(ax, ax, indexing="ij")
    env = np.exp(-((X - 0.5) ** 2 + (Z - 0.5) ** 2) / width2)
    ph = k0[0] * X + k0[1] * Z
    u0 = env * np.cos(ph)
    if with_u1:
        # one-way in the direction of k0: u1 = -c (k0/|k0|) . grad u0
        kn = math.hypot(*k0)
        gx = env * (-2.0 * (X - 0.5) / width2 * np.cos(ph) - k0[0] * np.sin(ph))
        gz = env * (-2.0 * (Z - 0.5) / width2 * np.cos(ph) - k0[1] * np.sin(ph))
        u1 = -c * (k0[0] * gx + k0[1] * gz) / kn
    else:
        u1 = np.zeros_like(u0)
    shot = Shot(eps=eps, u0=u0, u1=u1, q_stride=(s, s), box=(N, N))
    return Problem(name="periodic_2d", dim=2, n=(N, N), h=(h, h), origin=(0.0, 0.0),
                   periodic=(True, True), velocity=np.full((N, N), c), shots=[shot], T=T,
                   dt=dt, kappa=kappa, tau=tau)


# ---------------------------------------------------------------------------
# Layered model (a synthetic stand-in for the smoothed Marmousi model)
# ---------------------------------------------------------------------------

LAYERED_SHAPE = (737, 241)
LAYERED_H = 0.0125  # km


def gen_layered(seed: int = 1304, shape: Tuple[int, int] = LAYERED_SHAPE,
                h: float = LAYERED_H) -> np.ndarray:
    """9.2 km x 3 km layered model, 12 dipping interfaces and 3 normal faults,
    1.5-5.5 km/s, Gaussian-smoothed (sigma = 100 m), stored as float32."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.Generator(np.random.PCG64(seed))
    nx, nz = shape
    x = h * np.arange(nx)
    z = h * np.arange(nz)
    X, Z = np.meshgrid(x, z, indexing="ij")
    nif = 12
    depths = np.sort(rng.uniform(0.1, 2.9, size=nif))
    dips = np.deg2rad(rng.uniform(-8.0, 8.0, size=nif))
    vel = np.empty(nif + 1)
    vel[0] = 1.5
    for k in range(1, nif + 1):
        vel[k] = np.clip(1.5 + 4.0 * k / nif + rng.uniform(-0.15, 0.15), 1.5, 5.5)
    zeff = Z.copy()
    for _ in range(3):
        xf = rng.uniform(1.5, 7.7)
        dip = np.deg2rad(rng.uniform(55.0, 80.0))
        facing = 1.0 if rng.uniform() < 0.5 else -1.0
        throw = rng.uniform(0.05, 0.25)
        xplane = xf + facing * Z / math.tan(dip)
        hanging = facing * (X - xplane) > 0
        zeff = np.where(hanging, zeff - throw, zeff)
    layer = np.zeros(X.shape, dtype=np.int64)
    for i in range(nif):
        zi = depths[i] + np.tan(dips[i]) * (X - 4.6)
        layer += (zeff >= zi).astype(np.int64)
    c = vel[layer]
    c = gaussian_filter(c, sigma=0.1 / h, mode="reflect")
    return c.astype(np.float32)


def ricker(tau: np.ndarray, f: float) -> np.ndarray:
    a = (math.pi * f) ** 2
    return (1.0 - 2.0 * a * tau ** 2) * np.exp(-a * tau ** 2)


def ricker_dt(tau: np.ndarray, f: float) -> np.ndarray:
    a = (math.pi * f) ** 2
    return 2.0 * a * tau * np.exp(-a * tau ** 2) * (2.0 * a * tau ** 2 - 3.0)


def ricker_ring_shot(velocity: np.ndarray, h: float, src: Tuple[float, float], f: float,
                     periodic=(False, False)) -> Shot:
    """Outgoing Ricker ring at t0 = 1/f around src: u0 = R(t0 - r/c_s),
    u1 = R'(t0 - r/c_s), c_s = velocity at the grid point nearest the source;
    eps = c_s/(2 pi f) so that |p| is about 1 at the peak frequency."""
    nx, nz = velocity.shape
    ix = min(max(int(round(src[0] / h)), 0), nx - 1)
    iz = min(max(int(round(src[1] / h)), 0), nz - 1)
    cs = float(velocity[ix, iz])
    x = h * np.arange(nx)
    z = h * np.arange(nz)
    X, Z = np.meshgrid(x, z, indexing="ij")
    r = np.sqrt((X - src[0]) ** 2 + (Z - src[1]) ** 2)
    t0 = 1.0 / f
    u0 = ricker(t0 - r / cs, f)
    u1 = ricker_dt(t0 - r / cs, f)
    eps = cs / (2.0 * math.pi * f)
    s, nb = default_stride_box(eps, (h, h), (nx, nz), periodic)
    return Shot(eps=eps, u0=u0, u1=u1, q_stride=s, box=nb, source=tuple(src), freq=f)


def layered_single(T: float = 2.0, dt: float = 1e-3, f: float = 15.0,
                   src: Tuple[float, float] = (4.6, 0.01), kappa: float = 6.0,
                   tau: float = 1e-3, seed: int = 1304) -> Problem:
    """Layered model, one 15 Hz Ricker-ring source at 10 m depth, T = 2 s."""
    c = gen_layered(seed).astype(np.float64)
    shot = ricker_ring_shot(c, LAYERED_H, src, f)
    return Problem(name="layered_single", dim=2, n=LAYERED_SHAPE, h=(LAYERED_H, LAYERED_H),
                   origin=(0.0, 0.0), periodic=(False, False), velocity=c, shots=[shot], T=T,
                   dt=dt, kappa=kappa, tau=tau)


def layered_batch(nshots: int = 64, seed: int = 3542, T: float = 2.0, dt: float = 1e-3,
                  kappa: float = 6.0, tau: float = 1e-3, model_seed: int = 1304) -> Problem:
    """Layered model, nshots sources with x ~ U(1.0, 8.2) km, depth ~ U(0.01, 0.5) km,
    peak frequency ~ U(8, 25) Hz, each with its own eps."""
    c = gen_layered(model_seed).astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = rng.uniform(1.0, 8.2, size=nshots)
    zs = rng.uniform(0.01, 0.5, size=nshots)
    fs = rng.uniform(8.0, 25.0, size=nshots)
    shots = [ricker_ring_shot(c, LAYERED_H, (float(xs[i]), float(zs[i])), float(fs[i]))
             for i in range(nshots)]
    return Problem(name="layered_batch", dim=2, n=LAYERED_SHAPE, h=(LAYERED_H, LAYERED_H),
                   origin=(0.0, 0.0), periodic=(False, False), velocity=c, shots=shots, T=T,
                   dt=dt, kappa=kappa, tau=tau)


def layered_adjoint(nshots: int = 16, T: float = 2.0, dt: float = 1e-3, f: float = 15.0,
                    kappa: float = 6.0, tau: float = 1e-3, anomaly: float = 0.05,
                    model_seed: int = 1304) -> Tuple[Problem, np.ndarray]:
    """Layered model with nshots 15 Hz sources at 10 m depth spaced 0.575 km, 368
    receivers at z = 0 every 25 m, traces every 4 ms. Returns the problem on the
    background model and the 'true' model c (1 + anomaly exp(-|x-(4.6,1.5)|^2/(2 0.3^2)))."""
    c = gen_layered(model_seed).astype(np.float64)
    shots = [ricker_ring_shot(c, LAYERED_H, ((k + 0.5) * 0.575, 0.01), f) for k in range(nshots)]
    rx = np.stack([0.025 * np.arange(368), np.zeros(368)], axis=1)
    nx, nz = LAYERED_SHAPE
    X, Z = np.meshgrid(LAYERED_H * np.arange(nx), LAYERED_H * np.arange(nz), indexing="ij")
    ctrue = c * (1.0 + anomaly * np.exp(-((X - 4.6) ** 2 + (Z - 1.5) ** 2) / (2 * 0.3 ** 2)))
    rec_every = int(round(0.004 / dt))
    prob = Problem(name="layered_adjoint", dim=2, n=LAYERED_SHAPE, h=(LAYERED_H, LAYERED_H),
                   origin=(0.0, 0.0), periodic=(False, False), velocity=c, shots=shots, T=T,
                   dt=dt, kappa=kappa, tau=tau, receivers=rx, record_every=rec_every)
    return prob, ctrue


def by_name(name: str, **kw) -> Problem:
    table = {
        "periodic_1d": periodic_1d,
        "lens_2d": lens_2d,
        "lens_3d": lens_3d,
        "periodic_2d": periodic_2d,
        "layered_single": layered_single,
        "layered_batch": layered_batch,
    }
    return table[name](**kw)


def window_evals(prob, Q, eps):
    """Grid points inside the kappa sqrt(eps) square window of each centre, summed."""
    cut = prob.kappa * math.sqrt(eps)
    tot = np.ones(Q.shape[0])
    for k in range(prob.dim):
        lo = np.ceil((Q[:, k] - cut - prob.origin[k]) / prob.h[k])
        hi = np.floor((Q[:, k] + cut - prob.origin[k]) / prob.h[k])
        lo = np.clip(lo, 0, prob.n[k] - 1)
        hi = np.clip(hi, 0, prob.n[k] - 1)
        cnt = np.where((Q[:, k] + cut >= prob.origin[k]) &
                       (Q[:, k] - cut <= prob.origin[k] + (prob.n[k] - 1) * prob.h[k]),
                       hi - lo + 1, 0)
        tot *= np.maximum(cnt, 0)
    return float(tot.sum())
