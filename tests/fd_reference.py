"""Finite-difference reference for the 2D acoustic wave equation u_tt = c(x)^2 (u_xx + u_zz).

Not the method: the accuracy-versus-N sweep of the paper's numerical section compares
FGA fields with a fine-grid solve of the PDE, and this is that solve (test
infrastructure: numpy/scipy set-up, the time loop in plain PyTorch CPU tensor operations
so that it uses the host's cores; shares nothing with the CUDA path).

* Space: 8th-order central second differences on a grid refined `refine` times.
* Time: fourth-order two-step scheme (leapfrog with the modified-equation correction),
  u^{n+1} = 2 u^n - u^{n-1} + dt^2 M u^n + dt^4/12 M M u^n, M = c^2 L, stable while
  dt^2 |lambda(M)| <= 12; the first step from the Taylor expansion to dt^4.
* Medium: the cubic B-spline whose coefficients are the velocity samples with clamped
  indices (the FGA's medium), evaluated by scipy's spline evaluation without prefilter.
* The domain is padded on every side with that medium's own extension; the padded edge
  holds u = 0 and is far enough that nothing reflected there comes back by time T
  (pad >= c T / 2 on every side, checked).
"""

from __future__ import annotations

import math

import numpy as np
import torch
from scipy import ndimage

# 8th-order central weights of the second derivative: w0, w1..w4 (times 1/h^2)
W8 = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


def spline_velocity(coef: np.ndarray, h, x: np.ndarray, z: np.ndarray) -> np.ndarray:
    """c at points (x, z) (origin 0): sum_ij c_ij beta3(x/h0 - i) beta3(z/h1 - j),
    indices clamped to the grid."""
    return ndimage.map_coordinates(coef, [x / h[0], z / h[1]], order=3, mode="nearest",
                                   prefilter=False)


def laplacian8(u: torch.Tensor, inv_h2: float, out: torch.Tensor) -> torch.Tensor:
    """8th-order Laplacian of u with u = 0 beyond the array (Dirichlet)."""
    torch.mul(u, 2.0 * W8[0], out=out)
    for k in range(1, 5):
        w = W8[k]
        out[k:, :].add_(u[:-k, :], alpha=w)
        out[:-k, :].add_(u[k:, :], alpha=w)
        out[:, k:].add_(u[:, :-k], alpha=w)
        out[:, :-k].add_(u[:, k:], alpha=w)
    out.mul_(inv_h2)
    return out


def leapfrog_limit(cmax: float, hf: float) -> float:
    """Largest stable plain-leapfrog step for the 2D 8th-order Laplacian, c dt sqrt(lambda)
    <= 2, lambda the largest eigenvalue of -L (the Nyquist mode on both axes); the
    fourth-order scheme allows sqrt(12) instead of 2."""
    sym = -(W8[0] + 2.0 * sum(W8[k] * math.cos(k * math.pi) for k in range(1, 5)))
    lam = 2.0 * sym / (hf * hf)
    return 2.0 / (cmax * math.sqrt(lam))


def solve(coef: np.ndarray, h, n, f0, f1, T: float, refine: int = 2, pad: float = 1.0,
          courant: float = 0.5):
    """u(T) on the grid points i h (origin 0, shape n) from initial data given as callables
    f0(X, Z), f1(X, Z), evaluated on the refined grid and set to zero outside the original
    domain (where the grid data end). Returns (u on the grid, info)."""
    h = (float(h[0]), float(h[1]))
    assert abs(h[0] - h[1]) <= 1e-12 * h[0], "square cells only"
    hf = h[0] / refine
    npad = int(math.ceil(pad / h[0])) * refine  # padding in fine cells (whole coarse cells)
    nf = tuple((n[k] - 1) * refine + 1 + 2 * npad for k in range(2))
    x = (np.arange(nf[0]) - npad) * hf
    z = (np.arange(nf[1]) - npad) * hf
    X, Z = np.meshgrid(x, z, indexing="ij")
    c = spline_velocity(coef, h, X, Z)
    cmax = float(c.max())
    # a wave that reaches an edge of the original domain crosses the padding and back
    edge_c = max(float(c[0, :].max()), float(c[-1, :].max()), float(c[:, 0].max()),
                 float(c[:, -1].max()))
    assert npad * hf >= 0.5 * edge_c * T, "padding too thin for T"
    dt0 = courant * leapfrog_limit(cmax, hf)
    nsteps = max(int(math.ceil(T / dt0)), 1)
    dt = T / nsteps
    half = 0.5 * hf
    inside = ((X >= -half) & (X <= (n[0] - 1) * h[0] + half) & (Z >= -half)
              & (Z <= (n[1] - 1) * h[1] + half))
    u0 = torch.from_numpy(np.where(inside, f0(X, Z), 0.0))
    u1 = torch.from_numpy(np.where(inside, f1(X, Z), 0.0))
    c2 = torch.from_numpy(c * c)
    inv_h2 = 1.0 / (hf * hf)
    lap = torch.empty_like(u0)

    def M(u):
        return c2 * laplacian8(u, inv_h2, lap)

    Mu0 = M(u0)
    Mu1 = M(u1)
    prev = u0
    cur = u0 + dt * u1 + (0.5 * dt ** 2) * Mu0 + (dt ** 3 / 6.0) * Mu1 + (dt ** 4 / 24.0) * M(Mu0)
    a2, a4 = dt * dt, dt ** 4 / 12.0
    for _ in range(1, nsteps):
        Mc = M(cur)
        nxt = 2.0 * cur - prev + a2 * Mc + a4 * M(Mc)
        prev, cur = cur, nxt
    cur = cur.numpy()
    uc = cur[npad:npad + (n[0] - 1) * refine + 1:refine, npad:npad + (n[1] - 1) * refine + 1:refine]
    return np.ascontiguousarray(uc), {"fine_shape": nf, "dt": dt, "steps": nsteps, "cmax": cmax}
