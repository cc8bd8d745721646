"""Plain FP64 CPU oracle for the frozen Gaussian approximation (FGA).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module. It shares no code with the CUDA path
and never imports the product package; its inputs are plain numpy arrays and
numbers.

The three steps of the paper's algorithm (Algorithm section):
  1. decompose: the FBI transform of f0 and f1 on a small box around every q
     (Initial wavefield decomposition section), evaluated, as the paper does,
     with an FFT of g_q(r) = f(q + r) exp(-|r|^2/(2 eps)) on the box
     (numpy.fft is the library step); the branch split of Eq. psi; selection
     of the sets G+- by thresholding |psi+-};
  2. propagate: RK4 on the ray, dynamic-ray, amplitude and action equations
     (C++ part, fga_oracle.cpp); propagate_dd takes d_z Q, d_z P from divided
     differences across auxiliary rays instead (the alternative named after
     Eq. op_zZ);
  3. reconstruct: the sum of Eq. recons (C++ part), term by term.

Discretisation (the paper leaves these open; each is a reading):
  * q-grid: q = origin + s*m*h per axis, m = 0..n_q-1 (all grid points on a
    periodic axis, whose length must be a multiple of s);
  * box: r_j = (j - n_b/2) h, j = 0..n_b-1; samples outside an open axis are 0;
    on a periodic axis the box is one period and the window is periodised
    (sum over images |l| <= 2);
  * p-grid: p_m = 2 pi eps m/(n_b h), m = -n_b/2+1 .. n_b/2-1 (the unpaired
    Nyquist value m = -n_b/2 is left out so that the grid is symmetric under
    p -> -p), and the point p = 0, where u+-,0 is singular, is left out;
  * each term of the reconstruction carries the quadrature weight
    W = prod_k (s_k h_k)(2 pi eps/(n_b,k h_k)), without which the prefactors
    2^{d/2} and (2 pi eps)^{-3d/2} do not give back f0 at t = 0.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fga_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C++ part (g++, -O2, OpenMP, IEEE arithmetic) into oracle/_build."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        ci = ctypes.c_int
        lib.orc_medium_eval.argtypes = [ci, P, P, P, P, P, i64, P, P, P, P, P]
        lib.orc_hamiltonian.argtypes = [ci, P, P, P, P, P, ci, P, P, P]
        lib.orc_propagate.argtypes = [ci, P, P, P, P, P, i64, d, i64, P, P, P, P, P, P, P, P, P,
                                      ci]
        lib.orc_propagate_dd.argtypes = [ci, P, P, P, P, P, i64, d, i64, P, P, P, P, P, P, P,
                                         P, P, P, P, ci]
        lib.orc_reconstruct.argtypes = [ci, P, d, d, d, i64, P, P, P, P, P, i64, P, P, P, ci]
        lib.orc_fbi_direct.argtypes = [ci, P, P, P, P, d, P, i64, P, P, P]
        lib.orc_traces.argtypes = [ci, P, P, P, P, P, i64, d, i64, i64, P, P, P, P, d, d, d, i64,
                                   P, P, ci]
        lib.orc_propagate_tangent.argtypes = [ci, P, P, P, P, P, P, i64, d, i64, P, P, P, P, P,
                                              P, P, P, P, P, P, P, P, P, P, ci]
        lib.orc_traces_tangent.argtypes = [ci, P, P, P, P, P, P, i64, d, i64, i64, P, P, P, P,
                                           P, d, d, d, i64, P, P, P, ci]
        lib.orc_num_threads_available.restype = ci
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """Axis description: x_i = o + i h per axis; periodic axes wrap."""

    def __init__(self, n: Sequence[int], h: Sequence[float], o: Sequence[float],
                 periodic: Sequence[bool]):
        self.dim = len(n)
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.h = _f64(h)
        self.o = _f64(o)
        self.periodic = np.ascontiguousarray([1 if p else 0 for p in periodic], dtype=np.int32)

    @property
    def period(self) -> np.ndarray:
        return np.where(self.periodic > 0, self.n * self.h, 0.0)

    def args(self):
        return (self.dim, _ptr(self.n), _ptr(self.h), _ptr(self.o), _ptr(self.periodic))


def default_threads() -> int:
    return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# Medium (cubic B-spline of the velocity samples) -- C++ part
# ---------------------------------------------------------------------------

def medium_eval(grid: Grid, coef: np.ndarray, x: np.ndarray, order: int = 2):
    """c, grad c, Hessian (and third derivatives if order >= 3) at points x[npts][dim]."""
    lib = _load()
    coef = _f64(coef)
    x = _f64(x).reshape(-1, grid.dim)
    npts = x.shape[0]
    d = grid.dim
    c = np.empty(npts)
    g = np.empty((npts, d)) if order >= 1 else None
    hs = np.empty((npts, d, d)) if order >= 2 else None
    d3 = np.empty((npts, d, d, d)) if order >= 3 else None
    rc = lib.orc_medium_eval(*grid.args(), _ptr(coef), npts, _ptr(x), _ptr(c),
                             _ptr(g) if g is not None else None,
                             _ptr(hs) if hs is not None else None,
                             _ptr(d3) if d3 is not None else None)
    assert rc == 0
    return c, g, hs, d3


def interp_coefficients(grid: Grid, samples: np.ndarray) -> np.ndarray:
    """Coefficients C of the medium's spline (clamped indices on open axes, wrapped on
    periodic ones) that interpolate the samples: c(x_i) = c_i at every grid point. The
    tensor-product spline samples separably, so along each axis the grid values are
    B_k C with B_k[i][j] = sum of beta3(i - t) over the taps t = i-1, i, i+1 whose
    clamped (or wrapped) index is j; each B_k is solved densely (numpy.linalg.solve)."""
    c = _f64(samples).reshape(tuple(int(v) for v in grid.n))
    w = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}  # beta3 at the integer offsets
    for k in range(grid.dim):
        n = int(grid.n[k])
        B = np.zeros((n, n))
        for i in range(n):
            for off, wt in w.items():
                t = i + off
                j = t % n if grid.periodic[k] else min(max(t, 0), n - 1)
                B[i, j] += wt
        c = np.moveaxis(np.linalg.solve(B, np.moveaxis(c, k, 0).reshape(n, -1)).reshape(
            np.moveaxis(c, k, 0).shape), 0, k)
    return np.ascontiguousarray(c)


def hamiltonian(grid: Grid, coef: np.ndarray, sigma: int, Q, P) -> Dict[str, np.ndarray]:
    lib = _load()
    d = grid.dim
    out = np.empty(1 + 2 * d + 4 * d * d)
    Q = _f64(Q)
    P = _f64(P)
    rc = lib.orc_hamiltonian(*grid.args(), _ptr(_f64(coef)), int(sigma), _ptr(Q), _ptr(P),
                             _ptr(out))
    assert rc == 0
    i = 1
    res = {"H": out[0]}
    res["dHdQ"] = out[i:i + d].copy(); i += d
    res["dHdP"] = out[i:i + d].copy(); i += d
    for name in ("HQQ", "HQP", "HPP", "HPQ"):
        res[name] = out[i:i + d * d].reshape(d, d).copy()
        i += d * d
    return res


# ---------------------------------------------------------------------------
# Step 1: decomposition
# ---------------------------------------------------------------------------

def q_counts(grid: Grid, stride: Sequence[int]) -> np.ndarray:
    out = []
    for k in range(grid.dim):
        n, s = int(grid.n[k]), int(stride[k])
        if grid.periodic[k]:
            assert n % s == 0, "periodic axis length must be a multiple of the q-stride"
            out.append(n // s)
        else:
            out.append((n - 1) // s + 1)
    return np.array(out, dtype=np.int64)


def q_points(grid: Grid, stride: Sequence[int]) -> np.ndarray:
    """q-grid points in C order, [n_q total][dim]."""
    nq = q_counts(grid, stride)
    axes = [grid.o[k] + stride[k] * np.arange(nq[k]) * grid.h[k] for k in range(grid.dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def p_axis(grid: Grid, eps: float, box: Sequence[int], k: int) -> np.ndarray:
    """p values of axis k indexed by j = m + n_b/2, m = -n_b/2 .. n_b/2-1."""
    nb = int(box[k])
    m = np.arange(nb) - nb // 2
    return 2.0 * math.pi * eps * m / (nb * grid.h[k])


def p_points(grid: Grid, eps: float, box: Sequence[int]) -> np.ndarray:
    axes = [p_axis(grid, eps, box, k) for k in range(grid.dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def p_valid(box: Sequence[int]) -> np.ndarray:
    """Mask over the p-grid: False on the Nyquist index m = -n_b/2 of any axis and at p = 0."""
    masks = []
    for nb in box:
        v = np.ones(int(nb), dtype=bool)
        v[0] = False
        masks.append(v)
    mesh = np.meshgrid(*masks, indexing="ij")
    ok = np.logical_and.reduce([m.ravel() for m in mesh])
    zero = np.ravel_multi_index(tuple(int(nb) // 2 for nb in box), tuple(int(b) for b in box))
    ok[zero] = False
    return ok


def window_axis(grid: Grid, eps: float, box: Sequence[int], k: int) -> np.ndarray:
    nb = int(box[k])
    r = (np.arange(nb) - nb // 2) * grid.h[k]
    if grid.periodic[k]:
        L = grid.n[k] * grid.h[k]
        return sum(np.exp(-((r + l * L) ** 2) / (2.0 * eps)) for l in range(-2, 3))
    return np.exp(-(r ** 2) / (2.0 * eps))


def fbi(grid: Grid, f: np.ndarray, eps: float, stride: Sequence[int], box: Sequence[int],
        q_chunk: int = 256, q_subset: Optional[np.ndarray] = None) -> np.ndarray:
    """psi(q, p) for every q on the q-grid and every p on the box DFT grid
    (Initial wavefield decomposition section):
        psi(q, p) = prod_k h_k * sum_{j in box} f(q + r_j) w(r_j) e^{-i p.r_j/eps},
    evaluated per q as the FFT of g_q = f(q + r) w(r) on the box. With
    p_m r_j/eps = 2 pi m (j - n_b/2)/n_b the phase is e^{-2 pi i m j/n_b} (-1)^m,
    so psi(q, p_m) = prod h * (-1)^m * FFT(g_q)[m mod n_b].
    Returns a complex array [n_q total][n_p total], p in C order over j = m + n_b/2;
    with q_subset (flat q-grid indices) only those rows, in that order."""
    d = grid.dim
    f = _f64(f).reshape(tuple(int(v) for v in grid.n))
    nq = q_counts(grid, stride)
    box = [int(b) for b in box]
    for k in range(d):
        assert box[k] % 2 == 0
        if grid.periodic[k]:
            assert box[k] == grid.n[k], "on a periodic axis the box is one period"
    # per-axis sample indices [n_q,k][n_b,k] and validity
    idx, inside = [], []
    for k in range(d):
        m = np.arange(nq[k])[:, None]
        j = np.arange(box[k])[None, :]
        i = stride[k] * m + j - box[k] // 2
        if grid.periodic[k]:
            idx.append(np.mod(i, grid.n[k]))
            inside.append(np.ones_like(i, dtype=bool))
        else:
            inside.append((i >= 0) & (i < grid.n[k]))
            idx.append(np.clip(i, 0, grid.n[k] - 1))
    w = [window_axis(grid, eps, box, k) for k in range(d)]
    sign = [np.where((np.arange(box[k]) - box[k] // 2) % 2 == 0, 1.0, -1.0) for k in range(d)]
    # index maps from m = j - n_b/2 to the FFT bin (m mod n_b)
    fft_bin = [np.mod(np.arange(box[k]) - box[k] // 2, box[k]) for k in range(d)]
    hv = float(np.prod(grid.h))
    nqt = int(np.prod(nq))
    npt = int(np.prod(box))
    rows = np.arange(nqt) if q_subset is None else np.asarray(q_subset, dtype=np.int64)
    out = np.empty((rows.size, npt), dtype=np.complex128)
    qmulti = np.stack(np.unravel_index(rows, tuple(nq)), axis=1)
    nqt = rows.size
    for start in range(0, nqt, q_chunk):
        qs = qmulti[start:start + q_chunk]
        B = qs.shape[0]
        if d == 1:
            ii = idx[0][qs[:, 0]]
            ok = inside[0][qs[:, 0]]
            g = np.where(ok, f[ii], 0.0) * w[0][None, :]
            G = np.fft.fft(g, axis=1)
            psi = G[:, fft_bin[0]] * sign[0][None, :]
        elif d == 2:
            i0 = idx[0][qs[:, 0]][:, :, None]
            i1 = idx[1][qs[:, 1]][:, None, :]
            ok = inside[0][qs[:, 0]][:, :, None] & inside[1][qs[:, 1]][:, None, :]
            g = np.where(ok, f[i0, i1], 0.0) * (w[0][:, None] * w[1][None, :])[None]
            G = np.fft.fft2(g, axes=(1, 2))
            psi = G[:, fft_bin[0]][:, :, fft_bin[1]] * (sign[0][:, None] * sign[1][None, :])[None]
        else:
            i0 = idx[0][qs[:, 0]][:, :, None, None]
            i1 = idx[1][qs[:, 1]][:, None, :, None]
            i2 = idx[2][qs[:, 2]][:, None, None, :]
            ok = (inside[0][qs[:, 0]][:, :, None, None] & inside[1][qs[:, 1]][:, None, :, None]
                  & inside[2][qs[:, 2]][:, None, None, :])
            wt = w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]
            g = np.where(ok, f[i0, i1, i2], 0.0) * wt[None]
            G = np.fft.fftn(g, axes=(1, 2, 3))
            G = G[:, fft_bin[0]][:, :, fft_bin[1]][:, :, :, fft_bin[2]]
            sg = sign[0][:, None, None] * sign[1][None, :, None] * sign[2][None, None, :]
            psi = G * sg[None]
        out[start:start + B] = hv * psi.reshape(B, npt)
    return out


def fbi_direct(grid: Grid, f: np.ndarray, eps: float, box: Sequence[int], qi: np.ndarray,
               pv: np.ndarray) -> np.ndarray:
    """Brute-force FBI direct sum at the (q grid index, p value) pairs given (C++ part)."""
    lib = _load()
    qi = np.ascontiguousarray(qi, dtype=np.int64).reshape(-1, grid.dim)
    pv = _f64(pv).reshape(-1, grid.dim)
    nbx = np.ascontiguousarray(box, dtype=np.int64)
    out = np.empty((qi.shape[0], 2))
    rc = lib.orc_fbi_direct(grid.dim, _ptr(grid.n), _ptr(grid.h), _ptr(grid.periodic),
                            _ptr(_f64(f)), float(eps), _ptr(nbx), qi.shape[0], _ptr(qi),
                            _ptr(pv), _ptr(out))
    assert rc == 0
    return out[:, 0] + 1j * out[:, 1]


def branch_split(grid: Grid, coef: np.ndarray, eps: float, stride, box, psi0: np.ndarray,
                 psi1: np.ndarray, q_subset: Optional[np.ndarray] = None):
    """psi+- = 1/2 (psi0 +- i eps psi1/(c(q)|p|)) (Eq. psi, u+-,0), on valid (q,p) only;
    zero on the left-out p values. Returns (psi_plus, psi_minus, valid_mask[n_p])."""
    qpts = q_points(grid, stride)
    if q_subset is not None:
        qpts = qpts[np.asarray(q_subset, dtype=np.int64)]
    cq, _, _, _ = medium_eval(grid, coef, qpts, order=0)
    pp = p_points(grid, eps, box)
    pn = np.sqrt(np.sum(pp * pp, axis=1))
    valid = p_valid(box)
    inv = np.zeros_like(pn)
    inv[valid] = 1.0 / pn[valid]
    ratio = 1j * eps * inv[None, :] / cq[:, None]
    plus = 0.5 * (psi0 + ratio * psi1)
    minus = 0.5 * (psi0 - ratio * psi1)
    plus[:, ~valid] = 0.0
    minus[:, ~valid] = 0.0
    return plus, minus, valid


def select(psi_plus: np.ndarray, psi_minus: np.ndarray, valid: np.ndarray, tau: float,
           keep_n: int = 0):
    """Choose G+ and G- (thresholding of |psi+-|): keep the valid (q,p) with
    |psi| >= tau * M, M the largest |psi+-| over both branches; or, with keep_n > 0,
    the keep_n largest |psi| of each branch (ties broken by q index, then p index).
    Returns two arrays of flat (q,p) indices and M."""
    ap = np.abs(psi_plus)
    am = np.abs(psi_minus)
    vmask = np.broadcast_to(valid[None, :], ap.shape)
    M = max(ap[vmask].max(initial=0.0), am[vmask].max(initial=0.0))
    sel = []
    for a in (ap, am):
        flat = np.flatnonzero(vmask.ravel())
        vals = a.ravel()[flat]
        if keep_n > 0:
            order = np.lexsort((flat, -vals))  # by -|psi|, then flat index (q-major, p-minor)
            chosen = np.sort(flat[order[:keep_n]])
        else:
            chosen = flat[vals >= tau * M]
        sel.append(chosen)
    return sel[0], sel[1], M


def quadrature_weight(grid: Grid, eps: float, stride, box) -> float:
    W = 1.0
    for k in range(grid.dim):
        W *= stride[k] * grid.h[k] * (2.0 * math.pi * eps / (box[k] * grid.h[k]))
    return W


# ---------------------------------------------------------------------------
# Steps 2 and 3 -- C++ part
# ---------------------------------------------------------------------------

def propagate(grid: Grid, coef: np.ndarray, nsteps: int, dt: float, sigma: np.ndarray,
              q: np.ndarray, p: np.ndarray, nthreads: Optional[int] = None) -> Dict[str, np.ndarray]:
    lib = _load()
    d = grid.dim
    sigma = np.ascontiguousarray(sigma, dtype=np.int32)
    q = _f64(q).reshape(-1, d)
    p = _f64(p).reshape(-1, d)
    nG = q.shape[0]
    Q = np.empty((nG, d)); P = np.empty((nG, d))
    A = np.empty((nG, d, d, 2)); B = np.empty((nG, d, d, 2))
    a = np.empty((nG, 2)); S = np.empty(nG)
    rc = lib.orc_propagate(*grid.args(), _ptr(_f64(coef)), int(nsteps), float(dt), nG,
                           _ptr(sigma), _ptr(q), _ptr(p), _ptr(Q), _ptr(P), _ptr(A), _ptr(B),
                           _ptr(a), _ptr(S), int(nthreads or default_threads()))
    assert rc == 0, "orc_propagate failed (%d)" % rc
    return {"Q": Q, "P": P, "A": A[..., 0] + 1j * A[..., 1], "B": B[..., 0] + 1j * B[..., 1],
            "a": a[:, 0] + 1j * a[:, 1], "S": S}


def propagate_dd(grid: Grid, coef: np.ndarray, nsteps: int, dt: float, sigma: np.ndarray,
                 q: np.ndarray, p: np.ndarray, dq, dp, nthreads: Optional[int] = None):
    """propagate() with d_z Q, d_z P from central divided differences across auxiliary rays
    offset by dq[k] in q and dp[k] in p (the alternative named after Eq. op_zZ)."""
    lib = _load()
    d = grid.dim
    sigma = np.ascontiguousarray(sigma, dtype=np.int32)
    q = _f64(q).reshape(-1, d)
    p = _f64(p).reshape(-1, d)
    dq = _f64(np.broadcast_to(np.asarray(dq, dtype=np.float64), (d,)))
    dp = _f64(np.broadcast_to(np.asarray(dp, dtype=np.float64), (d,)))
    nG = q.shape[0]
    Q = np.empty((nG, d)); P = np.empty((nG, d))
    A = np.empty((nG, d, d, 2)); B = np.empty((nG, d, d, 2))
    a = np.empty((nG, 2)); S = np.empty(nG)
    rc = lib.orc_propagate_dd(*grid.args(), _ptr(_f64(coef)), int(nsteps), float(dt), nG,
                              _ptr(sigma), _ptr(q), _ptr(p), _ptr(dq), _ptr(dp), _ptr(Q), _ptr(P),
                              _ptr(A), _ptr(B), _ptr(a), _ptr(S), int(nthreads or default_threads()))
    assert rc == 0, "orc_propagate_dd failed (%d)" % rc
    return {"Q": Q, "P": P, "A": A[..., 0] + 1j * A[..., 1], "B": B[..., 0] + 1j * B[..., 1],
            "a": a[:, 0] + 1j * a[:, 1], "S": S}


def reconstruct(grid: Grid, eps: float, kappa: float, W: float, Q, P, a, psi, S, x,
                nthreads: Optional[int] = None):
    """Complex u at points x[npts][dim] (Eq. recons, windowed, periodic images)."""
    lib = _load()
    d = grid.dim
    Q = _f64(Q).reshape(-1, d)
    P = _f64(P).reshape(-1, d)
    nG = Q.shape[0]
    a2 = _f64(np.stack([np.real(a), np.imag(a)], axis=1)) if nG else np.empty((0, 2))
    s2 = _f64(np.stack([np.real(psi), np.imag(psi)], axis=1)) if nG else np.empty((0, 2))
    S = _f64(S)
    x = _f64(x).reshape(-1, d)
    npts = x.shape[0]
    ure = np.empty(npts); uim = np.empty(npts)
    L = _f64(grid.period)
    rc = lib.orc_reconstruct(d, _ptr(L), float(eps), float(kappa), float(W), nG, _ptr(Q),
                             _ptr(P), _ptr(a2), _ptr(s2), _ptr(S), npts, _ptr(x), _ptr(ure),
                             _ptr(uim), int(nthreads or default_threads()))
    assert rc == 0
    return ure + 1j * uim


def traces(grid: Grid, coef, nsteps: int, dt: float, record_every: int, sigma, q, p, psi,
           eps: float, kappa: float, W: float, xr, nthreads: Optional[int] = None):
    """Complex field at receivers xr[nrx][dim] at t_m = m*record_every*dt (m = 0..nsteps/
    record_every), every Gaussian propagated by RK4. Returns [nrec][nrx] complex."""
    lib = _load()
    d = grid.dim
    sigma = np.ascontiguousarray(sigma, dtype=np.int32)
    q = _f64(q).reshape(-1, d)
    p = _f64(p).reshape(-1, d)
    nG = q.shape[0]
    ps = _f64(np.stack([np.real(psi), np.imag(psi)], axis=1)) if nG else np.empty((0, 2))
    xr = _f64(xr).reshape(-1, d)
    nrec = nsteps // record_every + 1
    out = np.empty((nrec, xr.shape[0], 2))
    rc = lib.orc_traces(*grid.args(), _ptr(_f64(coef)), int(nsteps), float(dt), int(record_every),
                        nG, _ptr(sigma), _ptr(q), _ptr(p), _ptr(ps), float(eps), float(kappa),
                        float(W), xr.shape[0], _ptr(xr), _ptr(out), int(nthreads or default_threads()))
    assert rc == 0, "orc_traces failed (%d)" % rc
    return out[..., 0] + 1j * out[..., 1]


def frozen_set_traces(grid: Grid, coef, f0, f1, eps, stride, box, keys, nsteps, dt, record_every,
                      kappa, xr, nthreads=None):
    """Traces for a fixed set of Gaussians keys = (sigma, q index, p index) arrays, with the
    weights psi+- recomputed for the velocity coef (the FBI of the data does not depend on
    c; the branch split does, through c(q)). Used for derivatives with the set frozen."""
    sigma, qidx, pidx = keys
    rows, inv = np.unique(qidx, return_inverse=True)
    psi0 = fbi(grid, f0, eps, stride, box, q_subset=rows)
    psi1 = fbi(grid, f1, eps, stride, box, q_subset=rows)
    plus, minus, _ = branch_split(grid, coef, eps, stride, box, psi0, psi1, q_subset=rows)
    psi = np.where(np.asarray(sigma) > 0, plus[inv, pidx], minus[inv, pidx])
    qpts = q_points(grid, stride)[qidx]
    ppts = p_points(grid, eps, box)[pidx]
    W = quadrature_weight(grid, eps, stride, box)
    return traces(grid, coef, nsteps, dt, record_every, sigma, qpts, ppts, psi, eps, kappa, W, xr,
                  nthreads)


# ---------------------------------------------------------------------------
# Forward-mode (tangent-linear) derivatives along a change V of the velocity
# coefficients, with the set of Gaussians held fixed. The C++ part evaluates the same
# RK4 and reconstruction sum on dual numbers (value + derivative); the branch split's
# derivative through c(q) is written out here.
# ---------------------------------------------------------------------------

def propagate_tangent(grid: Grid, coef: np.ndarray, dcoef: np.ndarray, nsteps: int, dt: float,
                      sigma: np.ndarray, q: np.ndarray, p: np.ndarray,
                      nthreads: Optional[int] = None):
    """propagate() and the derivative of its outputs along dcoef: returns (state, dstate),
    dstate[k] = d state[k](coef + e dcoef)/de at e = 0 (q, p fixed)."""
    lib = _load()
    d = grid.dim
    sigma = np.ascontiguousarray(sigma, dtype=np.int32)
    q = _f64(q).reshape(-1, d)
    p = _f64(p).reshape(-1, d)
    nG = q.shape[0]
    bufs = [np.empty((nG, d)), np.empty((nG, d)), np.empty((nG, d, d, 2)), np.empty((nG, d, d, 2)),
            np.empty((nG, 2)), np.empty(nG)]
    dbufs = [np.empty_like(b) for b in bufs]
    rc = lib.orc_propagate_tangent(*grid.args(), _ptr(_f64(coef)), _ptr(_f64(dcoef)), int(nsteps),
                                   float(dt), nG, _ptr(sigma), _ptr(q), _ptr(p),
                                   *[_ptr(b) for b in bufs], *[_ptr(b) for b in dbufs],
                                   int(nthreads or default_threads()))
    assert rc == 0, "orc_propagate_tangent failed (%d)" % rc

    def pack(b):
        return {"Q": b[0], "P": b[1], "A": b[2][..., 0] + 1j * b[2][..., 1],
                "B": b[3][..., 0] + 1j * b[3][..., 1], "a": b[4][:, 0] + 1j * b[4][:, 1],
                "S": b[5]}

    return pack(bufs), pack(dbufs)


def branch_split_tangent(grid: Grid, coef: np.ndarray, dcoef: np.ndarray, eps: float, stride, box,
                         psi1: np.ndarray, q_subset: Optional[np.ndarray] = None):
    """Derivative of psi+- = 1/2 (psi0 +- i eps psi1/(c(q)|p|)) (Eq. psi, u+-,0) along
    dcoef: psi0 and psi1 do not depend on c, and the spline is linear in its
    coefficients, so d c(q) is the spline of dcoef at q and
        d psi+- = -+ 1/2 i eps psi1 d c(q)/(c(q)^2 |p|).
    Zero on the left-out p values. Returns (d psi_plus, d psi_minus)."""
    qpts = q_points(grid, stride)
    if q_subset is not None:
        qpts = qpts[np.asarray(q_subset, dtype=np.int64)]
    cq, _, _, _ = medium_eval(grid, coef, qpts, order=0)
    dcq, _, _, _ = medium_eval(grid, dcoef, qpts, order=0)
    pp = p_points(grid, eps, box)
    pn = np.sqrt(np.sum(pp * pp, axis=1))
    valid = p_valid(box)
    inv = np.zeros_like(pn)
    inv[valid] = 1.0 / pn[valid]
    dratio = -1j * eps * inv[None, :] * (dcq / (cq * cq))[:, None]
    dplus = 0.5 * dratio * psi1
    dminus = -0.5 * dratio * psi1
    dplus[:, ~valid] = 0.0
    dminus[:, ~valid] = 0.0
    return dplus, dminus


def traces_tangent(grid: Grid, coef, dcoef, nsteps: int, dt: float, record_every: int, sigma, q, p,
                   psi, dpsi, eps: float, kappa: float, W: float, xr, nthreads: Optional[int] = None):
    """traces() and its derivative along (dcoef, dpsi): returns two [nrec][nrx] complex
    arrays, the traces (equal to traces()) and d traces(coef + e dcoef, psi + e dpsi)/de."""
    lib = _load()
    d = grid.dim
    sigma = np.ascontiguousarray(sigma, dtype=np.int32)
    q = _f64(q).reshape(-1, d)
    p = _f64(p).reshape(-1, d)
    nG = q.shape[0]

    def c2(z):
        return _f64(np.stack([np.real(z), np.imag(z)], axis=1)) if nG else np.empty((0, 2))

    ps, dps = c2(psi), c2(dpsi)
    xr = _f64(xr).reshape(-1, d)
    nrec = nsteps // record_every + 1
    out = np.empty((nrec, xr.shape[0], 2))
    dout = np.empty_like(out)
    rc = lib.orc_traces_tangent(*grid.args(), _ptr(_f64(coef)), _ptr(_f64(dcoef)), int(nsteps),
                                float(dt), int(record_every), nG, _ptr(sigma), _ptr(q), _ptr(p),
                                _ptr(ps), _ptr(dps), float(eps), float(kappa), float(W),
                                xr.shape[0], _ptr(xr), _ptr(out), _ptr(dout),
                                int(nthreads or default_threads()))
    assert rc == 0, "orc_traces_tangent failed (%d)" % rc
    return out[..., 0] + 1j * out[..., 1], dout[..., 0] + 1j * dout[..., 1]


def frozen_set_traces_tangent(grid: Grid, coef, dcoef, f0, f1, eps, stride, box, keys, nsteps, dt,
                              record_every, kappa, xr, nthreads=None):
    """frozen_set_traces() and its directional derivative along dcoef (a change of the
    velocity coefficients): the rays and amplitudes through the dual-number RK4, the
    weights psi+- through c(q) in the branch split. Returns (traces, d traces), complex
    [nrec][nrx] each; the real parts are the recorded field and its derivative."""
    sigma, qidx, pidx = keys
    rows, inv = np.unique(qidx, return_inverse=True)
    psi0 = fbi(grid, f0, eps, stride, box, q_subset=rows)
    psi1 = fbi(grid, f1, eps, stride, box, q_subset=rows)
    plus, minus, _ = branch_split(grid, coef, eps, stride, box, psi0, psi1, q_subset=rows)
    dplus, dminus = branch_split_tangent(grid, coef, dcoef, eps, stride, box, psi1, q_subset=rows)
    pos = np.asarray(sigma) > 0
    psi = np.where(pos, plus[inv, pidx], minus[inv, pidx])
    dpsi = np.where(pos, dplus[inv, pidx], dminus[inv, pidx])
    qpts = q_points(grid, stride)[qidx]
    ppts = p_points(grid, eps, box)[pidx]
    W = quadrature_weight(grid, eps, stride, box)
    return traces_tangent(grid, coef, dcoef, nsteps, dt, record_every, sigma, qpts, ppts, psi, dpsi,
                          eps, kappa, W, xr, nthreads)


# ---------------------------------------------------------------------------
# The whole algorithm for one set of initial data
# ---------------------------------------------------------------------------

def decompose(grid: Grid, coef, f0, f1, eps, stride, box, tau, keep_n=0, q_subset=None):
    """Step 1. With q_subset (flat q indices), psi is computed for those q only: the
    rows left out are taken as psi = 0 (exact when their boxes hold no data)."""
    psi0 = fbi(grid, f0, eps, stride, box, q_subset=q_subset)
    psi1 = fbi(grid, f1, eps, stride, box, q_subset=q_subset)
    plus, minus, valid = branch_split(grid, coef, eps, stride, box, psi0, psi1, q_subset)
    sel_p, sel_m, M = select(plus, minus, valid, tau, keep_n)
    npt = plus.shape[1]
    qpts = q_points(grid, stride)
    ppts = p_points(grid, eps, box)
    rows = np.arange(qpts.shape[0]) if q_subset is None else np.asarray(q_subset, dtype=np.int64)
    gs = []
    for sigma, sel, arr in ((1, sel_p, plus), (-1, sel_m, minus)):
        ri, pi = np.divmod(sel, npt)
        qi = rows[ri]
        gs.append({"sigma": np.full(sel.size, sigma, dtype=np.int32), "qidx": qi, "pidx": pi,
                   "q": qpts[qi], "p": ppts[pi], "psi": arr.ravel()[sel]})
    gauss = {k: np.concatenate([gs[0][k], gs[1][k]]) for k in gs[0]}
    return {"psi0": psi0, "psi1": psi1, "psi_plus": plus, "psi_minus": minus, "valid": valid,
            "M": M, "gauss": gauss, "rows": rows}


def fga(grid: Grid, coef, f0, f1, eps, stride, box, tau, kappa, nsteps, dt, x=None, keep_n=0,
        nthreads=None, q_subset=None) -> Dict[str, object]:
    """Decompose, propagate to nsteps*dt, reconstruct at x (default: the grid)."""
    dec = decompose(grid, coef, f0, f1, eps, stride, box, tau, keep_n, q_subset)
    g = dec["gauss"]
    st = propagate(grid, coef, nsteps, dt, g["sigma"], g["q"], g["p"], nthreads)
    W = quadrature_weight(grid, eps, stride, box)
    if x is None:
        axes = [grid.o[k] + grid.h[k] * np.arange(grid.n[k]) for k in range(grid.dim)]
        mesh = np.meshgrid(*axes, indexing="ij")
        x = np.stack([m.ravel() for m in mesh], axis=1)
    u = reconstruct(grid, eps, kappa, W, st["Q"], st["P"], st["a"], g["psi"], st["S"], x,
                    nthreads)
    return {"dec": dec, "state": st, "u": u, "W": W}
