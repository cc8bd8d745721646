"""Python binding of libfga (include/fga.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of libfga; this module only
turns numpy arrays / torch tensors into pointers, calls the C ABI, and raises
FGAError when a call fails. There is no fallback path: if libfga.so cannot be
loaded, every call raises.

Pointers may be host (numpy, CPU tensors) or device (CUDA tensors on the
current device); device tensors must be contiguous float64.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

FGA_OK = 0
FGA_ERR_INVALID = 1
FGA_ERR_OOM = 2
FGA_ERR_CUDA = 3
FGA_ERR_TIMEOUT = 4
FGA_ERR_STATE = 5
FGA_ERR_NUMERIC = 6
FGA_ERR_CAPACITY = 7
FGA_FP64 = 0
FGA_MIXED_TF32X3 = 1
FGA_MIXED_BF16X3 = 2
FGA_Z_DYNAMIC = 0
FGA_Z_DIVIDED = 1
FGA_BSPLINE_APPROX = 0
FGA_BSPLINE_INTERP = 1

STATUS = {0: "FGA_OK", 1: "FGA_ERR_INVALID", 2: "FGA_ERR_OOM", 3: "FGA_ERR_CUDA",
          4: "FGA_ERR_TIMEOUT", 5: "FGA_ERR_STATE", 6: "FGA_ERR_NUMERIC", 7: "FGA_ERR_CAPACITY"}


class FGAError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, STATUS.get(status, status), message))


class Config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int64 * 3),
        ("h", ctypes.c_double * 3),
        ("origin", ctypes.c_double * 3),
        ("periodic", ctypes.c_int * 3),
        ("nshots", ctypes.c_int),
        ("eps", ctypes.POINTER(ctypes.c_double)),
        ("q_stride", ctypes.POINTER(ctypes.c_int)),
        ("box", ctypes.POINTER(ctypes.c_int)),
        ("T", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("integrate_exited", ctypes.c_int),
        ("keep_n", ctypes.c_int64),
        ("z_method", ctypes.c_int),
        ("dz_eta", ctypes.c_double),
        ("interp", ctypes.c_int),
    ]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfga.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libfga.so is missing; run paper_1304_3542_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    L.fga_plan.argtypes = [ctypes.POINTER(Config), P, P, ctypes.POINTER(P)]
    L.fga_decompose.argtypes = [P, P, P, P]
    L.fga_propagate.argtypes = [P]
    L.fga_reconstruct.argtypes = [P, P]
    L.fga_sync.argtypes = [P]
    L.fga_destroy.argtypes = [P]
    L.fga_status_string.argtypes = [ci]
    L.fga_status_string.restype = ctypes.c_char_p
    L.fga_last_error.argtypes = [P]
    L.fga_last_error.restype = ctypes.c_char_p
    L.fga_count.argtypes = [P, ci]
    L.fga_count.restype = i64
    L.fga_shot_grid.argtypes = [P, ci, P, P, P, P]
    L.fga_psi.argtypes = [P, ci, P, P]
    L.fga_gaussians.argtypes = [P, ci, P, P, P]
    L.fga_state.argtypes = [P, ci, P, P, P, P, P, P]
    L.fga_stage_times.argtypes = [P, P, P]
    L.fga_ray_steps.argtypes = [P]
    L.fga_ray_steps.restype = i64
    L.fga_set_receivers.argtypes = [P, i64, P, i64]
    L.fga_set_receivers.restype = ci
    L.fga_traces.argtypes = [P, P]
    L.fga_traces.restype = ci
    L.fga_autotune.argtypes = [P, P, P]
    L.fga_autotune.restype = ci
    L.fga_tuning.argtypes = [P, P]
    L.fga_tuning.restype = ci
    L.fga_set_tuning.argtypes = [P, P]
    L.fga_set_tuning.restype = ci
    L.fga_run_graph.argtypes = [P, P]
    L.fga_run_graph.restype = ci
    L.fga_run_pipeline.argtypes = [P, P, P, P]
    L.fga_run_pipeline.restype = ci
    L.fga_set_wait_budget.argtypes = [P, i64]
    L.fga_set_wait_budget.restype = ci
    L.fga_set_adjoint_checkpointing.argtypes = [P, ci]
    L.fga_set_adjoint_checkpointing.restype = ci
    L.fga_grad.argtypes = [P, P, P]
    L.fga_grad.restype = ci
    L.fga_reconstruct_static.argtypes = [ci, P, P, P, P, ctypes.c_double, ctypes.c_double, i64,
                                         P, P, P, P]
    L.fga_reconstruct_static.restype = ci
    L.fga_spline_prefilter.argtypes = [ci, P, P, P, P]
    L.fga_spline_prefilter.restype = ci
    L.fga_fma_peak.argtypes = [ci, ci, P, P]
    L.fga_fma_peak.restype = ci
    for name in ("fga_plan", "fga_decompose", "fga_propagate", "fga_reconstruct", "fga_sync",
                 "fga_destroy", "fga_shot_grid", "fga_psi", "fga_gaussians", "fga_state",
                 "fga_stage_times"):
        getattr(L, name).restype = ci
    _lib = L
    return L


def _ptr(x) -> Optional[int]:
    """Raw address of a contiguous float64/int buffer (numpy array or torch tensor)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(x))


def _check_f64(x, n, name):
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64:
            raise TypeError("%s must be float64" % name)
        if x.size != n:
            raise ValueError("%s has %d values, expected %d" % (name, x.size, n))
    elif hasattr(x, "dtype"):
        import torch

        if x.dtype != torch.float64:
            raise TypeError("%s must be float64" % name)
        if x.numel() != n:
            raise ValueError("%s has %d values, expected %d" % (name, x.numel(), n))


class Plan:
    """One FGA plan: grid, velocity, per-shot eps/q-stride/box, T, dt, kappa, tau."""

    def __init__(self, dim: int, n: Sequence[int], h: Sequence[float], origin: Sequence[float],
                 periodic: Sequence[bool], velocity, eps: Sequence[float], T: float, dt: float,
                 kappa: float, tau: float, q_stride=None, box=None, precision: int = FGA_FP64,
                 stream: Optional[int] = None, integrate_exited: bool = False,
                 keep_n: int = 0, z_method: int = 0, dz_eta: float = 0.0,
                 interp: int = FGA_BSPLINE_APPROX):
        self._L = load()
        self.dim = dim
        self.n = tuple(int(v) for v in n)
        self.npts = int(np.prod(self.n))
        self.nshots = len(eps)
        cfg = Config()
        cfg.dim = dim
        for k in range(3):
            cfg.n[k] = self.n[k] if k < dim else 1
            cfg.h[k] = float(h[k]) if k < dim else 1.0
            cfg.origin[k] = float(origin[k]) if k < dim else 0.0
            cfg.periodic[k] = int(bool(periodic[k])) if k < dim else 0
        cfg.nshots = self.nshots
        self._eps = np.ascontiguousarray(eps, dtype=np.float64)
        cfg.eps = self._eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._qs = None if q_stride is None else np.ascontiguousarray(q_stride, dtype=np.int32).ravel()
        self._box = None if box is None else np.ascontiguousarray(box, dtype=np.int32).ravel()
        cfg.q_stride = (self._qs.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
                        if self._qs is not None else None)
        cfg.box = (self._box.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
                   if self._box is not None else None)
        cfg.T, cfg.dt, cfg.kappa, cfg.tau = float(T), float(dt), float(kappa), float(tau)
        self._T, self._dt = float(T), float(dt)
        cfg.precision = int(precision)
        cfg.integrate_exited = int(bool(integrate_exited))
        cfg.keep_n = int(keep_n)
        cfg.z_method = int(z_method)
        cfg.dz_eta = float(dz_eta)
        cfg.interp = int(interp)
        _check_f64(velocity, self.npts, "velocity")
        self._keep = [velocity]
        out = ctypes.c_void_p()
        st = self._L.fga_plan(ctypes.byref(cfg), _ptr(velocity), stream, ctypes.byref(out))
        if st != FGA_OK:
            raise FGAError(st, "fga_plan", self._L.fga_last_error(None).decode())
        self._h = out

    # -- helpers -----------------------------------------------------------
    def _check(self, st, where):
        if st != FGA_OK:
            raise FGAError(st, where, self._L.fga_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.fga_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the three steps ---------------------------------------------------
    def decompose(self, u0, u1) -> np.ndarray:
        n = self.nshots * self.npts
        _check_f64(u0, n, "u0")
        _check_f64(u1, n, "u1")
        self._keep_in = (u0, u1)
        counts = np.zeros(self.nshots, dtype=np.int64)
        self._check(self._L.fga_decompose(self._h, _ptr(u0), _ptr(u1), counts.ctypes.data),
                    "fga_decompose")
        return counts

    def propagate(self):
        self._check(self._L.fga_propagate(self._h), "fga_propagate")

    def reconstruct(self, out=None):
        if out is None:
            out = np.empty((self.nshots,) + self.n)
        _check_f64(out, self.nshots * self.npts, "out")
        self._check(self._L.fga_reconstruct(self._h, _ptr(out)), "fga_reconstruct")
        return out

    def run_graph(self, out):
        """propagate + reconstruct into the device tensor out, as one CUDA graph replay."""
        self._check(self._L.fga_run_graph(self._h, _ptr(out)), "fga_run_graph")
        return out

    def set_wait_budget(self, tries: int):
        """fga_set_wait_budget: polls of a tensor-core completion wait before giving up
        (< 0: defaults; 0: give up at once)."""
        self._check(self._L.fga_set_wait_budget(self._h, int(tries)), "fga_set_wait_budget")

    def set_adjoint_checkpointing(self, mode: int):
        """fga_set_adjoint_checkpointing: 0 = record every ray state when it fits in half
        of the free device memory, 1 = always checkpoint segments and recompute them."""
        self._check(self._L.fga_set_adjoint_checkpointing(self._h, int(mode)),
                    "fga_set_adjoint_checkpointing")

    def run_pipeline(self, u0, u1, out):
        """decompose + propagate + reconstruct of every shot as one CUDA graph replay
        (fga_run_pipeline): device tensors u0, u1 in, out overwritten."""
        n = self.nshots * self.npts
        _check_f64(u0, n, "u0")
        _check_f64(u1, n, "u1")
        _check_f64(out, n, "out")
        self._check(self._L.fga_run_pipeline(self._h, _ptr(u0), _ptr(u1), _ptr(out)),
                    "fga_run_pipeline")
        return out

    def autotune(self, out):
        """Tune the ray kernel (blocks per SM, register budget) and the gather's segment
        length on this plan's data, then propagate and reconstruct into the device tensor
        out. Returns the choice (blocks per SM, segment length, ray kernel variant)."""
        ch = np.zeros(3, dtype=np.int64)
        self._check(self._L.fga_autotune(self._h, _ptr(out), ch.ctypes.data), "fga_autotune")
        return tuple(int(v) for v in ch)

    def tuning(self):
        ch = np.zeros(3, dtype=np.int64)
        self._check(self._L.fga_tuning(self._h, ch.ctypes.data), "fga_tuning")
        return tuple(int(v) for v in ch)

    def set_tuning(self, blocks_per_sm: int, segment: int, variant: int = 0):
        ch = np.array([blocks_per_sm, segment, variant], dtype=np.int64)
        self._check(self._L.fga_set_tuning(self._h, ch.ctypes.data), "fga_set_tuning")

    def sync(self):
        self._check(self._L.fga_sync(self._h), "fga_sync")

    # -- inspection --------------------------------------------------------
    def count(self, shot: int = 0) -> int:
        return int(self._L.fga_count(self._h, shot))

    def shot_grid(self, shot: int = 0):
        nq = np.zeros(self.dim, dtype=np.int64)
        nb = np.zeros(self.dim, dtype=np.int64)
        s = np.zeros(self.dim, dtype=np.int64)
        self._check(self._L.fga_shot_grid(self._h, shot, nq.ctypes.data, None, nb.ctypes.data,
                                          s.ctypes.data), "fga_shot_grid")
        return nq, nb, s

    def psi(self, shot: int = 0):
        nq, nb, _ = self.shot_grid(shot)
        out = np.zeros((int(np.prod(nq)), int(np.prod(nb)), 2))
        m = ctypes.c_double(0.0)
        self._check(self._L.fga_psi(self._h, shot, out.ctypes.data, ctypes.addressof(m)), "fga_psi")
        return out[..., 0] + 1j * out[..., 1], m.value

    def gaussians(self, shot: int = 0):
        G = self.count(shot)
        qi = np.zeros(G, dtype=np.int64)
        pi = np.zeros(G, dtype=np.int64)
        ps = np.zeros((G, 2))
        self._check(self._L.fga_gaussians(self._h, shot, qi.ctypes.data, pi.ctypes.data,
                                          ps.ctypes.data), "fga_gaussians")
        return qi, pi, ps[:, 0] + 1j * ps[:, 1]

    def state(self, shot: int = 0):
        G = self.count(shot)
        d = self.dim
        Q = np.zeros((G, d)); P = np.zeros((G, d))
        A = np.zeros((G, d, d, 2)); B = np.zeros((G, d, d, 2))
        a = np.zeros((G, 2)); S = np.zeros(G)
        self._check(self._L.fga_state(self._h, shot, Q.ctypes.data, P.ctypes.data, A.ctypes.data,
                                      B.ctypes.data, a.ctypes.data, S.ctypes.data), "fga_state")
        return {"Q": Q, "P": P, "A": A[..., 0] + 1j * A[..., 1], "B": B[..., 0] + 1j * B[..., 1],
                "a": a[:, 0] + 1j * a[:, 1], "S": S}

    def set_receivers(self, xr, record_every: int):
        xr = np.ascontiguousarray(xr, dtype=np.float64)
        self._rx = xr
        self._record_every = int(record_every)
        self._check(self._L.fga_set_receivers(self._h, xr.shape[0] if xr.size else 0,
                                              xr.ctypes.data if xr.size else None,
                                              int(record_every)), "fga_set_receivers")

    def traces(self, out=None):
        nrx = self._rx.shape[0]
        nrec = int(round(self._T / self._dt)) // self._record_every + 1
        if out is None:
            out = np.empty((self.nshots, nrec, nrx))
        self._check(self._L.fga_traces(self._h, _ptr(out)), "fga_traces")
        return out

    def grad(self, residual, out=None):
        """(d traces / d c)^T residual on the velocity grid (the set of Gaussians fixed)."""
        if out is None:
            out = np.empty(self.n)
        self._check(self._L.fga_grad(self._h, _ptr(residual), _ptr(out)), "fga_grad")
        return out

    def ray_steps(self) -> int:
        return int(self._L.fga_ray_steps(self._h))

    def stage_times(self):
        ms = np.zeros(5)
        n = ctypes.c_int64(0)
        self._check(self._L.fga_stage_times(self._h, ms.ctypes.data, ctypes.addressof(n)),
                    "fga_stage_times")
        return {"fbi": ms[0], "select": ms[1], "rays": ms[2], "binning": ms[3],
                "reconstruct": ms[4]}, int(n.value)


def reconstruct_static(dim: int, n: Sequence[int], h: Sequence[float], origin: Sequence[float],
                       periodic: Sequence[bool], eps: float, kappa: float, qp, coef, u,
                       stream: Optional[int] = None):
    """fga_reconstruct_static: the reconstruction without any device allocation.
    qp: device float64 [2*dim][nG] (Q rows then P rows); coef: device float64 [nG][2];
    u: device float64 grid, overwritten. The C side cannot see buffer sizes, so every
    size is checked here before the call."""
    L = load()
    npts = int(np.prod(np.asarray(n, dtype=np.int64)))
    nG = 0
    if qp is not None:
        nq = qp.numel() if hasattr(qp, "numel") else qp.size
        if nq % (2 * dim) != 0:
            raise ValueError("qp has %d values, not a multiple of 2*dim = %d" % (nq, 2 * dim))
        nG = nq // (2 * dim)
        _check_f64(qp, 2 * dim * nG, "qp")
        _check_f64(coef, 2 * nG, "coef")
    _check_f64(u, npts, "u")
    n_ = np.ascontiguousarray(n, dtype=np.int64)
    h_ = np.ascontiguousarray(h, dtype=np.float64)
    o_ = np.ascontiguousarray(origin, dtype=np.float64)
    p_ = np.ascontiguousarray([1 if v else 0 for v in periodic], dtype=np.int32)
    st = L.fga_reconstruct_static(dim, n_.ctypes.data, h_.ctypes.data, o_.ctypes.data,
                                  p_.ctypes.data, float(eps), float(kappa), nG, _ptr(qp),
                                  _ptr(coef), _ptr(u), stream)
    if st != FGA_OK:
        raise FGAError(st, "fga_reconstruct_static", L.fga_last_error(None).decode())
    return u


def spline_prefilter(samples: np.ndarray, periodic: Sequence[bool]) -> np.ndarray:
    """fga_spline_prefilter on the host: the coefficients of the clamped / wrapped cubic
    B-spline that interpolates the samples (C-order float64 grid, 1 to 3 axes)."""
    L = load()
    a = np.ascontiguousarray(samples, dtype=np.float64)
    out = np.empty_like(a)
    n = np.ascontiguousarray(a.shape, dtype=np.int64)
    per = np.ascontiguousarray([int(bool(v)) for v in periodic], dtype=np.int32)
    st = L.fga_spline_prefilter(a.ndim, n.ctypes.data, per.ctypes.data, a.ctypes.data,
                                out.ctypes.data)
    if st != FGA_OK:
        raise FGAError(st, "fga_spline_prefilter", L.fga_last_error(None).decode())
    return out


def fma_peak(bits: int = 64, iters: int = 4096):
    """fga_fma_peak: measured FMA throughput of the current GPU, (TFLOP/s, ms)."""
    L = load()
    tf = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    st = L.fga_fma_peak(int(bits), int(iters), ctypes.addressof(tf), ctypes.addressof(ms))
    if st != FGA_OK:
        raise FGAError(st, "fga_fma_peak", L.fga_last_error(None).decode())
    return tf.value, ms.value


def plan_from_problem(prob, velocity=None, stream=None, precision: int = FGA_FP64,
                      integrate_exited: bool = False, z_method: int = 0,
                      dz_eta: float = 0.0, interp: int = FGA_BSPLINE_APPROX) -> Plan:
    """A Plan for a workloads.Problem (its grid, shots, T, dt, kappa, tau, keep_n)."""
    vel = prob.velocity if velocity is None else velocity
    if isinstance(vel, np.ndarray):
        vel = np.ascontiguousarray(vel, dtype=np.float64)
    return Plan(prob.dim, prob.n, prob.h, prob.origin, prob.periodic, vel,
                [s.eps for s in prob.shots], prob.T, prob.dt, prob.kappa, prob.tau,
                q_stride=[s.q_stride for s in prob.shots], box=[s.box for s in prob.shots],
                precision=precision, stream=stream, integrate_exited=integrate_exited,
                keep_n=getattr(prob, "keep_n", 0), z_method=z_method, dz_eta=dz_eta,
                interp=interp)


def stacked_initial_data(prob):
    u0 = np.ascontiguousarray(np.stack([s.u0 for s in prob.shots]), dtype=np.float64)
    u1 = np.ascontiguousarray(np.stack([s.u1 for s in prob.shots]), dtype=np.float64)
    return u0, u1
