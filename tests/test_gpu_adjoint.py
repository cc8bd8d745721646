"""Traces at receivers and the hand-written adjoint (d traces/d c)^T r.

* GPU traces against the oracle's traces (same Gaussians, both branches summed
  literally by the oracle): rel-L2 <= 1e-10.
* J = 1/2 |u(T)|^2 on the whole grid (the adjoint through the reconstruction sum):
  the field recorded by receivers on every grid point equals fga_reconstruct's, and
  <grad J, v> matches central differences of J through fga_reconstruct.
* <grad J, v> for J = 1/2 |traces|^2 against central differences of J on the GPU
  (<= 2e-6 relative), for random smooth v and for single grid cells.
* Against the oracle's own derivative: <fga_grad(w), v> = <w, J v>, with J v the
  oracle's tangent-linear traces (dual-number RK4 through the rays, the amplitude and
  the action, and the derivative of the branch split through c(q)) for the same
  frozen set. This is the dot-product test of the GPU's reverse mode against the
  oracle's forward mode: w = traces (so <w, J v> = <grad J, v>) and random w, smooth
  v and single cells, <= 1e-12 relative; also at the shape of the layered adjoint
  workload (T = 2 s, 368 receivers, 501 samples) with the N largest Gaussians.
kappa = 8 so that Gaussians crossing a window edge change J by e^{-32} only. The lens
centre is kept off the spline's knot lines: in the symmetric lens centred on a knot
line, rays with p_x = 0 started on that line stay on it, where the Hessian of the cubic
spline has a kink; the derivative is then one-sided (the adjoint returns the derivative
of the cell the ray is in) while a central difference averages both sides.
"""

import dataclasses
import functools
import math

import numpy as np
import pytest

import oracle as O
from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=1)
def _problem():
    """The lens problem with the threshold put where the selected set cannot change under
    the finite-difference steps below (the adjoint differentiates with the set held
    fixed). A change dc of c(q) moves psi+ by at most |psi+ - psi0/2| |dc|/c (Eq. psi,
    u+-,0) and M by about as much, so each |psi+|/M is known to within a relative shift
    s; tau goes into the gap between consecutive ratios in 0.2%..5% whose slack after
    both neighbours' shifts is largest."""
    prob = WL.lens_2d(N=64, eps=1.0 / 400, T=0.1, dt=2e-3, s=2, box=32, tau=1e-2, kappa=8.0,
                      k0=24 * math.pi, width2=0.004, x0=(0.4937, 0.3), center=(0.5071, 0.4963))
    sh = prob.shots[0]
    g = O.Grid(prob.n, prob.h, prob.origin, prob.periodic)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau)
    plus = dec["psi_plus"][:, dec["valid"]].ravel()
    psi0 = dec["psi0"][:, dec["valid"]].ravel()
    r = np.abs(plus) / dec["M"]
    rel_dc = 2e-4 / prob.velocity.min()  # |dc| <= 1e-4 * max|v| (v <= 1), spline gain < 2
    shift = (np.abs(plus - 0.5 * psi0) / np.maximum(np.abs(plus), 1e-300) + 1.0) * rel_dc
    keep = (r > 2e-3) & (r < 5e-2)
    order = np.argsort(r[keep])
    rs, ss = r[keep][order], shift[keep][order]
    lo, hi = rs[:-1] * (1 + ss[:-1]), rs[1:] * (1 - ss[1:])
    k = int(np.argmax(np.log(hi) - np.log(lo)))
    assert hi[k] > lo[k] * 1.0005, (lo[k], hi[k])
    return dataclasses.replace(prob, tau=float(np.sqrt(lo[k] * hi[k])))


def _receivers():
    x = np.linspace(0.15, 0.85, 29)
    return np.stack([x, np.full_like(x, 0.5)], axis=1)


REC = 5


def _gpu(prob, c, want_plan=False):
    import torch

    plan = F.plan_from_problem(prob, velocity=np.ascontiguousarray(c),
                               stream=torch.cuda.current_stream().cuda_stream,
                               integrate_exited=True)
    plan.set_receivers(_receivers(), REC)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    tr = plan.traces()
    qi, pi, _ = plan.gaussians(0)
    keys = set(zip(qi.tolist(), pi.tolist()))
    if want_plan:
        return tr, keys, plan
    plan.close()
    return tr, keys


def _smooth_direction(n, seed):
    rng = np.random.default_rng(seed)
    X, Z = np.meshgrid(np.linspace(0, 1, n[0]), np.linspace(0, 1, n[1]), indexing="ij")
    v = np.zeros(n)
    for _ in range(4):
        kx, kz = rng.uniform(1, 4, 2)
        v += rng.standard_normal() * np.sin(2 * np.pi * (kx * X + rng.uniform())) * np.cos(
            2 * np.pi * (kz * Z + rng.uniform()))
    return v / np.abs(v).max()


def test_traces_match_oracle():
    prob = _problem()
    tr, keys = _gpu(prob, prob.velocity)
    sh = prob.shots[0]
    g = O.Grid(prob.n, prob.h, prob.origin, prob.periodic)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau)
    gs = dec["gauss"]
    W = O.quadrature_weight(g, sh.eps, sh.q_stride, sh.box)
    ot = O.traces(g, prob.velocity, prob.nsteps, prob.dt, REC, gs["sigma"], gs["q"], gs["p"],
                  gs["psi"], sh.eps, prob.kappa, W, _receivers())
    assert np.linalg.norm(ot.imag) <= 1e-12 * np.linalg.norm(ot.real)
    err = np.linalg.norm(tr[0] - ot.real) / np.linalg.norm(ot.real)
    assert err <= 1e-10, err


def test_adjoint_directional_derivatives():
    prob = _problem()
    c = prob.velocity
    tr, keys, plan = _gpu(prob, c, want_plan=True)
    J0 = 0.5 * float(np.sum(tr ** 2))
    grad = plan.grad(np.ascontiguousarray(tr))  # residual = traces (data = 0)
    plan.close()
    assert np.all(np.isfinite(grad)) and np.abs(grad).max() > 0
    for seed in (1, 2):
        v = _smooth_direction(prob.n, seed)
        dg = float(np.sum(grad * v))
        # GPU central differences (the selected set must not change)
        hstep = 1e-4
        trp, kp = _gpu(prob, c + hstep * v)
        trm, km = _gpu(prob, c - hstep * v)
        assert kp == keys and km == keys
        fd = (0.5 * np.sum(trp ** 2) - 0.5 * np.sum(trm ** 2)) / (2 * hstep)
        assert abs(dg - fd) <= 2e-6 * abs(fd), (dg, fd)
    # single cells where the gradient is largest
    flat = np.argsort(-np.abs(grad.ravel()))[:3]
    for f in flat:
        e = np.zeros(prob.n)
        e.ravel()[f] = 1.0
        hstep = 1e-4
        trp, _ = _gpu(prob, c + hstep * e)
        trm, _ = _gpu(prob, c - hstep * e)
        fd = (0.5 * np.sum(trp ** 2) - 0.5 * np.sum(trm ** 2)) / (2 * hstep)
        assert abs(grad.ravel()[f] - fd) <= 1e-5 * abs(fd) + 1e-12 * J0, (grad.ravel()[f], fd)


DOT_TOL = 1e-12


def _oracle_keys(prob, c, shot=0, rows=None):
    sh = prob.shots[shot]
    g = O.Grid(prob.n, prob.h, prob.origin, prob.periodic)
    dec = O.decompose(g, c, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau,
                      keep_n=getattr(prob, "keep_n", 0), q_subset=rows)
    gk = dec["gauss"]
    return g, dec, (gk["sigma"], gk["qidx"], gk["pidx"])


def test_adjoint_against_oracle_tangent():
    """Reverse mode on the GPU against forward mode in the oracle, same frozen set:
    <fga_grad(w), v> = <w, Re J v> for w = traces and two random w, along two smooth
    directions and the three cells where the gradient is largest; both ways of keeping
    the ray states for the reverse sweep (all recorded, or checkpointed segments)."""
    prob = _problem()
    c = prob.velocity
    tr, keys, plan = _gpu(prob, c, want_plan=True)
    sh = prob.shots[0]
    g, dec, okeys = _oracle_keys(prob, c)
    plus = okeys[0] == 1
    assert set(zip(okeys[1][plus].tolist(), okeys[2][plus].tolist())) == keys
    rng = np.random.default_rng(7)
    ws = [np.ascontiguousarray(tr)] + [rng.standard_normal(tr.shape) for _ in range(2)]
    grads = [plan.grad(np.ascontiguousarray(w)) for w in ws]
    # the other way of keeping the ray states (checkpoints, segments recomputed) gives the
    # same gradient up to the order of the atomic additions
    plan.set_adjoint_checkpointing(1)
    seg = [plan.grad(np.ascontiguousarray(w)) for w in ws]
    plan.close()
    for a, b in zip(grads, seg):
        assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)
    dirs = [_smooth_direction(prob.n, seed) for seed in (1, 2)]
    for f in np.argsort(-np.abs(grads[0].ravel()))[:3]:
        e = np.zeros(prob.n)
        e.ravel()[f] = 1.0
        dirs.append(e)
    worst = 0.0
    for v in dirs:
        _, jv = O.frozen_set_traces_tangent(g, c, v, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box,
                                            okeys, prob.nsteps, prob.dt, REC, prob.kappa,
                                            _receivers())
        for w, gr in zip(ws, grads):
            lhs = float(np.sum(gr * v))
            rhs = float(np.sum(w[0] * jv.real))
            err = abs(lhs - rhs) / (np.linalg.norm(w) * np.linalg.norm(jv.real))
            worst = max(worst, err)
            assert err <= DOT_TOL, (lhs, rhs, err)
    print("adjoint vs oracle tangent, worst relative difference %.3e" % worst)


def test_adjoint_layered_shape_against_oracle_tangent():
    """The layered adjoint workload's shape (737 x 241 model, sources at 10 m depth,
    368 surface receivers every 25 m, 501 samples to T = 2 s) with the 120 largest
    |psi+| per branch of two shots, so that the oracle's forward mode covers every
    Gaussian: <fga_grad(w), v> = <w, Re J v> for the data residual and a smooth v
    that also moves c(q) under the sources."""
    import torch

    prob16, ctrue = WL.layered_adjoint()
    prob = dataclasses.replace(prob16, shots=prob16.shots[7:9], keep_n=120)
    rx, rec = prob.receivers, prob.record_every
    u0, u1 = F.stacked_initial_data(prob)

    def forward(cc, keep=False):
        plan = F.plan_from_problem(prob, velocity=np.ascontiguousarray(cc),
                                   stream=torch.cuda.current_stream().cuda_stream,
                                   integrate_exited=True)
        plan.set_receivers(rx, rec)
        plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
        plan.propagate()
        t = plan.traces()
        if keep:
            return t, plan
        plan.close()
        return t

    data = forward(ctrue)
    c = prob.velocity
    tr, plan = forward(c, keep=True)
    assert tr.shape == (2, 501, 368)
    w = np.ascontiguousarray(tr - data)
    grad = plan.grad(w)
    counts = [plan.count(s) for s in range(2)]
    plan.close()
    assert counts == [120, 120]
    v = _smooth_direction(prob.n, 9)
    lhs = float(np.sum(grad * v))
    rhs = 0.0
    jvs = []
    for s in range(2):
        sh = prob.shots[s]
        rows = _active_rows(prob, sh)
        g, dec, okeys = _oracle_keys(prob, c, shot=s, rows=rows)
        _, jv = O.frozen_set_traces_tangent(g, c, v, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box,
                                            okeys, prob.nsteps, prob.dt, rec, prob.kappa, rx)
        rhs += float(np.sum(w[s] * jv.real))
        jvs.append(jv.real)
    err = abs(lhs - rhs) / (np.linalg.norm(w) * np.linalg.norm(np.stack(jvs)))
    print("layered shape: <grad, v> %.12e, <w, Jv> %.12e, relative difference %.3e"
          % (lhs, rhs, err))
    assert err <= DOT_TOL, (lhs, rhs, err)


def _active_rows(prob, shot):
    """q-grid rows whose FBI box meets the nonzero data (the others have psi = 0)."""
    g = O.Grid(prob.n, prob.h, prob.origin, prob.periodic)
    nz = (shot.u0 != 0) | (shot.u1 != 0)
    nq = O.q_counts(g, shot.q_stride)
    keep = []
    for k in range(prob.dim):
        other = tuple(a for a in range(prob.dim) if a != k)
        idx = np.flatnonzero(np.any(nz, axis=other))
        m = np.arange(nq[k]) * shot.q_stride[k]
        half = shot.box[k] // 2
        keep.append((m - half <= idx.max()) & (m + half - 1 >= idx.min()))
    mesh = np.meshgrid(*keep, indexing="ij")
    return np.flatnonzero(np.logical_and.reduce([x.ravel() for x in mesh]))


def test_autograd_function_matches_fga_grad():
    import torch

    from paper_1304_3542_gb300 import autograd as FA

    prob = _problem()
    vel = torch.from_numpy(np.ascontiguousarray(prob.velocity)).cuda().requires_grad_(True)
    tr = FA.traces(vel, prob, _receivers(), REC, integrate_exited=True)
    loss = 0.5 * (tr ** 2).sum()
    loss.backward()
    tr_np, keys, plan = _gpu(prob, prob.velocity, want_plan=True)
    g = plan.grad(np.ascontiguousarray(tr_np))
    plan.close()
    got = vel.grad.cpu().numpy()
    assert np.linalg.norm(got - g) <= 1e-10 * np.linalg.norm(g)


def test_autograd_forward_without_grad_releases_its_plan():
    """A forward that cannot be differentiated destroys its plan at once and returns the
    same traces (to rounding: receivers sum their contributions with atomic reductions,
    whose order varies from run to run)."""
    import gc

    import torch

    from paper_1304_3542_gb300 import autograd as FA

    prob = _problem()
    vel = torch.from_numpy(np.ascontiguousarray(prob.velocity)).cuda()
    with_grad = FA.traces(vel.clone().requires_grad_(True), prob, _receivers(), REC,
                          integrate_exited=True)
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.no_grad():
        outs = [FA.traces(vel, prob, _receivers(), REC, integrate_exited=True) for _ in range(3)]
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    ref = with_grad.detach()
    for o in outs:
        assert float((o - ref).norm() / ref.norm()) <= 1e-13
    # three kept plans would hold their checkpoint buffers; released ones hold nothing
    # beyond the outputs (a few kB) and the caching allocator's slack
    assert free0 - free1 < 64 << 20, (free0 - free1)


def _field_gpu(prob, c):
    import torch

    plan = F.plan_from_problem(prob, velocity=np.ascontiguousarray(c),
                               stream=torch.cuda.current_stream().cuda_stream,
                               integrate_exited=True)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    u = plan.reconstruct()[0]
    qi, pi, _ = plan.gaussians(0)
    plan.close()
    return u, set(zip(qi.tolist(), pi.tolist()))


def test_field_misfit_gradient():
    """J = 1/2 |u(T)|^2 over the grid through autograd.field (a receiver on every grid
    point, one record at T): the recorded field equals fga_reconstruct's, and <grad J, v>
    matches central differences of J computed with fga_reconstruct (set unchanged)."""
    import torch

    from paper_1304_3542_gb300 import autograd as FA

    prob = _problem()
    c = prob.velocity
    vel = torch.from_numpy(np.ascontiguousarray(c)).cuda().requires_grad_(True)
    u = FA.field(vel, prob, integrate_exited=True)
    ref, keys = _field_gpu(prob, c)
    got = u[0].detach().cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
    (0.5 * (u ** 2).sum()).backward()
    grad = vel.grad.cpu().numpy()
    assert np.all(np.isfinite(grad)) and np.abs(grad).max() > 0
    for seed in (1, 2):
        v = _smooth_direction(prob.n, seed)
        dg = float(np.sum(grad * v))
        hstep = 1e-4
        up, kp = _field_gpu(prob, c + hstep * v)
        um, km = _field_gpu(prob, c - hstep * v)
        assert kp == keys and km == keys
        fd = (0.5 * np.sum(up ** 2) - 0.5 * np.sum(um ** 2)) / (2 * hstep)
        assert abs(dg - fd) <= 2e-6 * abs(fd), (dg, fd)


def _support_mask(prob):
    """True on the cells whose spline value c(q) can enter psi+ of some shot: the data's
    bounding box widened by half an FBI box and by the spline's 2-cell reach."""
    m = np.zeros(prob.n, dtype=bool)
    for sh in prob.shots:
        nz = (sh.u0 != 0) | (sh.u1 != 0)
        sl = []
        for k in range(prob.dim):
            other = tuple(a for a in range(prob.dim) if a != k)
            idx = np.flatnonzero(np.any(nz, axis=other))
            pad = sh.box[k] // 2 + sh.q_stride[k] + 3
            sl.append(slice(max(idx.min() - pad, 0), idx.max() + pad + 1))
        m[tuple(sl)] = True
    return m


def test_adjoint_layered_full_size():
    """The configuration of the layered adjoint workload (737 x 241 model, 15 Hz sources
    at 10 m depth, 368 surface receivers every 25 m, traces every 4 ms to T = 2 s, data
    from the +5 % anomaly model) with two of its sixteen shots. The directions vanish
    wherever c(q) enters psi+, so the selected set is exactly the same under the steps."""
    import torch

    prob16, ctrue = WL.layered_adjoint()
    prob = dataclasses.replace(prob16, shots=prob16.shots[7:9])
    rx, rec = prob.receivers, prob.record_every
    u0, u1 = F.stacked_initial_data(prob)
    d_u0, d_u1 = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()

    def forward(c, keep=False):
        plan = F.plan_from_problem(prob, velocity=np.ascontiguousarray(c),
                                   stream=torch.cuda.current_stream().cuda_stream)
        plan.set_receivers(rx, rec)
        plan.decompose(d_u0, d_u1)
        plan.propagate()
        tr = plan.traces()
        keys = [tuple(a.tolist() for a in plan.gaussians(s)[:2]) for s in range(len(prob.shots))]
        if keep:
            return tr, keys, plan
        plan.close()
        return tr, keys

    data, _ = forward(ctrue)
    c = prob.velocity
    tr, keys, plan = forward(c, keep=True)
    assert tr.shape == (2, 501, 368)
    res = np.ascontiguousarray(tr - data)
    J = lambda t: 0.5 * float(np.sum((t - data) ** 2))
    J0 = J(tr)
    assert J0 > 0
    grad = plan.grad(res)
    plan.close()
    assert grad.shape == prob.n and np.all(np.isfinite(grad))
    free = ~_support_mask(prob)
    assert free.sum() > 0.5 * free.size
    # J is strongly nonlinear here (a step of 1e-3 km/s along v already moves the central
    # difference by 17 %; the difference converges to the adjoint value, 6.6e-4 off at
    # 1e-4 and 1.3e-4 at 1e-5), and the C2 spline and the window cut limit how far central
    # differences can be pushed: step 2e-5, agreement within 5e-4.
    hstep = 2e-5
    for seed in (3, 4):
        v = _smooth_direction(prob.n, seed) * free
        dg = float(np.sum(grad * v))
        trp, kp = forward(c + hstep * v)
        trm, km = forward(c - hstep * v)
        assert kp == keys and km == keys
        fd = (J(trp) - J(trm)) / (2 * hstep)
        assert abs(dg - fd) <= 5e-4 * abs(fd), (dg, fd)
    g_free = np.where(free, np.abs(grad), 0.0).ravel()
    hstep = 1e-4
    for f in np.argsort(-g_free)[:2]:
        e = np.zeros(prob.n)
        e.ravel()[f] = 1.0
        trp, _ = forward(c + hstep * e)
        trm, _ = forward(c - hstep * e)
        fd = (J(trp) - J(trm)) / (2 * hstep)
        # A single cell moves few rays, so the jumps of J where a receiver crosses the
        # edge of a Gaussian's window (relative size e^{-kappa^2/2} = 1.5e-8 of that
        # Gaussian's term at kappa = 6, not part of the derivative) weigh more against
        # the small change of J than for the smooth directions: 5e-3.
        assert abs(grad.ravel()[f] - fd) <= 5e-3 * abs(fd) + 1e-12 * J0, (grad.ravel()[f], fd)


def test_adjoint_checkpointing_rejects_unknown_mode():
    plan = F.plan_from_problem(_problem())
    with pytest.raises(F.FGAError) as ei:
        plan.set_adjoint_checkpointing(2)
    assert ei.value.status == F.FGA_ERR_INVALID
    plan.set_adjoint_checkpointing(1)
    plan.set_adjoint_checkpointing(0)
    plan.close()
