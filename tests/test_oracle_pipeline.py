"""Pins of the whole oracle pipeline (decompose -> propagate -> reconstruct).

* Frame identity: with all p of the box DFT grid, the reconstruction of the FBI
  coefficients at t = 0 gives back the data for any grid function, up to a
  Poisson error exp(-pi^2 eps/dq^2), the window cut exp(-kappa^2) and, on a
  periodic axis of length L, the overlap 2 exp(-L^2/(4 eps)) of neighbouring
  images of the periodised window (1e-14 at eps = 1/128, L = 1). This pins the
  FBI/reconstruction pair, the quadrature weight and the prefactors 2^{d/2} and
  (2 pi eps)^{-3d/2} of Eqs. recons and a_formu (d = 1, 2, 3).
* Constant speed: the semi-analytic Fourier-space prediction derived from the
  exact rays and amplitude (the method, not the PDE) pins the whole pipeline,
  including the branch split of Eq. psi, in 1D and in 2D.
* Against the PDE: d'Alembert in 1D with the O(eps) error the method predicts, and
  O(eps) convergence against a fine pseudo-spectral solve in a variable medium.
* Real data give a real field (the two branches are complex conjugates).
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1304_3542_gb300 import workloads as WL


def _grid(pr):
    return O.Grid(pr.n, pr.h, pr.origin, pr.periodic)


def _all_p_frame(g, f, eps, s, box, kappa, x):
    """Reconstruct at t = 0 from every (q, p) of the q-grid x box DFT grid."""
    psi = O.fbi(g, f, eps, s, box)
    qp = O.q_points(g, s)
    pp = O.p_points(g, eps, box)
    nq, npp = psi.shape
    Q = np.repeat(qp, npp, axis=0)
    P = np.tile(pp, (nq, 1))
    a0 = np.full(nq * npp, 2.0 ** (g.dim / 2.0))  # a(0) = 2^{d/2}
    W = O.quadrature_weight(g, eps, s, box)
    return O.reconstruct(g, eps, kappa, W, Q, P, a0, psi.ravel(), np.zeros(nq * npp), x)


def test_frame_identity_random_data_1d_periodic():
    n = 128
    g = O.Grid((n,), (1.0 / n,), (0.0,), (True,))
    f = np.random.default_rng(1).standard_normal(n)
    x = (np.arange(n) / n)[:, None]
    u = _all_p_frame(g, f, 1.0 / 128, (2,), (n,), 8.0, x)
    assert np.linalg.norm(u - f) <= 1e-12 * np.linalg.norm(f)


def test_frame_identity_random_data_2d_periodic():
    n = 32
    g = O.Grid((n, n), (1.0 / n,) * 2, (0.0, 0.0), (True, True))
    f = np.random.default_rng(2).standard_normal((n, n))
    axes = np.meshgrid(np.arange(n) / n, np.arange(n) / n, indexing="ij")
    pick = np.random.default_rng(4).choice(n * n, size=48, replace=False)
    x = np.stack([a.ravel() for a in axes], axis=1)[pick]
    u = _all_p_frame(g, f, 1.0 / 128, (1, 1), (n, n), 6.0, x)
    assert np.linalg.norm(u - f.ravel()[pick]) <= 1e-10 * np.linalg.norm(f.ravel()[pick])


def test_frame_identity_random_data_2d_open():
    # open axes: data zero near the edges, box 12 sqrt(eps), q-stride 0.5 sqrt(eps)
    n = (40, 36)
    h = (1.0 / 40, 1.0 / 40)
    g = O.Grid(n, h, (0.0, 0.0), (False, False))
    eps = 1.0 / 400  # sqrt(eps) = 2 cells
    rng = np.random.default_rng(3)
    f = np.zeros(n)
    f[12:28, 10:26] = rng.standard_normal((16, 16))
    s, box = (1, 1), (24, 24)
    x = np.stack([a.ravel() for a in np.meshgrid(*[h[k] * np.arange(n[k]) for k in range(2)],
                                                indexing="ij")], axis=1)
    u = _all_p_frame(g, f, eps, s, box, 6.0, x)
    assert np.linalg.norm(u - f.ravel()) <= 1e-10 * np.linalg.norm(f)


def test_frame_identity_random_data_3d_periodic():
    # n = 12 per axis, q-stride 1, eps = 1.9 h^2, kappa = 4.3: the Poisson error
    # exp(-pi^2 eps/h^2) = 7e-9, the image overlap 2 exp(-L^2/(4 eps)) = 1.2e-8 and the
    # window cut exp(-kappa^2) = 9e-9 bound the identity at about 3e-8 (3M Gaussians)
    n = 12
    h = 1.0 / n
    g = O.Grid((n,) * 3, (h,) * 3, (0.0,) * 3, (True,) * 3)
    f = np.random.default_rng(7).standard_normal((n,) * 3)
    axes = np.meshgrid(*(np.arange(n) / n,) * 3, indexing="ij")
    pick = np.random.default_rng(8).choice(n ** 3, size=32, replace=False)
    x = np.stack([a.ravel() for a in axes], axis=1)[pick]
    u = _all_p_frame(g, f, 1.9 * h * h, (1, 1, 1), (n,) * 3, 4.3, x)
    assert np.linalg.norm(u - f.ravel()[pick]) <= 2e-7 * np.linalg.norm(f.ravel()[pick])


def test_frame_identity_pipeline_1d():
    # the full pipeline (p = 0 and the Nyquist value left out, tau = 0, f1 = 0, T = 0)
    # on data with no spectral content near k = 0
    pr = WL.periodic_1d(width2=0.01)
    sh = pr.shots[0]
    res = O.fga(_grid(pr), pr.velocity, sh.u0, np.zeros_like(sh.u0), sh.eps, sh.q_stride,
                sh.box, 0.0, pr.kappa, 0, pr.dt)
    u = res["u"]
    assert np.linalg.norm(u.real - sh.u0) <= 1e-10 * np.linalg.norm(sh.u0)
    assert np.linalg.norm(u.imag) <= 1e-12 * np.linalg.norm(sh.u0)


def _prediction(fh0, fh1, kvecs, eps, c, T, pvals, valid, dim):
    """Fourier coefficients of the FGA field for constant speed c and all valid p:
    u^(k) = sum_p dp^d (2 pi eps)^{-d/2} e^{-|p - eps k|^2/eps}
            sum_sigma a_sigma(T,p) 1/2 (f0^ + sigma i eps f1^/(c|p|)) e^{-i sigma c T k.p/|p|},
    a_sigma(T,p) = sqrt(2) (2 - i sigma c T/|p|)^{(d-1)/2}  (exact rays and amplitude)."""
    out = np.zeros(fh0.shape, dtype=complex)
    for pv in pvals[valid]:
        pn = np.linalg.norm(pv)
        nh = pv / pn
        wgt = np.exp(-np.sum((pv[None, :] - eps * kvecs) ** 2, axis=1) / eps)
        kn = kvecs @ nh
        tot = 0.0
        for sigma in (1, -1):
            a = math.sqrt(2.0) * (2.0 - 1j * sigma * c * T / pn) ** ((dim - 1) / 2.0)
            tot = tot + a * 0.5 * (fh0 + sigma * 1j * eps * fh1 / (c * pn)) * np.exp(-1j * sigma * c * T * kn)
        out += wgt * tot
    return out


def test_spectral_prediction_1d_periodic():
    pr = WL.periodic_1d()  # the 1D constant-speed problem, T = 0.25
    sh = pr.shots[0]
    g = _grid(pr)
    res = O.fga(g, pr.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, 0.0, pr.kappa,
                pr.nsteps, pr.dt)
    n = pr.n[0]
    k = 2 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    pv = O.p_points(g, sh.eps, sh.box)
    valid = O.p_valid(sh.box)
    dp = 2 * math.pi * sh.eps / (sh.box[0] * pr.h[0])
    uh = _prediction(np.fft.fft(sh.u0), np.fft.fft(sh.u1), k[:, None], sh.eps, 1.0,
                     pr.nsteps * pr.dt, pv, valid, 1)
    upred = np.fft.ifft(uh * dp / math.sqrt(2 * math.pi * sh.eps))
    err = np.linalg.norm(res["u"] - upred) / np.linalg.norm(upred)
    assert err <= 1e-10, err


def test_spectral_prediction_2d_periodic():
    n = 32
    eps = 1.0 / 64
    rng = np.random.default_rng(5)
    kk = np.fft.fftfreq(n, d=1.0 / n)
    KX, KZ = np.meshgrid(kk, kk, indexing="ij")
    band = (np.hypot(KX, KZ) >= 6) & (np.hypot(KX, KZ) <= 10)
    f0 = np.real(np.fft.ifft2(band * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))))
    f1 = np.real(np.fft.ifft2(band * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))))) * 40
    c = 1.3
    pr = WL.periodic_2d(N=n, eps=eps, T=0.02, dt=2e-3, s=2, kappa=8.0, c=c)
    g = _grid(pr)
    axes = np.meshgrid(np.arange(n) / n, np.arange(n) / n, indexing="ij")
    xall = np.stack([a.ravel() for a in axes], axis=1)
    pick = np.random.default_rng(6).choice(n * n, size=48, replace=False)
    res = O.fga(g, pr.velocity, f0, f1, eps, (2, 2), (n, n), 0.0, 8.0, pr.nsteps, pr.dt,
                x=xall[pick])
    kvec = 2 * np.pi * np.stack([KX.ravel(), KZ.ravel()], axis=1)
    pv = O.p_points(g, eps, (n, n))
    valid = O.p_valid((n, n))
    dp = 2 * math.pi * eps / (n / n)
    uh = _prediction(np.fft.fft2(f0).ravel(), np.fft.fft2(f1).ravel(), kvec, eps, c,
                     pr.nsteps * pr.dt, pv, valid, 2)
    upred = np.fft.ifft2((uh * dp ** 2 / (2 * math.pi * eps)).reshape(n, n)).ravel()[pick]
    err = np.linalg.norm(res["u"] - upred) / np.linalg.norm(upred)
    assert err <= 1e-9, err


@pytest.mark.slow
def test_dalembert_error_is_order_eps_1d():
    # right-going packet, constant c: exact u(T,x) = u0(x - cT); the FGA error of the
    # method is O(eps) and halves when eps halves at a fixed eps*k0 and envelope.
    errs = []
    for N, eps in ((512, 1.0 / 128), (1024, 1.0 / 256)):
        k0 = 40 * math.pi * (1.0 / 128) / eps
        stride, _ = WL.default_stride_box(eps, (1.0 / N,), (N,), (True,))
        pr = WL.periodic_1d(N=N, eps=eps, k0=k0, s=stride[0], tau=1e-12)
        sh = pr.shots[0]
        res = O.fga(_grid(pr), pr.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box,
                    pr.tau, pr.kappa, pr.nsteps, pr.dt)
        x = np.arange(N) / N
        xs = np.mod(x - pr.nsteps * pr.dt, 1.0)
        ex = np.exp(-((xs - 0.5) ** 2) / 0.005) * np.cos(k0 * (x - pr.nsteps * pr.dt))
        errs.append(np.linalg.norm(res["u"].real - ex) / np.linalg.norm(ex))
    assert errs[0] <= 1e-2
    assert 1.7 <= errs[0] / errs[1] <= 2.3, errs


def test_field_is_real_for_real_data():
    # the two branches are complex conjugates of each other (p -> -p), so Im u vanishes
    pr = WL.lens_2d(N=64, eps=1.0 / 256, T=0.05, dt=5e-3, s=2, box=48, tau=1e-3,
                    k0=24 * math.pi, width2=0.01, x0=(0.5, 0.4))
    sh = pr.shots[0]
    g = _grid(pr)
    dec = O.decompose(g, pr.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, pr.tau)
    # guard band: no |psi| within 1e-9 of the threshold, so both sets mirror exactly
    for arr in (dec["psi_plus"], dec["psi_minus"]):
        r = np.abs(arr[:, dec["valid"]]) / (pr.tau * dec["M"])
        assert not np.any(np.abs(r - 1.0) < 1e-9)
    res = O.fga(g, pr.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, pr.tau, pr.kappa,
                pr.nsteps, pr.dt)
    u = res["u"]
    gauss = res["dec"]["gauss"]
    assert np.sum(gauss["sigma"] == 1) == np.sum(gauss["sigma"] == -1)
    assert np.linalg.norm(u.imag) <= 1e-12 * np.linalg.norm(u.real)


def test_keep_n_selection():
    rng = np.random.default_rng(9)
    plus = rng.standard_normal((6, 20)) + 1j * rng.standard_normal((6, 20))
    minus = rng.standard_normal((6, 20)) + 1j * rng.standard_normal((6, 20))
    valid = np.ones(20, dtype=bool)
    valid[[0, 7]] = False
    sp, sm, M = O.select(plus, minus, valid, 0.0, keep_n=11)
    for sel, arr in ((sp, plus), (sm, minus)):
        assert sel.size == 11
        a = np.abs(arr).ravel()
        mask = np.zeros(a.size, dtype=bool)
        mask[sel] = True
        vm = np.broadcast_to(valid[None, :], arr.shape).ravel()
        assert np.all(vm[sel])
        assert a[mask].min() >= a[~mask & vm].max()
    sp, sm, M = O.select(plus, minus, valid, 0.5)
    assert M == max(np.abs(plus[:, valid]).max(), np.abs(minus[:, valid]).max())
    assert np.all(np.abs(plus.ravel()[sp]) >= 0.5 * M)


def _pseudo_spectral_1d(c, u0, u1, T, nsub):
    """u_tt = c(x)^2 u_xx on the periodic unit interval: Fourier second derivative in x,
    classical RK4 in t on (u, u_t)."""
    n = u0.size
    k = 2 * np.pi * np.fft.fftfreq(n, d=1.0 / n)
    c2 = c ** 2

    def f(u, v):
        return v, c2 * np.real(np.fft.ifft(-(k ** 2) * np.fft.fft(u)))

    u, v = u0.copy(), u1.copy()
    dt = T / nsub
    for _ in range(nsub):
        k1 = f(u, v)
        k2 = f(u + 0.5 * dt * k1[0], v + 0.5 * dt * k1[1])
        k3 = f(u + 0.5 * dt * k2[0], v + 0.5 * dt * k2[1])
        k4 = f(u + dt * k3[0], v + dt * k3[1])
        u = u + dt / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        v = v + dt / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return u


@pytest.mark.slow
def test_order_eps_convergence_variable_medium_1d():
    # c = 1 + 0.2 sin(2 pi x) (its cubic spline, evaluated by the oracle, is used by both
    # solvers); packet with eps*k0 fixed and a fixed envelope; the FGA error against a fine
    # pseudo-spectral solve must fall like eps (log-log slope in [0.8, 1.2]).
    T = 0.25
    errs, epss = [], []
    for eps in (1.0 / 32, 1.0 / 64, 1.0 / 128, 1.0 / 256):
        N = 1024
        h = 1.0 / N
        g = O.Grid((N,), (h,), (0.0,), (True,))
        x = h * np.arange(N)
        coef = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        cgrid, _, _, _ = O.medium_eval(g, coef, x[:, None], order=0)
        k0 = 1.0 / eps
        env = np.exp(-((x - 0.5) ** 2) / 0.01)
        u0 = env * np.cos(k0 * x)
        du0 = env * (-2 * (x - 0.5) / 0.01 * np.cos(k0 * x) - k0 * np.sin(k0 * x))
        u1 = -cgrid * du0
        s = max(1, int(round(0.5 * math.sqrt(eps) / h)))
        while N % s:
            s -= 1
        res = O.fga(g, coef, u0, u1, eps, (s,), (N,), 1e-12, 8.0, 500, T / 500)
        ref = _pseudo_spectral_1d(cgrid, u0, u1, T, 4000)
        errs.append(np.linalg.norm(res["u"].real - ref) / np.linalg.norm(ref))
        epss.append(eps)
    slope = np.polyfit(np.log(epss), np.log(errs), 1)[0]
    assert 0.8 <= slope <= 1.2, (errs, slope)


def test_traces_equal_the_reconstruction_at_every_record():
    # the oracle's receiver traces (rays and the sum at the receivers in one pass) against
    # the separate propagate + reconstruct of the same Gaussians stopped at each record time
    pr = WL.lens_2d(N=64, eps=1.0 / 256, T=0.04, dt=5e-3, s=2, box=48, tau=1e-2,
                    k0=24 * math.pi, width2=0.01, x0=(0.5, 0.4))
    sh = pr.shots[0]
    g = _grid(pr)
    dec = O.decompose(g, pr.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, pr.tau)
    gs = dec["gauss"]
    W = O.quadrature_weight(g, sh.eps, sh.q_stride, sh.box)
    xr = np.stack([np.linspace(0.2, 0.8, 9), np.full(9, 0.45)], axis=1)
    every = 2
    tr = O.traces(g, pr.velocity, pr.nsteps, pr.dt, every, gs["sigma"], gs["q"], gs["p"], gs["psi"],
                  sh.eps, pr.kappa, W, xr)
    assert tr.shape == (pr.nsteps // every + 1, len(xr))
    for m in range(tr.shape[0]):
        st = O.propagate(g, pr.velocity, m * every, pr.dt, gs["sigma"], gs["q"], gs["p"])
        u = O.reconstruct(g, sh.eps, pr.kappa, W, st["Q"], st["P"], st["a"], gs["psi"], st["S"], xr)
        np.testing.assert_allclose(tr[m], u, rtol=0, atol=1e-12 * max(1.0, np.abs(u).max()))


def test_keep_n_ties_go_to_the_lower_q_then_p_index():
    # equal |psi| everywhere but one entry: the N - 1 remaining picks are the first valid
    # (q, p) in q-major, p-minor order
    plus = np.full((4, 10), 1.0 + 0j)
    plus[2, 5] = 3.0
    valid = np.ones(10, dtype=bool)
    valid[[0, 3]] = False
    sp, _, _ = O.select(plus, plus.copy(), valid, 0.0, keep_n=5)
    flat_valid = [q * 10 + p for q in range(4) for p in range(10) if valid[p]]
    expect = sorted([2 * 10 + 5] + [f for f in flat_valid if f != 25][:4])
    assert sp.tolist() == expect
