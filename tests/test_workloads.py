"""The seeded synthetic inputs: reproducible, shaped as the design notes state, and with
initial data u1 that is the time derivative of the outgoing ring u0."""

import math

import numpy as np

from paper_1304_3542_gb300 import workloads as WL


def test_layered_model_is_seeded_and_in_range():
    a = WL.gen_layered(1304)
    b = WL.gen_layered(1304)
    assert a.dtype == np.float32 and a.shape == WL.LAYERED_SHAPE == (737, 241)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, WL.gen_layered(1305))
    assert a.min() >= 1.5 - 1e-5 and a.max() <= 5.5 + 1e-5
    assert float(np.median(a[:, 0])) < 1.55  # the top layer is 1.5 km/s
    assert float(a[:, -1].mean()) > 3.5  # faster at depth


def test_ricker_dt_is_the_derivative_of_ricker():
    f = 15.0
    t = np.linspace(-0.2, 0.2, 401)
    h = 1e-6
    fd = (WL.ricker(t + h, f) - WL.ricker(t - h, f)) / (2 * h)
    np.testing.assert_allclose(WL.ricker_dt(t, f), fd, rtol=0, atol=1e-6 * np.abs(fd).max())


def test_ring_shot_is_an_outgoing_ring_with_eps_from_the_frequency():
    c = WL.gen_layered(1304).astype(np.float64)
    src, f = (4.6, 0.01), 15.0
    sh = WL.ricker_ring_shot(c, WL.LAYERED_H, src, f)
    cs = float(c[int(round(src[0] / WL.LAYERED_H)), int(round(src[1] / WL.LAYERED_H))])
    assert abs(sh.eps - cs / (2 * math.pi * f)) <= 1e-15
    s, nb = WL.default_stride_box(sh.eps, (WL.LAYERED_H,) * 2, c.shape, (False, False))
    assert tuple(sh.q_stride) == s and tuple(sh.box) == nb
    # u(t, r) = R(t - r/cs) around t0 = 1/f: u1 = du/dt at t0
    x = WL.LAYERED_H * np.arange(c.shape[0])
    z = WL.LAYERED_H * np.arange(c.shape[1])
    X, Z = np.meshgrid(x, z, indexing="ij")
    r = np.hypot(X - src[0], Z - src[1])
    h = 1e-7
    dudt = (WL.ricker(1.0 / f + h - r / cs, f) - WL.ricker(1.0 / f - h - r / cs, f)) / (2 * h)
    np.testing.assert_allclose(sh.u1, dudt, rtol=0, atol=1e-5 * np.abs(dudt).max())


def test_default_stride_and_box():
    for eps in (1.0 / 256, 0.016, 0.05):
        se = math.sqrt(eps)
        s, nb = WL.default_stride_box(eps, (0.0125, 0.01), (737, 241), (False, False))
        for k, hk in enumerate((0.0125, 0.01)):
            assert s[k] == max(1, int(round(0.5 * se / hk)))
            assert nb[k] % 32 == 0 and nb[k] >= 12 * se / hk and nb[k] - 32 < 12 * se / hk
    s, nb = WL.default_stride_box(1.0 / 128, (1.0 / 96,), (96,), (True,))
    assert nb == (96,) and 96 % s[0] == 0


def test_batch_shots_follow_their_ranges():
    prob = WL.layered_batch(nshots=16)
    assert len(prob.shots) == 16
    for sh in prob.shots:
        assert 1.0 <= sh.source[0] <= 8.2 and 0.01 <= sh.source[1] <= 0.5
        assert 8.0 <= sh.freq <= 25.0
    again = WL.layered_batch(nshots=16)
    assert [sh.source for sh in again.shots] == [sh.source for sh in prob.shots]
