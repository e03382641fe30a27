"""Pins of the oracle's linear field and 2LPT initial conditions (closed forms
for plane waves, power statistics, exact adjoint of the quadratic map)."""

import numpy as np
import pytest

from oracle import lpt, pm
from oracle.cosmology import Cosmology, linear_power, lpt_growth
from oracle.pm import Setup


def _grid(n, box):
    return np.arange(n) * box / n


def test_single_plane_wave_is_pure_zeldovich():
    n, box, amp, m = 16, 50.0, 0.3, 2
    st = Setup(n, n, box)
    k = 2 * np.pi * m / box
    qx = _grid(n, box)[:, None, None] * np.ones((n, n, n))
    s1, s2, _ = lpt.lpt_fields(amp * np.cos(k * qx), st)
    np.testing.assert_allclose(s1[:, 0], (-amp * np.sin(k * qx) / k).ravel(), atol=1e-13)
    np.testing.assert_allclose(s1[:, 1:], 0.0, atol=1e-13)
    np.testing.assert_allclose(s2, 0.0, atol=1e-13)        # 1D flow has no 2LPT term


def test_two_orthogonal_waves_second_order_closed_form():
    n, box, a1, a2, m1, m2 = 16, 40.0, 0.4, 0.25, 1, 3
    st = Setup(n, n, box)
    k1, k2 = 2 * np.pi * m1 / box, 2 * np.pi * m2 / box
    g = _grid(n, box)
    qx, qy = g[:, None, None] * np.ones((n, n, n)), g[None, :, None] * np.ones((n, n, n))
    _, s2, _ = lpt.lpt_fields(a1 * np.cos(k1 * qx) + a2 * np.cos(k2 * qy), st)
    # S = a1 a2 cos(k1 x) cos(k2 y); phi2 = -S / (k1^2 + k2^2); s2 = grad phi2
    c = a1 * a2 / (k1 ** 2 + k2 ** 2)
    np.testing.assert_allclose(s2[:, 0], (c * k1 * np.sin(k1 * qx) * np.cos(k2 * qy)).ravel(), atol=1e-13)
    np.testing.assert_allclose(s2[:, 1], (c * k2 * np.cos(k1 * qx) * np.sin(k2 * qy)).ravel(), atol=1e-13)
    np.testing.assert_allclose(s2[:, 2], 0.0, atol=1e-13)


def test_linear_field_single_mode_amplitude():
    n, box, m = 16, 64.0, 3
    st = Setup(n, 2 * n, box)
    k = 2 * np.pi * m / box
    qx = _grid(n, box)[:, None, None] * np.ones((n, n, n))
    dl = lpt.linear_field(np.cos(k * qx), st)
    amp = np.sqrt(linear_power(np.array(k), st.cosmo) / st.spacing ** 3)
    np.testing.assert_allclose(dl, amp * np.cos(k * qx), atol=1e-12 * amp)


def test_linear_field_reproduces_power_spectrum():
    n, box = 64, 256.0
    st = Setup(n, n, box)
    rng = np.random.default_rng(11)
    ratios, weights = [], []
    for _ in range(3):
        dl = lpt.linear_field(rng.standard_normal((n, n, n)), st)
        kmean, p, nm = pm.power_of_mesh(dl, box)
        # mode-averaged expectation in each bin
        (kx, ky, kz), _ = pm.rfft_wavenumbers(n, box)
        kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
        _, pexp, _ = pm.power_of_mesh(np.zeros((n, n, n)), box)
        ok = nm > 500
        ratios.append(p[ok] / linear_power(kmean[ok], st.cosmo))
        weights.append(nm[ok])
    r = np.average(np.concatenate(ratios), weights=np.concatenate(weights))
    assert abs(r - 1.0) < 0.03


def test_initial_momentum_is_growth_rate_times_displacement():
    st = Setup(8, 16, 64.0)
    noise = np.random.default_rng(1).standard_normal((8, 8, 8))
    s, p = lpt.initial_conditions(noise, st)
    d1, d2, g1, g2 = lpt_growth(st.cosmo, st.a_init)
    s1, s2, _ = lpt.lpt_fields(lpt.linear_field(noise, st), st)
    np.testing.assert_allclose(s, d1 * s1 + d2 * s2, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(p, g1 * s1 + g2 * s2, rtol=1e-14, atol=1e-14)
    assert d2 < 0 and abs(d2 / d1 ** 2 + 3 / 7) < 1e-3     # matter era


def test_initial_momentum_is_the_time_derivative_of_the_displacement():
    # p = a^3 E(a) ds/da with s(a) = D1(a) s1 + D2(a) s2: central differences
    # of the 2LPT displacement in a_init, on the same noise, give p at both
    # orders (g1 = a^3 E D1', g2 = a^3 E D2').
    noise = np.random.default_rng(4).standard_normal((8, 8, 8))
    a0, eps = 1.0 / 64, 1e-6
    st = Setup(8, 16, 64.0, a_init=a0)
    _, p = lpt.initial_conditions(noise, st)
    s_up, _ = lpt.initial_conditions(noise, Setup(8, 16, 64.0, a_init=a0 + eps))
    s_dn, _ = lpt.initial_conditions(noise, Setup(8, 16, 64.0, a_init=a0 - eps))
    e = np.sqrt(st.cosmo.omega_m * a0 ** -3 + 1 - st.cosmo.omega_m)
    p_fd = a0 ** 3 * e * (s_up - s_dn) / (2 * eps)
    np.testing.assert_allclose(p_fd, p, rtol=0, atol=1e-7 * np.abs(p).max())
    # the second order alone: its share of p is ~D1, so check it separately
    s1, s2, _ = lpt.lpt_fields(lpt.linear_field(noise, st), st)
    g2 = lpt_growth(st.cosmo, a0)[3]
    g2_fd = a0 ** 3 * e * (lpt_growth(st.cosmo, a0 + eps)[1] - lpt_growth(st.cosmo, a0 - eps)[1]) / (2 * eps)
    assert abs(g2 / g2_fd - 1) < 1e-7, (g2, g2_fd)


def _ic_objective(noise, st, lam, mu):
    s, p = lpt.initial_conditions(noise, st)
    return np.sum(lam * s) + np.sum(mu * p)


def test_initial_conditions_vjp_finite_difference():
    rng = np.random.default_rng(2)
    n = 8
    st = Setup(n, 16, 40.0, Cosmology(0.3, 0.8))
    noise = rng.standard_normal((n, n, n))
    lam, mu = rng.standard_normal((n ** 3, 3)), rng.standard_normal((n ** 3, 3))
    g_noise, g_om, g_s8 = lpt.initial_conditions_vjp(noise, lam, mu, st)
    for _ in range(3):
        v = rng.standard_normal((n, n, n))
        eps = 1e-3          # the map is quadratic: central differences are exact
        fd = (_ic_objective(noise + eps * v, st, lam, mu) - _ic_objective(noise - eps * v, st, lam, mu)) / (2 * eps)
        assert abs(fd - np.sum(g_noise * v)) < 1e-9 * max(1.0, abs(fd))
    for name, grad in (("omega_m", g_om), ("sigma8", g_s8)):
        eps = 1e-5
        vals = []
        for sgn in (1, -1):
            c = st.cosmo
            c = Cosmology(c.omega_m + sgn * eps, c.sigma8, c.h, c.n_s) if name == "omega_m" else \
                Cosmology(c.omega_m, c.sigma8 + sgn * eps, c.h, c.n_s)
            vals.append(_ic_objective(noise, Setup(n, 16, 40.0, c), lam, mu))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grad) < 1e-6 * max(1.0, abs(fd)), (name, fd, grad)
